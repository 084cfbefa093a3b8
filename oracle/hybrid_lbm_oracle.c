/*
 * hybrid_lbm_oracle.c -- plain, slow FP64 CPU oracle of the hybrid
 * free-energy lattice Boltzmann scheme for binary mixtures of Tiribocchi,
 * Stella, Gonnella and Lamura (arXiv:0902.3921).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path calls, links or
 * loads this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA library: the lattice tables below are typed in
 * again from the paper, by design.
 *
 * Every function follows one passage of the paper, named in its comment,
 * in the paper's order and notation.  No blocking, no fusion, no
 * reordering: each operator is applied to a whole field before the next one
 * starts.  All arithmetic is IEEE double, round-to-nearest; the build uses
 * -ffp-contract=off so x86-64 and AArch64 give the same bits.  The site loops
 * carry OpenMP pragmas: every site's value is computed by the same
 * operations whichever thread runs it (no reduction crosses sites), so any
 * thread count gives the same bits as one thread (orc_set_threads).
 *
 * Conventions (the paper is silent on them; the readings are listed in the
 * design notes of the repository):
 *   - lattice spacing and LB time step are 1 (Sec. III), so c = 1, c_s^2 = 1/3;
 *   - periodic boundaries on every axis;
 *   - fields are row-major [z][y][x], site s = (z*Ly + y)*Lx + x;
 *   - populations are [i][s], vector fields [alpha][s];
 *   - the FD time step is dt_FD = dt_LB / m = 1/m (Sec. II C);
 *   - within one LB step both halves read the state at time t: the LB update
 *     uses phi(t), the FD update uses u*(t) (explicit operator splitting).
 *
 * The D3Q19 stencil weights of orc_stencil_weights (3D branch) generalise
 * Eqs. 30-31, which the paper gives in 2D only, so no printed 3D value exists.
 * The 3D operators are pinned by closed forms instead: exact first and second
 * derivatives of low-order polynomials, their Fourier symbols, and the flat
 * interface relaxing to phi0 tanh(x/xi) of Eq. 2 in 3D.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int dims;            /* 2 (D2Q9) or 3 (D3Q19)                               */
  int Lx, Ly, Lz;      /* periodic lattice; Lz = 1 in 2D                      */
  double a, b, kappa;  /* Ginzburg-Landau free energy, Eq. 1                  */
  double T;            /* temperature of the ideal-gas term n T ln n, Eq. 1   */
  double tau;          /* BGK relaxation time, Eq. 11                         */
  double Gamma;        /* mobility, Eq. 10                                    */
  double N, Q;         /* stencil parameters, Eqs. 30-31                      */
  int m;               /* FD substeps per LB step, Sec. II C                  */
  int adv_variant;     /* 0: Eqs. 32-35 as printed; 1: upwind flux form      */
  int cubic_at_half;   /* 0: b lap (phi^n)^3 as printed in Eq. 36; 1: cube of
                          phi^{n+1/2} (an option for experiments)             */
  double g[3];         /* body force per unit density, Sec. III (G = n g)     */
  long force_steps;    /* G acts for LB steps t = 0 .. force_steps-1          */
  int stencil_fd;      /* 0: Eqs. 33 and 36 as printed (central d u, 5-point
                          Laplacian); 1: the stencil operators of Eqs. 30-31
                          with (N, Q) in their place, the "more general
                          stencil" of Sec. II C (after Eq. 36) and Sec. IV    */
} orc_params;

/* ---- lattices (Sec. II A, Fig. 1; D3Q19 is the 3D generalisation) -------- */

static const int E2Q9[9][3] = {
    {0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W2Q9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                               1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int E3Q19[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W3Q19[19] = {
    1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2/3, Sec. II A */

int orc_nq(int dims) { return dims == 3 ? 19 : 9; }

/* Threads of the site loops (n <= 0: all cores); returns the count in use.
 * The result of every function is the same for any count. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n <= 0) n = omp_get_num_procs();
  omp_set_num_threads(n);
  return n;
#else
  (void)n;
  return 1;
#endif
}

static const int *orc_e(int dims, int i) {
  return dims == 3 ? E3Q19[i] : E2Q9[i];
}
static double orc_w(int dims, int i) {
  return dims == 3 ? W3Q19[i] : W2Q9[i];
}

/* Copies the lattice vectors (q x 3 ints) and weights (q doubles). */
void orc_lattice(int dims, int *e, double *w) {
  int q = orc_nq(dims);
  for (int i = 0; i < q; i++) {
    for (int k = 0; k < 3; k++) e[3 * i + k] = orc_e(dims, i)[k];
    w[i] = orc_w(dims, i);
  }
}

static long orc_sites(const orc_params *p) {
  return (long)p->Lx * p->Ly * (p->dims == 3 ? p->Lz : 1);
}

static int wrap(int x, int L) { return ((x % L) + L) % L; }

/* Site index of (x + dx, y + dy, z + dz) with periodic wrap. */
static long nbr(const orc_params *p, int x, int y, int z, int dx, int dy,
                int dz) {
  int Lz = p->dims == 3 ? p->Lz : 1;
  return ((long)wrap(z + dz, Lz) * p->Ly + wrap(y + dy, p->Ly)) * p->Lx +
         wrap(x + dx, p->Lx);
}

/* ---- stencils, Sec. II B, Eqs. 30-31 ------------------------------------- */

/*
 * Weight cubes w[(dz+1)*9 + (dy+1)*3 + (dx+1)] of the discrete operators.
 *   grad[alpha] : d_{D,alpha}, Eq. 30 (d_Dy is the transpose of d_Dx).
 *   lap         : lap_D, Eq. 31.
 * 2D: d_Dx = [[-M,0,M],[-N,0,N],[-M,0,M]], M = (1-2N)/4 so 2N + 4M = 1;
 *     lap_D = [[R,Q,R],[Q,-4(Q+R),Q],[R,Q,R]], R = (1-Q)/2 so Q + 2R = 1.
 * 3D (D3Q19 neighbourhood): N on the two face neighbours along alpha, M on
 *     the eight edge neighbours with e_alpha != 0 (2N + 8M = 1); Q on the six
 *     faces, R on the twelve edges, centre -(6Q+12R) (Q + 4R = 1).
 */
void orc_stencil_weights(int dims, double N, double Q, double *grad /*3*27*/,
                         double *lap /*27*/) {
  double M = dims == 3 ? (1.0 - 2.0 * N) / 8.0 : (1.0 - 2.0 * N) / 4.0;
  double R = dims == 3 ? (1.0 - Q) / 4.0 : (1.0 - Q) / 2.0;
  memset(grad, 0, sizeof(double) * 3 * 27);
  memset(lap, 0, sizeof(double) * 27);
  int zlo = dims == 3 ? -1 : 0, zhi = dims == 3 ? 1 : 0;
  double centre = 0.0;
  for (int dz = zlo; dz <= zhi; dz++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dx = -1; dx <= 1; dx++) {
        int d[3] = {dx, dy, dz};
        int nn = dx * dx + dy * dy + dz * dz;
        int k = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
        if (nn == 1) {
          lap[k] = Q;
          centre += Q;
        } else if (nn == 2) {
          lap[k] = R;
          centre += R;
        }
        for (int al = 0; al < dims; al++) {
          if (d[al] == 0) continue;
          if (nn == 1) grad[al * 27 + k] = N * d[al];
          else if (nn == 2) grad[al * 27 + k] = M * d[al];
        }
      }
  lap[13] = -centre;
}

/* out = sum over the 3x3(x3) neighbourhood of w * field (periodic). */
static void apply_stencil(const orc_params *p, const double *w,
                          const double *field, double *out) {
  int Lz = p->dims == 3 ? p->Lz : 1;
  int zlo = p->dims == 3 ? -1 : 0, zhi = p->dims == 3 ? 1 : 0;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < Lz; z++)
    for (int y = 0; y < p->Ly; y++)
      for (int x = 0; x < p->Lx; x++) {
        double acc = 0.0;
        for (int dz = zlo; dz <= zhi; dz++)
          for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
              double wk = w[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
              if (wk != 0.0) acc += wk * field[nbr(p, x, y, z, dx, dy, dz)];
            }
        out[((long)z * p->Ly + y) * p->Lx + x] = acc;
      }
}

/* Discrete gradient d_D (Eq. 30) of a scalar field; out is [dims][S]. */
void orc_grad_D(const orc_params *p, const double *field, double *out) {
  double grad[81], lap[27];
  orc_stencil_weights(p->dims, p->N, p->Q, grad, lap);
  long S = orc_sites(p);
  for (int al = 0; al < p->dims; al++)
    apply_stencil(p, grad + 27 * al, field, out + al * S);
}

/* Discrete Laplacian lap_D (Eq. 31) with the stencil's (Q, R). */
void orc_lap_D(const orc_params *p, const double *field, double *out) {
  double grad[81], lap[27];
  orc_stencil_weights(p->dims, p->N, p->Q, grad, lap);
  apply_stencil(p, lap, field, out);
}

/* Standard Laplacian of the FD scheme: Eq. 31 with Q = 1, R = 0 (Eq. 36). */
void orc_lap_std(const orc_params *p, const double *field, double *out) {
  double grad[81], lap[27];
  orc_stencil_weights(p->dims, 0.5, 1.0, grad, lap);
  apply_stencil(p, lap, field, out);
}

/* ---- thermodynamics, Sec. II ---------------------------------------------- */

/* Chemical potential mu = a phi + b phi^3 - kappa lap_D phi, Eq. 5. */
void orc_mu(const orc_params *p, const double *phi, double *mu) {
  long S = orc_sites(p);
  double *lap = malloc(sizeof(double) * S);
  orc_lap_D(p, phi, lap);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S; s++)
    mu[s] = p->a * phi[s] + p->b * phi[s] * phi[s] * phi[s] -
            p->kappa * lap[s];
  free(lap);
}

/*
 * Force density F, Eq. 28: F = grad(n c_s^2 - p^i) - phi grad mu with the
 * ideal-gas pressure p^i = n T (Eq. 1).  For T = c_s^2 the first term
 * vanishes (the second form of Eq. 28).  The external force G = n g of
 * Sec. III is added while t < force_steps.  n is the density at time t.
 * out is [dims][S].
 */
void orc_force(const orc_params *p, const double *phi, const double *n, long t,
               double *F) {
  long S = orc_sites(p);
  int d = p->dims;
  double *mu = malloc(sizeof(double) * S);
  double *gmu = malloc(sizeof(double) * S * d);
  orc_mu(p, phi, mu);
  orc_grad_D(p, mu, gmu);
  for (int al = 0; al < d; al++)
    for (long s = 0; s < S; s++) F[al * S + s] = -phi[s] * gmu[al * S + s];
  if (p->T != CS2) {
    double *pn = malloc(sizeof(double) * S);
    double *gpn = malloc(sizeof(double) * S * d);
    for (long s = 0; s < S; s++) pn[s] = (CS2 - p->T) * n[s];
    orc_grad_D(p, pn, gpn);
    for (long k = 0; k < S * d; k++) F[k] += gpn[k];
    free(pn);
    free(gpn);
  }
  if (t < p->force_steps)
    for (int al = 0; al < d; al++)
      for (long s = 0; s < S; s++) F[al * S + s] += n[s] * p->g[al];
  free(mu);
  free(gmu);
}

/* ---- LB with forcing term, Sec. II A -------------------------------------- */

/* Second-order equilibrium, Eq. 15: feq_i = w_i n [1 + e.u/cs2 +
 * uu:(ee - cs2 I)/(2 cs2^2)]. */
void orc_feq(int dims, double n, const double *u, double *feq) {
  int q = orc_nq(dims);
  for (int i = 0; i < q; i++) {
    const int *e = orc_e(dims, i);
    double eu = 0.0, uu = 0.0;
    for (int al = 0; al < dims; al++) {
      eu += e[al] * u[al];
      uu += u[al] * u[al];
    }
    /* uu:(ee - cs2 I) = (e.u)^2 - cs2 |u|^2 */
    feq[i] = orc_w(dims, i) * n *
             (1.0 + eu / CS2 + (eu * eu - CS2 * uu) / (2.0 * CS2 * CS2));
  }
}

/* Lattice forcing term, Eq. 29 (A = 0, B and C of Eq. 26):
 * F_i = (1 - 1/(2 tau)) w_i [(e_i - u*)/cs2 + (e_i.u*) e_i / cs2^2] . F */
void orc_forcing_term(int dims, double tau, const double *u, const double *F,
                      double *Fi) {
  int q = orc_nq(dims);
  double pref = 1.0 - 1.0 / (2.0 * tau);
  for (int i = 0; i < q; i++) {
    const int *e = orc_e(dims, i);
    double eu = 0.0, acc = 0.0;
    for (int al = 0; al < dims; al++) eu += e[al] * u[al];
    for (int al = 0; al < dims; al++)
      acc += ((e[al] - u[al]) / CS2 + eu * e[al] / (CS2 * CS2)) * F[al];
    Fi[i] = pref * orc_w(dims, i) * acc;
  }
}

/* Density n = sum_i f_i (Eq. 12) at every site. */
void orc_density(const orc_params *p, const double *f, double *n) {
  long S = orc_sites(p);
  int q = orc_nq(p->dims);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S; s++) {
    double acc = 0.0;
    for (int i = 0; i < q; i++) acc += f[i * S + s];
    n[s] = acc;
  }
}

/* n = sum f_i (Eq. 12) and u* from n u* = sum f_i e_i + F/2 (Eq. 18). */
void orc_moments(const orc_params *p, const double *f, const double *F,
                 double *n, double *u) {
  long S = orc_sites(p);
  int q = orc_nq(p->dims), d = p->dims;
  orc_density(p, f, n);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S; s++)
    for (int al = 0; al < d; al++) {
      double j = 0.0;
      for (int i = 0; i < q; i++) j += f[i * S + s] * orc_e(d, i)[al];
      u[al * S + s] = (j + 0.5 * F[al * S + s]) / n[s];
    }
}

/*
 * Initial populations f_i = feq_i(n, u - F/(2n)) (Eqs. 15, 18), so that the
 * u* of Eq. 18 at t = 0 equals the given u.  F is evaluated at t = 0.
 */
void orc_init(const orc_params *p, const double *n, const double *phi,
              const double *u, double *f) {
  long S = orc_sites(p);
  int q = orc_nq(p->dims), d = p->dims;
  double *F = malloc(sizeof(double) * S * d);
  orc_force(p, phi, n, 0, F);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S; s++) {
    double us[3] = {0, 0, 0}, feq[19];
    for (int al = 0; al < d; al++)
      us[al] = u[al * S + s] - F[al * S + s] / (2.0 * n[s]);
    orc_feq(d, n[s], us, feq);
    for (int i = 0; i < q; i++) f[i * S + s] = feq[i];
  }
  free(F);
}

/*
 * One LB step, Eq. 17 with Eqs. 15, 18, 28, 29:
 *   f_i(r + e_i, t+1) = f_i(r,t) - [f_i - feq_i(n, u*)]/tau + F_i.
 * f holds the pre-collision populations at t on entry and at t+1 on return.
 * Returns n(t) and u*(t) (the velocity the FD step of the same LB step uses).
 */
void orc_lb_step(const orc_params *p, double *f, const double *phi, long t,
                 double *n_out, double *u_out) {
  long S = orc_sites(p);
  int q = orc_nq(p->dims), d = p->dims;
  int Lz = p->dims == 3 ? p->Lz : 1;
  double *n = malloc(sizeof(double) * S);
  double *F = malloc(sizeof(double) * S * d);
  double *u = malloc(sizeof(double) * S * d);
  double *fpost = malloc(sizeof(double) * S * q);
  orc_density(p, f, n);
  orc_force(p, phi, n, t, F);
  orc_moments(p, f, F, n, u);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S; s++) {
    double us[3] = {0, 0, 0}, Fs[3] = {0, 0, 0}, feq[19], Fi[19];
    for (int al = 0; al < d; al++) {
      us[al] = u[al * S + s];
      Fs[al] = F[al * S + s];
    }
    orc_feq(d, n[s], us, feq);
    orc_forcing_term(d, p->tau, us, Fs, Fi);
    for (int i = 0; i < q; i++)
      fpost[i * S + s] =
          f[i * S + s] - (f[i * S + s] - feq[i]) / p->tau + Fi[i];
  }
  /* streaming: the left-hand side of Eq. 17, periodic */
  for (int i = 0; i < q; i++) {
    const int *e = orc_e(d, i);
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < Lz; z++)
      for (int y = 0; y < p->Ly; y++)
        for (int x = 0; x < p->Lx; x++)
          f[i * S + nbr(p, x, y, z, e[0], e[1], e[2])] =
              fpost[i * S + ((long)z * p->Ly + y) * p->Lx + x];
  }
  if (n_out) memcpy(n_out, n, sizeof(double) * S);
  if (u_out) memcpy(u_out, u, sizeof(double) * S * d);
  free(n);
  free(F);
  free(u);
  free(fpost);
}

/* ---- convection-diffusion by finite differences, Sec. II C --------------- */

/*
 * Convective half step, Eq. 32, with the central derivative of u (Eq. 33)
 * and the upwind derivative of phi chosen by the sign of u at the site
 * (Eqs. 34-35; u = 0 takes the backward difference, the product is 0 then).
 * adv_variant 1 replaces it by the conservative upwind flux form
 * phi - dt sum_alpha [J(i+1/2) - J(i-1/2)], J = U phi_upwind, U the mean of
 * the two site velocities.
 */
void orc_advect(const orc_params *p, const double *phi, const double *u,
                double dt, double *out) {
  long S = orc_sites(p);
  int d = p->dims;
  int Lz = p->dims == 3 ? p->Lz : 1;
  /* stencil_fd: d_alpha u_alpha by the stencil derivative of Eq. 30 */
  double *du_st = NULL;
  if (p->stencil_fd && p->adv_variant == 0) {
    double *g = malloc(sizeof(double) * 3 * S);
    du_st = malloc(sizeof(double) * 3 * S);
    for (int al = 0; al < d; al++) {
      orc_grad_D(p, u + al * S, g);
      memcpy(du_st + al * S, g + al * S, sizeof(double) * S);
    }
    free(g);
  }
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < Lz; z++)
    for (int y = 0; y < p->Ly; y++)
      for (int x = 0; x < p->Lx; x++) {
        long s = ((long)z * p->Ly + y) * p->Lx + x;
        double tend = 0.0;
        for (int al = 0; al < d; al++) {
          int dp[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
          dp[al] = 1;
          dm[al] = -1;
          long sp = nbr(p, x, y, z, dp[0], dp[1], dp[2]);
          long sm = nbr(p, x, y, z, dm[0], dm[1], dm[2]);
          const double *ua = u + al * S;
          if (p->adv_variant == 0) {
            double du = du_st ? du_st[al * S + s]          /* Eq. 30 */
                              : (ua[sp] - ua[sm]) / 2.0;   /* Eq. 33 */
            double dphi = ua[s] < 0.0 ? phi[sp] - phi[s]  /* Eq. 35 */
                                      : phi[s] - phi[sm]; /* Eq. 34 */
            tend += phi[s] * du + ua[s] * dphi;
          } else {
            double Up = 0.5 * (ua[s] + ua[sp]);
            double Um = 0.5 * (ua[sm] + ua[s]);
            double Jp = Up > 0.0 ? Up * phi[s] : Up * phi[sp];
            double Jm = Um > 0.0 ? Um * phi[sm] : Um * phi[s];
            tend += Jp - Jm;
          }
        }
        out[s] = phi[s] - dt * tend;
      }
  free(du_st);
}

/*
 * Diffusive half step, Eq. 36:
 *   phi^{n+1} = phi^{n+1/2} + dt Gamma [a lap phi^{n+1/2} + b lap (phi^n)^3
 *                                       - kappa lap(lap phi^{n+1/2})]
 * with the standard Laplacian (Eq. 31 with Q = 1, R = 0), or with lap_D of
 * Eq. 31 at the stencil's (Q, R) when stencil_fd is set (Sec. II C, the
 * sentence after Eq. 36: other stencils for this Laplacian are possible).
 */
void orc_diffuse(const orc_params *p, const double *phi_half,
                 const double *phi_old, double dt, double *out) {
  long S = orc_sites(p);
  double *cube = malloc(sizeof(double) * S);
  double *lap_h = malloc(sizeof(double) * S);
  double *lap_c = malloc(sizeof(double) * S);
  double *lap_lap = malloc(sizeof(double) * S);
  const double *src = p->cubic_at_half ? phi_half : phi_old;
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S; s++) cube[s] = src[s] * src[s] * src[s];
  void (*lap)(const orc_params *, const double *, double *) = p->stencil_fd ? orc_lap_D : orc_lap_std;
  lap(p, phi_half, lap_h);
  lap(p, cube, lap_c);
  lap(p, lap_h, lap_lap);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < S; s++)
    out[s] = phi_half[s] + dt * p->Gamma *
                               (p->a * lap_h[s] + p->b * lap_c[s] -
                                p->kappa * lap_lap[s]);
  free(cube);
  free(lap_h);
  free(lap_c);
  free(lap_lap);
}

/* One LB step of the FD scheme: m substeps of dt = 1/m, u* frozen. */
void orc_fd_step(const orc_params *p, double *phi, const double *u) {
  long S = orc_sites(p);
  double dt = 1.0 / p->m;
  double *half = malloc(sizeof(double) * S);
  double *next = malloc(sizeof(double) * S);
  for (int k = 0; k < p->m; k++) {
    orc_advect(p, phi, u, dt, half);
    orc_diffuse(p, half, phi, dt, next);
    memcpy(phi, next, sizeof(double) * S);
  }
  free(half);
  free(next);
}

/* nsteps full hybrid steps from time t0: LB step (Eq. 17) then FD step
 * (Eqs. 32-36) with the u*(t) it produced.  Optionally returns n and u* of
 * the last step. */
void orc_run(const orc_params *p, double *f, double *phi, long t0, long nsteps,
             double *n_last, double *u_last) {
  long S = orc_sites(p);
  double *n = malloc(sizeof(double) * S);
  double *u = malloc(sizeof(double) * S * p->dims);
  for (long t = t0; t < t0 + nsteps; t++) {
    orc_lb_step(p, f, phi, t, n, u);
    orc_fd_step(p, phi, u);
  }
  if (n_last) memcpy(n_last, n, sizeof(double) * S);
  if (u_last) memcpy(u_last, u, sizeof(double) * S * p->dims);
  free(n);
  free(u);
}

/*
 * Observables at time t from the pre-collision populations and phi(t):
 * n, u* (Eq. 18) and the diagonal pressure p0 of Eq. 6,
 *   p0 = n T + a phi^2/2 + 3 b phi^4/4 - kappa phi lap phi - kappa |grad phi|^2/2,
 * with the stencil operators of Eqs. 30-31.
 */
void orc_observe(const orc_params *p, const double *f, const double *phi,
                 long t, double *n, double *u, double *p0) {
  long S = orc_sites(p);
  int d = p->dims;
  double *F = malloc(sizeof(double) * S * d);
  double *lap = malloc(sizeof(double) * S);
  double *grad = malloc(sizeof(double) * S * d);
  orc_density(p, f, n);
  orc_force(p, phi, n, t, F);
  orc_moments(p, f, F, n, u);
  orc_lap_D(p, phi, lap);
  orc_grad_D(p, phi, grad);
  for (long s = 0; s < S; s++) {
    double g2 = 0.0;
    for (int al = 0; al < d; al++) g2 += grad[al * S + s] * grad[al * S + s];
    double ph = phi[s];
    p0[s] = n[s] * p->T + p->a * ph * ph / 2.0 +
            3.0 * p->b * ph * ph * ph * ph / 4.0 - p->kappa * ph * lap[s] -
            p->kappa * g2 / 2.0;
  }
  free(F);
  free(lap);
  free(grad);
}
