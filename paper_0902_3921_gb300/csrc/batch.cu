// batch.cu -- many independent 2D lattices (uneven sizes, per-instance body
// force schedules) advanced together: by one persistent launch, or on the
// tiled path described below.
//
// Persistent path: every instance is owned by exactly one CTA (instances are assigned to CTAs
// longest-first on the host), and a CTA advances each of its instances
// through all requested LB steps before it moves to the next one, so CTAs
// never wait for one another: the only synchronisation is __syncthreads
// between the phases of a step.  Per step and instance:
//   mu    = a phi + b phi^3 - kappa lap_D phi                      (Eq. 5)
//   collide: F = -phi d_D mu + n g, pull streaming, n, u*, BGK + Guo F_i
//                                                  (Eqs. 12, 15, 17, 18, 28, 29)
//   m FD substeps: phih (Eqs. 32-35), psi, new phi (Eq. 36)
// Per-site arrays of all instances are packed end to end (offset off_k; the
// instances grouped by shape), one plane per population:
// h[i * ST + off_k + y * Lx + x].  The instance's neighbours stay in L1/L2
// while the CTA works on it.
//
// Tiled path (FP32 deviations, printed advection form, even m, Lx % 4 == 0):
// the step is instead the collide over a table of (instance, 32 x 16 tile)
// items -- the persistent TMA-staged kernel, through one set of tensor maps
// per instance shape, for the instances at least 64 on a side, the tile
// kernel for the rest -- and m / 2 launches of the two-substep wavefront FD
// kernel over a table of (instance, strip, segment of at most 48 rows) items
// (longest first; HLBM_BATCH_FD_ROWS changes the 48),
// per LB step, captured in a CUDA graph: every population and phi value is
// read and written once per step as on a single lattice.  The launches are
// plain (no programmatic dependent launch: an early-scheduled grid would hold
// the SM slots that the previous grid's later CTAs need).  The autotuner
// times both paths on the zeroed state and keeps the faster
// (HLBM_BATCH_PATH=tiled or persistent fixes the choice).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "lbm_common.cuh"

namespace {

using namespace hlbm;

struct DevInst {
  int Lx, Ly;
  long long off;
  double gx, gy;
  long long force_steps;
};

template <typename C>
struct BatchArgs {
  const DevInst *inst;
  const int *order;      // instance ids grouped by CTA
  const int *cta_first;  // first index into order for each CTA (count + 1 entries)
  C *h[2];               // populations (deviations), planes of ST sites
  C *phi[3];             // phi(t), phi(t+1), FD scratch
  C *u;                  // u* planes (2 x ST)
  C *mu;                 // chemical potential
  C *fa, *fq;            // FD phih and psi
  long long ST;
  C a, b, kappa, tau_inv, pref, N, M, Q, R, C0, dt, dtG;
  int m, adv_variant, cubic_at_half;
};

__device__ __forceinline__ int wrp(int x, int L) { return x < 0 ? x + L : (x >= L ? x - L : x); }

template <typename C>
__device__ void batch_instance_step(const BatchArgs<C> &A, const DevInst &I, long long t) {
  const int Lx = I.Lx, Ly = I.Ly;
  const long long off = I.off, ST = A.ST;
  const int in = (int)(t & 1), out = 1 - in;
  const C *hin = A.h[in] + off;
  C *hout = A.h[out] + off;
  const C *phi = A.phi[in] + off;
  C *mu = A.mu + off, *ux = A.u + off, *uy = A.u + ST + off;
  const int tx = threadIdx.x, ty = threadIdx.y, bx = blockDim.x, by = blockDim.y;
  // mu on every site (Eq. 5)
  for (int y = ty; y < Ly; y += by) {
    const int ym = wrp(y - 1, Ly), yp = wrp(y + 1, Ly);
    for (int x = tx; x < Lx; x += bx) {
      const int xm = wrp(x - 1, Lx), xp = wrp(x + 1, Lx);
      const C c = phi[y * Lx + x];
      C lap = A.R * phi[ym * Lx + xm];
      lap += A.Q * phi[ym * Lx + x];
      lap += A.R * phi[ym * Lx + xp];
      lap += A.Q * phi[y * Lx + xm];
      lap += A.C0 * c;
      lap += A.Q * phi[y * Lx + xp];
      lap += A.R * phi[yp * Lx + xm];
      lap += A.Q * phi[yp * Lx + x];
      lap += A.R * phi[yp * Lx + xp];
      mu[y * Lx + x] = A.a * c + A.b * c * c * c - A.kappa * lap;
    }
  }
  __syncthreads();
  const bool on = t < I.force_steps;
  const C gx = on ? (C)I.gx : C(0), gy = on ? (C)I.gy : C(0);
  for (int y = ty; y < Ly; y += by) {
    const int ym = wrp(y - 1, Ly), yp = wrp(y + 1, Ly);
    for (int x = tx; x < Lx; x += bx) {
      const int xm = wrp(x - 1, Lx), xp = wrp(x + 1, Lx);
      const int rc = y * Lx, rm = ym * Lx, rp = yp * Lx;
      C gmx = -A.M * mu[rm + xm];
      gmx += A.M * mu[rm + xp];
      gmx += -A.N * mu[rc + xm];
      gmx += A.N * mu[rc + xp];
      gmx += -A.M * mu[rp + xm];
      gmx += A.M * mu[rp + xp];
      C gmy = -A.M * mu[rm + xm];
      gmy += -A.N * mu[rm + x];
      gmy += -A.M * mu[rm + xp];
      gmy += A.M * mu[rp + xm];
      gmy += A.N * mu[rp + x];
      gmy += A.M * mu[rp + xp];
      const C ph = phi[rc + x];
      C Fx = -ph * gmx, Fy = -ph * gmy;
      C h[9];
      h[0] = hin[0 * ST + rc + x];
      h[1] = hin[1 * ST + rc + xm];
      h[2] = hin[2 * ST + rm + x];
      h[3] = hin[3 * ST + rc + xp];
      h[4] = hin[4 * ST + rp + x];
      h[5] = hin[5 * ST + rm + xm];
      h[6] = hin[6 * ST + rm + xp];
      h[7] = hin[7 * ST + rp + xp];
      h[8] = hin[8 * ST + rp + xm];
      C dens = h[0];
#pragma unroll
      for (int i = 1; i < 9; ++i) dens += h[i];
      const C jx = ((h[1] - h[3]) + (h[5] - h[7])) + (h[8] - h[6]);
      const C jy = ((h[2] - h[4]) + (h[5] - h[7])) + (h[6] - h[8]);
      const C n = C(1) + dens;
      Fx += n * gx;
      Fy += n * gy;
      const C vx = (jx + C(0.5) * Fx) / n;
      const C vy = (jy + C(0.5) * Fy) / n;
      const C usq = vx * vx + vy * vy, uF = vx * Fx + vy * Fy;
      const C om = A.tau_inv, keep = C(1) - A.tau_inv;
      const int s = rc + x;
      {
        const C w = C(q9_w(0));
        hout[s] = keep * h[0] + om * (w * (dens - n * (C(1.5) * usq))) +
                  A.pref * w * (C(-3) * uF);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = k < 2 ? k + 1 : k + 3, ib = i + 2;
        const C w = C(q9_w(i));
        const C eu = C(q9_ex(i)) * vx + C(q9_ey(i)) * vy;
        const C eF = C(q9_ex(i)) * Fx + C(q9_ey(i)) * Fy;
        const C even = w * (dens + n * (C(4.5) * eu * eu - C(1.5) * usq));
        const C odd = w * (n * (C(3) * eu));
        const C Fe = A.pref * w * (C(9) * eu * eF - C(3) * uF);
        const C Fo = A.pref * w * (C(3) * eF);
        hout[i * ST + s] = keep * h[i] + om * (even + odd) + (Fe + Fo);
        hout[ib * ST + s] = keep * h[ib] + om * (even - odd) + (Fe - Fo);
      }
      ux[s] = vx;
      uy[s] = vy;
    }
  }
  __syncthreads();
  // m FD substeps; the last one writes phi(t+1)
  const C *src = phi;
  C *fa = A.fa + off, *fq = A.fq + off;
  for (int j = 0; j < A.m; ++j) {
    C *dst = (((A.m - 1 - j) % 2) == 0 ? A.phi[out] : A.phi[2]) + off;
    for (int y = ty; y < Ly; y += by) {
      const int ym = wrp(y - 1, Ly), yp = wrp(y + 1, Ly);
      for (int x = tx; x < Lx; x += bx) {
        const int xm = wrp(x - 1, Lx), xp = wrp(x + 1, Lx);
        const int s = y * Lx + x;
        const C pc = src[s], uc = ux[s], vc = uy[s];
        C tend;
        if (A.adv_variant == LBM_ADV_PAPER) {
          const C dux = (ux[y * Lx + xp] - ux[y * Lx + xm]) / C(2);
          const C dpx = uc < C(0) ? src[y * Lx + xp] - pc : pc - src[y * Lx + xm];
          const C duy = (uy[yp * Lx + x] - uy[ym * Lx + x]) / C(2);
          const C dpy = vc < C(0) ? src[yp * Lx + x] - pc : pc - src[ym * Lx + x];
          tend = (pc * dux + uc * dpx);
          tend += (pc * duy + vc * dpy);
        } else {
          const C Upx = C(0.5) * (uc + ux[y * Lx + xp]), Umx = C(0.5) * (ux[y * Lx + xm] + uc);
          const C Upy = C(0.5) * (vc + uy[yp * Lx + x]), Umy = C(0.5) * (uy[ym * Lx + x] + vc);
          const C Jpx = Upx > C(0) ? Upx * pc : Upx * src[y * Lx + xp];
          const C Jmx = Umx > C(0) ? Umx * src[y * Lx + xm] : Umx * pc;
          const C Jpy = Upy > C(0) ? Upy * pc : Upy * src[yp * Lx + x];
          const C Jmy = Umy > C(0) ? Umy * src[ym * Lx + x] : Umy * pc;
          tend = Jpx - Jmx;
          tend += Jpy - Jmy;
        }
        fa[s] = pc - A.dt * tend;
      }
    }
    __syncthreads();
    for (int y = ty; y < Ly; y += by) {
      const int ym = wrp(y - 1, Ly), yp = wrp(y + 1, Ly);
      for (int x = tx; x < Lx; x += bx) {
        const int xm = wrp(x - 1, Lx), xp = wrp(x + 1, Lx);
        const int s = y * Lx + x;
        const C hk = fa[s];
        const C c = A.cubic_at_half ? hk : src[s];
        C lap = fa[ym * Lx + x];
        lap += fa[y * Lx + xm];
        lap += C(-4) * hk;
        lap += fa[y * Lx + xp];
        lap += fa[yp * Lx + x];
        fq[s] = A.a * hk + A.b * (c * c * c) - A.kappa * lap;
      }
    }
    __syncthreads();
    for (int y = ty; y < Ly; y += by) {
      const int ym = wrp(y - 1, Ly), yp = wrp(y + 1, Ly);
      for (int x = tx; x < Lx; x += bx) {
        const int xm = wrp(x - 1, Lx), xp = wrp(x + 1, Lx);
        const int s = y * Lx + x;
        C lap = fq[ym * Lx + x];
        lap += fq[y * Lx + xm];
        lap += C(-4) * fq[s];
        lap += fq[y * Lx + xp];
        lap += fq[yp * Lx + x];
        dst[s] = fa[s] + A.dtG * lap;
      }
    }
    __syncthreads();
    src = dst;
  }
}

template <typename C>
__global__ void __launch_bounds__(1024) batch_kernel(BatchArgs<C> A, long long t0, int nsteps) {
  const int first = A.cta_first[blockIdx.x], last = A.cta_first[blockIdx.x + 1];
  for (int k = first; k < last; ++k) {
    const DevInst I = A.inst[A.order[k]];
    for (int s = 0; s < nsteps; ++s) batch_instance_step<C>(A, I, t0 + s);
  }
}

// Initial populations of one instance from FP64 staging (n, phi, ux, uy):
// f_i = feq_i(n, u - F/(2n)) with F = -phi d_D mu + n g at t = 0, stored at
// r - e_i (pull layout), and phi.
template <typename C>
__global__ void batch_init_kernel(BatchArgs<C> A, DevInst I, const double *stg, double N, double M,
                                  double Q, double R, double C0, double a, double b, double kappa) {
  const int Lx = I.Lx, Ly = I.Ly;
  const long long S = (long long)Lx * Ly;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int x = s % Lx, y = s / Lx;
  const double *n = stg, *phi = stg + S, *u0 = stg + 2 * S, *u1 = stg + 3 * S;
  auto at = [&](const double *f, int dx, int dy) { return f[wrp(y + dy, Ly) * Lx + wrp(x + dx, Lx)]; };
  auto muat = [&](int dx, int dy) {
    const int xx = wrp(x + dx, Lx), yy = wrp(y + dy, Ly);
    double lap = 0.0;
    for (int ey = -1; ey <= 1; ey++)
      for (int ex = -1; ex <= 1; ex++) {
        const int nn = ex * ex + ey * ey;
        const double w = nn == 0 ? C0 : (nn == 1 ? Q : R);
        lap += w * phi[wrp(yy + ey, Ly) * Lx + wrp(xx + ex, Lx)];
      }
    const double c = phi[yy * Lx + xx];
    return a * c + b * c * c * c - kappa * lap;
  };
  const double gmx = N * (muat(1, 0) - muat(-1, 0)) +
                     M * ((muat(1, -1) - muat(-1, -1)) + (muat(1, 1) - muat(-1, 1)));
  const double gmy = N * (muat(0, 1) - muat(0, -1)) +
                     M * ((muat(-1, 1) - muat(-1, -1)) + (muat(1, 1) - muat(1, -1)));
  const double nv = n[s], ph = phi[s];
  const bool on = I.force_steps > 0;
  const double Fx = -ph * gmx + (on ? nv * I.gx : 0.0), Fy = -ph * gmy + (on ? nv * I.gy : 0.0);
  const double ux = u0[s] - Fx / (2.0 * nv), uy = u1[s] - Fy / (2.0 * nv);
  const double cs2 = 1.0 / 3.0, uu = ux * ux + uy * uy;
  for (int i = 0; i < 9; i++) {
    const int ex = q9_ex(i), ey = q9_ey(i);
    const double eu = ex * ux + ey * uy;
    const double h = q9_w(i) * ((nv - 1.0) + nv * (eu / cs2 + (eu * eu - cs2 * uu) / (2.0 * cs2 * cs2)));
    A.h[0][i * A.ST + I.off + wrp(y - ey, Ly) * Lx + wrp(x - ex, Lx)] = (C)h;
  }
  A.phi[0][I.off + s] = (C)ph;
  (void)at;
}

// n, phi, u* of one instance at time t into FP64 staging (same arithmetic
// as the collide phase, without the collision).
template <typename C>
__global__ void batch_moments_kernel(BatchArgs<C> A, DevInst I, long long t, double *stg) {
  const int Lx = I.Lx, Ly = I.Ly;
  const long long S = (long long)Lx * Ly, ST = A.ST;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int x = s % Lx, y = s / Lx;
  const int in = (int)(t & 1);
  const C *hin = A.h[in] + I.off, *phi = A.phi[in] + I.off;
  auto muat = [&](int dx, int dy) {
    const int xx = wrp(x + dx, Lx), yy = wrp(y + dy, Ly);
    C lap = C(0);
    for (int ey = -1; ey <= 1; ey++)
      for (int ex = -1; ex <= 1; ex++) {
        const int nn = ex * ex + ey * ey;
        const C w = nn == 0 ? A.C0 : (nn == 1 ? A.Q : A.R);
        lap += w * phi[wrp(yy + ey, Ly) * Lx + wrp(xx + ex, Lx)];
      }
    const C c = phi[yy * Lx + xx];
    return A.a * c + A.b * c * c * c - A.kappa * lap;
  };
  const C gmx = A.N * (muat(1, 0) - muat(-1, 0)) +
                A.M * ((muat(1, -1) - muat(-1, -1)) + (muat(1, 1) - muat(-1, 1)));
  const C gmy = A.N * (muat(0, 1) - muat(0, -1)) +
                A.M * ((muat(-1, 1) - muat(-1, -1)) + (muat(1, 1) - muat(1, -1)));
  const C ph = phi[s];
  C h[9], dens = C(0);
  for (int i = 0; i < 9; i++) {
    h[i] = hin[i * ST + wrp(y - q9_ey(i), Ly) * Lx + wrp(x - q9_ex(i), Lx)];
    dens += h[i];
  }
  const C jx = ((h[1] - h[3]) + (h[5] - h[7])) + (h[8] - h[6]);
  const C jy = ((h[2] - h[4]) + (h[5] - h[7])) + (h[6] - h[8]);
  const C n = C(1) + dens;
  const bool on = t < I.force_steps;
  const C Fx = -ph * gmx + (on ? n * (C)I.gx : C(0)), Fy = -ph * gmy + (on ? n * (C)I.gy : C(0));
  stg[s] = (double)n;
  stg[S + s] = (double)ph;
  stg[2 * S + s] = (double)((jx + C(0.5) * Fx) / n);
  stg[3 * S + s] = (double)((jy + C(0.5) * Fy) / n);
}

}  // namespace

struct lbm_batch {
  lbm_params P;
  int count = 0, m = 1, ctas = 0, threads = 256;
  long long ST = 0, t = 0, maxS = 0;
  bool inited = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<DevInst> inst;
  DevInst *d_inst = nullptr;
  int *d_order = nullptr, *d_first = nullptr;
  void *h[2] = {nullptr, nullptr}, *phi[3] = {nullptr, nullptr, nullptr};
  void *u = nullptr, *mu = nullptr, *fa = nullptr, *fq = nullptr;
  double *staging = nullptr;
  int err = 0;
  std::string msg;
  cudaGraphExec_t graph = nullptr;
  long long graph_steps = -1, graph_t0 = -1;
  bool use_graphs = true;
  // tiled path
  bool tiled = false;
  TiledInst *d_tinst = nullptr;
  int4 *d_citems = nullptr, *d_fitems = nullptr, *d_titems = nullptr;
  int ncitems = 0, nfitems = 0, ntitems = 0;  // collide tiles (tile kernel), FD items, collide tiles (TMA)
  struct TmaChunk {                           // one launch of the TMA collide
    int begin = 0, n = 0, shapes = 0;          // its items in d_titems, shape slots used
    TmaShapeMaps maps[2];                      // per buffer parity
  };
  std::vector<TmaChunk> tchunks;
  float persistent_ms = -1.f;  // the persistent kernel's time per LB step at its tuned shape
};

namespace {

thread_local std::string g_batch_error;

int bfail(lbm_batch *b, int code, const std::string &msg) {
  if (b == nullptr) {
    g_batch_error = msg;
  } else if (b->err == 0) {
    b->err = code;
    b->msg = msg;
  }
  return code;
}

#define BCK(b, call, what)                                                             \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,        \
                   std::string(what) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

template <typename C>
BatchArgs<C> batch_args(const lbm_batch *b) {
  BatchArgs<C> A;
  A.inst = b->d_inst;
  A.order = b->d_order;
  A.cta_first = b->d_first;
  for (int k = 0; k < 2; k++) A.h[k] = static_cast<C *>(b->h[k]);
  for (int k = 0; k < 3; k++) A.phi[k] = static_cast<C *>(b->phi[k]);
  A.u = static_cast<C *>(b->u);
  A.mu = static_cast<C *>(b->mu);
  A.fa = static_cast<C *>(b->fa);
  A.fq = static_cast<C *>(b->fq);
  A.ST = b->ST;
  const lbm_params &P = b->P;
  A.a = (C)P.a;
  A.b = (C)P.b;
  A.kappa = (C)P.kappa;
  A.tau_inv = (C)(1.0 / P.tau);
  A.pref = (C)(1.0 - 1.0 / (2.0 * P.tau));
  A.N = (C)P.N;
  A.M = (C)((1.0 - 2.0 * P.N) / 4.0);
  A.Q = (C)P.Q;
  A.R = (C)((1.0 - P.Q) / 2.0);
  A.C0 = (C)(-4.0 * (P.Q + (1.0 - P.Q) / 2.0));
  A.dt = (C)(1.0 / b->m);
  A.dtG = (C)(P.Gamma / b->m);
  A.m = b->m;
  A.adv_variant = P.adv_variant;
  A.cubic_at_half = P.cubic_at_half;
  return A;
}

// Kernel constants of the tiled path (FP32, D2Q9, T = 1/3; the body force comes
// from the instance table).
KParams<float> tiled_params(const lbm_batch *b) {
  const lbm_params &P = b->P;
  KParams<float> p{};
  p.Lx = p.Ly = p.Lz = 1;
  p.a = (float)P.a;
  p.b = (float)P.b;
  p.kappa = (float)P.kappa;
  p.tau_inv = (float)(1.0 / P.tau);
  p.pref = (float)(1.0 - 1.0 / (2.0 * P.tau));
  p.N = (float)P.N;
  p.Q = (float)P.Q;
  p.M = (float)((1.0 - 2.0 * P.N) / 4.0);
  p.R = (float)((1.0 - P.Q) / 2.0);
  p.C0 = (float)(-4.0 * (P.Q + (1.0 - P.Q) / 2.0));
  p.cs2mT = 0.f;
  p.dt = (float)(1.0 / b->m);
  p.dtG = (float)(P.Gamma / b->m);
  p.scale = p.inv_scale = 1.f;
  p.adv_variant = P.adv_variant;
  p.cubic_at_half = P.cubic_at_half;
  p.stencil_fd = 0;
  return p;
}

// One LB step per iteration: the collide of every tile (TMA launches, then the
// tile kernel), then m / 2 two-substep FD launches (phi(t) -> phi[2] ->
// phi[out] ... ending in phi[out]).
cudaError_t launch_tiled(lbm_batch *b, long long t0, int nsteps) {
  const KParams<float> p = tiled_params(b);
  float *h[2] = {static_cast<float *>(b->h[0]), static_cast<float *>(b->h[1])};
  float *ph[3] = {static_cast<float *>(b->phi[0]), static_cast<float *>(b->phi[1]),
                  static_cast<float *>(b->phi[2])};
  float *u = static_cast<float *>(b->u);
  const int launches = b->m / 2;
  for (int s = 0; s < nsteps; ++s) {
    const long long t = t0 + s;
    const int in = (int)(t & 1), out = 1 - in;
    cudaError_t e = cudaSuccess;
    for (const auto &c : b->tchunks) {
      if (e != cudaSuccess) break;
      e = collide2d_tma_batch(c.maps[in], h[in], h[out], ph[in], u, b->ST, b->d_tinst, b->d_titems + c.begin, c.n,
                              p, t, b->stream, false);
    }
    if (e == cudaSuccess && b->ncitems > 0)
      e = collide2d_batch(h[in], h[out], ph[in], u, b->ST, b->d_tinst, b->d_citems, b->ncitems, p, t,
                          b->stream);
    if (e != cudaSuccess) return e;
    const float *src = ph[in];
    for (int j = 0; j < launches; ++j) {
      float *dst = ((launches - 1 - j) % 2 == 0) ? ph[out] : ph[2];
      e = fd2d_wave_batch(src, u, dst, b->ST, b->d_tinst, b->d_fitems, b->nfitems, p, b->stream, false);
      if (e != cudaSuccess) return e;
      src = dst;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_batch(lbm_batch *b, long long t0, int nsteps) {
  if (b->tiled) return launch_tiled(b, t0, nsteps);
  dim3 block(32, b->threads / 32);
  if (b->P.precision == LBM_F64)
    batch_kernel<double><<<b->ctas, block, 0, b->stream>>>(batch_args<double>(b), t0, nsteps);
  else
    batch_kernel<float><<<b->ctas, block, 0, b->stream>>>(batch_args<float>(b), t0, nsteps);
  return cudaGetLastError();
}

// Longest-processing-time assignment of instances to `ctas` CTAs.
void assign(lbm_batch *b, int ctas, std::vector<int> &order, std::vector<int> &first) {
  std::vector<int> ids(b->count);
  std::iota(ids.begin(), ids.end(), 0);
  std::stable_sort(ids.begin(), ids.end(), [&](int p, int q) {
    return (long long)b->inst[p].Lx * b->inst[p].Ly > (long long)b->inst[q].Lx * b->inst[q].Ly;
  });
  std::vector<long long> load(ctas, 0);
  std::vector<std::vector<int>> lists(ctas);
  for (int id : ids) {
    const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lists[c].push_back(id);
    load[c] += (long long)b->inst[id].Lx * b->inst[id].Ly;
  }
  order.clear();
  first.assign(1, 0);
  for (auto &l : lists) {
    order.insert(order.end(), l.begin(), l.end());
    first.push_back((int)order.size());
  }
}

int upload_assignment(lbm_batch *b, int ctas) {
  std::vector<int> order, first;
  assign(b, ctas, order, first);
  if (b->d_order) cudaFree(b->d_order);
  if (b->d_first) cudaFree(b->d_first);
  b->d_order = b->d_first = nullptr;
  BCK(b, cudaMalloc(&b->d_order, sizeof(int) * order.size()), "cudaMalloc");
  BCK(b, cudaMalloc(&b->d_first, sizeof(int) * first.size()), "cudaMalloc");
  BCK(b, cudaMemcpy(b->d_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice),
      "host-to-device copy");
  BCK(b, cudaMemcpy(b->d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice),
      "host-to-device copy");
  b->ctas = ctas;
  return LBM_OK;
}

// Autotuner of the CTA shape (threads per CTA x CTAs per SM) on the zeroed
// state: every candidate runs `steps` steps and the fastest is kept.
int tune_batch(lbm_batch *b, int steps) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int shapes[4][2] = {{1024, 1}, {512, 2}, {256, 4}, {512, 1}};
  float best = 1e30f;
  int bt = b->threads, bc = b->ctas;
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0), "cudaEventCreate");
  BCK(b, cudaEventCreate(&e1), "cudaEventCreate");
  for (auto &sh : shapes) {
    b->threads = sh[0];
    int rc = upload_assignment(b, std::min(b->count, sms * sh[1]));
    if (rc) return rc;
    float ms = 0.f;
    BCK(b, launch_batch(b, 0, steps), "batch kernel");  // warm-up
    BCK(b, cudaEventRecord(e0, b->stream), "cudaEventRecord");
    BCK(b, launch_batch(b, 0, steps), "batch kernel");
    BCK(b, cudaEventRecord(e1, b->stream), "cudaEventRecord");
    BCK(b, cudaEventSynchronize(e1), "cudaEventSynchronize");
    BCK(b, cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (std::getenv("HLBM_TUNE_VERBOSE"))
      std::fprintf(stderr, "hlbm tune batch threads=%d ctas=%d: %.1f us/step\n", sh[0], b->ctas,
                   ms * 1000.f / steps);
    if (ms < best) {
      best = ms;
      bt = sh[0];
      bc = b->ctas;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->threads = bt;
  b->persistent_ms = best / steps;
  return upload_assignment(b, bc);
}

bool tiled_eligible(const lbm_batch *b) {
  if (b->P.precision != LBM_F32DEV || b->P.adv_variant != LBM_ADV_PAPER || b->m % 2 != 0) return false;
  for (const DevInst &d : b->inst)
    if (d.Lx % 4 != 0) return false;
  return true;
}

// The item tables of the tiled path: 32 x 16 collide tiles (TMA chunks of
// shape slots for the instances at least collide2d_tma_batch_min_side() on a
// side, a slot per run of equal shapes in storage order of up to 0xffff
// instances; the tile kernel for the rest, or for every instance without the
// driver's tensor-map encoder or with HLBM_BATCH_NO_TMA set) and FD strips
// split into segments of at most 48 rows (HLBM_BATCH_FD_ROWS).
int build_tiles(lbm_batch *b) {
  std::vector<TiledInst> ti;
  std::vector<int4> ci, fi, tmi;
  const int TX = fd2d_wave_batch_strip_columns();
  for (const DevInst &d : b->inst)
    ti.push_back(TiledInst{d.Lx, d.Ly, d.off, (float)d.gx, (float)d.gy, d.force_steps});
  const bool tma = !std::getenv("HLBM_BATCH_NO_TMA");
  const int tma_min = collide2d_tma_batch_min_side();
  std::vector<int> ord(b->count);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int p, int q) { return b->inst[p].off < b->inst[q].off; });
  struct Shape {
    int chunk, slot, Lx, Ly, n;
    long long off0;
  };
  std::vector<Shape> shapes;
  b->tchunks.clear();
  for (int k : ord) {
    const DevInst &d = b->inst[k];
    if (tma && d.Lx >= tma_min && d.Ly >= tma_min) {
      if (shapes.empty() || shapes.back().Lx != d.Lx || shapes.back().Ly != d.Ly || shapes.back().n == 0xffff ||
          shapes.back().off0 + (long long)shapes.back().n * d.Lx * d.Ly != d.off) {
        if (b->tchunks.empty() || b->tchunks.back().shapes == TMA_BATCH_SHAPES) {
          b->tchunks.emplace_back();
          b->tchunks.back().begin = (int)tmi.size();
        }
        shapes.push_back(Shape{(int)b->tchunks.size() - 1, b->tchunks.back().shapes++, d.Lx, d.Ly, 0, d.off});
      }
      Shape &sh = shapes.back();
      const int j = sh.n++;
      for (int y0 = 0; y0 < d.Ly; y0 += BATCH_TILE_ROWS)
        for (int x0 = 0; x0 < d.Lx; x0 += 32) tmi.push_back(make_int4(k, x0, y0, (sh.slot << 16) | j));
    } else {
      for (int y0 = 0; y0 < d.Ly; y0 += BATCH_TILE_ROWS)
        for (int x0 = 0; x0 < d.Lx; x0 += 32) ci.push_back(make_int4(k, x0, y0, 0));
    }
  }
  for (size_t c = 0; c < b->tchunks.size(); ++c)
    b->tchunks[c].n = (c + 1 < b->tchunks.size() ? b->tchunks[c + 1].begin : (int)tmi.size()) - b->tchunks[c].begin;
  for (const Shape &sh : shapes) {
    bool ok = true;
    for (int par = 0; par < 2 && ok; ++par)
      ok = collide2d_tma_batch_shape(&b->tchunks[sh.chunk].maps[par], sh.slot, static_cast<float *>(b->h[par]),
                                     static_cast<float *>(b->phi[par]), b->ST, sh.Lx, sh.Ly, sh.off0, sh.n);
    if (!ok) {  // no encoder, or a shape it refuses: the tile kernel for every instance
      for (const int4 &it : tmi) ci.push_back(make_int4(it.x, it.y, it.z, 0));
      tmi.clear();
      b->tchunks.clear();
      break;
    }
  }
  const char *fr = std::getenv("HLBM_BATCH_FD_ROWS");
  const int max_rows = fr ? std::max(8, std::atoi(fr)) : 48;
  for (int k = 0; k < b->count; ++k) {
    const DevInst &d = b->inst[k];
    const int strips = (d.Lx + TX - 1) / TX;
    const int nseg = std::max(1, (d.Ly + max_rows - 1) / max_rows), ny = (d.Ly + nseg - 1) / nseg;
    for (int sx = 0; sx < strips; ++sx)
      for (int ys = 0; ys < d.Ly; ys += ny) fi.push_back(make_int4(k, sx, ys, std::min(ny, d.Ly - ys)));
  }
  // longest segments first: the CTAs are dispatched in item order
  std::stable_sort(fi.begin(), fi.end(), [](const int4 &p, const int4 &q) { return p.w > q.w; });
  auto upload = [&](auto **dst, const auto &v) -> int {
    if (v.empty()) return LBM_OK;
    using T = typename std::decay<decltype(v)>::type::value_type;
    BCK(b, cudaMalloc(dst, sizeof(T) * v.size()), "cudaMalloc");
    BCK(b, cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice), "host-to-device copy");
    return LBM_OK;
  };
  int rc = upload(&b->d_tinst, ti);
  if (!rc) rc = upload(&b->d_citems, ci);
  if (!rc) rc = upload(&b->d_titems, tmi);
  if (!rc) rc = upload(&b->d_fitems, fi);
  b->ncitems = (int)ci.size();
  b->ntitems = (int)tmi.size();
  b->nfitems = (int)fi.size();
  return rc;
}

// Times `steps` LB steps of the current path (after one warm-up call), ms per step.
int time_path(lbm_batch *b, int steps, float *ms_per_step) {
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0), "cudaEventCreate");
  BCK(b, cudaEventCreate(&e1), "cudaEventCreate");
  float ms = 0.f;
  BCK(b, launch_batch(b, 0, steps), "batch step");
  BCK(b, cudaEventRecord(e0, b->stream), "cudaEventRecord");
  BCK(b, launch_batch(b, 0, steps), "batch step");
  BCK(b, cudaEventRecord(e1, b->stream), "cudaEventRecord");
  BCK(b, cudaEventSynchronize(e1), "cudaEventSynchronize");
  BCK(b, cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_per_step = ms / steps;
  return LBM_OK;
}

// After a synchronisation: a bounded wait of the TMA collide that gave up
// (its copies never completed) latches LBM_ETIMEOUT.
int check_waits(lbm_batch *b) {
  if (b->ntitems > 0 && collide2d_tma_error(true) > 0)
    return bfail(b, LBM_ETIMEOUT, "batched collide kernel: a TMA copy did not complete within its wait bound");
  return LBM_OK;
}

int zero_state(lbm_batch *b) {
  const size_t cb = b->P.precision == LBM_F64 ? 8 : 4;
  void *bufs[] = {b->h[0], b->h[1], b->phi[0], b->phi[1], b->phi[2], b->u, b->mu, b->fa, b->fq};
  const size_t sizes[] = {cb * 9 * b->ST, cb * 9 * b->ST, cb * b->ST, cb * b->ST, cb * b->ST,
                          cb * 2 * b->ST, cb * b->ST, cb * b->ST, cb * b->ST};
  for (int k = 0; k < 9; k++) BCK(b, cudaMemsetAsync(bufs[k], 0, sizes[k], b->stream), "cudaMemset");
  BCK(b, cudaStreamSynchronize(b->stream), "cudaMemset");
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_params *common, const lbm_instance *inst, int count,
                     void *cuda_stream, lbm_batch **out) {
  if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!common || !inst || count <= 0) return bfail(nullptr, LBM_EINVAL, "NULL or empty batch");
  const lbm_params &P = *common;
  if (P.dims != 2) return bfail(nullptr, LBM_EINVAL, "batches are 2D (D2Q9)");
  if (P.precision != LBM_F64 && P.precision != LBM_F32DEV)
    return bfail(nullptr, LBM_EINVAL, "batches store FP64 or FP32-deviation populations");
  if (!(P.tau > 0.5) || !(P.b > 0.0) || !(P.kappa >= 0.0) || !(P.Gamma >= 0.0) ||
      !std::isfinite(P.a) || !std::isfinite(P.N) || !std::isfinite(P.Q))
    return bfail(nullptr, LBM_EINVAL, "bad common parameters (tau > 1/2, b > 0, kappa, Gamma >= 0)");
  if (P.T != 1.0 / 3.0) return bfail(nullptr, LBM_EINVAL, "batches need T = 1/3");
  if (P.stencil_fd != 0) return bfail(nullptr, LBM_EINVAL, "batches run Eqs. 33 and 36 as printed (stencil_fd = 0)");
  if (P.adv_variant != LBM_ADV_PAPER && P.adv_variant != LBM_ADV_FLUX)
    return bfail(nullptr, LBM_EINVAL, "unknown adv_variant");
  // FD substeps as for a single lattice (Sec. II C)
  const double aeff = P.a < 0 ? -2.0 * P.a : P.a;
  const double stiff = P.Gamma * (aeff * 8.0 + P.kappa * 64.0);
  const int m_min = std::max(1, (int)std::ceil(stiff / 2.0 - 1e-12));
  int m = P.fd_substeps == 0 ? std::max(1, (int)std::ceil(stiff / 1.5 - 1e-12))
                             : std::abs(P.fd_substeps);
  if (P.fd_substeps > 0 && m < m_min) return bfail(nullptr, LBM_EINVAL, "fd_substeps below the Euler bound");
  lbm_batch *b = new lbm_batch();
  b->P = P;
  b->count = count;
  b->m = m;
  for (int k = 0; k < count; k++) {
    const lbm_instance &q = inst[k];
    if (q.Lx < 3 || q.Ly < 3 || (long long)q.Lx * q.Ly > (1LL << 30) || q.force_steps < 0 ||
        !std::isfinite(q.g[0]) || !std::isfinite(q.g[1])) {
      delete b;
      return bfail(nullptr, LBM_EINVAL, "bad instance " + std::to_string(k));
    }
    DevInst d;
    d.Lx = q.Lx;
    d.Ly = q.Ly;
    d.off = 0;
    d.gx = q.g[0];
    d.gy = q.g[1];
    d.force_steps = q.force_steps;
    b->inst.push_back(d);
    b->maxS = std::max(b->maxS, (long long)q.Lx * q.Ly);
  }
  // storage order: the instances grouped by shape (Lx, Ly), so that those of
  // one shape are equally spaced, as the tiled path's per-shape tensor maps need
  std::vector<int> ord(count);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int p, int q) {
    return std::make_pair(b->inst[p].Lx, b->inst[p].Ly) < std::make_pair(b->inst[q].Lx, b->inst[q].Ly);
  });
  long long ST = 0;
  for (int k : ord) {
    b->inst[k].off = ST;
    ST += (long long)b->inst[k].Lx * b->inst[k].Ly;
  }
  b->ST = ST;
  auto bail = [&](int code) {
    g_batch_error = b->msg;
    lbm_batch_free(b);
    return code;
  };
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(bfail(b, LBM_ECUDA, "cudaStreamCreate"));
    b->own_stream = true;
  }
  const size_t cb = P.precision == LBM_F64 ? 8 : 4;
  struct {
    void **p;
    size_t n;
  } al[] = {{&b->h[0], cb * 9 * ST},   {&b->h[1], cb * 9 * ST}, {&b->phi[0], cb * ST},
            {&b->phi[1], cb * ST},     {&b->phi[2], cb * ST},   {&b->u, cb * 2 * ST},
            {&b->mu, cb * ST},         {&b->fa, cb * ST},       {&b->fq, cb * ST},
            {(void **)&b->staging, sizeof(double) * 4 * b->maxS},
            {(void **)&b->d_inst, sizeof(DevInst) * count}};
  for (auto &a : al) {
    cudaError_t e = cudaMalloc(a.p, a.n);
    if (e != cudaSuccess)
      return bail(bfail(b, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "cudaMalloc"));
  }
  if (cudaMemcpy(b->d_inst, b->inst.data(), sizeof(DevInst) * count, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return bail(bfail(b, LBM_ECUDA, "host-to-device copy"));
  // CTA shape: 1024 threads and one CTA per SM unless the batch is small
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->threads = 1024;
  int rc = upload_assignment(b, std::min(count, sms));
  if (rc) return bail(rc);
  // every instance starts at rest (phi = 0, f = w) until it is initialised
  rc = zero_state(b);
  if (!rc && !std::getenv("HLBM_BATCH_SHAPE")) rc = tune_batch(b, 2);
  if (!rc && std::getenv("HLBM_BATCH_SHAPE")) {
    int th = 1024, per = 1;
    if (std::sscanf(std::getenv("HLBM_BATCH_SHAPE"), "%d,%d", &th, &per) != 2 ||
        (th != 256 && th != 512 && th != 1024) || per < 1 || per > 8)
      rc = bfail(b, LBM_EINVAL, "HLBM_BATCH_SHAPE must be 'threads,ctas_per_sm'");
    else {
      b->threads = th;
      rc = upload_assignment(b, std::min(count, sms * per));
    }
  }
  if (!rc) rc = zero_state(b);
  // the tiled path where eligible, if it is faster (or asked for)
  const char *path = std::getenv("HLBM_BATCH_PATH");
  if (!rc && path && std::strcmp(path, "tiled") != 0 && std::strcmp(path, "persistent") != 0)
    rc = bfail(b, LBM_EINVAL, "HLBM_BATCH_PATH must be 'tiled' or 'persistent'");
  if (!rc && tiled_eligible(b) && !(path && std::strcmp(path, "persistent") == 0)) {
    if (b->persistent_ms <= 0.f) rc = time_path(b, 2, &b->persistent_ms);  // a fixed CTA shape
    if (!rc && (fd2d_wave_configure() != cudaSuccess || collide2d_tma_configure(LBM_F32DEV) != cudaSuccess))
      rc = bfail(b, LBM_ECUDA, "tiled path: shared-memory attributes");
    if (!rc) rc = build_tiles(b);
    if (!rc) {
      b->tiled = true;
      float tiled_ms = 0.f;
      rc = time_path(b, 2, &tiled_ms);
      if (!rc) rc = check_waits(b);
      if (std::getenv("HLBM_TUNE_VERBOSE"))
        std::fprintf(stderr, "hlbm tune batch tiled: %.1f us/step (persistent %.1f)\n", tiled_ms * 1000.f,
                     b->persistent_ms * 1000.f);
      const bool forced = path && std::strcmp(path, "tiled") == 0;
      if (!rc && !forced && b->persistent_ms < tiled_ms) b->tiled = false;
    }
    if (!rc) rc = zero_state(b);
  }
  if (rc) return bail(rc);
  *out = b;
  return LBM_OK;
}

int lbm_batch_init_fields(lbm_batch *b, int k, const double *n, const double *phi,
                          const double *ux, const double *uy) {
  if (!b) return LBM_EINVAL;
  if (b->err) return b->err;
  if (k < 0 || k >= b->count || !n || !phi || !ux || !uy)
    return bfail(b, LBM_EINVAL, "lbm_batch_init_fields: bad instance or NULL array");
  const DevInst &I = b->inst[k];
  const long long S = (long long)I.Lx * I.Ly;
  const double *src[4] = {n, phi, ux, uy};
  for (int j = 0; j < 4; j++)
    BCK(b, cudaMemcpyAsync(b->staging + j * S, src[j], sizeof(double) * S, cudaMemcpyHostToDevice,
                           b->stream),
        "host-to-device copy");
  const lbm_params &P = b->P;
  const double M = (1.0 - 2.0 * P.N) / 4.0, R = (1.0 - P.Q) / 2.0, C0 = -4.0 * (P.Q + R);
  const unsigned nb = (unsigned)((S + 255) / 256);
  if (P.precision == LBM_F64)
    batch_init_kernel<double><<<nb, 256, 0, b->stream>>>(batch_args<double>(b), I, b->staging, P.N,
                                                         M, P.Q, R, C0, P.a, P.b, P.kappa);
  else
    batch_init_kernel<float><<<nb, 256, 0, b->stream>>>(batch_args<float>(b), I, b->staging, P.N,
                                                        M, P.Q, R, C0, P.a, P.b, P.kappa);
  BCK(b, cudaGetLastError(), "init kernel");
  BCK(b, cudaStreamSynchronize(b->stream), "lbm_batch_init_fields");
  b->t = 0;  // the batch clock restarts: initialise every instance before stepping
  b->inited = true;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, long long nsteps) {
  if (!b) return LBM_EINVAL;
  if (b->err) return b->err;
  if (!b->inited) return bfail(b, LBM_ESTATE, "fields are not initialised");
  if (nsteps < 0 || nsteps > (1LL << 30)) return bfail(b, LBM_EINVAL, "bad nsteps");
  if (nsteps == 0) return LBM_OK;
  if (!b->use_graphs) {
    BCK(b, launch_batch(b, b->t, (int)nsteps), "batch kernel");
  } else {
    // the call's launches captured once per (t0, nsteps) pair
    if (b->graph == nullptr || b->graph_steps != nsteps || b->graph_t0 != b->t) {
      if (b->graph) cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "capture");
      cudaError_t le = launch_batch(b, b->t, (int)nsteps);
      cudaGraph_t g = nullptr;
      cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
      BCK(b, le, "batch kernel");
      BCK(b, ee, "cudaStreamEndCapture");
      cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      BCK(b, ie, "cudaGraphInstantiate");
      b->graph_steps = nsteps;
      b->graph_t0 = b->t;
    }
    BCK(b, cudaGraphLaunch(b->graph, b->stream), "cudaGraphLaunch");
  }
  b->t += nsteps;
  return LBM_OK;
}

int lbm_batch_moments(lbm_batch *b, int k, double *n, double *phi, double *ux, double *uy) {
  if (!b) return LBM_EINVAL;
  if (b->err) return b->err;
  if (!b->inited) return bfail(b, LBM_ESTATE, "fields are not initialised");
  if (k < 0 || k >= b->count) return bfail(b, LBM_EINVAL, "bad instance");
  const DevInst &I = b->inst[k];
  const long long S = (long long)I.Lx * I.Ly;
  const unsigned nb = (unsigned)((S + 255) / 256);
  if (b->P.precision == LBM_F64)
    batch_moments_kernel<double><<<nb, 256, 0, b->stream>>>(batch_args<double>(b), I, b->t, b->staging);
  else
    batch_moments_kernel<float><<<nb, 256, 0, b->stream>>>(batch_args<float>(b), I, b->t, b->staging);
  BCK(b, cudaGetLastError(), "moments kernel");
  double *dst[4] = {n, phi, ux, uy};
  for (int j = 0; j < 4; j++)
    if (dst[j])
      BCK(b, cudaMemcpyAsync(dst[j], b->staging + j * S, sizeof(double) * S, cudaMemcpyDeviceToHost,
                             b->stream),
          "device-to-host copy");
  BCK(b, cudaStreamSynchronize(b->stream), "lbm_batch_moments");
  return check_waits(b);
}

int lbm_batch_set_graphs(lbm_batch *b, int enable) {
  if (!b) return LBM_EINVAL;
  b->use_graphs = enable != 0;
  return LBM_OK;
}

int lbm_batch_shape(const lbm_batch *b, int *threads, int *ctas, long long *sites) {
  if (!b) return LBM_EINVAL;
  if (threads) *threads = b->tiled ? 0 : b->threads;
  if (ctas) *ctas = b->tiled ? b->ncitems + b->ntitems : b->ctas;
  if (sites) *sites = b->ST;
  return LBM_OK;
}

int lbm_batch_synchronize(lbm_batch *b) {
  if (!b) return LBM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) bfail(b, LBM_ECUDA, std::string("lbm_batch_synchronize: ") + cudaGetErrorString(e));
  if (!b->err) check_waits(b);
  return b->err;
}

void lbm_batch_free(lbm_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  void *ptrs[] = {b->h[0], b->h[1], b->phi[0], b->phi[1], b->phi[2], b->u, b->mu,
                  b->fa,   b->fq,   b->staging, b->d_inst, b->d_order, b->d_first,
                  b->d_tinst, b->d_citems, b->d_fitems, b->d_titems};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char *lbm_batch_last_error(const lbm_batch *b) {
  return b ? b->msg.c_str() : g_batch_error.c_str();
}

}  // extern "C"
