// kernels_common.cu -- dimension-generic kernels off the per-step path:
// initial populations (Eqs. 15, 18, 28), population read-back, and the FP64
// diagnostics of Sec. III (warp-shuffle + block tree, fixed order, so the
// sums are bitwise reproducible for a given lattice).
//
// Staging buffer layout (FP64): [0] n, [1] phi, [2 .. 2+d) u components,
// [2+d] scratch (mu during initialisation).
#include "lbm_common.cuh"

namespace hlbm {

namespace {

struct Geo {
  int dims, Lx, Ly, Lz;
  long long S;
};

__device__ __forceinline__ long long site_of(const Geo &g, int x, int y, int z) {
  return ((long long)z * g.Ly + y) * g.Lx + x;
}

__device__ __forceinline__ void coords_of(const Geo &g, long long s, int &x, int &y, int &z) {
  x = (int)(s % g.Lx);
  long long r = s / g.Lx;
  y = (int)(r % g.Ly);
  z = (int)(r / g.Ly);
}

__device__ __forceinline__ int lat_e(int dims, int i, int a) {
  if (dims == 2) return a == 0 ? q9_ex(i) : (a == 1 ? q9_ey(i) : 0);
  return a == 0 ? q19_ex(i) : (a == 1 ? q19_ey(i) : q19_ez(i));
}
__device__ __forceinline__ double lat_w(int dims, int i) { return dims == 2 ? q9_w(i) : q19_w(i); }

struct Stencil {
  double N, M, Q, R, C0;
};

// sum over the 3x3(x3) neighbourhood of a weight(d) * field; grad component a
// (a >= 0) or the Laplacian (a < 0) with the stencil weights of Eqs. 30-31.
__device__ double apply(const Geo &g, const Stencil &st, const double *f, int x, int y, int z,
                        int a) {
  double acc = 0.0;
  const int zlo = g.dims == 3 ? -1 : 0, zhi = g.dims == 3 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; dz++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dx = -1; dx <= 1; dx++) {
        const int nn = dx * dx + dy * dy + dz * dz;
        double w = 0.0;
        if (a < 0) {
          w = nn == 0 ? st.C0 : (nn == 1 ? st.Q : (nn == 2 ? st.R : 0.0));
        } else {
          const int da = a == 0 ? dx : (a == 1 ? dy : dz);
          if (da != 0) w = (nn == 1 ? st.N : (nn == 2 ? st.M : 0.0)) * da;
        }
        if (w != 0.0)
          acc += w * f[site_of(g, wrapi(x + dx, g.Lx), wrapi(y + dy, g.Ly), wrapi(z + dz, g.Lz))];
      }
  return acc;
}

__global__ void init_mu_kernel(Geo g, Stencil st, double a, double b, double kappa,
                               double *stg) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.S) return;
  int x, y, z;
  coords_of(g, s, x, y, z);
  const double *phi = stg + g.S;
  const double c = phi[s];
  stg[(2 + g.dims) * g.S + s] = a * c + b * c * c * c - kappa * apply(g, st, phi, x, y, z, -1);
}

template <typename S>
__global__ void init_pop_kernel(Geo g, Stencil st, double cs2mT, double gx, double gy,
                                double gz, double scale, const double *stg, S *hout,
                                void *phiout, int phi_is_double) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.S) return;
  int x, y, z;
  coords_of(g, s, x, y, z);
  const int d = g.dims, q = d == 2 ? 9 : 19;
  const double *nn = stg, *phi = stg + g.S, *mu = stg + (2 + d) * g.S;
  const double n = nn[s], ph = phi[s];
  double F[3], us[3] = {0, 0, 0};
  const double gg[3] = {gx, gy, gz};
  // F at t = 0 (Eq. 28): -phi d_D mu [+ d_D((cs2 - T) n)] + n g
  for (int a = 0; a < d; a++) {
    F[a] = -ph * apply(g, st, mu, x, y, z, a);
    if (cs2mT != 0.0) {
      double acc = 0.0;
      const int zlo = d == 3 ? -1 : 0, zhi = d == 3 ? 1 : 0;
      for (int dz = zlo; dz <= zhi; dz++)
        for (int dy = -1; dy <= 1; dy++)
          for (int dx = -1; dx <= 1; dx++) {
            const int n2 = dx * dx + dy * dy + dz * dz;
            const int da = a == 0 ? dx : (a == 1 ? dy : dz);
            if (da == 0 || n2 > 2) continue;
            const double w = (n2 == 1 ? st.N : st.M) * da;
            acc += w * (cs2mT * nn[site_of(g, wrapi(x + dx, g.Lx), wrapi(y + dy, g.Ly),
                                            wrapi(z + dz, g.Lz))]);
          }
      F[a] += acc;
    }
    F[a] += n * gg[a];
    us[a] = stg[(2 + a) * g.S + s] - F[a] / (2.0 * n);
  }
  const double cs2 = 1.0 / 3.0;
  double uu = 0.0;
  for (int a = 0; a < d; a++) uu += us[a] * us[a];
  for (int i = 0; i < q; i++) {
    double eu = 0.0;
    for (int a = 0; a < d; a++) eu += lat_e(d, i, a) * us[a];
    const double w = lat_w(d, i);
    // feq_i - w_i of Eq. 15
    const double h = w * ((n - 1.0) + n * (eu / cs2 + (eu * eu - cs2 * uu) / (2.0 * cs2 * cs2)));
    // pull layout: the population that arrives at r came from r - e_i
    const long long src = site_of(g, wrapi(x - lat_e(d, i, 0), g.Lx),
                                  wrapi(y - lat_e(d, i, 1), g.Ly),
                                  wrapi(z - lat_e(d, i, 2), g.Lz));
    if constexpr (sizeof(S) == 2)
      hout[i * g.S + src] = __float2half_rn((float)(h * scale));
    else
      hout[i * g.S + src] = (S)h;
  }
  if (phi_is_double)
    static_cast<double *>(phiout)[s] = ph;
  else
    static_cast<float *>(phiout)[s] = (float)ph;
}

template <typename S>
__global__ void population_kernel(Geo g, int i, double inv_scale, const S *hin, double *out) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.S) return;
  int x, y, z;
  coords_of(g, s, x, y, z);
  const int d = g.dims;
  const long long src = site_of(g, wrapi(x - lat_e(d, i, 0), g.Lx), wrapi(y - lat_e(d, i, 1), g.Ly),
                                wrapi(z - lat_e(d, i, 2), g.Lz));
  double hv;
  if constexpr (sizeof(S) == 2)
    hv = (double)__half2float(hin[i * g.S + src]) * inv_scale;
  else
    hv = (double)hin[i * g.S + src];
  out[s] = lat_w(d, i) + hv;
}

// ---- diagnostics ------------------------------------------------------------------
constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Per block: partial sums of DIAG_NPART quantities over a fixed grid-stride
// assignment of sites, reduced in a fixed order.
__global__ void __launch_bounds__(DIAG_THREADS)
    diag_partial_kernel(Geo g, double phi0, double r0, double r1, double r2,
                        const double *__restrict__ stg, double *__restrict__ part) {
  const int d = g.dims;
  const double *nn = stg, *phi = stg + g.S;
  const double rref[3] = {r0, r1, r2};
  const double L[3] = {(double)g.Lx, (double)g.Ly, (double)g.Lz};
  double acc[DIAG_NPART];
  for (int k = 0; k < DIAG_NPART; k++) acc[k] = 0.0;
  for (long long s = blockIdx.x * (long long)DIAG_THREADS + threadIdx.x; s < g.S;
       s += (long long)gridDim.x * DIAG_THREADS) {
    const double n = nn[s], ph = phi[s];
    double u2 = 0.0;
    bool finite = isfinite(n) && isfinite(ph);
    acc[DIAG_SUM_N] += n;
    acc[DIAG_SUM_PHI] += ph;
    for (int a = 0; a < d; a++) {
      const double ua = stg[(2 + a) * g.S + s];
      finite = finite && isfinite(ua);
      acc[DIAG_MOM0 + a] += n * ua;
      u2 += ua * ua;
    }
    acc[DIAG_UMAX] = fmax(acc[DIAG_UMAX], sqrt(u2));
    acc[DIAG_AREA] += (1.0 + ph / phi0) / 2.0;
    if (ph > 0.0) {
      int c[3];
      coords_of(g, s, c[0], c[1], c[2]);
      acc[DIAG_CMW] += ph;
      for (int a = 0; a < d; a++) {
        double rel = c[a] - rref[a];
        rel -= L[a] * floor(rel / L[a] + 0.5);
        acc[DIAG_CM0 + a] += ph * rel;
      }
    }
    if (!finite) acc[DIAG_NONFINITE] = 1.0;
  }
  __shared__ double red[DIAG_THREADS / 32][DIAG_NPART];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < DIAG_NPART; k++) {
    const bool isMax = (k == DIAG_UMAX || k == DIAG_NONFINITE);
    const double v = isMax ? warp_max(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIAG_NPART) {
    const int k = threadIdx.x;
    const bool isMax = (k == DIAG_UMAX || k == DIAG_NONFINITE);
    double v = red[0][k];
    for (int w = 1; w < DIAG_THREADS / 32; w++) v = isMax ? fmax(v, red[w][k]) : v + red[w][k];
    part[blockIdx.x * DIAG_NPART + k] = v;
  }
}

// One block: folds the partials in a fixed order, then (thread 0) the centre
// of mass, u* at r_cm and the pressure jump from the stencil form of Eq. 6.
__global__ void __launch_bounds__(DIAG_THREADS)
    diag_finish_kernel(Geo g, Stencil st, double a, double b, double kappa, double T,
                       double r0, double r1, double r2, int nblocks,
                       const double *__restrict__ part, const double *__restrict__ stg,
                       double *__restrict__ res) {
  __shared__ double red[DIAG_THREADS / 32][DIAG_NPART];
  __shared__ double tot[DIAG_NPART];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < DIAG_NPART; k++) {
    const bool isMax = (k == DIAG_UMAX || k == DIAG_NONFINITE);
    double v = 0.0;
    for (int blk = threadIdx.x; blk < nblocks; blk += DIAG_THREADS) {
      const double x = part[blk * DIAG_NPART + k];
      v = isMax ? fmax(v, x) : v + x;
    }
    v = isMax ? warp_max(v) : warp_sum(v);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIAG_NPART) {
    const int k = threadIdx.x;
    const bool isMax = (k == DIAG_UMAX || k == DIAG_NONFINITE);
    double v = red[0][k];
    for (int w = 1; w < DIAG_THREADS / 32; w++) v = isMax ? fmax(v, red[w][k]) : v + red[w][k];
    tot[k] = v;
    res[k] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int d = g.dims;
  const double *nn = stg, *phi = stg + g.S;
  const double rref[3] = {r0, r1, r2};
  const int L[3] = {g.Lx, g.Ly, g.Lz};
  double rcm[3] = {0, 0, 0};
  for (int k = 0; k < d; k++)
    rcm[k] = tot[DIAG_CMW] > 0.0 ? rref[k] + tot[DIAG_CM0 + k] / tot[DIAG_CMW] : rref[k];
  // u* at r_cm, multilinear with periodic wrap
  int base[3] = {0, 0, 0};
  double frac[3] = {0, 0, 0};
  for (int k = 0; k < d; k++) {
    const double fl = floor(rcm[k]);
    base[k] = (int)fl;
    frac[k] = rcm[k] - fl;
  }
  double vf[3] = {0, 0, 0};
  for (int corner = 0; corner < (1 << d); corner++) {
    int idx[3] = {0, 0, 0};
    double wt = 1.0;
    for (int k = 0; k < d; k++) {
      const int bit = (corner >> k) & 1;
      idx[k] = wrapi(base[k] + bit, L[k]);
      wt *= bit ? frac[k] : 1.0 - frac[k];
    }
    const long long s = site_of(g, idx[0], idx[1], idx[2]);
    for (int c = 0; c < d; c++) vf[c] += wt * stg[(2 + c) * g.S + s];
  }
  // p0 of Eq. 6 at the centre site and at site 0
  double p0v[2];
  for (int which = 0; which < 2; which++) {
    const int x = which == 0 ? g.Lx / 2 : 0, y = which == 0 ? g.Ly / 2 : 0;
    const int z = (which == 0 && d == 3) ? g.Lz / 2 : 0;
    const long long s = site_of(g, x, y, z);
    const double ph = phi[s];
    double g2 = 0.0;
    for (int k = 0; k < d; k++) {
      const double gk = apply(g, st, phi, x, y, z, k);
      g2 += gk * gk;
    }
    const double lap = apply(g, st, phi, x, y, z, -1);
    p0v[which] = nn[s] * T + a * ph * ph / 2.0 + 3.0 * b * ph * ph * ph * ph / 4.0 -
                 kappa * ph * lap - kappa * g2 / 2.0;
  }
  res[DIAG_DP] = p0v[0] - p0v[1];
  for (int k = 0; k < 3; k++) {
    res[DIAG_RCM0 + k] = rcm[k];
    res[DIAG_VF0 + k] = vf[k];
  }
}

Geo geo_of(const lbm_handle *h) {
  Geo g;
  g.dims = h->dims;
  g.Lx = h->P.Lx;
  g.Ly = h->P.Ly;
  g.Lz = h->dims == 3 ? h->P.Lz : 1;
  g.S = h->S;
  return g;
}

Stencil stencil_of(const lbm_handle *h) {
  Stencil st;
  st.N = h->P.N;
  st.Q = h->P.Q;
  if (h->dims == 2) {
    st.M = (1.0 - 2.0 * h->P.N) / 4.0;
    st.R = (1.0 - h->P.Q) / 2.0;
    st.C0 = -4.0 * (st.Q + st.R);
  } else {
    st.M = (1.0 - 2.0 * h->P.N) / 8.0;
    st.R = (1.0 - h->P.Q) / 4.0;
    st.C0 = -(6.0 * st.Q + 12.0 * st.R);
  }
  return st;
}

unsigned blocks_for(long long S, int threads) { return (unsigned)((S + threads - 1) / threads); }

}  // namespace

cudaError_t launch_init(lbm_handle *h, int out) {
  const Geo g = geo_of(h);
  const Stencil st = stencil_of(h);
  const unsigned nb = blocks_for(g.S, 256);
  init_mu_kernel<<<nb, 256, 0, h->stream>>>(g, st, h->P.a, h->P.b, h->P.kappa, h->staging);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool on = h->P.force_steps > 0;
  const double gx = on ? h->P.g[0] : 0.0, gy = on ? h->P.g[1] : 0.0,
               gz = on && h->dims == 3 ? h->P.g[2] : 0.0;
  const double cs2mT = 1.0 / 3.0 - h->P.T;
  switch (h->P.precision) {
    case LBM_F64:
      init_pop_kernel<double><<<nb, 256, 0, h->stream>>>(g, st, cs2mT, gx, gy, gz, 1.0,
                                                         h->staging,
                                                         static_cast<double *>(h->h[out]),
                                                         h->phi[out], 1);
      break;
    case LBM_F32DEV:
      init_pop_kernel<float><<<nb, 256, 0, h->stream>>>(g, st, cs2mT, gx, gy, gz, 1.0,
                                                        h->staging,
                                                        static_cast<float *>(h->h[out]),
                                                        h->phi[out], 0);
      break;
    default:
      init_pop_kernel<__half><<<nb, 256, 0, h->stream>>>(
          g, st, cs2mT, gx, gy, gz, std::ldexp(1.0, h->P.f16_scale_log2), h->staging,
          static_cast<__half *>(h->h[out]), h->phi[out], 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_population(lbm_handle *h, int in, int i) {
  const Geo g = geo_of(h);
  const unsigned nb = blocks_for(g.S, 256);
  switch (h->P.precision) {
    case LBM_F64:
      population_kernel<double><<<nb, 256, 0, h->stream>>>(
          g, i, 1.0, static_cast<const double *>(h->h[in]), h->staging);
      break;
    case LBM_F32DEV:
      population_kernel<float><<<nb, 256, 0, h->stream>>>(
          g, i, 1.0, static_cast<const float *>(h->h[in]), h->staging);
      break;
    default:
      population_kernel<__half><<<nb, 256, 0, h->stream>>>(
          g, i, std::ldexp(1.0, -h->P.f16_scale_log2), static_cast<const __half *>(h->h[in]),
          h->staging);
  }
  return cudaGetLastError();
}

cudaError_t launch_diag(lbm_handle *h, const double *r_ref) {
  const Geo g = geo_of(h);
  const Stencil st = stencil_of(h);
  diag_partial_kernel<<<DIAG_BLOCKS, DIAG_THREADS, 0, h->stream>>>(
      g, h->phi0, r_ref[0], r_ref[1], r_ref[2], h->staging, h->partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_finish_kernel<<<1, DIAG_THREADS, 0, h->stream>>>(g, st, h->P.a, h->P.b, h->P.kappa,
                                                        h->P.T, r_ref[0], r_ref[1], r_ref[2],
                                                        DIAG_BLOCKS, h->partials, h->staging,
                                                        h->dres);
  return cudaGetLastError();
}

}  // namespace hlbm

namespace hlbm {

// The diagnostics kernels on caller-provided FP64 fields ([n | phi | u_x |
// u_y (| u_z)], S doubles each) with caller-provided partials/result storage
// and an explicit number of partial blocks.
cudaError_t launch_diag_raw(const lbm_params &P, double phi0, const double *r_ref,
                            const double *fields, double *partials, int nblocks, double *res,
                            cudaStream_t stream) {
  Geo g;
  g.dims = P.dims;
  g.Lx = P.Lx;
  g.Ly = P.Ly;
  g.Lz = P.dims == 3 ? P.Lz : 1;
  g.S = (long long)g.Lx * g.Ly * g.Lz;
  Stencil st;
  st.N = P.N;
  st.Q = P.Q;
  if (P.dims == 2) {
    st.M = (1.0 - 2.0 * P.N) / 4.0;
    st.R = (1.0 - P.Q) / 2.0;
    st.C0 = -4.0 * (st.Q + st.R);
  } else {
    st.M = (1.0 - 2.0 * P.N) / 8.0;
    st.R = (1.0 - P.Q) / 4.0;
    st.C0 = -(6.0 * st.Q + 12.0 * st.R);
  }
  diag_partial_kernel<<<nblocks, DIAG_THREADS, 0, stream>>>(g, phi0, r_ref[0], r_ref[1],
                                                            r_ref[2], fields, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_finish_kernel<<<1, DIAG_THREADS, 0, stream>>>(g, st, P.a, P.b, P.kappa, P.T, r_ref[0],
                                                     r_ref[1], r_ref[2], nblocks, partials,
                                                     fields, res);
  return cudaGetLastError();
}

}  // namespace hlbm
