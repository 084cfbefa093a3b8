// kernels_2d.cu -- D2Q9 hot path on sm_103a.
//
//   collide2d : phi tile + halo 2 staged in shared memory -> mu (Eq. 5) on the
//               tile + 1 -> F = -phi d_D mu (+ grad((cs2 - T) n)) + n g (Eq. 28)
//               -> pull-streamed populations -> n, u* (Eqs. 12, 18) -> BGK with
//               the Guo forcing term (Eqs. 15, 17, 29) -> populations and u*.
//   fd2d      : `sub` substeps of the convection-diffusion update (Eqs. 32-36)
//               temporally blocked in shared memory (halo 3 per substep).
//   density2d : n - 1 of every site (only for T != 1/3, whose extra force
//               needs n on the neighbours).
//
// Populations are stored as deviations h_i = f_i - w_i in [i][y][x] order and
// streamed with the "pull" pattern: the buffer of time t holds the
// post-collision values of step t-1 at their source site, so
// f_i(r, t) = buf_i(r - e_i) and the kernel writes its own site only.
#include "lbm_common.cuh"

namespace hlbm {

namespace {

constexpr int C2_TX = 32;  // tile width (one warp along x)
constexpr int C2_TY = 16;  // tile height (block of 32 x 8 threads, 2 rows each)
constexpr int C2_BY = 8;

template <typename S, typename C, bool TGEN, int MODE>
__global__ void __launch_bounds__(256)
    collide2d_kernel(const S *__restrict__ hin, S *__restrict__ hout, const C *__restrict__ phi,
                     const C *__restrict__ dn, C *__restrict__ uout, double *__restrict__ stg,
                     KParams<C> p) {
  constexpr int PX = C2_TX + 4, PY = C2_TY + 4;  // phi tile + halo 2
  constexpr int MX = C2_TX + 2, MY = C2_TY + 2;  // mu tile + halo 1
  __shared__ C sphi[PY][PX];
  __shared__ C smu[MY][MX];
  __shared__ C spn[TGEN ? MY : 1][TGEN ? MX : 1];
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int x0 = blockIdx.x * C2_TX, y0 = blockIdx.y * C2_TY;
  const int tid = threadIdx.y * 32 + threadIdx.x;

  for (int k = tid; k < PX * PY; k += 256) {
    const int ry = k / PX, rx = k - ry * PX;
    const int gx = wrapi(x0 + rx - 2, Lx), gy = wrapi(y0 + ry - 2, Ly);
    sphi[ry][rx] = phi[(long long)gy * Lx + gx];
  }
  if constexpr (TGEN) {
    for (int k = tid; k < MX * MY; k += 256) {
      const int ry = k / MX, rx = k - ry * MX;
      const int gx = wrapi(x0 + rx - 1, Lx), gy = wrapi(y0 + ry - 1, Ly);
      spn[ry][rx] = p.cs2mT * (C(1) + dn[(long long)gy * Lx + gx]);
    }
  }
  __syncthreads();
  // mu = a phi + b phi^3 - kappa lap_D phi on the tile + 1 (Eqs. 5, 31)
  for (int k = tid; k < MX * MY; k += 256) {
    const int my = k / MX, mx = k - my * MX;
    const int cy = my + 1, cx = mx + 1;
    const C c = sphi[cy][cx];
    C lap = p.R * sphi[cy - 1][cx - 1];
    lap += p.Q * sphi[cy - 1][cx];
    lap += p.R * sphi[cy - 1][cx + 1];
    lap += p.Q * sphi[cy][cx - 1];
    lap += p.C0 * c;
    lap += p.Q * sphi[cy][cx + 1];
    lap += p.R * sphi[cy + 1][cx - 1];
    lap += p.Q * sphi[cy + 1][cx];
    lap += p.R * sphi[cy + 1][cx + 1];
    smu[my][mx] = p.a * c + p.b * c * c * c - p.kappa * lap;
  }
  __syncthreads();

#pragma unroll 1
  for (int r = 0; r < C2_TY / C2_BY; ++r) {
    const int lx = threadIdx.x, ly = threadIdx.y + C2_BY * r;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= Lx || y >= Ly) continue;
    // F = -phi d_D mu (Eqs. 28, 30)
    const int mx = lx + 1, my = ly + 1;
    C gmx = -p.M * smu[my - 1][mx - 1];
    gmx += p.M * smu[my - 1][mx + 1];
    gmx += -p.N * smu[my][mx - 1];
    gmx += p.N * smu[my][mx + 1];
    gmx += -p.M * smu[my + 1][mx - 1];
    gmx += p.M * smu[my + 1][mx + 1];
    C gmy = -p.M * smu[my - 1][mx - 1];
    gmy += -p.N * smu[my - 1][mx];
    gmy += -p.M * smu[my - 1][mx + 1];
    gmy += p.M * smu[my + 1][mx - 1];
    gmy += p.N * smu[my + 1][mx];
    gmy += p.M * smu[my + 1][mx + 1];
    const C ph = sphi[ly + 2][lx + 2];
    C Fx = -ph * gmx, Fy = -ph * gmy;
    if constexpr (TGEN) {
      C px = -p.M * spn[my - 1][mx - 1];
      px += p.M * spn[my - 1][mx + 1];
      px += -p.N * spn[my][mx - 1];
      px += p.N * spn[my][mx + 1];
      px += -p.M * spn[my + 1][mx - 1];
      px += p.M * spn[my + 1][mx + 1];
      C py = -p.M * spn[my - 1][mx - 1];
      py += -p.N * spn[my - 1][mx];
      py += -p.M * spn[my - 1][mx + 1];
      py += p.M * spn[my + 1][mx - 1];
      py += p.N * spn[my + 1][mx];
      py += p.M * spn[my + 1][mx + 1];
      Fx += px;
      Fy += py;
    }
    // pull the populations f_i(r, t) = buf_i(r - e_i)
    const int xm = x == 0 ? Lx - 1 : x - 1, xp = x == Lx - 1 ? 0 : x + 1;
    const long long rowc = (long long)y * Lx;
    const long long rowm = (long long)(y == 0 ? Ly - 1 : y - 1) * Lx;
    const long long rowp = (long long)(y == Ly - 1 ? 0 : y + 1) * Lx;
    C hv[9];
    hv[0] = Store<S, C>::ld(hin + 0 * Sz + rowc + x, p.inv_scale);
    hv[1] = Store<S, C>::ld(hin + 1 * Sz + rowc + xm, p.inv_scale);
    hv[2] = Store<S, C>::ld(hin + 2 * Sz + rowm + x, p.inv_scale);
    hv[3] = Store<S, C>::ld(hin + 3 * Sz + rowc + xp, p.inv_scale);
    hv[4] = Store<S, C>::ld(hin + 4 * Sz + rowp + x, p.inv_scale);
    hv[5] = Store<S, C>::ld(hin + 5 * Sz + rowm + xm, p.inv_scale);
    hv[6] = Store<S, C>::ld(hin + 6 * Sz + rowm + xp, p.inv_scale);
    hv[7] = Store<S, C>::ld(hin + 7 * Sz + rowp + xp, p.inv_scale);
    hv[8] = Store<S, C>::ld(hin + 8 * Sz + rowp + xm, p.inv_scale);
    // n - 1 and the momentum of the deviations (sum w_i e_i = 0)
    C dens = hv[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) dens += hv[i];
    const C jx = ((hv[1] - hv[3]) + (hv[5] - hv[7])) + (hv[8] - hv[6]);
    const C jy = ((hv[2] - hv[4]) + (hv[5] - hv[7])) + (hv[6] - hv[8]);
    const C n = C(1) + dens;
    Fx += n * p.gx;
    Fy += n * p.gy;
    // u* (Eq. 18)
    const C ux = (jx + C(0.5) * Fx) / n;
    const C uy = (jy + C(0.5) * Fy) / n;
    const long long s = rowc + x;
    if constexpr (MODE == COLLIDE_MOMENTS) {
      stg[s] = (double)n;
      stg[Sz + s] = (double)ph;
      stg[2 * Sz + s] = (double)ux;
      stg[3 * Sz + s] = (double)uy;
      continue;
    }
    const C usq = ux * ux + uy * uy;
    const C uF = ux * Fx + uy * Fy;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      constexpr C three = C(3), four5 = C(4.5), one5 = C(1.5), nine = C(9);
      const int ex = q9_ex(i), ey = q9_ey(i);
      const C w = C(q9_w(i));
      const C eu = C(ex) * ux + C(ey) * uy;
      const C eF = C(ex) * Fx + C(ey) * Fy;
      // feq_i - w_i (Eq. 15) and the forcing term (Eq. 29)
      const C heq = w * (dens + n * (three * eu + four5 * eu * eu - one5 * usq));
      const C Fi = p.pref * w * (three * (eF - uF) + nine * eu * eF);
      const C post = hv[i] - (hv[i] - heq) * p.tau_inv + Fi;
      Store<S, C>::st(hout + i * Sz + s, post, p.scale);
    }
    uout[s] = ux;
    uout[Sz + s] = uy;
  }
}

// ---- FD convection-diffusion, temporally blocked ---------------------------------
// Tile TX x TY, `sub` substeps; each substep shrinks the valid region by 3:
// advection needs phi, u at radius 1, psi = a phih + b phi^3 - kappa lap phih at
// radius 1 of the output, and the output adds dt Gamma lap psi.  This is Eq. 36
// with the three Laplacians regrouped into lap(a phih + b phi^3 - kappa lap phih)
// (the operator is linear, so the two forms differ by rounding only).
template <typename C, int TX, int TY>
__global__ void __launch_bounds__(256)
    fd2d_kernel(const C *__restrict__ phi_in, const C *__restrict__ u, C *__restrict__ phi_out,
                KParams<C> p, int sub) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sm = reinterpret_cast<C *>(smem_raw);
  const int H = 3 * sub, RX = TX + 2 * H, RY = TY + 2 * H, R = RX * RY;
  C *sp = sm, *sh = sm + R, *sq = sm + 2 * R, *su = sm + 3 * R, *sv = sm + 4 * R;
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int x0 = blockIdx.x * TX - H, y0 = blockIdx.y * TY - H;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int ry = ty; ry < RY; ry += 8) {
    const long long row = (long long)wrapi(y0 + ry, Ly) * Lx;
    for (int rx = tx; rx < RX; rx += 32) {
      const long long g = row + wrapi(x0 + rx, Lx);
      sp[ry * RX + rx] = phi_in[g];
      su[ry * RX + rx] = u[g];
      sv[ry * RX + rx] = u[Sz + g];
    }
  }
  __syncthreads();
  const C dt = p.dt, dtG = p.dtG;
#pragma unroll 1
  for (int s = 1; s <= sub; ++s) {
    // convective half step (Eqs. 32-35) on the region shrunk by 3s - 2
    int lo = 3 * s - 2;
    for (int ry = lo + ty; ry < RY - lo; ry += 8)
      for (int rx = lo + tx; rx < RX - lo; rx += 32) {
        const int k = ry * RX + rx;
        const C ph = sp[k];
        C tend;
        if (p.adv_variant == LBM_ADV_PAPER) {
          const C ua = su[k], va = sv[k];
          const C dux = (su[k + 1] - su[k - 1]) / C(2);
          const C dpx = ua < C(0) ? sp[k + 1] - ph : ph - sp[k - 1];
          const C duy = (sv[k + RX] - sv[k - RX]) / C(2);
          const C dpy = va < C(0) ? sp[k + RX] - ph : ph - sp[k - RX];
          tend = (ph * dux + ua * dpx);
          tend += (ph * duy + va * dpy);
        } else {
          const C Upx = C(0.5) * (su[k] + su[k + 1]);
          const C Umx = C(0.5) * (su[k - 1] + su[k]);
          const C Jpx = Upx > C(0) ? Upx * ph : Upx * sp[k + 1];
          const C Jmx = Umx > C(0) ? Umx * sp[k - 1] : Umx * ph;
          const C Upy = C(0.5) * (sv[k] + sv[k + RX]);
          const C Umy = C(0.5) * (sv[k - RX] + sv[k]);
          const C Jpy = Upy > C(0) ? Upy * ph : Upy * sp[k + RX];
          const C Jmy = Umy > C(0) ? Umy * sp[k - RX] : Umy * ph;
          tend = Jpx - Jmx;
          tend += Jpy - Jmy;
        }
        sh[k] = ph - dt * tend;
      }
    __syncthreads();
    // psi = a phih + b (phi^n)^3 - kappa lap phih (5-point Laplacian, Eq. 36)
    lo = 3 * s - 1;
    for (int ry = lo + ty; ry < RY - lo; ry += 8)
      for (int rx = lo + tx; rx < RX - lo; rx += 32) {
        const int k = ry * RX + rx;
        const C hk = sh[k];
        const C c = p.cubic_at_half ? hk : sp[k];
        C lap = sh[k - RX];
        lap += sh[k - 1];
        lap += C(-4) * hk;
        lap += sh[k + 1];
        lap += sh[k + RX];
        sq[k] = p.a * hk + p.b * (c * c * c) - p.kappa * lap;
      }
    __syncthreads();
    // phi^{n+1} = phih + dt Gamma lap psi
    lo = 3 * s;
    for (int ry = lo + ty; ry < RY - lo; ry += 8)
      for (int rx = lo + tx; rx < RX - lo; rx += 32) {
        const int k = ry * RX + rx;
        C lap = sq[k - RX];
        lap += sq[k - 1];
        lap += C(-4) * sq[k];
        lap += sq[k + 1];
        lap += sq[k + RX];
        sp[k] = sh[k] + dtG * lap;
      }
    __syncthreads();
  }
  for (int ry = H + ty; ry < H + TY; ry += 8) {
    const int gy = y0 + ry;
    if (gy >= Ly) break;
    for (int rx = H + tx; rx < H + TX; rx += 32) {
      const int gx = x0 + rx;
      if (gx < Lx) phi_out[(long long)gy * Lx + gx] = sp[ry * RX + rx];
    }
  }
}

template <typename S, typename C>
__global__ void __launch_bounds__(256)
    density2d_kernel(const S *__restrict__ hin, C *__restrict__ dn, KParams<C> p) {
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  if (x >= Lx || y >= Ly) return;
  const int xm = x == 0 ? Lx - 1 : x - 1, xp = x == Lx - 1 ? 0 : x + 1;
  const long long rowc = (long long)y * Lx;
  const long long rowm = (long long)(y == 0 ? Ly - 1 : y - 1) * Lx;
  const long long rowp = (long long)(y == Ly - 1 ? 0 : y + 1) * Lx;
  C d = Store<S, C>::ld(hin + rowc + x, p.inv_scale);
  d += Store<S, C>::ld(hin + 1 * Sz + rowc + xm, p.inv_scale);
  d += Store<S, C>::ld(hin + 2 * Sz + rowm + x, p.inv_scale);
  d += Store<S, C>::ld(hin + 3 * Sz + rowc + xp, p.inv_scale);
  d += Store<S, C>::ld(hin + 4 * Sz + rowp + x, p.inv_scale);
  d += Store<S, C>::ld(hin + 5 * Sz + rowm + xm, p.inv_scale);
  d += Store<S, C>::ld(hin + 6 * Sz + rowm + xp, p.inv_scale);
  d += Store<S, C>::ld(hin + 7 * Sz + rowp + xp, p.inv_scale);
  d += Store<S, C>::ld(hin + 8 * Sz + rowp + xm, p.inv_scale);
  dn[rowc + x] = d;
}

template <typename S, typename C>
cudaError_t collide2d(lbm_handle *h, int in, int force_on, int mode) {
  KParams<C> p = make_params<C>(h, force_on);
  dim3 grid((p.Lx + C2_TX - 1) / C2_TX, (p.Ly + C2_TY - 1) / C2_TY), block(32, C2_BY);
  const S *hin = static_cast<const S *>(h->h[in]);
  S *hout = static_cast<S *>(h->h[1 - in]);
  const C *phi = static_cast<const C *>(h->phi[in]);
  const C *dn = static_cast<const C *>(h->dn);
  C *u = static_cast<C *>(h->u);
  const bool tgen = p.cs2mT != C(0);
  if (mode == COLLIDE_STEP) {
    if (tgen)
      collide2d_kernel<S, C, true, COLLIDE_STEP>
          <<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
    else
      collide2d_kernel<S, C, false, COLLIDE_STEP>
          <<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
  } else {
    if (tgen)
      collide2d_kernel<S, C, true, COLLIDE_MOMENTS>
          <<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
    else
      collide2d_kernel<S, C, false, COLLIDE_MOMENTS>
          <<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
  }
  return cudaGetLastError();
}

template <typename C, int TX, int TY>
cudaError_t fd2d(lbm_handle *h, int in) {
  KParams<C> p = make_params<C>(h, 0);
  dim3 grid((p.Lx + TX - 1) / TX, (p.Ly + TY - 1) / TY), block(32, 8);
  const int launches = (h->m + h->sub - 1) / h->sub;
  const C *u = static_cast<const C *>(h->u);
  const C *src = static_cast<const C *>(h->phi[in]);
  for (int j = 0; j < launches; ++j) {
    const int sub = (j == launches - 1) ? h->m - h->sub * (launches - 1) : h->sub;
    C *dst = static_cast<C *>(((launches - 1 - j) % 2 == 0) ? h->phi[1 - in] : h->phi[2]);
    const int H = 3 * sub;
    const size_t smem = sizeof(C) * 5 * (size_t)(TX + 2 * H) * (TY + 2 * H);
    fd2d_kernel<C, TX, TY><<<grid, block, smem, h->stream>>>(src, u, dst, p, sub);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = dst;
  }
  return cudaSuccess;
}

}  // namespace

// FD tile per compute type: FP32 64 x 32, FP64 32 x 32 (shared memory budget).
constexpr int FD2_TX_F = 64, FD2_TY_F = 32, FD2_TX_D = 32, FD2_TY_D = 32;

size_t fd2d_smem_bytes(int precision, int sub) {
  const int H = 3 * sub;
  if (precision == LBM_F64) return sizeof(double) * 5 * (size_t)(FD2_TX_D + 2 * H) * (FD2_TY_D + 2 * H);
  return sizeof(float) * 5 * (size_t)(FD2_TX_F + 2 * H) * (FD2_TY_F + 2 * H);
}

cudaError_t fd2d_configure(int precision, size_t smem) {
  if (precision == LBM_F64)
    return cudaFuncSetAttribute(fd2d_kernel<double, FD2_TX_D, FD2_TY_D>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaFuncSetAttribute(fd2d_kernel<float, FD2_TX_F, FD2_TY_F>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t collide2d_launch(lbm_handle *h, int in, int force_on, int mode) {
  switch (h->P.precision) {
    case LBM_F64: return collide2d<double, double>(h, in, force_on, mode);
    case LBM_F32DEV: return collide2d<float, float>(h, in, force_on, mode);
    default: return collide2d<__half, float>(h, in, force_on, mode);
  }
}

cudaError_t fd2d_launch(lbm_handle *h, int in) {
  if (h->P.precision == LBM_F64) return fd2d<double, FD2_TX_D, FD2_TY_D>(h, in);
  return fd2d<float, FD2_TX_F, FD2_TY_F>(h, in);
}

cudaError_t density2d_launch(lbm_handle *h, int in) {
  dim3 grid((h->P.Lx + 31) / 32, (h->P.Ly + 7) / 8), block(32, 8);
  switch (h->P.precision) {
    case LBM_F64: {
      KParams<double> p = make_params<double>(h, 0);
      density2d_kernel<double, double><<<grid, block, 0, h->stream>>>(
          static_cast<const double *>(h->h[in]), static_cast<double *>(h->dn), p);
      break;
    }
    case LBM_F32DEV: {
      KParams<float> p = make_params<float>(h, 0);
      density2d_kernel<float, float><<<grid, block, 0, h->stream>>>(
          static_cast<const float *>(h->h[in]), static_cast<float *>(h->dn), p);
      break;
    }
    default: {
      KParams<float> p = make_params<float>(h, 0);
      density2d_kernel<__half, float><<<grid, block, 0, h->stream>>>(
          static_cast<const __half *>(h->h[in]), static_cast<float *>(h->dn), p);
    }
  }
  return cudaGetLastError();
}

}  // namespace hlbm
