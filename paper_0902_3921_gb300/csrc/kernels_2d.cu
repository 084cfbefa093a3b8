// kernels_2d.cu -- D2Q9 hot path on sm_103a.
//
//   collide2d : phi tile + halo 2 staged in shared memory -> mu (Eq. 5) on the
//               tile + 1 -> F = -phi d_D mu (+ grad((cs2 - T) n)) + n g (Eq. 28)
//               -> pull-streamed populations -> n, u* (Eqs. 12, 18) -> BGK with
//               the Guo forcing term (Eqs. 15, 17, 29) -> populations and u*.
//   fd2d      : `sub` substeps of the convection-diffusion update (Eqs. 32-36)
//               per launch, pipelined over rows by marching warps (halo 3 per
//               substep), with the launch shape chosen by the runtime's autotuner.
//   density2d : n - 1 of every site (only for T != 1/3, whose extra force
//               needs n on the neighbours).
//
// Populations are stored as deviations h_i = f_i - w_i in [i][y][x] order and
// streamed with the "pull" pattern: the buffer of time t holds the
// post-collision values of step t-1 at their source site, so
// f_i(r, t) = buf_i(r - e_i) and the kernel writes its own site only.
#include <type_traits>

#include "lbm_common.cuh"

namespace hlbm {

namespace {

constexpr int C2_TX = 32;  // tile width (one warp along x)
constexpr int C2_BY = 8;   // block of 32 x 8 threads, RY rows each (tile height 8 RY)

// One 32 x 8 RY tile with origin (x0, y0) of an Lx x Ly periodic lattice whose
// population and velocity planes are Sz values apart (Lx Ly for one lattice,
// the total site count for a batch); gx, gy the body force per unit density.
template <typename S, typename C, bool TGEN, int MODE, int RY>
__device__ __forceinline__ void collide2d_tile(const S *__restrict__ hin, S *__restrict__ hout,
                                               const C *__restrict__ phi, const C *__restrict__ dn,
                                               C *__restrict__ uout, double *__restrict__ stg,
                                               const KParams<C> &p, const int Lx, const int Ly,
                                               const long long Sz, const int x0, const int y0, const C gx,
                                               const C gy) {
  constexpr int C2_TY = C2_BY * RY;              // tile height
  constexpr int PX = C2_TX + 4, PY = C2_TY + 4;  // phi tile + halo 2
  constexpr int MX = C2_TX + 2, MY = C2_TY + 2;  // mu tile + halo 1
  __shared__ C sphi[PY][PX];
  __shared__ C smu[MY][MX];
  __shared__ C spn[TGEN ? MY : 1][TGEN ? MX : 1];
  const int tx = threadIdx.x, tid = threadIdx.y * 32 + threadIdx.x;

  // 1. issue the pull loads f_i(r, t) = buf_i(r - e_i) of this thread's sites
  //    first, so that they are in flight during the stencil phase
  const int x = x0 + tx;
  const bool xin = x < Lx;
  const int xc = xin ? x : Lx - 1;
  const int xm = xc == 0 ? Lx - 1 : xc - 1, xp = xc == Lx - 1 ? 0 : xc + 1;
  C hv[RY][9];
  long long site[RY];
  bool ok[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int y = y0 + threadIdx.y + C2_BY * r;
    ok[r] = xin && y < Ly;
    const int yc = y < Ly ? y : Ly - 1;
    const long long rowc = (long long)yc * Lx;
    const long long rowm = (long long)(yc == 0 ? Ly - 1 : yc - 1) * Lx;
    const long long rowp = (long long)(yc == Ly - 1 ? 0 : yc + 1) * Lx;
    site[r] = rowc + xc;
    hv[r][0] = Store<S, C>::ld(hin + 0 * Sz + rowc + xc, p.inv_scale);
    hv[r][1] = Store<S, C>::ld(hin + 1 * Sz + rowc + xm, p.inv_scale);
    hv[r][2] = Store<S, C>::ld(hin + 2 * Sz + rowm + xc, p.inv_scale);
    hv[r][3] = Store<S, C>::ld(hin + 3 * Sz + rowc + xp, p.inv_scale);
    hv[r][4] = Store<S, C>::ld(hin + 4 * Sz + rowp + xc, p.inv_scale);
    hv[r][5] = Store<S, C>::ld(hin + 5 * Sz + rowm + xm, p.inv_scale);
    hv[r][6] = Store<S, C>::ld(hin + 6 * Sz + rowm + xp, p.inv_scale);
    hv[r][7] = Store<S, C>::ld(hin + 7 * Sz + rowp + xp, p.inv_scale);
    hv[r][8] = Store<S, C>::ld(hin + 8 * Sz + rowp + xm, p.inv_scale);
  }

  // 2. phi on the tile + halo 2 (periodic) and mu on the tile + 1
  const bool big = Lx >= PX && Ly >= PY;  // one conditional wrap suffices
  for (int ry = threadIdx.y; ry < PY; ry += C2_BY) {
    const int gy = big ? wrap1(y0 + ry - 2, Ly) : wrapi(y0 + ry - 2, Ly);
    const C *prow = phi + (long long)gy * Lx;
    for (int rx = tx; rx < PX; rx += 32) {
      const int gx = big ? wrap1(x0 + rx - 2, Lx) : wrapi(x0 + rx - 2, Lx);
      sphi[ry][rx] = prow[gx];
    }
  }
  if constexpr (TGEN) {
    for (int k = tid; k < MX * MY; k += 256) {
      const int ry = k / MX, rx = k - ry * MX;
      const int gx = wrapi(x0 + rx - 1, Lx), gy = wrapi(y0 + ry - 1, Ly);
      spn[ry][rx] = p.cs2mT * (C(1) + dn[(long long)gy * Lx + gx]);
    }
  }
  __syncthreads();
  // mu = a phi + b phi^3 - kappa lap_D phi (Eqs. 5, 31)
  for (int my = threadIdx.y; my < MY; my += C2_BY)
    for (int mx = tx; mx < MX; mx += 32) {
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

  // 3. force, moments, collision and the writes of each site
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    if (!ok[r]) continue;
    const int lx = tx, ly = threadIdx.y + C2_BY * r;
    const int mx = lx + 1, my = ly + 1;
    // F = -phi d_D mu (Eqs. 28, 30)
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
    const C *h = hv[r];
    // n - 1 and the momentum of the deviations (sum w_i e_i = 0)
    C dens = h[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) dens += h[i];
    const C jx = ((h[1] - h[3]) + (h[5] - h[7])) + (h[8] - h[6]);
    const C jy = ((h[2] - h[4]) + (h[5] - h[7])) + (h[6] - h[8]);
    const C n = C(1) + dens;
    Fx += n * gx;
    Fy += n * gy;
    // u* (Eq. 18)
    const C ux = (jx + C(0.5) * Fx) / n;
    const C uy = (jy + C(0.5) * Fy) / n;
    const long long s = site[r];
    if constexpr (MODE == COLLIDE_MOMENTS) {
      stg[s] = (double)n;
      stg[Sz + s] = (double)ph;
      stg[2 * Sz + s] = (double)ux;
      stg[3 * Sz + s] = (double)uy;
      continue;
    }
    const C usq = ux * ux + uy * uy;
    const C uF = ux * Fx + uy * Fy;
    const C om = p.tau_inv, keep = C(1) - p.tau_inv;
    // rest population: feq_0 - w_0 (Eq. 15) and F_0 (Eq. 29)
    {
      const C w = C(q9_w(0));
      const C heq = w * (dens - n * (C(1.5) * usq));
      const C Fi = p.pref * w * (C(-3) * uF);
      Store<S, C>::st(hout + s, keep * h[0] + om * heq + Fi, p.scale);
    }
    // opposite pairs (i, ibar) share the even parts of feq and F_i and have
    // odd parts of opposite sign
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = k < 2 ? k + 1 : k + 3, ib = i + 2;  // (1,3) (2,4) (5,7) (6,8)
      const C w = C(q9_w(i));
      const C eu = C(q9_ex(i)) * ux + C(q9_ey(i)) * uy;
      const C eF = C(q9_ex(i)) * Fx + C(q9_ey(i)) * Fy;
      const C even = w * (dens + n * (C(4.5) * eu * eu - C(1.5) * usq));
      const C odd = w * (n * (C(3) * eu));
      const C Feven = p.pref * w * (C(9) * eu * eF - C(3) * uF);
      const C Fodd = p.pref * w * (C(3) * eF);
      Store<S, C>::st(hout + i * Sz + s, keep * h[i] + om * (even + odd) + (Feven + Fodd),
                      p.scale);
      Store<S, C>::st(hout + ib * Sz + s, keep * h[ib] + om * (even - odd) + (Feven - Fodd),
                      p.scale);
    }
    uout[s] = ux;
    uout[Sz + s] = uy;
  }
}

template <typename S, typename C, bool TGEN, int MODE, int RY>
__global__ void __launch_bounds__(256, 2)
    collide2d_kernel(const S *__restrict__ hin, S *__restrict__ hout, const C *__restrict__ phi,
                     const C *__restrict__ dn, C *__restrict__ uout, double *__restrict__ stg,
                     KParams<C> p) {
  collide2d_tile<S, C, TGEN, MODE, RY>(hin, hout, phi, dn, uout, stg, p, p.Lx, p.Ly, (long long)p.Lx * p.Ly,
                                       blockIdx.x * C2_TX, blockIdx.y * (C2_BY * RY), p.gx, p.gy);
}

// The same tile step for many independent lattices packed end to end (one
// plane per population over all of them, ST sites): CTA b takes the 32 x 16
// tile items[b] = (instance, x0, y0) and the instance's size, offset and body
// force (on while t < force_steps).  FP32 deviations, T = 1/3.
__global__ void __launch_bounds__(256, 2)
    collide2d_batch_kernel(const float *__restrict__ hin, float *__restrict__ hout,
                           const float *__restrict__ phi, float *__restrict__ u, long long ST,
                           const TiledInst *__restrict__ inst, const int4 *__restrict__ items,
                           KParams<float> p, long long t) {
  const int4 it = items[blockIdx.x];
  const TiledInst I = inst[it.x];
  const bool on = t < I.force_steps;
  collide2d_tile<float, float, false, COLLIDE_STEP, BATCH_TILE_ROWS / C2_BY>(
      hin + I.off, hout + I.off, phi + I.off, nullptr, u + I.off, nullptr, p, I.Lx, I.Ly, ST, it.y, it.z,
      on ? I.gx : 0.f, on ? I.gy : 0.f);
}

// ---- collide with asynchronous staging (FP32 / FP64 populations) ----------------
// The same arithmetic as collide2d_kernel, but every pulled population and the
// phi tile are copied global -> shared with cp.async, so that the whole tile
// (9 planes of 32 x 32 sites) is in flight at once without holding registers;
// 4 CTAs per SM keep about 150 KB of loads outstanding per SM.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gsrc), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

constexpr int CA_TX = 32, CA_TY = 32, CA_RY = CA_TY / C2_BY;

template <typename C>
constexpr size_t collide_async_smem() {
  return sizeof(C) * (9 * CA_TX * CA_TY + (CA_TX + 4) * (CA_TY + 4) + 2 * (CA_TX + 2) * (CA_TY + 2));
}

template <typename C, bool TGEN, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB)
    collide2d_async_kernel(const C *__restrict__ hin, C *__restrict__ hout,
                           const C *__restrict__ phi, const C *__restrict__ dn,
                           C *__restrict__ uout, double *__restrict__ stg, KParams<C> p) {
  // thread (tx, ty) owns column tx, rows 4 ty .. 4 ty + 3 of the 32 x 32 tile,
  // so the 3 x 3 stencils reuse rows from registers
  constexpr int PX = CA_TX + 4, PY = CA_TY + 4, MX = CA_TX + 2, MY = CA_TY + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C(*pops)[CA_TY][CA_TX] = reinterpret_cast<C(*)[CA_TY][CA_TX]>(smem_raw);
  C(*sphi)[PX] = reinterpret_cast<C(*)[PX]>(smem_raw + sizeof(C) * 9 * CA_TX * CA_TY);
  C(*smu)[MX] = reinterpret_cast<C(*)[MX]>(smem_raw + sizeof(C) * (9 * CA_TX * CA_TY + PX * PY));
  C(*spn)[MX] = smu + MY;
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int x0 = blockIdx.x * CA_TX, y0 = blockIdx.y * CA_TY;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int ly0 = 4 * ty;
  const int x = x0 + tx;
  const int xm = x == 0 ? Lx - 1 : x - 1, xp = x >= Lx - 1 ? 0 : x + 1;
  pdl_wait();  // phi(t) comes from the previous kernel
  pdl_trigger();
  // 1. every pulled population f_i(r, t) = buf_i(r - e_i) of the tile
#pragma unroll
  for (int r = 0; r < CA_RY; ++r) {
    const int ly = ly0 + r, y = y0 + ly;
    if (x >= Lx || y >= Ly) continue;
    const long long rowc = (long long)y * Lx;
    const long long rowm = (long long)(y == 0 ? Ly - 1 : y - 1) * Lx;
    const long long rowp = (long long)(y == Ly - 1 ? 0 : y + 1) * Lx;
    cp_async<sizeof(C)>(&pops[0][ly][tx], hin + 0 * Sz + rowc + x);
    cp_async<sizeof(C)>(&pops[1][ly][tx], hin + 1 * Sz + rowc + xm);
    cp_async<sizeof(C)>(&pops[2][ly][tx], hin + 2 * Sz + rowm + x);
    cp_async<sizeof(C)>(&pops[3][ly][tx], hin + 3 * Sz + rowc + xp);
    cp_async<sizeof(C)>(&pops[4][ly][tx], hin + 4 * Sz + rowp + x);
    cp_async<sizeof(C)>(&pops[5][ly][tx], hin + 5 * Sz + rowm + xm);
    cp_async<sizeof(C)>(&pops[6][ly][tx], hin + 6 * Sz + rowm + xp);
    cp_async<sizeof(C)>(&pops[7][ly][tx], hin + 7 * Sz + rowp + xp);
    cp_async<sizeof(C)>(&pops[8][ly][tx], hin + 8 * Sz + rowp + xm);
  }
  // 2. phi on the tile + halo 2 (periodic)
  const bool big = Lx >= PX && Ly >= PY;
  for (int ry = ty; ry < PY; ry += C2_BY) {
    const int gy = big ? wrap1(y0 + ry - 2, Ly) : wrapi(y0 + ry - 2, Ly);
    const C *prow = phi + (long long)gy * Lx;
    for (int rx = tx; rx < PX; rx += 32) {
      const int gx = big ? wrap1(x0 + rx - 2, Lx) : wrapi(x0 + rx - 2, Lx);
      cp_async<sizeof(C)>(&sphi[ry][rx], prow + gx);
    }
  }
  if constexpr (TGEN) {
    for (int k = tid; k < MX * MY; k += 256) {
      const int ry = k / MX, rx = k - ry * MX;
      const int gx = wrapi(x0 + rx - 1, Lx), gy = wrapi(y0 + ry - 1, Ly);
      spn[ry][rx] = p.cs2mT * (C(1) + dn[(long long)gy * Lx + gx]);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // mu = a phi + b phi^3 - kappa lap_D phi (Eqs. 5, 31) on the tile + 1:
  // the 32 x 32 interior four rows per thread with rows reused from
  // registers, then the one-site frame (132 sites) flat
  auto mu_at = [&](C (&w)[3][3]) {  // explicitly rounded: evaluated in two places
    C lap = rn_mul(p.R, w[0][0]);
    lap = rn_fma(p.Q, w[0][1], lap);
    lap = rn_fma(p.R, w[0][2], lap);
    lap = rn_fma(p.Q, w[1][0], lap);
    lap = rn_fma(p.C0, w[1][1], lap);
    lap = rn_fma(p.Q, w[1][2], lap);
    lap = rn_fma(p.R, w[2][0], lap);
    lap = rn_fma(p.Q, w[2][1], lap);
    lap = rn_fma(p.R, w[2][2], lap);
    const C c = w[1][1];
    const C c3 = rn_mul(rn_mul(c, c), c);
    return rn_fma(p.a, c, rn_fma(p.b, c3, rn_mul(-p.kappa, lap)));
  };
  {
    // interior mu rows my = ly0 + 1 .. ly0 + 4, column mx = tx + 1 (phi rows my - 1 .. my + 1
    // of the phi tile are rows my .. my + 2, columns tx + 1 .. tx + 3)
    C w[3][3];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) w[k + 1][j] = sphi[ly0 + 1 + k][tx + 1 + j];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        w[0][j] = w[1][j];
        w[1][j] = w[2][j];
        w[2][j] = sphi[ly0 + 3 + r][tx + 1 + j];
      }
      smu[ly0 + 1 + r][tx + 1] = mu_at(w);
    }
    for (int k = tid; k < 2 * MX + 2 * (MY - 2); k += 256) {
      int my, mx;
      if (k < MX) { my = 0; mx = k; }
      else if (k < 2 * MX) { my = MY - 1; mx = k - MX; }
      else { const int q = k - 2 * MX; my = 1 + (q >> 1); mx = (q & 1) ? MX - 1 : 0; }
      C v[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2) v[a][b2] = sphi[my + a][mx + b2];
      smu[my][mx] = mu_at(v);
    }
  }
  __syncthreads();
  // 3. force, moments, collision; mu rows reused from registers
  C m3[3][3];  // mu rows (ly - 1 .. ly + 1) x columns (tx - 1 .. tx + 1), tile + 1 coordinates
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) m3[k + 1][j] = smu[ly0 + k][tx + j];
  const C om = p.tau_inv, keep = C(1) - p.tau_inv;
#pragma unroll 1
  for (int r = 0; r < CA_RY; ++r) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      m3[0][j] = m3[1][j];
      m3[1][j] = m3[2][j];
      m3[2][j] = smu[ly0 + r + 2][tx + j];
    }
    const int lx = tx, ly = ly0 + r, y = y0 + ly;
    if (x >= Lx || y >= Ly) continue;
    C gmx = -p.M * m3[0][0];
    gmx += p.M * m3[0][2];
    gmx += -p.N * m3[1][0];
    gmx += p.N * m3[1][2];
    gmx += -p.M * m3[2][0];
    gmx += p.M * m3[2][2];
    C gmy = -p.M * m3[0][0];
    gmy += -p.N * m3[0][1];
    gmy += -p.M * m3[0][2];
    gmy += p.M * m3[2][0];
    gmy += p.N * m3[2][1];
    gmy += p.M * m3[2][2];
    const C ph = sphi[ly + 2][lx + 2];
    C Fx = -ph * gmx, Fy = -ph * gmy;
    if constexpr (TGEN) {
      const int mx = lx + 1, my = ly + 1;
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
    C h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = pops[i][ly][lx];
    C dens = h[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) dens += h[i];
    const C jx = ((h[1] - h[3]) + (h[5] - h[7])) + (h[8] - h[6]);
    const C jy = ((h[2] - h[4]) + (h[5] - h[7])) + (h[6] - h[8]);
    const C n = C(1) + dens;
    Fx += n * p.gx;
    Fy += n * p.gy;
    const C inv_n = C(1) / n;
    const C ux = (jx + C(0.5) * Fx) * inv_n;
    const C uy = (jy + C(0.5) * Fy) * inv_n;
    const long long s = (long long)y * Lx + x;
    if constexpr (MODE == COLLIDE_MOMENTS) {
      stg[s] = (double)n;
      stg[Sz + s] = (double)ph;
      stg[2 * Sz + s] = (double)ux;
      stg[3 * Sz + s] = (double)uy;
      continue;
    }
    const C usq = ux * ux + uy * uy;
    const C uF = ux * Fx + uy * Fy;
    {
      const C w = C(q9_w(0));
      const C heq = w * (dens - n * (C(1.5) * usq));
      const C Fi = p.pref * w * (C(-3) * uF);
      hout[s] = keep * h[0] + om * heq + Fi;
    }
    const C base = dens - n * (C(1.5) * usq);  // the u-independent and |u|^2 parts
    const C n3 = C(3) * n, n45 = C(4.5) * n;
    const C pF3 = C(3) * p.pref, pF9 = C(9) * p.pref, puF = C(3) * p.pref * uF;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = k < 2 ? k + 1 : k + 3, ib = i + 2;  // (1,3) (2,4) (5,7) (6,8)
      const C w = C(q9_w(i));
      const C eu = C(q9_ex(i)) * ux + C(q9_ey(i)) * uy;
      const C eF = C(q9_ex(i)) * Fx + C(q9_ey(i)) * Fy;
      const C even = w * (base + n45 * eu * eu);
      const C odd = w * (n3 * eu);
      const C Feven = w * (pF9 * eu * eF - puF);
      const C Fodd = w * (pF3 * eF);
      hout[i * Sz + s] = keep * h[i] + om * (even + odd) + (Feven + Fodd);
      hout[ib * Sz + s] = keep * h[ib] + om * (even - odd) + (Feven - Fodd);
    }
    uout[s] = ux;
    uout[Sz + s] = uy;
  }
}

// ---- FD convection-diffusion: warp-marching temporal blocking -------------------
// One warp owns a strip of W = 32 V columns (V consecutive columns per lane)
// and marches down a tile of TY output rows, running SUB substeps of Eqs.
// 32-36 as a software pipeline over rows.  When row r of phi is loaded:
//   substep s advects row r - 1 - 3s, forms psi = a phih + b phi^3 -
//   kappa lap phih on row r - 2 - 3s and the new phi on row r - 3 - 3s,
// so every value lives in a 3-row register ring and the x neighbours come
// from the adjacent lane by warp shuffles.  Each substep loses one column
// (row) of validity per stencil, i.e. 3 per substep: the strip outputs its
// middle OW = W - 2 HX columns and the tile reads 3 SUB extra rows on both
// sides.  Eq. 36's three Laplacians are regrouped as
// lap(a phih + b phi^3 - kappa lap phih) (the operator is linear).
// The advection terms of a row (d_x u and d_y v of Eq. 33, u and v, or the
// face velocities of the flux form) are computed once per launch and kept in
// a per-lane shared-memory ring until the last substep has used them.
// packed FP32 pairs (two columns of a lane) for the FD stages
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename C, int V>
struct VecT;
template <>
struct VecT<float, 4> {
  using T = float4;
};
template <>
struct VecT<float, 2> {
  using T = float2;
};
template <>
struct VecT<double, 2> {
  using T = double2;
};

template <typename C, int V>
__device__ __forceinline__ void load_row(const C *__restrict__ row, const int (&gx)[V],
                                         bool vec, C (&out)[V]) {
  if (vec) {
    using T = typename VecT<C, V>::T;
    const T t = __ldg(reinterpret_cast<const T *>(row + gx[0]));
    const C *tc = reinterpret_cast<const C *>(&t);
#pragma unroll
    for (int j = 0; j < V; ++j) out[j] = tc[j];
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) out[j] = __ldg(row + gx[j]);
  }
}

template <typename C, int V, int SUB>
__global__ void __launch_bounds__(64)
    fd2d_march_kernel(const C *__restrict__ phi_in, const C *__restrict__ u,
                      C *__restrict__ phi_out, KParams<C> p, int TY, int nstrips, int ntiles) {
  constexpr int H = 3 * SUB;                    // rows of halo per side
  constexpr int HX = (H + V - 1) / V * V;       // columns of halo, a multiple of V
  constexpr int W = 32 * V, OW = W - 2 * HX;    // strip width and output width
  constexpr int RD = 3 * SUB - 2;               // rows of advection terms kept
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ __align__(16) C terms[2][RD][4][W];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wid = blockIdx.x * 2 + warp;
  if (wid >= nstrips * ntiles) return;  // whole warp: no block barriers are used
  const int sx = wid % nstrips, tyi = wid / nstrips;
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int xs = sx * OW - HX;  // global column of local column 0
  const int y0 = tyi * TY;
  const int NR = TY + 2 * H;
  int gx[V];
#pragma unroll
  for (int j = 0; j < V; ++j) gx[j] = wrapi(xs + V * lane + j, Lx);
  const bool vec = (Lx % V) == 0;  // then a lane's V columns are contiguous and aligned
  C (*T)[4][W] = terms[warp];

  C ph[SUB][3][V], A[SUB][3][V], P[SUB][3][V], vr[3][V], ur[V];
#pragma unroll
  for (int s = 0; s < SUB; ++s)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < V; ++j) ph[s][k][j] = A[s][k][j] = P[s][k][j] = C(0);
#pragma unroll
  for (int j = 0; j < V; ++j) {
    ur[j] = C(0);
    vr[0][j] = vr[1][j] = vr[2][j] = C(0);
  }
  const C dt = p.dt, dtG = p.dtG, a = p.a, b = p.b, kappa = p.kappa;
  const bool paper = p.adv_variant == LBM_ADV_PAPER, cubic_half = p.cubic_at_half != 0;
  int tw = RD - 1;  // terms slot of row r - 1
  int gy = wrapi(y0 - H, Ly);  // global row of the next load

  // row r + 1 is loaded while row r is processed
  C nph[V], nu[V], nv[V];
  {
    const long long grow = (long long)gy * Lx;
    load_row<C, V>(phi_in + grow, gx, vec, nph);
    load_row<C, V>(u + grow, gx, vec, nu);
    load_row<C, V>(u + Sz + grow, gx, vec, nv);
  }
  auto row = [&](auto R3c, int r) {
    constexpr int R3 = decltype(R3c)::value;
    constexpr int S0 = R3, S1 = (R3 + 1) % 3, S2 = (R3 + 2) % 3;
    // slots: row r -> S0, r - 1 -> S2, r - 2 -> S1 (rows are stored at row % 3)
    C un[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      ph[0][S0][j] = nph[j];
      un[j] = nu[j];
      vr[S0][j] = nv[j];
    }
    if (r + 1 < NR) {
      gy = gy + 1 == Ly ? 0 : gy + 1;
      const long long grow = (long long)gy * Lx;
      load_row<C, V>(phi_in + grow, gx, vec, nph);
      load_row<C, V>(u + grow, gx, vec, nu);
      load_row<C, V>(u + Sz + grow, gx, vec, nv);
    }
    tw = tw + 1 == RD ? 0 : tw + 1;
    {  // advection terms of row r - 1
      const C uL0 = __shfl_up_sync(FULL, ur[V - 1], 1);
      const C uRV = __shfl_down_sync(FULL, ur[0], 1);
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const C uc = ur[j], uL = j == 0 ? uL0 : ur[j - 1], uR = j == V - 1 ? uRV : ur[j + 1];
        const C vm = vr[S1][j], vc = vr[S2][j], vp = vr[S0][j];
        C t0, t1, t2, t3 = C(0);
        if (paper) {
          // Eqs. 32-35 as phih = c0 phi + |dt u| phi_upx + |dt v| phi_upy with
          // c0 = 1 - dt (d_x u + d_y v + |u| + |v|); the upwind side is the
          // sign of dt u (dt v): positive -> x - 1 (y - 1), else x + 1 (y + 1)
          const C div = (uR - uL) / C(2) + (vp - vm) / C(2);
          t0 = C(1) - dt * (div + (fabs(uc) + fabs(vc)));
          t1 = dt * uc;
          t2 = dt * vc;
        } else {
          t0 = C(0.5) * (uc + uR);
          t1 = C(0.5) * (uL + uc);
          t2 = C(0.5) * (vc + vp);
          t3 = C(0.5) * (vm + vc);
        }
        T[tw][0][V * lane + j] = t0;
        T[tw][1][V * lane + j] = t1;
        T[tw][2][V * lane + j] = t2;
        if (!paper) T[tw][3][V * lane + j] = t3;
      }
#pragma unroll
      for (int j = 0; j < V; ++j) ur[j] = un[j];
    }
#pragma unroll
    for (int s = 0; s < SUB; ++s) {
      const int nw = r - 3 * s;  // newest row of the input of substep s
      // rows of substep s outside [3s + 1, NR - 3s - 1) never reach the output
      if (nw - 1 >= 3 * s + 1) {  // convective half step (Eqs. 32-35) on row nw - 1
        int ts = tw - 3 * s;
        if (ts < 0) ts += RD;
        const C(&cur)[V] = ph[s][S2];
        const C(&up)[V] = ph[s][S1];
        const C(&dn)[V] = ph[s][S0];
        const C l0 = __shfl_up_sync(FULL, cur[V - 1], 1);
        const C rV = __shfl_down_sync(FULL, cur[0], 1);
        bool packed = false;
        if constexpr (std::is_same<C, float>::value) {
          if (paper) {  // two columns per packed FP32x2 instruction
            packed = true;
#pragma unroll
            for (int j = 0; j < V; j += 2) {
              const float2 t0 = *reinterpret_cast<const float2 *>(&T[ts][0][V * lane + j]);
              const float2 t1 = *reinterpret_cast<const float2 *>(&T[ts][1][V * lane + j]);
              const float2 t2 = *reinterpret_cast<const float2 *>(&T[ts][2][V * lane + j]);
              const float pl = j == 0 ? l0 : cur[j - 1], pr = j + 1 == V - 1 ? rV : cur[j + 2];
              const float2 upx = f2(t1.x > 0.f ? pl : cur[j + 1], t1.y > 0.f ? cur[j] : pr);
              const float2 upy = f2(t2.x > 0.f ? up[j] : dn[j], t2.y > 0.f ? up[j + 1] : dn[j + 1]);
              const float2 r = fma2(f2(fabsf(t2.x), fabsf(t2.y)), upy,
                                    fma2(f2(fabsf(t1.x), fabsf(t1.y)), upx,
                                         mul2(t0, f2(cur[j], cur[j + 1]))));
              A[s][S2][j] = r.x;
              A[s][S2][j + 1] = r.y;
            }
          }
        }
        if (!packed) {
#pragma unroll
          for (int j = 0; j < V; ++j) {
            const C pc = cur[j], pl = j == 0 ? l0 : cur[j - 1], pr = j == V - 1 ? rV : cur[j + 1];
            const C t0 = T[ts][0][V * lane + j], t1 = T[ts][1][V * lane + j];
            const C t2 = T[ts][2][V * lane + j];
            if (paper) {
              const C upx = t1 > C(0) ? pl : pr;  // u = 0 contributes nothing
              const C upy = t2 > C(0) ? up[j] : dn[j];
              A[s][S2][j] = t0 * pc + fabs(t1) * upx + fabs(t2) * upy;
            } else {
              const C t3 = T[ts][3][V * lane + j];
              const C Jpx = t0 > C(0) ? t0 * pc : t0 * pr;
              const C Jmx = t1 > C(0) ? t1 * pl : t1 * pc;
              const C Jpy = t2 > C(0) ? t2 * pc : t2 * dn[j];
              const C Jmy = t3 > C(0) ? t3 * up[j] : t3 * pc;
              C tend = Jpx - Jmx;
              tend += Jpy - Jmy;
              A[s][S2][j] = pc - dt * tend;
            }
          }
        }
      }
      if (nw - 2 >= 3 * s + 2) {  // psi on row nw - 2 (Eq. 36)
        const C(&Ac)[V] = A[s][S1];
        const C l0 = __shfl_up_sync(FULL, Ac[V - 1], 1);
        const C rV = __shfl_down_sync(FULL, Ac[0], 1);
        if constexpr (std::is_same<C, float>::value) {
          const float2 a2 = f2(a, a), b2 = f2(b, b), mk2 = f2(-kappa, -kappa), m4 = f2(-4.f, -4.f);
#pragma unroll
          for (int j = 0; j < V; j += 2) {
            const float2 hk = f2(Ac[j], Ac[j + 1]);
            const float2 left = f2(j == 0 ? l0 : Ac[j - 1], Ac[j]);
            const float2 right = f2(Ac[j + 1], j + 1 == V - 1 ? rV : Ac[j + 2]);
            float2 lap = add2(f2(A[s][S0][j], A[s][S0][j + 1]), left);
            lap = fma2(m4, hk, lap);
            lap = add2(lap, right);
            lap = add2(lap, f2(A[s][S2][j], A[s][S2][j + 1]));
            const float2 c = cubic_half ? hk : f2(ph[s][S1][j], ph[s][S1][j + 1]);
            const float2 r = fma2(a2, hk, fma2(b2, mul2(mul2(c, c), c), mul2(mk2, lap)));
            P[s][S1][j] = r.x;
            P[s][S1][j + 1] = r.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < V; ++j) {
            const C hk = Ac[j];
            C lap = A[s][S0][j];
            lap += j == 0 ? l0 : Ac[j - 1];
            lap += C(-4) * hk;
            lap += j == V - 1 ? rV : Ac[j + 1];
            lap += A[s][S2][j];
            const C c = cubic_half ? hk : ph[s][S1][j];
            P[s][S1][j] = a * hk + b * (c * c * c) - kappa * lap;
          }
        }
      }
      if (nw - 3 >= 3 * s + 3) {  // phi of the next substep on row nw - 3
        const C(&Pc)[V] = P[s][S0];
        const C l0 = __shfl_up_sync(FULL, Pc[V - 1], 1);
        const C rV = __shfl_down_sync(FULL, Pc[0], 1);
        C F[V];
        if constexpr (std::is_same<C, float>::value) {
          const float2 g2 = f2(dtG, dtG), m4 = f2(-4.f, -4.f);
#pragma unroll
          for (int j = 0; j < V; j += 2) {
            const float2 pc = f2(Pc[j], Pc[j + 1]);
            float2 lap = add2(f2(P[s][S2][j], P[s][S2][j + 1]), f2(j == 0 ? l0 : Pc[j - 1], Pc[j]));
            lap = fma2(m4, pc, lap);
            lap = add2(lap, f2(Pc[j + 1], j + 1 == V - 1 ? rV : Pc[j + 2]));
            lap = add2(lap, f2(P[s][S1][j], P[s][S1][j + 1]));
            const float2 r = fma2(g2, lap, f2(A[s][S0][j], A[s][S0][j + 1]));
            F[j] = r.x;
            F[j + 1] = r.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < V; ++j) {
            C lap = P[s][S2][j];
            lap += j == 0 ? l0 : Pc[j - 1];
            lap += C(-4) * Pc[j];
            lap += j == V - 1 ? rV : Pc[j + 1];
            lap += P[s][S1][j];
            F[j] = A[s][S0][j] + dtG * lap;
          }
        }
        if (s + 1 < SUB) {
#pragma unroll
          for (int j = 0; j < V; ++j) ph[s + 1 < SUB ? s + 1 : 0][S0][j] = F[j];
        } else {
          const int orow = nw - 3 - H;  // output row within the tile
          const int gy = y0 + orow;
          if (orow >= 0 && orow < TY && gy < Ly) {
            C *dst = phi_out + (long long)gy * Lx;
#pragma unroll
            for (int j = 0; j < V; ++j) {
              const int c = V * lane + j;
              const int x = sx * OW + c - HX;
              if (c >= HX && c < HX + OW && x < Lx) dst[x] = F[j];
            }
          }
        }
      }
    }
  };
  for (int r = 0; r < NR; r += 3) {
    row(std::integral_constant<int, 0>{}, r);
    if (r + 1 < NR) row(std::integral_constant<int, 1>{}, r + 1);
    if (r + 2 < NR) row(std::integral_constant<int, 2>{}, r + 2);
  }
}

// ---- FD convection-diffusion: shared-memory tile, SUB substeps per launch ----------
// A block of 32 x 8 threads owns a region RXW (a multiple of 32) wide and
// TY + 2H high (H = 3 SUB) whose inner TX = RXW - 2H columns are written.
// phi, u and v are staged once; the advection coefficients of Eqs. 32-35
// (printed form: c0, dt u, dt v; flux form: the four face velocities) are
// kept in registers for the thread's sites, and each substep runs three
// phases (phih, psi, new phi) over a region that shrinks by one site per
// phase, with a block barrier between phases.
template <typename C, int RXW, int SUB>
struct FDTile {
  static constexpr int H = 3 * SUB, TX = RXW - 2 * H, TY = 32, RY = TY + 2 * H;
  static constexpr int NXI = RXW / 32, NYI = (RY + 7) / 8;
  static constexpr size_t smem = sizeof(C) * 3 * (size_t)RXW * RY;
};

template <typename C, int RXW, int SUB>
__global__ void __launch_bounds__(256)
    fd2d_tile_kernel(const C *__restrict__ phi_in, const C *__restrict__ u,
                     C *__restrict__ phi_out, KParams<C> p) {
  using G = FDTile<C, RXW, SUB>;
  constexpr int H = G::H, TX = G::TX, TY = G::TY, RY = G::RY, NXI = G::NXI, NYI = G::NYI;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sp = reinterpret_cast<C *>(smem_raw);
  C *sa = sp + RXW * RY;
  C *sq = sa + RXW * RY;
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int x0 = blockIdx.x * TX - H, y0 = blockIdx.y * TY - H;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool big = Lx >= RXW && Ly >= RY;
  // 1. stage phi -> sp, u -> sa, v -> sq on the whole region
  for (int ry = ty; ry < RY; ry += 8) {
    const int gy = big ? wrap1(y0 + ry, Ly) : wrapi(y0 + ry, Ly);
    const long long row = (long long)gy * Lx;
#pragma unroll
    for (int xi = 0; xi < NXI; ++xi) {
      const int rx = tx + 32 * xi;
      const int gx = big ? wrap1(x0 + rx, Lx) : wrapi(x0 + rx, Lx);
      const int k = ry * RXW + rx;
      sp[k] = __ldg(phi_in + row + gx);
      sa[k] = __ldg(u + row + gx);
      sq[k] = __ldg(u + Sz + row + gx);
    }
  }
  __syncthreads();
  // 2. advection coefficients of this thread's sites (registers)
  const bool paper = p.adv_variant == LBM_ADV_PAPER, cubic_half = p.cubic_at_half != 0;
  const bool stencil = p.stencil_fd != 0;  // Eqs. 30-31 in place of Eq. 33 and the 5-point Laplacian
  const C dt = p.dt, dtG = p.dtG, a = p.a, b = p.b, kappa = p.kappa;
  // lap of Eq. 36: the 5-point Laplacian, or lap_D of Eq. 31 (stencil_fd)
  auto lap_at = [&](const C *f, int k) {
    if (stencil) {
      const C faces = (f[k - RXW] + f[k + RXW]) + (f[k - 1] + f[k + 1]);
      const C corners = (f[k - RXW - 1] + f[k - RXW + 1]) + (f[k + RXW - 1] + f[k + RXW + 1]);
      return p.Q * faces + p.R * corners + p.C0 * f[k];
    }
    C l = f[k - RXW];
    l += f[k - 1];
    l += C(-4) * f[k];
    l += f[k + 1];
    l += f[k + RXW];
    return l;
  };
  C c0[NYI][NXI], c1[NYI][NXI], c2[NYI][NXI], c3[NYI][NXI];
#pragma unroll
  for (int yi = 0; yi < NYI; ++yi)
#pragma unroll
    for (int xi = 0; xi < NXI; ++xi) {
      const int ry = ty + 8 * yi, rx = tx + 32 * xi;
      c0[yi][xi] = c1[yi][xi] = c2[yi][xi] = c3[yi][xi] = C(0);
      if (ry < 1 || ry >= RY - 1 || rx < 1 || rx >= RXW - 1) continue;
      const int k = ry * RXW + rx;
      const C uc = sa[k], uL = sa[k - 1], uR = sa[k + 1];
      const C vc = sq[k], vm = sq[k - RXW], vp = sq[k + RXW];
      if (paper) {
        // phih = c0 phi + |dt u| phi_upx + |dt v| phi_upy (Eqs. 32-35); with
        // stencil_fd the divergence by the stencil derivative of Eq. 30
        C div = (uR - uL) / C(2) + (vp - vm) / C(2);
        if (stencil) {
          const C dux = p.N * (uR - uL) + p.M * ((sa[k - RXW + 1] - sa[k - RXW - 1]) + (sa[k + RXW + 1] - sa[k + RXW - 1]));
          const C dvy = p.N * (vp - vm) + p.M * ((sq[k + RXW + 1] - sq[k - RXW + 1]) + (sq[k + RXW - 1] - sq[k - RXW - 1]));
          div = dux + dvy;
        }
        c0[yi][xi] = C(1) - dt * (div + (fabs(uc) + fabs(vc)));
        c1[yi][xi] = dt * uc;
        c2[yi][xi] = dt * vc;
      } else {
        c0[yi][xi] = C(0.5) * (uc + uR);
        c1[yi][xi] = C(0.5) * (uL + uc);
        c2[yi][xi] = C(0.5) * (vc + vp);
        c3[yi][xi] = C(0.5) * (vm + vc);
      }
    }
  __syncthreads();
  // 3. SUB substeps of Eqs. 32-36
#pragma unroll
  for (int s = 1; s <= SUB; ++s) {
    int lo = 3 * s - 2;
#pragma unroll
    for (int yi = 0; yi < NYI; ++yi)
#pragma unroll
      for (int xi = 0; xi < NXI; ++xi) {
        const int ry = ty + 8 * yi, rx = tx + 32 * xi;
        if (ry < lo || ry >= RY - lo || rx < lo || rx >= RXW - lo) continue;
        const int k = ry * RXW + rx;
        const C pc = sp[k];
        if (paper) {
          const C t1 = c1[yi][xi], t2 = c2[yi][xi];
          const C upx = t1 > C(0) ? sp[k - 1] : sp[k + 1];
          const C upy = t2 > C(0) ? sp[k - RXW] : sp[k + RXW];
          sa[k] = c0[yi][xi] * pc + fabs(t1) * upx + fabs(t2) * upy;
        } else {
          const C Upx = c0[yi][xi], Umx = c1[yi][xi], Upy = c2[yi][xi], Umy = c3[yi][xi];
          const C Jpx = Upx > C(0) ? Upx * pc : Upx * sp[k + 1];
          const C Jmx = Umx > C(0) ? Umx * sp[k - 1] : Umx * pc;
          const C Jpy = Upy > C(0) ? Upy * pc : Upy * sp[k + RXW];
          const C Jmy = Umy > C(0) ? Umy * sp[k - RXW] : Umy * pc;
          C tend = Jpx - Jmx;
          tend += Jpy - Jmy;
          sa[k] = pc - dt * tend;
        }
      }
    __syncthreads();
    lo = 3 * s - 1;  // psi = a phih + b phi^3 - kappa lap phih (Eq. 36)
#pragma unroll
    for (int yi = 0; yi < NYI; ++yi)
#pragma unroll
      for (int xi = 0; xi < NXI; ++xi) {
        const int ry = ty + 8 * yi, rx = tx + 32 * xi;
        if (ry < lo || ry >= RY - lo || rx < lo || rx >= RXW - lo) continue;
        const int k = ry * RXW + rx;
        const C hk = sa[k];
        const C c = cubic_half ? hk : sp[k];
        const C lap = lap_at(sa, k);
        sq[k] = a * hk + b * (c * c * c) - kappa * lap;
      }
    __syncthreads();
    lo = 3 * s;  // phi^{n+1} = phih + dt Gamma lap psi
#pragma unroll
    for (int yi = 0; yi < NYI; ++yi)
#pragma unroll
      for (int xi = 0; xi < NXI; ++xi) {
        const int ry = ty + 8 * yi, rx = tx + 32 * xi;
        if (ry < lo || ry >= RY - lo || rx < lo || rx >= RXW - lo) continue;
        const int k = ry * RXW + rx;
        const C lap = lap_at(sq, k);
        sp[k] = sa[k] + dtG * lap;
      }
    __syncthreads();
  }
  // 4. write the inner TX x TY sites
#pragma unroll
  for (int yi = 0; yi < NYI; ++yi)
#pragma unroll
    for (int xi = 0; xi < NXI; ++xi) {
      const int ry = ty + 8 * yi, rx = tx + 32 * xi;
      if (ry < H || ry >= H + TY || rx < H || rx >= H + TX) continue;
      const int gx = x0 + rx, gy = y0 + ry;
      if (gx < Lx && gy < Ly) phi_out[(long long)gy * Lx + gx] = sp[ry * RXW + rx];
    }
}

// ---- FD convection-diffusion: block kernel, one 128-column region per CTA ----
// FP32 only.  A CTA of NW warps owns a region 128 columns wide and RY =
// K NW rows high, whose inner (128 - 2H) x (RY - 2H) sites are written
// (H = 3 SUB).  Warp w owns the K consecutive rows wK .. wK + K - 1; lane l
// owns the four columns 4l .. 4l + 3 of each, so every shared-memory access
// is one float4 per lane (row pitch 128 floats: a warp reads 512 contiguous
// bytes) and the x neighbours come from the adjacent lanes by shuffles.
// Columns 0 and 127 are never valid, so lanes 0 and 31 need no neighbour
// outside the warp.  A phase walks the warp's rows top to bottom and passes
// the stencil rows r - 1, r, r + 1 on in registers, so each input row is
// read from shared memory once (shared-memory bandwidth bounds the kernel).
// The advection coefficients of Eqs. 32-35 depend only on u*(t): they are
// computed once per launch and kept in registers for all SUB substeps.
// Shared memory: phi, phih and psi planes of RY x 128 floats; each substep
// is three phases over a region that shrinks by one site per phase.  The
// diffusion phases use packed FP32 pairs.
constexpr int FDB_RX = 128;

template <int SUB, int K, int NW>
struct FDBlock {
  static constexpr int H = 3 * SUB, RY = K * NW, TX = FDB_RX - 2 * H, TY = RY - 2 * H;
  // phi, phih, psi planes, and (printed advection form) the c0 plane
  static constexpr size_t smem_of(bool flux) { return sizeof(float) * (flux ? 3 : 4) * (size_t)RY * FDB_RX; }
  static constexpr size_t smem = smem_of(false);
};

__device__ __forceinline__ float4 ld4(const float *a, int r, int c) {
  return *reinterpret_cast<const float4 *>(a + r * FDB_RX + c);
}
__device__ __forceinline__ void st4(float *a, int r, int c, float4 v) {
  *reinterpret_cast<float4 *>(a + r * FDB_RX + c) = v;
}
__device__ __forceinline__ float comp(const float4 &v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 mk4(const float (&e)[4]) { return make_float4(e[0], e[1], e[2], e[3]); }

template <bool FLUX, int SUB, int K, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    fd2d_block_kernel(const float *__restrict__ phi_in, const float *__restrict__ u,
                      float *__restrict__ phi_out, KParams<float> p) {
  using G = FDBlock<SUB, K, NW>;
  constexpr int H = G::H, RY = G::RY, TX = G::TX, TY = G::TY, NC = FLUX ? 4 : 2;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) float fdb_smem[];
  float *sp = fdb_smem, *sa = sp + RY * FDB_RX, *sq = sa + RY * FDB_RX, *st0 = sq + RY * FDB_RX;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, c = 4 * lane;
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int x0 = blockIdx.x * TX - H, y0 = blockIdx.y * TY - H;
  int gx[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) gx[j] = wrapi(x0 + c + j, Lx);
  // a lane's four columns are one aligned float4 of the lattice when the
  // region origin and Lx are multiples of 4 (then they never straddle the wrap)
  const bool vec = H % 4 == 0 && (Lx & 3) == 0;
  // 1. phi -> sp, v -> sq (only until the coefficients are in registers);
  //    u stays in registers in the printed form (a thread needs only its own
  //    rows of it), the flux form (more coefficients) stores it to sa
  // (all rows are loaded into registers before any is stored, so that the
  // loads are in flight together)
  long long rowo[K];
#pragma unroll
  for (int k = 0; k < K; ++k) rowo[k] = (long long)wrapi(y0 + warp * K + k, Ly) * Lx;
  auto ldrow = [&](const float *f, int k) {
    if (vec) return __ldg(reinterpret_cast<const float4 *>(f + rowo[k] + gx[0]));
    float e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) e[j] = __ldg(f + rowo[k] + gx[j]);
    return mk4(e);
  };
  float4 rp[K], ru[K], rv[K];
  pdl_wait();  // u*(t) comes from the previous kernel
  pdl_trigger();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    rp[k] = ldrow(phi_in, k);
    ru[k] = ldrow(u, k);
    rv[k] = ldrow(u + Sz, k);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int r = warp * K + k;
    st4(sp, r, c, rp[k]);
    if constexpr (FLUX) st4(sa, r, c, ru[k]);
    st4(sq, r, c, rv[k]);
  }
  __syncthreads();
  // 2. advection coefficients (printed form: c0, dt u, dt v; flux form: the
  //    four face velocities) of this thread's sites
  const float dt = p.dt, dtG = p.dtG, a = p.a, b = p.b, kappa = p.kappa;
  const bool cubic_half = p.cubic_at_half != 0;
  float T[K][NC][4];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int r = warp * K + k;
    const int rm = r > 0 ? r - 1 : r, rp = r < RY - 1 ? r + 1 : r;  // row 0 / RY-1: never valid
    const float4 uc = FLUX ? ld4(sa, r, c) : ru[k], vc = ld4(sq, r, c), vm = ld4(sq, rm, c), vp = ld4(sq, rp, c);
    const float uL0 = __shfl_up_sync(FULL, uc.w, 1), uR3 = __shfl_down_sync(FULL, uc.x, 1);
    float c0[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float ucj = comp(uc, j), uL = j == 0 ? uL0 : comp(uc, j - 1), uR = j == 3 ? uR3 : comp(uc, j + 1);
      const float vcj = comp(vc, j), vmj = comp(vm, j), vpj = comp(vp, j);
      if constexpr (!FLUX) {
        const float div = (uR - uL) / 2.f + (vpj - vmj) / 2.f;
        c0[j] = 1.f - dt * (div + (fabsf(ucj) + fabsf(vcj)));  // kept in shared memory
        T[k][0][j] = dt * ucj;
        T[k][1][j] = dt * vcj;
      } else {
        T[k][0][j] = 0.5f * (ucj + uR);
        T[k][1][j] = 0.5f * (uL + ucj);
        T[k][2][j] = 0.5f * (vcj + vpj);
        T[k][3][j] = 0.5f * (vmj + vcj);
      }
    }
    if constexpr (!FLUX) st4(st0, r, c, mk4(c0));
  }
  // printed form: no barrier here (the first advection sweep reads the phi
  // plane stored before the last one and this thread's own c0, and writes
  // sa, which no thread reads until the barrier after it; sq, read above, is
  // first overwritten after that barrier too); the flux form read sa above
  if constexpr (FLUX) __syncthreads();
  // 3. SUB substeps of Eqs. 32-36.  sweep(in, lo, fn) runs one stencil phase
  //    over this warp's K consecutive rows r (lo <= r < RY - lo, a
  //    warp-uniform test): fn(k, r, row r - 1, row r, row r + 1 of plane
  //    `in`), each row of `in` loaded once and passed on in registers
  auto sweep = [&](const float *in, int lo, auto &&fn) {
    const int rb = warp * K;
    float4 up = ld4(in, rb > 0 ? rb - 1 : 0, c), cen = ld4(in, rb, c);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int r = rb + k;
      const float4 dn = ld4(in, r < RY - 1 ? r + 1 : r, c);
      if (r >= lo && r < RY - lo) fn(k, r, up, cen, dn);
      up = cen;
      cen = dn;
    }
  };
  // phi^n and phi^{n+1} alternate between two planes (the psi of Eq. 36
  // never reaches shared memory)
  float *pin = sp, *pout = sq;
  auto clampr = [](int r) { return r < 0 ? 0 : (r > RY - 1 ? RY - 1 : r); };
#pragma unroll
  for (int s = 0; s < SUB; ++s) {
    // phih = advected phi (Eqs. 32-35)
    sweep(pin, 3 * s + 1, [&](int k, int r, const float4 &pu, const float4 &pc, const float4 &pd) {
      float4 t0v = make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (!FLUX) t0v = ld4(st0, r, c);
      const float l0 = __shfl_up_sync(FULL, pc.w, 1), r3 = __shfl_down_sync(FULL, pc.x, 1);
      float e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float pcj = comp(pc, j), pl = j == 0 ? l0 : comp(pc, j - 1), pr = j == 3 ? r3 : comp(pc, j + 1);
        if constexpr (!FLUX) {
          const float t1 = T[k][0][j], t2 = T[k][1][j];
          const float upx = t1 > 0.f ? pl : pr;  // u = 0 contributes nothing
          const float upy = t2 > 0.f ? comp(pu, j) : comp(pd, j);
          e[j] = comp(t0v, j) * pcj + fabsf(t1) * upx + fabsf(t2) * upy;
        } else {
          const float t0 = T[k][0][j], t1 = T[k][1][j], t2 = T[k][2][j], t3 = T[k][3][j];
          const float Jpx = t0 > 0.f ? t0 * pcj : t0 * pr;
          const float Jmx = t1 > 0.f ? t1 * pl : t1 * pcj;
          const float Jpy = t2 > 0.f ? t2 * pcj : t2 * comp(pd, j);
          const float Jmy = t3 > 0.f ? t3 * comp(pu, j) : t3 * pcj;
          float tend = Jpx - Jmx;
          tend += Jpy - Jmy;
          e[j] = pcj - dt * tend;
        }
      }
      st4(sa, r, c, mk4(e));
    });
    __syncthreads();
    // psi = a phih + b phi^3 - kappa lap phih and phi^{n+1} = phih + dt Gamma
    // lap psi (Eq. 36), fused: the warp computes psi on its rows and one row
    // either side, keeps the last three psi rows in registers and writes
    // phi^{n+1} of row r as soon as psi of row r + 1 is known
    const bool last = s == SUB - 1;
    const int lo3 = 3 * s + 3, rb = warp * K;
    if (rb + K > lo3 && rb < RY - lo3) {  // warp-uniform: some row of this warp is valid
      float4 hu = ld4(sa, clampr(rb - 2), c), hc = ld4(sa, clampr(rb - 1), c);
      float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
#pragma unroll
      for (int j = 0; j < K + 2; ++j) {
        const int rr = rb - 1 + j;  // psi row computed now
        const float4 hd = ld4(sa, clampr(rr + 1), c), pc = ld4(pin, clampr(rr), c);
        float4 q2;
        {
          const float l0 = __shfl_up_sync(FULL, hc.w, 1), r3 = __shfl_down_sync(FULL, hc.x, 1);
          // packed pairs (sites 0,1) and (2,3): vertical and centre terms as
          // pairs, the horizontal neighbour sums (which straddle pairs) scalar
          float2 o[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float2 hk = q ? f2(hc.z, hc.w) : f2(hc.x, hc.y);
            const float2 vs = add2(q ? f2(hu.z, hu.w) : f2(hu.x, hu.y), q ? f2(hd.z, hd.w) : f2(hd.x, hd.y));
            const float2 hs = q ? f2(hc.y + hc.w, hc.z + r3) : f2(l0 + hc.y, hc.x + hc.z);
            const float2 lap = fma2(f2(-4.f, -4.f), hk, add2(vs, hs));
            const float2 cb = cubic_half ? hk : (q ? f2(pc.z, pc.w) : f2(pc.x, pc.y));
            o[q] = fma2(f2(a, a), hk, fma2(f2(b, b), mul2(mul2(cb, cb), cb), mul2(f2(-kappa, -kappa), lap)));
          }
          q2 = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        }
        const int r = rr - 1;  // phi^{n+1} row: psi rows r - 1, r, r + 1 = q0, q1, q2; phih row r = hu
        if (j >= 2 && r >= lo3 && r < RY - lo3) {
          const float l0 = __shfl_up_sync(FULL, q1.w, 1), r3 = __shfl_down_sync(FULL, q1.x, 1);
          float e[4];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float2 qk = q ? f2(q1.z, q1.w) : f2(q1.x, q1.y);
            const float2 vs = add2(q ? f2(q0.z, q0.w) : f2(q0.x, q0.y), q ? f2(q2.z, q2.w) : f2(q2.x, q2.y));
            const float2 hs = q ? f2(q1.y + q1.w, q1.z + r3) : f2(l0 + q1.y, q1.x + q1.z);
            const float2 lap = fma2(f2(-4.f, -4.f), qk, add2(vs, hs));
            const float2 o = fma2(f2(dtG, dtG), lap, q ? f2(hu.z, hu.w) : f2(hu.x, hu.y));
            e[2 * q] = o.x;
            e[2 * q + 1] = o.y;
          }
          if (!last) {
            st4(pout, r, c, mk4(e));
          } else if (r >= H && r < H + TY && y0 + r < Ly) {
            const long long row = (long long)(y0 + r) * Lx;
            if (vec) {  // the group is wholly inside or outside the written range
              if (c >= H && c < H + TX && x0 + c < Lx)
                *reinterpret_cast<float4 *>(phi_out + row + x0 + c) = mk4(e);
            } else {
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                const int cc = c + jj, xg = x0 + cc;
                if (cc >= H && cc < H + TX && xg < Lx) phi_out[row + xg] = e[jj];
              }
            }
          }
        }
        q0 = q1;
        q1 = q2;
        hu = hc;
        hc = hd;
      }
    }
    if (!last) {
      __syncthreads();
      float *t = pin;
      pin = pout;
      pout = t;
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

template <typename S, typename C, int RY>
cudaError_t collide2d_ry(lbm_handle *h, int in, int force_on, int mode) {
  constexpr int C2_TY = C2_BY * RY;
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
      collide2d_kernel<S, C, true, COLLIDE_STEP, RY>
          <<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
    else
      collide2d_kernel<S, C, false, COLLIDE_STEP, RY>
          <<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
  } else {
    if (tgen)
      collide2d_kernel<S, C, true, COLLIDE_MOMENTS, RY>
          <<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
    else
      collide2d_kernel<S, C, false, COLLIDE_MOMENTS, RY>
          <<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
  }
  return cudaGetLastError();
}

// MINB: CTAs per SM the register budget is sized for (4: no headroom, 3: none
// of the FP32 variants spill)
template <typename C, int MINB>
cudaError_t collide2d_async(lbm_handle *h, int in, int force_on, int mode) {
  KParams<C> p = make_params<C>(h, force_on);
  dim3 grid((p.Lx + CA_TX - 1) / CA_TX, (p.Ly + CA_TY - 1) / CA_TY), block(32, C2_BY);
  const C *hin = static_cast<const C *>(h->h[in]);
  C *hout = static_cast<C *>(h->h[1 - in]);
  const C *phi = static_cast<const C *>(h->phi[in]);
  const C *dn = static_cast<const C *>(h->dn);
  C *u = static_cast<C *>(h->u);
  const size_t smem = collide_async_smem<C>();
  const bool tgen = p.cs2mT != C(0);
  if (mode == COLLIDE_STEP) {
    if (tgen)
      return launch_pdl(collide2d_async_kernel<C, true, COLLIDE_STEP, MINB>, grid, block, smem,
                        h->stream, hin, hout, phi, dn, u, h->staging, p);
    return launch_pdl(collide2d_async_kernel<C, false, COLLIDE_STEP, MINB>, grid, block, smem,
                      h->stream, hin, hout, phi, dn, u, h->staging, p);
  } else {
    if (tgen)
      collide2d_async_kernel<C, true, COLLIDE_MOMENTS, MINB>
          <<<grid, block, smem, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
    else
      collide2d_async_kernel<C, false, COLLIDE_MOMENTS, MINB>
          <<<grid, block, smem, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
  }
  return cudaGetLastError();
}

template <typename C, int MINB>
cudaError_t collide2d_async_configure_one() {
  const int smem = (int)collide_async_smem<C>();
  cudaError_t e = cudaSuccess;
  for (auto fn : {collide2d_async_kernel<C, true, COLLIDE_STEP, MINB>,
                  collide2d_async_kernel<C, false, COLLIDE_STEP, MINB>,
                  collide2d_async_kernel<C, true, COLLIDE_MOMENTS, MINB>,
                  collide2d_async_kernel<C, false, COLLIDE_MOMENTS, MINB>})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

template <typename C>
cudaError_t collide2d_async_configure() {
  cudaError_t e = collide2d_async_configure_one<C, 2>();
  if (e == cudaSuccess) e = collide2d_async_configure_one<C, 3>();
  if (e == cudaSuccess && sizeof(C) == 4) e = collide2d_async_configure_one<C, 4>();
  return e;
}

template <typename S, typename C>
cudaError_t collide2d(lbm_handle *h, int in, int force_on, int mode) {
  if constexpr (sizeof(C) == 4) {
    // 3, 5, 6, 7: TMA staging (scalar, packed-pair 4 CTAs/SM, packed-pair 3
    // CTAs/SM, persistent pipelined; FP32 and FP16 storage, 7 FP32 only)
    if (h->collide_rows == 3 || (h->collide_rows >= 5 && h->collide_rows <= 7))
      return collide2d_tma(h, in, force_on, mode, h->collide_rows);
  }
  if constexpr (std::is_same<S, C>::value) {
    // 0: asynchronous staging sized for 4 CTAs per SM (FP64: 2), 1: for 3
    if (h->collide_rows == 0)
      return sizeof(C) == 4 ? collide2d_async<C, 4>(h, in, force_on, mode)
                            : collide2d_async<C, 2>(h, in, force_on, mode);
    if (h->collide_rows == 1) return collide2d_async<C, 3>(h, in, force_on, mode);
  }
  return h->collide_rows == 4 ? collide2d_ry<S, C, 4>(h, in, force_on, mode)
                              : collide2d_ry<S, C, 2>(h, in, force_on, mode);
}

template <typename C, int V, int SUB>
cudaError_t fd2d_launch_one(lbm_handle *h, const KParams<C> &p, const C *src, C *dst, int TY) {
  constexpr int H = 3 * SUB, HX = (H + V - 1) / V * V, OW = 32 * V - 2 * HX;
  const int nstrips = (p.Lx + OW - 1) / OW, ntiles = (p.Ly + TY - 1) / TY;
  const int warps = nstrips * ntiles;
  fd2d_march_kernel<C, V, SUB><<<(warps + 1) / 2, 64, 0, h->stream>>>(
      src, static_cast<const C *>(h->u), dst, p, TY, nstrips, ntiles);
  return cudaGetLastError();
}

template <typename C, int RXW, int SUB>
cudaError_t fd2d_tile_one(lbm_handle *h, const KParams<C> &p, const C *src, C *dst) {
  using G = FDTile<C, RXW, SUB>;
  dim3 grid((p.Lx + G::TX - 1) / G::TX, (p.Ly + G::TY - 1) / G::TY), block(32, 8);
  fd2d_tile_kernel<C, RXW, SUB><<<grid, block, G::smem, h->stream>>>(
      src, static_cast<const C *>(h->u), dst, p);
  return cudaGetLastError();
}

template <bool FLUX, int SUB, int K, int NW>
cudaError_t fd2d_block_one(lbm_handle *h, const KParams<float> &p, const float *src, float *dst) {
  using G = FDBlock<SUB, K, NW>;
  dim3 grid((p.Lx + G::TX - 1) / G::TX, (p.Ly + G::TY - 1) / G::TY);
  return launch_pdl(fd2d_block_kernel<FLUX, SUB, K, NW>, grid, dim3(NW * 32), G::smem_of(FLUX), h->stream,
                    src, static_cast<const float *>(h->u), dst, p);
}

// block kernel shapes (substeps per launch, region rows RY, warps); the
// tuning fields carry them as sub, rows = RY, cols = warps / 8
#define FDB_SHAPES(X) X(1, 64, 16) X(2, 64, 16) X(2, 80, 16) X(4, 80, 16) X(4, 96, 16) X(4, 96, 32) X(2, 96, 32)

template <typename C>
cudaError_t fd2d_block(lbm_handle *h, const KParams<C> &p, const C *src, C *dst, int sub) {
  if constexpr (std::is_same<C, float>::value) {
    const bool flux = p.adv_variant == LBM_ADV_FLUX;
#define FDB_CASE(SB, RYY, NWW)                                                      \
  if (sub == SB && h->fd_rows == RYY && h->fd_cols * 8 == NWW)                     \
    return flux ? fd2d_block_one<true, SB, RYY / NWW, NWW>(h, p, src, dst)         \
                : fd2d_block_one<false, SB, RYY / NWW, NWW>(h, p, src, dst);
    FDB_SHAPES(FDB_CASE)
#undef FDB_CASE
    // a remainder launch with fewer substeps than the shape
    if (sub == 1) return flux ? fd2d_block_one<true, 1, 4, 16>(h, p, src, dst) : fd2d_block_one<false, 1, 4, 16>(h, p, src, dst);
    if (sub == 2) return flux ? fd2d_block_one<true, 2, 4, 16>(h, p, src, dst) : fd2d_block_one<false, 2, 4, 16>(h, p, src, dst);
    if (sub == 3) return flux ? fd2d_block_one<true, 3, 4, 16>(h, p, src, dst) : fd2d_block_one<false, 3, 4, 16>(h, p, src, dst);
    return flux ? fd2d_block_one<true, 4, 5, 16>(h, p, src, dst) : fd2d_block_one<false, 4, 5, 16>(h, p, src, dst);
  }
  return cudaErrorInvalidValue;
}

template <typename C>
cudaError_t fd2d_tile(lbm_handle *h, const KParams<C> &p, const C *src, C *dst, int sub) {
  if (h->fd_tile_w == 32) return fd2d_tile_one<C, 32, 1>(h, p, src, dst);  // one substep
  return sub >= 2 ? fd2d_tile_one<C, 64, 2>(h, p, src, dst) : fd2d_tile_one<C, 64, 1>(h, p, src, dst);
}

cudaError_t fd2d_block_configure() {
  cudaError_t e = cudaSuccess;
#define FDB_CFG(SB, RYY, NWW)                                                                   \
  if (e == cudaSuccess)                                                                         \
    e = cudaFuncSetAttribute(fd2d_block_kernel<false, SB, RYY / NWW, NWW>,                      \
                             cudaFuncAttributeMaxDynamicSharedMemorySize,                        \
                             (int)FDBlock<SB, RYY / NWW, NWW>::smem_of(false));                  \
  if (e == cudaSuccess)                                                                         \
    e = cudaFuncSetAttribute(fd2d_block_kernel<true, SB, RYY / NWW, NWW>,                       \
                             cudaFuncAttributeMaxDynamicSharedMemorySize,                        \
                             (int)FDBlock<SB, RYY / NWW, NWW>::smem_of(true));
  FDB_SHAPES(FDB_CFG)
  FDB_CFG(3, 64, 16)  // the remainder launch of m = 3 (mod 4)
#undef FDB_CFG
  return e;
}

template <typename C>
cudaError_t fd2d_tile_configure() {
  cudaError_t e = cudaFuncSetAttribute(fd2d_tile_kernel<C, 32, 1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)FDTile<C, 32, 1>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd2d_tile_kernel<C, 64, 1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FDTile<C, 64, 1>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd2d_tile_kernel<C, 64, 2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FDTile<C, 64, 2>::smem);
  return e;
}

template <typename C, int V>
cudaError_t fd2d_sub(lbm_handle *h, const KParams<C> &p, const C *src, C *dst, int sub, int TY) {
  if constexpr (std::is_same<C, float>::value) {
    // wavefront kernel: 2 or 4 substeps; an odd remainder goes to the block kernel
    if (h->fd_tile_w == 1) {
      if (sub == 2 || sub == 4) return fd2d_wave(h, p, src, dst, sub, h->fd_rows);
      return fd2d_block<C>(h, p, src, dst, sub);
    }
  }
  if (h->fd_tile_w == 128) return fd2d_block<C>(h, p, src, dst, sub);
  if (h->fd_tile_w > 0) return fd2d_tile<C>(h, p, src, dst, sub);
  switch (sub) {
    case 1: return fd2d_launch_one<C, V, 1>(h, p, src, dst, TY);
    case 2: return fd2d_launch_one<C, V, 2>(h, p, src, dst, TY);
    case 3: return fd2d_launch_one<C, V, 3>(h, p, src, dst, TY);
    default: return fd2d_launch_one<C, V, 4>(h, p, src, dst, TY);
  }
}

// m substeps as ceil(m / sub) launches; the last launch takes the remainder.
template <typename C, int V>
cudaError_t fd2d(lbm_handle *h, int in) {
  KParams<C> p = make_params<C>(h, 0);
  const int launches = (h->m + h->sub - 1) / h->sub;
  const C *src = static_cast<const C *>(h->phi[in]);
  for (int j = 0; j < launches; ++j) {
    const int sub = (j == launches - 1) ? h->m - h->sub * (launches - 1) : h->sub;
    C *dst = static_cast<C *>(((launches - 1 - j) % 2 == 0) ? h->phi[1 - in] : h->phi[2]);
    cudaError_t e = fd2d_sub<C, V>(h, p, src, dst, sub, h->fd_rows);
    if (e != cudaSuccess) return e;
    src = dst;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t collide2d_launch(lbm_handle *h, int in, int force_on, int mode) {
  switch (h->P.precision) {
    case LBM_F64: return collide2d<double, double>(h, in, force_on, mode);
    case LBM_F32DEV: return collide2d<float, float>(h, in, force_on, mode);
    default: return collide2d<__half, float>(h, in, force_on, mode);
  }
}

cudaError_t collide2d_configure(int precision) {
  cudaError_t e = precision == LBM_F64 ? fd2d_tile_configure<double>() : fd2d_tile_configure<float>();
  if (e == cudaSuccess && precision != LBM_F64) e = fd2d_block_configure();
  if (e == cudaSuccess && precision != LBM_F64) e = fd2d_wave_configure();
  if (e != cudaSuccess) return e;
  if (precision == LBM_F64) return collide2d_async_configure<double>();
  if (precision == LBM_F32DEV) {
    e = collide2d_async_configure<float>();
    return e == cudaSuccess ? collide2d_tma_configure(precision) : e;
  }
  return collide2d_tma_configure(precision);  // FP16 deviations
}

cudaError_t fd2d_launch(lbm_handle *h, int in) {
  if (h->P.precision == LBM_F64) return fd2d<double, 2>(h, in);
  return h->fd_cols == 2 ? fd2d<float, 2>(h, in) : fd2d<float, 4>(h, in);
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

cudaError_t collide2d_batch(const float *hin, float *hout, const float *phi, float *u, long long ST,
                            const TiledInst *inst, const int4 *items, int nitems, const KParams<float> &p,
                            long long t, cudaStream_t s) {
  collide2d_batch_kernel<<<nitems, dim3(32, C2_BY), 0, s>>>(hin, hout, phi, u, ST, inst, items, p, t);
  return cudaGetLastError();
}

}  // namespace hlbm
