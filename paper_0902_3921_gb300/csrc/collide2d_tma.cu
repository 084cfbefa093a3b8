// collide2d_tma.cu -- D2Q9 collide-and-stream with its inputs staged in shared
// memory by the tensor memory accelerator (FP32 deviation storage).
//
// The arithmetic is that of the shared-memory collide kernels of
// kernels_2d.cu: mu = a phi + b phi^3 - kappa lap_D phi (Eqs. 5, 31) on the
// tile + 1, F = -phi d_D mu (Eqs. 28, 30) plus n g (and grad((c_s^2 - T) n)
// when T != 1/3), n and u* (Eqs. 12, 18), BGK with the forcing term (Eqs. 15,
// 17, 29).  What differs is how a 32 x 32 tile's inputs reach shared memory:
// thread 0 issues ten tiled TMA copies that complete on one mbarrier,
//   plane i with e_x =  0: columns x0 .. x0 + 31      (x sits at column tx)
//   plane i with e_x = +1: columns x0 - 4 .. x0 + 31  (x - 1 sits at column tx + 3)
//   plane i with e_x = -1: columns x0 .. x0 + 35      (x + 1 sits at column tx + 1)
//   (rows y0 - e_y .. y0 - e_y + 31: the pull f_i(r, t) = buf_i(r - e_i))
//   phi: columns x0 - 4 .. x0 + 35, rows y0 - 2 .. y0 + 33 (halo 2 for mu and d_D mu)
// A copy's x origin must be a multiple of 16 bytes, hence the 36- and
// 40-column boxes.  The copies do not wrap around the periodic lattice:
// cells outside it arrive as zeros, and the CTAs on the lattice's edges
// reload the cells they use from the periodic images before computing.
//
// PACK evaluates the collision of a thread's two rows at a time with packed
// FP32 pair instructions (add/mul/fma .f32x2); MINB is the number of CTAs
// per SM the registers are budgeted for.  Variants (the collide_rows value of
// the handle's launch shapes): 3 scalar (3 CTAs/SM), 5 packed (4), 6 packed (3),
// 7 persistent and pipelined (below; packed, 4 CTAs/SM).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "lbm_common.cuh"

namespace hlbm {

namespace {

constexpr int TT = 32;                // tile side in sites
constexpr int TR = 4;                 // rows per thread (32 x 8 threads)
constexpr int PHW = 40, PHH = 36;     // phi box
constexpr int MUW = TT + 2;           // mu on the tile + 1
constexpr int TMA_MIN_SIDE = 64;

// number of planes j < i pulled along x (e_x != 0): 0 0 1 1 2 2 3 4 5 6
__host__ __device__ constexpr int nshift(int i) { return i <= 5 ? i / 2 : i - 3; }
__host__ __device__ constexpr int plane_w(int i) { return q9_ex(i) == 0 ? TT : TT + 4; }
__host__ __device__ constexpr int plane_off(int i) { return TT * (TT * i + 4 * nshift(i)); }
__host__ __device__ constexpr int col_off(int i) { return q9_ex(i) > 0 ? 3 : (q9_ex(i) < 0 ? 1 : 0); }
__host__ __device__ constexpr int box_dx(int i) { return q9_ex(i) > 0 ? -4 : 0; }

constexpr int POP_FLOATS = plane_off(9);

// Population planes of a 32 x 32 tile for storage type S (FP32 or FP16
// deviations): a copy's x origin must be a multiple of A = 16 / sizeof(S)
// elements, so planes pulled from x - 1 start A columns left of the tile and
// planes pulled from x +- 1 are TT + A wide.  (FP32: the functions above.)
template <typename S>
struct TmaGeo {
  static constexpr int A = 16 / (int)sizeof(S);
  __host__ __device__ static constexpr int w(int i) { return q9_ex(i) == 0 ? TT : TT + A; }
  __host__ __device__ static constexpr int off(int i) { return TT * (TT * i + A * nshift(i)); }  // elements
  __host__ __device__ static constexpr int col(int i) { return q9_ex(i) > 0 ? A - 1 : (q9_ex(i) < 0 ? 1 : 0); }
  __host__ __device__ static constexpr int dx(int i) { return q9_ex(i) > 0 ? -A : 0; }
  static constexpr int POP_BYTES = (int)sizeof(S) * off(9);
  static constexpr int OFF_POP = 128;  // bytes [0, 128): the mbarrier
  static constexpr int OFF_PHI = OFF_POP + POP_BYTES;
  static constexpr int OFF_MU = OFF_PHI + 4 * PHW * PHH;
  static constexpr int OFF_PN = OFF_MU + 4 * MUW * MUW;
  static constexpr uint32_t TX_BYTES = (uint32_t)(POP_BYTES + 4 * PHW * PHH);
  static_assert(OFF_PHI % 128 == 0 && ((int)sizeof(S) * off(1)) % 128 == 0 &&
                    ((int)sizeof(S) * off(2)) % 128 == 0,
                "TMA destinations must be 128-byte aligned");
};
static_assert(TmaGeo<float>::off(9) == POP_FLOATS && TmaGeo<float>::col(1) == col_off(1) &&
                  TmaGeo<float>::dx(1) == box_dx(1),
              "FP32 geometry");

// + 128: room to align the dynamic shared-memory base to 128 bytes
template <typename S, bool TGEN>
constexpr size_t tma_smem() {
  return 128 + TmaGeo<S>::OFF_PN + (TGEN ? 4 * MUW * MUW : 0);
}

// storage <-> compute conversions (FP16 deviations carry the scale 2^s)
__device__ __forceinline__ float cvt_ld(float v, float) { return v; }
__device__ __forceinline__ float cvt_ld(__half v, float inv_scale) { return __half2float(v) * inv_scale; }
__device__ __forceinline__ void cvt_st(float *d, float v, float) { *d = v; }
__device__ __forceinline__ void cvt_st(__half *d, float v, float scale) { *d = __float2half_rn(v * scale); }

__device__ int g_collide_tma_err = 0;
// bound of the waits for a tile's copies (the drain waits of the give-up path
// keep 0.5 s); the host shortens it only to exercise the give-up path
__device__ unsigned long long g_collide_tma_wait_ns = 500000000ull;

__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                       uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float2 s2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, s2(-1.f), a); }

// mu at the centre of a 3 x 3 window of phi (explicitly rounded: the same
// site's mu is evaluated by the interior and the frame code)
__device__ __forceinline__ float mu_at(const KParams<float> &p, const float (&w)[3][3]) {
  float lap = rn_mul(p.R, w[0][0]);
  lap = rn_fma(p.Q, w[0][1], lap);
  lap = rn_fma(p.R, w[0][2], lap);
  lap = rn_fma(p.Q, w[1][0], lap);
  lap = rn_fma(p.C0, w[1][1], lap);
  lap = rn_fma(p.Q, w[1][2], lap);
  lap = rn_fma(p.R, w[2][0], lap);
  lap = rn_fma(p.Q, w[2][1], lap);
  lap = rn_fma(p.R, w[2][2], lap);
  const float c = w[1][1];
  const float c3 = rn_mul(rn_mul(c, c), c);
  return rn_fma(p.a, c, rn_fma(p.b, c3, rn_mul(-p.kappa, lap)));
}

template <typename S, bool TGEN, int MODE, bool PACK, int MINB>
__global__ void __launch_bounds__(256, MINB)
    collide2d_tma_kernel(const __grid_constant__ CUtensorMap map_p32,
                         const __grid_constant__ CUtensorMap map_p36,
                         const __grid_constant__ CUtensorMap map_phi, const S *__restrict__ hin,
                         S *__restrict__ hout, const float *__restrict__ phi,
                         const float *__restrict__ dn, float *__restrict__ uout,
                         double *__restrict__ stg, KParams<float> p) {
  using G = TmaGeo<S>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *base = smem_raw + ((128u - (su32(smem_raw) & 127u)) & 127u);
  const uint32_t bar = su32(base);
  S *pops = reinterpret_cast<S *>(base + G::OFF_POP);
  float(*sphi)[PHW] = reinterpret_cast<float(*)[PHW]>(base + G::OFF_PHI);
  float(*smu)[MUW] = reinterpret_cast<float(*)[MUW]>(base + G::OFF_MU);
  float(*spn)[MUW] = reinterpret_cast<float(*)[MUW]>(base + G::OFF_PN);
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int x0 = blockIdx.x * TT, y0 = blockIdx.y * TT;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int ly0 = TR * ty, x = x0 + tx;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();  // phi(t) and the populations come from the previous kernels
  pdl_trigger();
  // 1. the ten copies (one thread), the T != 1/3 pressure by plain loads meanwhile
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(G::TX_BYTES)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 9; ++i)
      tma_3d(su32(pops + G::off(i)), G::w(i) == TT ? &map_p32 : &map_p36, x0 + G::dx(i),
             y0 - q9_ey(i), i, bar);
    tma_2d(su32(&sphi[0][0]), &map_phi, x0 - 4, y0 - 2, bar);
  }
  if constexpr (TGEN) {
    for (int k = tid; k < MUW * MUW; k += 256) {
      const int ry = k / MUW, rx = k - ry * MUW;
      const int gx = wrapi(x0 + rx - 1, Lx), gy = wrapi(y0 + ry - 1, Ly);
      spn[ry][rx] = p.cs2mT * (1.f + dn[(long long)gy * Lx + gx]);
    }
  }
  // 2. periodic images of the cells the copies left as zeros (edge CTAs only;
  //    Lx, Ly >= 64, so one conditional wrap suffices).  phi: only the cells
  //    of the 36 x 36 box beyond the lattice are visited (the column strips,
  //    then the row strips between them); populations: the pulls from outside
  //    the lattice start at the first or last column or row.  The first
  //    round of loads (one phi cell and two population candidates a thread)
  //    is issued before the wait for the copies, so that it overlaps them.
  const int rxr = Lx - x0 + 2, ryb = Ly - y0 + 2;  // first box column / row beyond the lattice
  const int wl = x0 == 0 ? 2 : 0, wr = max(0, TT + 4 - rxr), ht = y0 == 0 ? 2 : 0, hb = max(0, TT + 4 - ryb);
  const bool edge = wl + wr + ht + hb > 0;
  const int ncol = (TT + 4) * (wl + wr), wc = TT + 4 - wl - wr, ntot = ncol + (ht + hb) * wc;
  // phi cell q of the box: its place in sphi (row-major, PHW floats a row) and its value
  auto phi_cell = [&](int q, float &v) {
    int rx, ry;
    if (q < ncol) {
      const int c = q / (TT + 4);
      ry = q - c * (TT + 4);
      rx = c < wl ? c : rxr + (c - wl);
    } else {
      const int q2 = q - ncol, r = q2 / wc;
      rx = wl + (q2 - r * wc);
      ry = r < ht ? r : ryb + (r - ht);
    }
    v = phi[(long long)wrap1(y0 - 2 + ry, Ly) * Lx + wrap1(x0 - 2 + rx, Lx)];
    return ry * PHW + rx + 2;
  };
  float pv0 = 0.f;
  int pd0 = -1;
  S hv2[2];
  int hd2[2] = {-1, -1};
  if (edge) {
    if (tid < ntot) pd0 = phi_cell(tid, pv0);
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      const int k = tid + 256 * sl;
      if (k >= 8 * 2 * TT) continue;
      const int i = 1 + k / (2 * TT), j = k % (2 * TT);
      const int ex = q9_ex(i), ey = q9_ey(i);
      int xs, ys;
      if (j < TT) {
        if (ex == 0) continue;
        xs = ex > 0 ? 0 : Lx - 1;
        ys = y0 + j;
      } else {
        if (ey == 0) continue;
        ys = ey > 0 ? 0 : Ly - 1;
        xs = x0 + j - TT;
      }
      if (xs < x0 || xs >= x0 + TT || xs >= Lx || ys < y0 || ys >= y0 + TT || ys >= Ly) continue;
      const int sx = wrap1(xs - ex, Lx), sy = wrap1(ys - ey, Ly);
      hd2[sl] = G::off(i) + (ys - y0) * G::w(i) + (xs - x0) + G::col(i);
      hv2[sl] = hin[i * Sz + (long long)sy * Lx + sx];
    }
  }
  const bool arrived = bar_wait(bar, 0, g_collide_tma_wait_ns);
  if (!__syncthreads_and(arrived)) {
    // the copies did not complete within the wait bound: report, let them land
    // (that drain keeps the 0.5 s bound), leave
    if (tid == 0) {
      atomicExch(&g_collide_tma_err, 1);
      bar_wait(bar, 0, 500000000ull);
    }
    return;
  }
  if (edge) {
    float *sphi_flat = &sphi[0][0];
    if (pd0 >= 0) sphi_flat[pd0] = pv0;
#pragma unroll
    for (int sl = 0; sl < 2; ++sl)
      if (hd2[sl] >= 0) pops[hd2[sl]] = hv2[sl];
    for (int q = 256 + tid; q < ntot; q += 256) {  // ragged tiles: the rest of the phi cells
      float v;
      const int d = phi_cell(q, v);
      sphi_flat[d] = v;
    }
  }
  __syncthreads();
  // 3. mu on the tile + 1: the interior four rows per thread with rows reused
  //    from registers, then the one-site frame
  {
    float w[3][3];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) w[k + 1][j] = sphi[ly0 + 1 + k][tx + 3 + j];
#pragma unroll
    for (int r = 0; r < TR; ++r) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        w[0][j] = w[1][j];
        w[1][j] = w[2][j];
        w[2][j] = sphi[ly0 + 3 + r][tx + 3 + j];
      }
      smu[ly0 + 1 + r][tx + 1] = mu_at(p, w);
    }
    for (int k = tid; k < 2 * MUW + 2 * (MUW - 2); k += 256) {
      int my, mx;
      if (k < MUW) {
        my = 0;
        mx = k;
      } else if (k < 2 * MUW) {
        my = MUW - 1;
        mx = k - MUW;
      } else {
        const int q = k - 2 * MUW;
        my = 1 + (q >> 1);
        mx = (q & 1) ? MUW - 1 : 0;
      }
      float v[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2) v[a][b2] = sphi[my + a][mx + b2 + 2];
      smu[my][mx] = mu_at(p, v);
    }
  }
  __syncthreads();

  // 4. force, moments and collision; mu rows reused from registers
  float m3[3][3];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) m3[k + 1][j] = smu[ly0 + k][tx + j];
  // F = -phi d_D mu (+ d_D((c_s^2 - T) n)) at tile row ly, m3 = mu rows ly-1 .. ly+1
  auto force_at = [&](int ly, float &Fx, float &Fy) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      m3[0][j] = m3[1][j];
      m3[1][j] = m3[2][j];
      m3[2][j] = smu[ly + 2][tx + j];
    }
    float gmx = -p.M * m3[0][0];
    gmx += p.M * m3[0][2];
    gmx += -p.N * m3[1][0];
    gmx += p.N * m3[1][2];
    gmx += -p.M * m3[2][0];
    gmx += p.M * m3[2][2];
    float gmy = -p.M * m3[0][0];
    gmy += -p.N * m3[0][1];
    gmy += -p.M * m3[0][2];
    gmy += p.M * m3[2][0];
    gmy += p.N * m3[2][1];
    gmy += p.M * m3[2][2];
    const float ph = sphi[ly + 2][tx + 4];
    Fx = -ph * gmx;
    Fy = -ph * gmy;
    if constexpr (TGEN) {
      const int mx = tx + 1, my = ly + 1;
      float px = -p.M * spn[my - 1][mx - 1];
      px += p.M * spn[my - 1][mx + 1];
      px += -p.N * spn[my][mx - 1];
      px += p.N * spn[my][mx + 1];
      px += -p.M * spn[my + 1][mx - 1];
      px += p.M * spn[my + 1][mx + 1];
      float py = -p.M * spn[my - 1][mx - 1];
      py += -p.N * spn[my - 1][mx];
      py += -p.M * spn[my - 1][mx + 1];
      py += p.M * spn[my + 1][mx - 1];
      py += p.N * spn[my + 1][mx];
      py += p.M * spn[my + 1][mx + 1];
      Fx += px;
      Fy += py;
    }
  };
  auto pop = [&](int i, int ly) { return cvt_ld(pops[G::off(i) + ly * G::w(i) + tx + G::col(i)], p.inv_scale); };
  const float om = p.tau_inv, keep = 1.f - p.tau_inv;

  if constexpr (!PACK) {
#pragma unroll 1
    for (int r = 0; r < TR; ++r) {
      const int ly = ly0 + r, y = y0 + ly;
      float Fx, Fy;
      force_at(ly, Fx, Fy);
      if (x >= Lx || y >= Ly) continue;
      float h[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) h[i] = pop(i, ly);
      float dens = h[0];
#pragma unroll
      for (int i = 1; i < 9; ++i) dens += h[i];
      const float jx = ((h[1] - h[3]) + (h[5] - h[7])) + (h[8] - h[6]);
      const float jy = ((h[2] - h[4]) + (h[5] - h[7])) + (h[6] - h[8]);
      const float n = 1.f + dens;
      Fx += n * p.gx;
      Fy += n * p.gy;
      const float inv_n = 1.f / n;
      const float ux = (jx + 0.5f * Fx) * inv_n;
      const float uy = (jy + 0.5f * Fy) * inv_n;
      const long long s = (long long)y * Lx + x;
      if constexpr (MODE == COLLIDE_MOMENTS) {
        stg[s] = (double)n;
        stg[Sz + s] = (double)sphi[ly + 2][tx + 4];
        stg[2 * Sz + s] = (double)ux;
        stg[3 * Sz + s] = (double)uy;
        continue;
      }
      const float usq = ux * ux + uy * uy;
      const float uF = ux * Fx + uy * Fy;
      {
        const float w = float(q9_w(0));
        const float heq = w * (dens - n * (1.5f * usq));
        const float Fi = p.pref * w * (-3.f * uF);
        cvt_st(hout + s, keep * h[0] + om * heq + Fi, p.scale);
      }
      const float base = dens - n * (1.5f * usq);
      const float n3 = 3.f * n, n45 = 4.5f * n;
      const float pF3 = 3.f * p.pref, pF9 = 9.f * p.pref, puF = 3.f * p.pref * uF;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = k < 2 ? k + 1 : k + 3, ib = i + 2;  // (1,3) (2,4) (5,7) (6,8)
        const float w = float(q9_w(i));
        const float eu = float(q9_ex(i)) * ux + float(q9_ey(i)) * uy;
        const float eF = float(q9_ex(i)) * Fx + float(q9_ey(i)) * Fy;
        const float even = w * (base + n45 * eu * eu);
        const float odd = w * (n3 * eu);
        const float Feven = w * (pF9 * eu * eF - puF);
        const float Fodd = w * (pF3 * eF);
        cvt_st(hout + i * Sz + s, keep * h[i] + om * (even + odd) + (Feven + Fodd), p.scale);
        cvt_st(hout + ib * Sz + s, keep * h[ib] + om * (even - odd) + (Feven - Fodd), p.scale);
      }
      uout[s] = ux;
      uout[Sz + s] = uy;
    }
  } else {
    static_assert(MODE == COLLIDE_STEP, "the packed collision is a step kernel");
    // FP16 storage: the populations stay in the stored scale 2^s; only the
    // moments are brought back, and the weights carry the scale, so that the
    // new populations come out already scaled (power-of-two factors: exact)
    constexpr bool FOLD = !std::is_same<S, float>::value;
    const float wsc = FOLD ? p.scale : 1.f;
    auto popr = [&](int i, int ly) {
      return FOLD ? float(pops[G::off(i) + ly * G::w(i) + tx + G::col(i)]) : pop(i, ly);
    };
    // per weight class w: A = w / tau, B = w (1 - 1/2tau) (Eqs. 17, 29)
    const float A0 = om * float(q9_w(0)) * wsc, B0 = p.pref * float(q9_w(0)) * wsc;
    const float A1 = om * float(q9_w(1)) * wsc, B1 = p.pref * float(q9_w(1)) * wsc;
    const float A2 = om * float(q9_w(5)) * wsc, B2 = p.pref * float(q9_w(5)) * wsc;
#pragma unroll
    for (int r = 0; r < TR; r += 2) {
      const int lya = ly0 + r, ya = y0 + lya;
      float2 Fx, Fy;
      force_at(lya, Fx.x, Fy.x);
      force_at(lya + 1, Fx.y, Fy.y);
      if (x >= Lx || ya >= Ly) continue;
      const bool row_b = ya + 1 < Ly;
      float2 h[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) h[i] = make_float2(popr(i, lya), popr(i, lya + 1));
      float2 dens = h[0];
#pragma unroll
      for (int i = 1; i < 9; ++i) dens = add2(dens, h[i]);
      float2 jx = add2(add2(sub2(h[1], h[3]), sub2(h[5], h[7])), sub2(h[8], h[6]));
      float2 jy = add2(add2(sub2(h[2], h[4]), sub2(h[5], h[7])), sub2(h[6], h[8]));
      if constexpr (FOLD) {
        dens = mul2(dens, s2(p.inv_scale));
        jx = mul2(jx, s2(p.inv_scale));
        jy = mul2(jy, s2(p.inv_scale));
      }
      const float2 n = add2(s2(1.f), dens);
      Fx = fma2(n, s2(p.gx), Fx);
      Fy = fma2(n, s2(p.gy), Fy);
      const float2 inv_n = make_float2(1.f / n.x, 1.f / n.y);
      const float2 ux = mul2(fma2(s2(0.5f), Fx, jx), inv_n);
      const float2 uy = mul2(fma2(s2(0.5f), Fy, jy), inv_n);
      const float2 usq = fma2(ux, ux, mul2(uy, uy));
      const float2 uF = fma2(ux, Fx, mul2(uy, Fy));
      // w (base + 4.5 n eu^2) / tau + w pref (9 eu eF - 3 uF) = A se + B fe  (even part)
      // w 3 n eu / tau + w pref 3 eF                         = An3 eu + 3B eF (odd part)
      const float2 base = fma2(n, mul2(usq, s2(-1.5f)), dens);
      const float2 n45 = mul2(n, s2(4.5f)), m3uF = mul2(uF, s2(-3.f));
      const float2 An3_1 = mul2(n, s2(3.f * A1)), An3_2 = mul2(n, s2(3.f * A2));
      float2 o[9];
      o[0] = fma2(s2(keep), h[0], fma2(s2(A0), base, mul2(s2(-3.f * B0), uF)));
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = k < 2 ? k + 1 : k + 3, ib = i + 2;
        const float A = k < 2 ? A1 : A2, B = k < 2 ? B1 : B2;
        const float2 An3 = k < 2 ? An3_1 : An3_2;
        float2 eu, eF;
        if (k == 0) { eu = ux; eF = Fx; }
        else if (k == 1) { eu = uy; eF = Fy; }
        else if (k == 2) { eu = add2(ux, uy); eF = add2(Fx, Fy); }
        else { eu = sub2(uy, ux); eF = sub2(Fy, Fx); }
        const float2 se = fma2(mul2(n45, eu), eu, base);
        const float2 fe = fma2(mul2(eu, s2(9.f)), eF, m3uF);
        const float2 E = fma2(s2(A), se, mul2(s2(B), fe));
        const float2 O = fma2(eu, An3, mul2(s2(3.f * B), eF));
        o[i] = add2(fma2(s2(keep), h[i], E), O);
        o[ib] = sub2(fma2(s2(keep), h[ib], E), O);
      }
      const long long s = (long long)ya * Lx + x;
#pragma unroll
      for (int i = 0; i < 9; ++i) cvt_st(hout + i * Sz + s, o[i].x, FOLD ? 1.f : p.scale);
      uout[s] = ux.x;
      uout[Sz + s] = uy.x;
      if (row_b) {
#pragma unroll
        for (int i = 0; i < 9; ++i) cvt_st(hout + i * Sz + s + Lx, o[i].y, FOLD ? 1.f : p.scale);
        uout[s + Lx] = ux.y;
        uout[Sz + s + Lx] = uy.y;
      }
    }
  }
}

// ---- persistent, pipelined variant ------------------------------------------------
// The same arithmetic on 32 x 16 tiles, but each CTA stays resident and takes
// tiles from a per-handle counter (atomicAdd), with two shared-memory stages:
// while one tile is computed, the ten copies of the next are in flight.  The
// last CTA to finish resets the counter for the next launch.  A thread owns
// one column and two rows, whose collisions it evaluates as packed pairs.
constexpr int PY = 16;            // tile rows
constexpr int PPHH = PY + 4;      // phi box rows
constexpr int PMUH = PY + 2;      // mu rows
__host__ __device__ constexpr int pplane_off(int i) { return PY * (TT * i + 4 * nshift(i)); }
constexpr int PPOP_FLOATS = pplane_off(9);
constexpr int PSTAGE = 4 * (PPOP_FLOATS + PHW * PPHH);  // bytes of one stage (= its copies)
constexpr int P_OFF_STAGE = 128;                        // [0, 128): two mbarriers, two tile slots
constexpr int P_OFF_MU = P_OFF_STAGE + 2 * PSTAGE;
constexpr int P_OFF_PN = P_OFF_MU + 4 * MUW * PMUH;
static_assert(PSTAGE % 128 == 0 && (4 * PPOP_FLOATS) % 128 == 0 && (4 * pplane_off(1)) % 128 == 0 &&
                  (4 * pplane_off(2)) % 128 == 0,
              "TMA destinations must be 128-byte aligned");
template <bool TGEN>
constexpr size_t pipe_smem() {
  return 128 + P_OFF_PN + (TGEN ? 4 * MUW * PMUH : 0);
}

// The cells of an edge tile that its copies leave as zeros (the copies do not
// wrap around the periodic lattice): phi outside the lattice in the 36 x 20
// box, and the populations pulled across the lattice's edges.  Each thread
// loads its share (at most 3 + 2 cells) into registers before the copies are
// waited for, so that these loads overlap them; pipe_fix_store writes them
// into the stage once the copies have landed.  The float offsets in the stage
// (< 2^16) are packed two to a word, 0xffff for none.
struct PipeFix {
  float v[5];
  unsigned dst[3];
  __device__ __forceinline__ void set(int s, int off) {
    dst[s >> 1] = (s & 1) ? (dst[s >> 1] & 0xffffu) | ((unsigned)off << 16)
                          : (dst[s >> 1] & 0xffff0000u) | (unsigned)off;
  }
  __device__ __forceinline__ unsigned get(int s) const { return (s & 1) ? dst[s >> 1] >> 16 : dst[s >> 1] & 0xffffu; }
};
static_assert(PPOP_FLOATS + PHW * PPHH < 0xffff, "stage offsets fit 16 bits");
__device__ __forceinline__ void pipe_fix_load(PipeFix &f, const float *__restrict__ hin,
                                              const float *__restrict__ phi, const int Lx, const int Ly,
                                              const long long Sz, const int x0, const int y0) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
#pragma unroll
  for (int s = 0; s < 3; ++s) f.dst[s] = 0xffffffffu;
  // box column rxr and row ryb are the first beyond the lattice (Lx, Ly >= 64,
  // so one conditional wrap suffices below)
  const int rxr = Lx - x0 + 2, ryb = Ly - y0 + 2;
  const int wl = x0 == 0 ? 2 : 0, wr = max(0, TT + 4 - rxr), ht = y0 == 0 ? 2 : 0, hb = max(0, PPHH - ryb);
  if (wl + wr + ht + hb == 0) return;
  // phi outside the lattice: the column strips (all PPHH rows), then the row
  // strips between them
  const int ncol = PPHH * (wl + wr), wc = TT + 4 - wl - wr, ntot = ncol + (ht + hb) * wc;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int q = tid + 256 * s;
    if (q >= ntot) continue;
    int rx, ry;
    if (q < ncol) {
      const int c = q / PPHH;
      ry = q - c * PPHH;
      rx = c < wl ? c : rxr + (c - wl);
    } else {
      const int q2 = q - ncol, r = q2 / wc;
      rx = wl + (q2 - r * wc);
      ry = r < ht ? r : ryb + (r - ht);
    }
    f.set(s, PPOP_FLOATS + ry * PHW + rx + 2);
    f.v[s] = phi[(long long)wrap1(y0 - 2 + ry, Ly) * Lx + wrap1(x0 - 2 + rx, Lx)];
  }
  // populations whose pull buf_i(r - e_i) crosses an edge of the lattice
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int q = tid + 256 * s;
    if (q >= 8 * (PY + TT)) continue;
    const int i = 1 + q / (PY + TT), j = q % (PY + TT);
    const int ex = q9_ex(i), ey = q9_ey(i);
    int xs, ys;
    if (j < PY) {
      if (ex == 0) continue;
      xs = ex > 0 ? 0 : Lx - 1;
      ys = y0 + j;
    } else {
      if (ey == 0) continue;
      ys = ey > 0 ? 0 : Ly - 1;
      xs = x0 + j - PY;
    }
    if (xs < x0 || xs >= x0 + TT || xs >= Lx || ys < y0 || ys >= y0 + PY || ys >= Ly) continue;
    const int sx = wrap1(xs - ex, Lx), sy = wrap1(ys - ey, Ly);
    f.set(3 + s, pplane_off(i) + (ys - y0) * plane_w(i) + (xs - x0) + col_off(i));
    f.v[3 + s] = hin[i * Sz + (long long)sy * Lx + sx];
  }
}
__device__ __forceinline__ void pipe_fix_store(const PipeFix &f, float *pops) {
#pragma unroll
  for (int s = 0; s < 5; ++s)
    if (f.get(s) != 0xffffu) pops[f.get(s)] = f.v[s];
}

// One 32 x 16 tile of the pipelined kernels once its copies have landed in the
// stage at `pops`: the periodic images the copies left as zeros (from `fix`),
// mu on the tile + 1, the force and the packed collision of each thread's two
// rows (Lx x Ly lattice whose planes are Sz values apart; gx, gy the body
// force per unit density).
template <bool TGEN>
__device__ __forceinline__ void pipe_tile(float *pops, float (*smu)[MUW], float (*spn)[MUW], const PipeFix &fix,
                                          const float *__restrict__ hin, float *__restrict__ hout,
                                          const float *__restrict__ phi, float *__restrict__ uout,
                                          const KParams<float> &p, const int Lx, const int Ly,
                                          const long long Sz, const int x0, const int y0, const float gx,
                                          const float gy) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int ly0 = 2 * ty, x = x0 + tx;
  float(*sphi)[PHW] = reinterpret_cast<float(*)[PHW]>(pops + PPOP_FLOATS);
  const float om = p.tau_inv, keep = 1.f - p.tau_inv;
  const float A0 = om * float(q9_w(0)), B0 = p.pref * float(q9_w(0));
  const float A1 = om * float(q9_w(1)), B1 = p.pref * float(q9_w(1));
  const float A2 = om * float(q9_w(5)), B2 = p.pref * float(q9_w(5));
  pipe_fix_store(fix, pops);  // the periodic images loaded before the copies were waited for
  __syncthreads();
  // mu on the tile + 1: this thread's two rows, then the frame
  {
    // site row ly is phi row ly + 2 and mu row ly + 1
    float w[3][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j) w[a + 1][j] = sphi[ly0 + 1 + a][tx + 3 + j];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        w[0][j] = w[1][j];
        w[1][j] = w[2][j];
        w[2][j] = sphi[ly0 + 3 + r][tx + 3 + j];
      }
      smu[ly0 + 1 + r][tx + 1] = mu_at(p, w);
    }
    if (tid < 2 * MUW + 2 * PY) {
      int my, mx;
      if (tid < MUW) {
        my = 0;
        mx = tid;
      } else if (tid < 2 * MUW) {
        my = PMUH - 1;
        mx = tid - MUW;
      } else {
        const int q = tid - 2 * MUW;
        my = 1 + (q >> 1);
        mx = (q & 1) ? MUW - 1 : 0;
      }
      float v[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2) v[a][b2] = sphi[my + a][mx + b2 + 2];
      smu[my][mx] = mu_at(p, v);
    }
  }
  __syncthreads();
  // force (Eqs. 28, 30) of the two rows, then the packed collision
  float2 Fx, Fy;
  {
    float m[4][3];  // mu rows ly0 .. ly0 + 3 (tile + 1 coordinates), columns tx .. tx + 2
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j) m[a][j] = smu[ly0 + a][tx + j];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float gmx = -p.M * m[r][0];
      gmx += p.M * m[r][2];
      gmx += -p.N * m[r + 1][0];
      gmx += p.N * m[r + 1][2];
      gmx += -p.M * m[r + 2][0];
      gmx += p.M * m[r + 2][2];
      float gmy = -p.M * m[r][0];
      gmy += -p.N * m[r][1];
      gmy += -p.M * m[r][2];
      gmy += p.M * m[r + 2][0];
      gmy += p.N * m[r + 2][1];
      gmy += p.M * m[r + 2][2];
      const float ph = sphi[ly0 + r + 2][tx + 4];
      float fx = -ph * gmx, fy = -ph * gmy;
      if constexpr (TGEN) {
        const int mx = tx + 1, my = ly0 + r + 1;
        float px = -p.M * spn[my - 1][mx - 1];
        px += p.M * spn[my - 1][mx + 1];
        px += -p.N * spn[my][mx - 1];
        px += p.N * spn[my][mx + 1];
        px += -p.M * spn[my + 1][mx - 1];
        px += p.M * spn[my + 1][mx + 1];
        float py = -p.M * spn[my - 1][mx - 1];
        py += -p.N * spn[my - 1][mx];
        py += -p.M * spn[my - 1][mx + 1];
        py += p.M * spn[my + 1][mx - 1];
        py += p.N * spn[my + 1][mx];
        py += p.M * spn[my + 1][mx + 1];
        fx += px;
        fy += py;
      }
      if (r == 0) {
        Fx.x = fx;
        Fy.x = fy;
      } else {
        Fx.y = fx;
        Fy.y = fy;
      }
    }
  }
  const int ya = y0 + ly0;
  if (x < Lx && ya < Ly) {
    const bool row_b = ya + 1 < Ly;
    auto pop = [&](int i, int ly) { return pops[pplane_off(i) + ly * plane_w(i) + tx + col_off(i)]; };
    float2 h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = make_float2(pop(i, ly0), pop(i, ly0 + 1));
    float2 dens = h[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) dens = add2(dens, h[i]);
    const float2 jx = add2(add2(sub2(h[1], h[3]), sub2(h[5], h[7])), sub2(h[8], h[6]));
    const float2 jy = add2(add2(sub2(h[2], h[4]), sub2(h[5], h[7])), sub2(h[6], h[8]));
    const float2 n = add2(s2(1.f), dens);
    Fx = fma2(n, s2(gx), Fx);
    Fy = fma2(n, s2(gy), Fy);
    const float2 inv_n = make_float2(1.f / n.x, 1.f / n.y);
    const float2 ux = mul2(fma2(s2(0.5f), Fx, jx), inv_n);
    const float2 uy = mul2(fma2(s2(0.5f), Fy, jy), inv_n);
    const float2 usq = fma2(ux, ux, mul2(uy, uy));
    const float2 uF = fma2(ux, Fx, mul2(uy, Fy));
    const float2 base2 = fma2(n, mul2(usq, s2(-1.5f)), dens);
    const float2 n45 = mul2(n, s2(4.5f)), m3uF = mul2(uF, s2(-3.f));
    const float2 An3_1 = mul2(n, s2(3.f * A1)), An3_2 = mul2(n, s2(3.f * A2));
    float2 o[9];
    o[0] = fma2(s2(keep), h[0], fma2(s2(A0), base2, mul2(s2(-3.f * B0), uF)));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = q < 2 ? q + 1 : q + 3, ib = i + 2;
      const float A = q < 2 ? A1 : A2, B = q < 2 ? B1 : B2;
      const float2 An3 = q < 2 ? An3_1 : An3_2;
      float2 eu, eF;
      if (q == 0) {
        eu = ux;
        eF = Fx;
      } else if (q == 1) {
        eu = uy;
        eF = Fy;
      } else if (q == 2) {
        eu = add2(ux, uy);
        eF = add2(Fx, Fy);
      } else {
        eu = sub2(uy, ux);
        eF = sub2(Fy, Fx);
      }
      const float2 se = fma2(mul2(n45, eu), eu, base2);
      const float2 fe = fma2(mul2(eu, s2(9.f)), eF, m3uF);
      const float2 E = fma2(s2(A), se, mul2(s2(B), fe));
      const float2 O = fma2(eu, An3, mul2(s2(3.f * B), eF));
      o[i] = add2(fma2(s2(keep), h[i], E), O);
      o[ib] = sub2(fma2(s2(keep), h[ib], E), O);
    }
    const long long sa = (long long)ya * Lx + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) hout[i * Sz + sa] = o[i].x;
    uout[sa] = ux.x;
    uout[Sz + sa] = uy.x;
    if (row_b) {
#pragma unroll
      for (int i = 0; i < 9; ++i) hout[i * Sz + sa + Lx] = o[i].y;
      uout[sa + Lx] = ux.y;
      uout[Sz + sa + Lx] = uy.y;
    }
  }
}
template <bool TGEN, int MINB>
__global__ void __launch_bounds__(256, MINB)
    collide2d_tma_pipe_kernel(const __grid_constant__ CUtensorMap map_p32,
                              const __grid_constant__ CUtensorMap map_p36,
                              const __grid_constant__ CUtensorMap map_phi, const float *__restrict__ hin,
                              float *__restrict__ hout, const float *__restrict__ phi,
                              const float *__restrict__ dn, float *__restrict__ uout,
                              unsigned *__restrict__ sched, KParams<float> p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *base = smem_raw + ((128u - (su32(smem_raw) & 127u)) & 127u);
  const uint32_t bar0 = su32(base);
  volatile int *stile = reinterpret_cast<volatile int *>(base + 16);  // tile of stage 0 / 1
  float(*smu)[MUW] = reinterpret_cast<float(*)[MUW]>(base + P_OFF_MU);
  float(*spn)[MUW] = reinterpret_cast<float(*)[MUW]>(base + P_OFF_PN);
  const int Lx = p.Lx, Ly = p.Ly;
  const long long Sz = (long long)Lx * Ly;
  const int ntx = (Lx + TT - 1) / TT, ntiles = ntx * ((Ly + PY - 1) / PY);
  const int tid = threadIdx.y * 32 + threadIdx.x;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();  // phi(t), the populations and the reset counter come from earlier kernels
  pdl_trigger();
  // thread 0: the ten copies of `tile` into stage st, completing on its mbarrier
  auto issue = [&](int tile, int st) {
    const int x0 = (tile % ntx) * TT, y0 = (tile / ntx) * PY;
    unsigned char *sb = base + P_OFF_STAGE + st * PSTAGE;
    const uint32_t bar = bar0 + 8 * st;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic accesses first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)PSTAGE)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 9; ++i)
      tma_3d(su32(sb + 4 * pplane_off(i)), plane_w(i) == TT ? &map_p32 : &map_p36, x0 + box_dx(i), y0 - q9_ey(i),
             i, bar);
    tma_2d(su32(sb + 4 * PPOP_FLOATS), &map_phi, x0 - 4, y0 - 2, bar);
  };
  if (tid == 0) {
    const int t0 = (int)atomicAdd(sched, 1u);
    stile[0] = t0;
    if (t0 < ntiles) issue(t0, 0);
  }
  __syncthreads();
  int k = 0;
  bool failed = false;
  while (true) {
    const int st = k & 1;
    const int tile = stile[st];
    if (tile >= ntiles) break;
    // claim the next tile and start its copies into the other stage (free
    // since the end of the previous iteration)
    if (tid == 0) {
      const int tn = (int)atomicAdd(sched, 1u);
      stile[st ^ 1] = tn;
      if (tn < ntiles) issue(tn, st ^ 1);
    }
    const int x0 = (tile % ntx) * TT, y0 = (tile / ntx) * PY;
    float *pops = reinterpret_cast<float *>(base + P_OFF_STAGE + st * PSTAGE);
    if constexpr (TGEN) {
      for (int q = tid; q < MUW * PMUH; q += 256) {
        const int ry = q / MUW, rx = q - ry * MUW;
        const int gx = wrapi(x0 + rx - 1, Lx), gy = wrapi(y0 + ry - 1, Ly);
        spn[ry][rx] = p.cs2mT * (1.f + dn[(long long)gy * Lx + gx]);
      }
    }
    PipeFix fix;
    pipe_fix_load(fix, hin, phi, Lx, Ly, Sz, x0, y0);
    const bool arrived = bar_wait(bar0 + 8 * st, (uint32_t)(k >> 1) & 1u, g_collide_tma_wait_ns);
    if (!__syncthreads_and(arrived)) {
      failed = true;
      break;
    }
    pipe_tile<TGEN>(pops, smu, spn, fix, hin, hout, phi, uout, p, Lx, Ly, Sz, x0, y0, p.gx, p.gy);
    __syncthreads();  // stage st, smu and spn are free again; the next tile's slot is visible
    ++k;
  }
  if (tid == 0) {
    if (failed) {
      // a copy did not complete within the wait bound: report it and let the copies
      // still in flight land before the CTA's shared memory is released
      atomicExch(&g_collide_tma_err, 1);
      const int st = k & 1;
      bar_wait(bar0 + 8 * st, (uint32_t)(k >> 1) & 1u, 500000000ull);
      if (stile[st ^ 1] < ntiles) bar_wait(bar0 + 8 * (st ^ 1), (uint32_t)((k + 1) >> 1) & 1u, 500000000ull);
    }
    // every CTA has made its last claim before it counts itself out; the last
    // one resets the counter for the next launch
    __threadfence();
    if (atomicAdd(sched + 1, 1u) == gridDim.x - 1) {
      atomicExch(sched, 0u);
      atomicExch(sched + 1, 0u);
      __threadfence();
    }
  }
}

__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int w,
                                       uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

// The pipelined kernel over the 32 x 16 tiles of many independent lattices
// packed end to end (one plane per population over all of them, ST sites):
// tile k is items[k] = (instance, x0, y0, shape slot << 16 | index j within
// the shape), copied through the slot's tensor maps in the kernel parameter
// (populations at (x, y, j, plane), phi at (x, y, j)); the instance's body
// force is on while t < force_steps.  T = 1/3.  Instances are at least
// TMA_MIN_SIDE on a side.  Static schedule: CTA c takes items c, c + G,
// c + 2G, ... (G CTAs, G <= nitems), and thread 0 loads the item after next
// one tile ahead, so that no claim or dependent load stands between a tile
// and the copies of the next.
__global__ void __launch_bounds__(256, 4)
    collide2d_tma_batch_kernel(const __grid_constant__ TmaShapeMaps maps, const float *__restrict__ hin,
                               float *__restrict__ hout, const float *__restrict__ phi,
                               float *__restrict__ uout, long long ST, const TiledInst *__restrict__ inst,
                               const int4 *__restrict__ items, int nitems, KParams<float> p, long long t) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *base = smem_raw + ((128u - (su32(smem_raw) & 127u)) & 127u);
  const uint32_t bar0 = su32(base);
  float(*smu)[MUW] = reinterpret_cast<float(*)[MUW]>(base + P_OFF_MU);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int G = gridDim.x;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();  // phi(t) and the populations come from earlier kernels
  pdl_trigger();
  // thread 0: the ten copies of item `it` into stage st, completing on its mbarrier
  auto issue = [&](const int4 it, int st) {
    const int slot = it.w >> 16, j = it.w & 0xffff;
    const CUtensorMap *m = reinterpret_cast<const CUtensorMap *>(&maps.map[slot][0][0]);
    unsigned char *sb = base + P_OFF_STAGE + st * PSTAGE;
    const uint32_t bar = bar0 + 8 * st;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic accesses first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)PSTAGE)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 9; ++i)
      tma_4d(su32(sb + 4 * pplane_off(i)), plane_w(i) == TT ? m : m + 1, it.y + box_dx(i), it.z - q9_ey(i), j, i,
             bar);
    tma_3d(su32(sb + 4 * PPOP_FLOATS), m + 2, it.y - 4, it.z - 2, j, bar);
  };
  int4 nxt = make_int4(0, 0, 0, 0);  // thread 0: the item after the one in flight
  if (tid == 0) {
    issue(items[blockIdx.x], 0);
    if (blockIdx.x + G < nitems) nxt = items[blockIdx.x + G];
  }
  int k = 0, tile = blockIdx.x;
  bool failed = false;
  for (; tile < nitems; tile += G, ++k) {
    const int st = k & 1;
    // the copies of the next item go into the other stage (free since the end
    // of the previous iteration)
    if (tid == 0 && tile + G < nitems) {
      issue(nxt, st ^ 1);
      if (tile + 2 * G < nitems) nxt = items[tile + 2 * G];
    }
    const int4 it = items[tile];
    const int slot = it.w >> 16, j = it.w & 0xffff;
    const int Lx = maps.Lx[slot], Ly = maps.Ly[slot];
    const long long off = maps.off0[slot] + (long long)j * Lx * Ly;
    float *pops = reinterpret_cast<float *>(base + P_OFF_STAGE + st * PSTAGE);
    PipeFix fix;
    pipe_fix_load(fix, hin + off, phi + off, Lx, Ly, ST, it.y, it.z);
    const bool arrived = bar_wait(bar0 + 8 * st, (uint32_t)(k >> 1) & 1u, g_collide_tma_wait_ns);
    if (!__syncthreads_and(arrived)) {
      failed = true;
      break;
    }
    const TiledInst &I = inst[it.x];
    const bool on = t < I.force_steps;
    pipe_tile<false>(pops, smu, nullptr, fix, hin + off, hout + off, phi + off, uout + off, p, Lx, Ly, ST, it.y,
                     it.z, on ? I.gx : 0.f, on ? I.gy : 0.f);
    __syncthreads();  // stage st and smu are free again
  }
  if (tid == 0 && failed) {
    // a copy did not complete within the wait bound: report it and let the copies
    // still in flight land before the CTA's shared memory is released
    atomicExch(&g_collide_tma_err, 1);
    const int st = k & 1;
    bar_wait(bar0 + 8 * st, (uint32_t)(k >> 1) & 1u, 500000000ull);
    if (tile + G < nitems) bar_wait(bar0 + 8 * (st ^ 1), (uint32_t)((k + 1) >> 1) & 1u, 500000000ull);
  }
}

// ---- host side -------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

bool encode(CUtensorMap *map, CUtensorMapDataType type, void *ptr, int rank, const cuuint64_t *dims,
            const cuuint64_t *strides, const cuuint32_t *box) {
  auto fn = encode_fn();
  if (fn == nullptr) return false;
  const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
  return fn(map, type, rank, ptr, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// maps per buffer parity b, [6 b + j]: 32 x 32 tiles: j = 0 populations 32 wide, 1 populations
// 32 + A wide (A = 4 FP32, 8 FP16), 2 phi 40 x 36; 32 x 16 tiles (pipelined kernel, FP32
// only): 3, 4 populations, 5 phi 40 x 20
CUtensorMap *maps_of(lbm_handle *h) { return reinterpret_cast<CUtensorMap *>(h->tma_maps); }

bool prepare(lbm_handle *h) {
  if (h->tma_ready) return true;
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  const bool half = h->P.precision == LBM_F16DEV;
  const cuuint64_t es = half ? 2 : 4;
  const CUtensorMapDataType pt = half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint32_t A = (cuuint32_t)(16 / es);
  const cuuint64_t Lx = (cuuint64_t)h->P.Lx, Ly = (cuuint64_t)h->P.Ly;
  const cuuint64_t pd[3] = {Lx, Ly, 9}, ps[2] = {es * Lx, es * Lx * Ly};
  const cuuint64_t fd[2] = {Lx, Ly}, fs[1] = {4 * Lx};
  const cuuint32_t b32[3] = {TT, TT, 1}, bw[3] = {TT + A, TT, 1}, bphi[2] = {PHW, PHH};
  const cuuint32_t q32[3] = {TT, PY, 1}, q36[3] = {TT + 4, PY, 1}, qphi[2] = {PHW, PPHH};
  const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUtensorMap *m = maps_of(h);
  for (int b = 0; b < 2; ++b) {
    CUtensorMap *mb = m + 6 * b;
    if (!encode(&mb[0], pt, h->h[b], 3, pd, ps, b32) || !encode(&mb[1], pt, h->h[b], 3, pd, ps, bw) ||
        !encode(&mb[2], f32, h->phi[b], 2, fd, fs, bphi))
      return false;
    if (!half && (!encode(&mb[3], f32, h->h[b], 3, pd, ps, q32) || !encode(&mb[4], f32, h->h[b], 3, pd, ps, q36) ||
                  !encode(&mb[5], f32, h->phi[b], 2, fd, fs, qphi)))
      return false;
  }
  h->tma_ready = true;
  return true;
}

template <typename S, bool TGEN, int MODE, bool PACK, int MINB>
cudaError_t launch_one(lbm_handle *h, int in, const KParams<float> &p) {
  const CUtensorMap *m = maps_of(h) + 6 * in;
  dim3 grid((p.Lx + TT - 1) / TT, (p.Ly + TT - 1) / TT), block(32, 256 / 32);
  const S *hin = static_cast<const S *>(h->h[in]);
  S *hout = static_cast<S *>(h->h[1 - in]);
  const float *phi = static_cast<const float *>(h->phi[in]);
  const float *dn = static_cast<const float *>(h->dn);
  float *u = static_cast<float *>(h->u);
  auto kern = collide2d_tma_kernel<S, TGEN, MODE, PACK, MINB>;
  if (MODE == COLLIDE_STEP)
    return launch_pdl(kern, grid, block, tma_smem<S, TGEN>(), h->stream, m[0], m[1], m[2], hin, hout, phi, dn,
                      u, h->staging, p);
  kern<<<grid, block, tma_smem<S, TGEN>(), h->stream>>>(m[0], m[1], m[2], hin, hout, phi, dn, u, h->staging, p);
  return cudaGetLastError();
}

// resident CTAs of a pipelined kernel on this device (queried once per kernel)
template <bool TGEN, int MINB>
int pipe_grid() {
  static const int g = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, collide2d_tma_pipe_kernel<TGEN, MINB>, 256,
                                                  pipe_smem<TGEN>());
    return std::max(1, sms * std::max(per, 1));
  }();
  return g;
}

template <bool TGEN, int MINB>
cudaError_t launch_pipe(lbm_handle *h, int in, const KParams<float> &p) {
  const CUtensorMap *m = maps_of(h) + 6 * in + 3;
  const int ntiles = ((p.Lx + TT - 1) / TT) * ((p.Ly + PY - 1) / PY);
  const int grid = std::min(ntiles, pipe_grid<TGEN, MINB>());
  return launch_pdl(collide2d_tma_pipe_kernel<TGEN, MINB>, dim3(grid), dim3(32, 256 / 32), pipe_smem<TGEN>(),
                    h->stream, m[0], m[1], m[2], static_cast<const float *>(h->h[in]),
                    static_cast<float *>(h->h[1 - in]), static_cast<const float *>(h->phi[in]),
                    static_cast<const float *>(h->dn), static_cast<float *>(h->u), h->sched, p);
}

template <typename S, bool TGEN>
cudaError_t launch_step(lbm_handle *h, int in, const KParams<float> &p, int variant) {
  if constexpr (std::is_same<S, float>::value)
    if (variant == 7) return launch_pipe<TGEN, 4>(h, in, p);
  switch (variant) {
    case 5: return launch_one<S, TGEN, COLLIDE_STEP, true, 4>(h, in, p);
    case 6: return launch_one<S, TGEN, COLLIDE_STEP, true, 3>(h, in, p);
    default: return launch_one<S, TGEN, COLLIDE_STEP, false, 3>(h, in, p);
  }
}

template <typename S>
cudaError_t collide2d_tma_s(lbm_handle *h, int in, int force_on, int mode, int variant) {
  const KParams<float> p = make_params<float>(h, force_on);
  const bool tgen = p.cs2mT != 0.f;
  if (mode == COLLIDE_STEP)
    return tgen ? launch_step<S, true>(h, in, p, variant) : launch_step<S, false>(h, in, p, variant);
  return tgen ? launch_one<S, true, COLLIDE_MOMENTS, false, 3>(h, in, p)
              : launch_one<S, false, COLLIDE_MOMENTS, false, 3>(h, in, p);
}

template <typename S>
void configure_s(cudaError_t &e) {
  auto set = [&](auto fn, size_t smem) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  };
  set(collide2d_tma_kernel<S, false, COLLIDE_STEP, false, 3>, tma_smem<S, false>());
  set(collide2d_tma_kernel<S, false, COLLIDE_STEP, true, 4>, tma_smem<S, false>());
  set(collide2d_tma_kernel<S, false, COLLIDE_STEP, true, 3>, tma_smem<S, false>());
  set(collide2d_tma_kernel<S, true, COLLIDE_STEP, false, 3>, tma_smem<S, true>());
  set(collide2d_tma_kernel<S, true, COLLIDE_STEP, true, 4>, tma_smem<S, true>());
  set(collide2d_tma_kernel<S, true, COLLIDE_STEP, true, 3>, tma_smem<S, true>());
  set(collide2d_tma_kernel<S, false, COLLIDE_MOMENTS, false, 3>, tma_smem<S, false>());
  set(collide2d_tma_kernel<S, true, COLLIDE_MOMENTS, false, 3>, tma_smem<S, true>());
}

}  // namespace

bool collide2d_tma_eligible(const lbm_handle *h, int variant) {
  const bool half = h->P.precision == LBM_F16DEV;
  if (h->dims != 2 || (h->P.precision != LBM_F32DEV && !half)) return false;
  if (variant != 3 && variant != 5 && variant != 6 && variant != 7) return false;
  if (variant == 7 && (half || h->sched == nullptr)) return false;  // the pipelined kernel is FP32
  return h->P.Lx % (half ? 8 : 4) == 0 && h->P.Lx >= TMA_MIN_SIDE && h->P.Ly >= TMA_MIN_SIDE &&
         encode_fn() != nullptr;
}

cudaError_t collide2d_tma(lbm_handle *h, int in, int force_on, int mode, int variant) {
  if (!collide2d_tma_eligible(h, variant)) return cudaErrorInvalidValue;
  if (!prepare(h)) return cudaErrorInvalidValue;
  return h->P.precision == LBM_F16DEV ? collide2d_tma_s<__half>(h, in, force_on, mode, variant)
                                      : collide2d_tma_s<float>(h, in, force_on, mode, variant);
}

cudaError_t collide2d_tma_configure(int precision) {
  cudaError_t e = cudaSuccess;
  if (precision == LBM_F16DEV) {
    configure_s<__half>(e);
    return e;
  }
  configure_s<float>(e);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(collide2d_tma_pipe_kernel<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pipe_smem<false>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(collide2d_tma_pipe_kernel<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pipe_smem<true>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(collide2d_tma_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pipe_smem<false>());
  return e;
}

int collide2d_tma_set_wait_ns(unsigned long long ns) {
  return cudaMemcpyToSymbol(g_collide_tma_wait_ns, &ns, sizeof ns) == cudaSuccess ? 0 : -1;
}

int collide2d_tma_error(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_collide_tma_err, sizeof v) != cudaSuccess) return -1;
  if (reset && v != 0) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_collide_tma_err, &zero, sizeof zero);
  }
  return v;
}


int collide2d_tma_batch_min_side() { return TMA_MIN_SIDE; }

bool collide2d_tma_batch_shape(TmaShapeMaps *m, int slot, float *h, float *phi, long long ST, int Lx, int Ly,
                               long long off0, int n) {
  static_assert(sizeof(CUtensorMap) == 128 && alignof(TmaShapeMaps) >= 64, "tensor map size and alignment");
  if (slot < 0 || slot >= TMA_BATCH_SHAPES || n < 1 || n > 0xffff || Lx < TMA_MIN_SIDE || Ly < TMA_MIN_SIDE ||
      Lx % 4 != 0 || off0 % 4 != 0 || ST % 4 != 0)
    return false;
  CUtensorMap *mk = reinterpret_cast<CUtensorMap *>(&m->map[slot][0][0]);
  const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t S = (cuuint64_t)Lx * Ly;
  const cuuint64_t pd[4] = {(cuuint64_t)Lx, (cuuint64_t)Ly, (cuuint64_t)n, 9};
  const cuuint64_t ps[3] = {4 * (cuuint64_t)Lx, 4 * S, 4 * (cuuint64_t)ST};
  const cuuint64_t fd[3] = {(cuuint64_t)Lx, (cuuint64_t)Ly, (cuuint64_t)n}, fs[2] = {4 * (cuuint64_t)Lx, 4 * S};
  const cuuint32_t q32[4] = {TT, PY, 1, 1}, q36[4] = {TT + 4, PY, 1, 1}, qphi[3] = {PHW, PPHH, 1};
  if (!encode(&mk[0], f32, h + off0, 4, pd, ps, q32) || !encode(&mk[1], f32, h + off0, 4, pd, ps, q36) ||
      !encode(&mk[2], f32, phi + off0, 3, fd, fs, qphi))
    return false;
  m->Lx[slot] = Lx;
  m->Ly[slot] = Ly;
  m->off0[slot] = off0;
  return true;
}

cudaError_t collide2d_tma_batch(const TmaShapeMaps &maps, const float *hin, float *hout, const float *phi,
                                float *u, long long ST, const TiledInst *inst, const int4 *items, int nitems,
                                const KParams<float> &p, long long t, cudaStream_t s, bool pdl) {
  static const int resident = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, collide2d_tma_batch_kernel, 256, pipe_smem<false>());
    return std::max(1, sms * std::max(per, 1));
  }();
  if (nitems <= 0) return cudaSuccess;
  const int grid = std::min(nitems, resident);
  return launch_ex(pdl, collide2d_tma_batch_kernel, dim3(grid), dim3(32, 256 / 32), pipe_smem<false>(), s, maps,
                   hin, hout, phi, u, ST, inst, items, nitems, p, t);
}

}  // namespace hlbm
