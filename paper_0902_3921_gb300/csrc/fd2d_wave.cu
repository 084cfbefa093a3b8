// fd2d_wave.cu -- FP32 convection-diffusion update of phi (Sec. II C,
// Eqs. 32-36) in y-marching ("wavefront") form, for large 2D lattices.
//
// One CTA owns a strip of 128 computed columns (x0 .. x0 + 127, wrapped; the
// inner 128 - 2 HX are written) and marches down a segment of NY output rows,
// reading HY = 3 SUB input rows above and below it.  Input row j of the
// segment arrives at tick j; every tick each warp advances its part of the
// row pipeline by one row:
//
//   warp A (substeps 1 and 2), a = t - 1:
//     advection coefficients of row a (Eqs. 32-35, from u*, v* of rows
//     a - 1 .. a + 1), phih_1(a), psi_1(a - 1), phi_1(a - 2),
//     phih_2(a - 3), psi_2(a - 4), phi_2(a - 5);
//   warp B (substeps 3 and 4, SUB = 4 only), b = t - 9:
//     phih_3(b) .. phi_3(b - 2), phih_4(b - 3) .. phi_4(b - 5), reading
//     phi_2 that warp A handed over before the last barrier and the
//     coefficients warp A wrote to a shared ring.
//
// A stencil input is consumed three rows at a time (r - 1, r, r + 1): each
// warp keeps the two older rows of every input in registers and receives one
// new row per tick, so nothing is read twice.  Lane l holds the four columns
// 4l .. 4l + 3 of a row (one float4) and takes its x neighbours from lanes
// l -/+ 1 by shuffles; columns 0 and 127 lose validity first and are never
// written.  Warp A writes the coefficients of each row to a 16-row shared
// ring, from which the later substeps read them (3, 7 and 10 ticks later).
// Inputs (phi, u, v) are prefetched D rows ahead by cp.async into per-lane
// rings (a lane reads back only the 16 bytes it copied, so no barrier guards
// them); one named barrier per pair of ticks orders the hand-over between
// the warps.
//
// Per site and LB step the kernel reads phi and u* once and writes phi once
// (16 B), plus the strip's x halo (128 / (128 - 2 HX) of the columns) and the
// segment's y halo ((NY + 2 HY) / NY of the rows), which are re-read from L2.
// The arithmetic is that of the block kernel (Eq. 36 regrouped as
// lap(a phih + b phi^3 - kappa lap phih), the advection as
// c0 phi + |dt u| phi_up,x + |dt v| phi_up,y), explicitly rounded so that every
// site gets the same bits wherever it falls in the strip or the segment.
#include <cstdint>
#include <type_traits>

#include "lbm_common.cuh"

namespace hlbm {
namespace {

constexpr int WV_W = 128;   // computed columns of a strip
constexpr int WV_IR = 8;    // input ring rows (per lane)
constexpr int WV_D = 6;     // input prefetch distance in rows (<= WV_IR - 2)
constexpr unsigned WV_FULL = 0xffffffffu;

template <int SUB>
struct Wave {
  static_assert(SUB == 2 || SUB == 4, "two substeps per warp");
  static constexpr int NWARP = SUB / 2;
  static constexpr int NT = 32 * NWARP;
  static constexpr int HY = 3 * SUB;                // rows of reach of SUB substeps
  static constexpr int HX = (3 * SUB + 3) / 4 * 4;  // columns, rounded to whole float4 groups
  static constexpr int TX = WV_W - 2 * HX;          // written columns of a strip
  // warp A's output row lags its input by 6 rows; warp B's by 14 (it works on
  // row b = t - 9, two ticks behind warp A's phi_2, so that one barrier per
  // pair of ticks orders the hand-over)
  static constexpr int LAG = SUB == 4 ? 14 : 6;
  // coefficient ring rows: written for row a at tick a + 1, read for row a - 3
  // (warp A) and rows t - 9, t - 12 (warp B); hand-over ring rows
  static constexpr int CR = SUB == 4 ? 16 : 4;
  static constexpr int HR = 4;
  // shared memory (floats): phi, u, v rings of warp A, the coefficient ring
  // (c0, dt u, dt v) and the two-row phi_2 hand-over (SUB = 4)
  static constexpr int OFF_PHI = 0, OFF_U = WV_IR * WV_W, OFF_V = 2 * WV_IR * WV_W;
  static constexpr int OFF_C = 3 * WV_IR * WV_W;
  static constexpr int OFF_H = OFF_C + 3 * CR * WV_W;
  static constexpr int FLOATS = OFF_H + (SUB == 4 ? HR * WV_W : 0);
  static constexpr size_t smem = sizeof(float) * FLOATS;
  // ticks for a segment of NY output rows, rounded up to whole pairs
  static __host__ __device__ int ticks(int NY) { return (NY + HY + LAG + 1) / 2 * 2; }
};

__device__ __forceinline__ float4 wv_ld(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void wv_st(float *p, const float4 &v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float wv_c(const float4 &v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ float2 wv_lo(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 wv_hi(const float4 &v) { return make_float2(v.z, v.w); }

__device__ __forceinline__ void wv_cp16(float *sdst, const float *gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void wv_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void wv_wait_d() { asm volatile("cp.async.wait_group %0;" ::"n"(WV_D) : "memory"); }
template <int NT>
__device__ __forceinline__ void wv_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

struct WvCoef {
  float4 c0, t1, t2;  // c0 = 1 - dt (d_x u + d_y v + |u| + |v|), dt u, dt v of one row
};

// state of one substep's row pipeline: the two older rows of each stencil input
struct WvSub {
  float4 pm, pc;  // phi^n rows a - 1, a
  float4 hu, hc;  // phih rows a - 2, a - 1
  float4 qu, qc;  // psi rows a - 3, a - 2
};

struct WvConst {
  float dt, dtG, a, b, kappa;
  bool cubic_half;
};

// advection coefficients of row r (Eq. 33: central d_x u and d_y v; Eqs. 34-35:
// upwind by the sign of u, v) from u of row r and v of rows r - 1, r, r + 1
__device__ __forceinline__ WvCoef wv_coef(const float4 &uc, const float4 &vm, const float4 &vc,
                                          const float4 &vp, float dt) {
  const float uL = __shfl_up_sync(WV_FULL, uc.w, 1), uR = __shfl_down_sync(WV_FULL, uc.x, 1);
  float c0[4], t1[4], t2[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float ucj = wv_c(uc, j), vcj = wv_c(vc, j);
    const float ul = j == 0 ? uL : wv_c(uc, j - 1), ur = j == 3 ? uR : wv_c(uc, j + 1);
    const float div = __fadd_rn(__fmul_rn(__fsub_rn(ur, ul), 0.5f),
                                __fmul_rn(__fsub_rn(wv_c(vp, j), wv_c(vm, j)), 0.5f));
    c0[j] = __fmaf_rn(-dt, __fadd_rn(div, __fadd_rn(fabsf(ucj), fabsf(vcj))), 1.f);
    t1[j] = __fmul_rn(dt, ucj);
    t2[j] = __fmul_rn(dt, vcj);
  }
  return {make_float4(c0[0], c0[1], c0[2], c0[3]), make_float4(t1[0], t1[1], t1[2], t1[3]),
          make_float4(t2[0], t2[1], t2[2], t2[3])};
}

// One tick of one substep: pn = phi^n of row a + 1 and the coefficients of
// row a.  Computes phih(a) (Eqs. 32-35), psi(a - 1) = a phih + b phi^3 -
// kappa lap phih, and returns phi^{n+1}(a - 2) = phih + dt Gamma lap psi
// (Eq. 36); then shifts the row windows by one.
__device__ __forceinline__ float4 wv_substep(WvSub &st, const float4 &pn, const WvCoef &cf,
                                             const WvConst &k) {
  // phih of row a
  float4 hn;
  {
    const float pl = __shfl_up_sync(WV_FULL, st.pc.w, 1), pr = __shfl_down_sync(WV_FULL, st.pc.x, 1);
    float e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float pcj = wv_c(st.pc, j);
      const float plj = j == 0 ? pl : wv_c(st.pc, j - 1), prj = j == 3 ? pr : wv_c(st.pc, j + 1);
      const float t1 = wv_c(cf.t1, j), t2 = wv_c(cf.t2, j);
      const float upx = t1 > 0.f ? plj : prj;  // u = 0 contributes nothing
      const float upy = t2 > 0.f ? wv_c(st.pm, j) : wv_c(pn, j);
      e[j] = __fmaf_rn(fabsf(t2), upy, __fmaf_rn(fabsf(t1), upx, __fmul_rn(wv_c(cf.c0, j), pcj)));
    }
    hn = make_float4(e[0], e[1], e[2], e[3]);
  }
  // psi of row a - 1 (phih rows a - 2, a - 1, a); phi^3 of phi^n (or of phih)
  float4 qn;
  {
    const float hl = __shfl_up_sync(WV_FULL, st.hc.w, 1), hr = __shfl_down_sync(WV_FULL, st.hc.x, 1);
    const float4 &cb4 = k.cubic_half ? st.hc : st.pm;
    float2 o[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2 hk = q ? wv_hi(st.hc) : wv_lo(st.hc);
      const float2 vs = __fadd2_rn(q ? wv_hi(st.hu) : wv_lo(st.hu), q ? wv_hi(hn) : wv_lo(hn));
      const float2 hs = q ? make_float2(__fadd_rn(st.hc.y, st.hc.w), __fadd_rn(st.hc.z, hr))
                          : make_float2(__fadd_rn(hl, st.hc.y), __fadd_rn(st.hc.x, st.hc.z));
      const float2 lap = __ffma2_rn(make_float2(-4.f, -4.f), hk, __fadd2_rn(vs, hs));
      const float2 cb = q ? wv_hi(cb4) : wv_lo(cb4);
      o[q] = __ffma2_rn(make_float2(k.a, k.a), hk,
                        __ffma2_rn(make_float2(k.b, k.b), __fmul2_rn(__fmul2_rn(cb, cb), cb),
                                   __fmul2_rn(make_float2(-k.kappa, -k.kappa), lap)));
    }
    qn = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
  }
  // phi^{n+1} of row a - 2 (psi rows a - 3, a - 2, a - 1; phih row a - 2)
  float4 out;
  {
    const float ql = __shfl_up_sync(WV_FULL, st.qc.w, 1), qr = __shfl_down_sync(WV_FULL, st.qc.x, 1);
    float2 o[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2 qk = q ? wv_hi(st.qc) : wv_lo(st.qc);
      const float2 vs = __fadd2_rn(q ? wv_hi(st.qu) : wv_lo(st.qu), q ? wv_hi(qn) : wv_lo(qn));
      const float2 hs = q ? make_float2(__fadd_rn(st.qc.y, st.qc.w), __fadd_rn(st.qc.z, qr))
                          : make_float2(__fadd_rn(ql, st.qc.y), __fadd_rn(st.qc.x, st.qc.z));
      const float2 lap = __ffma2_rn(make_float2(-4.f, -4.f), qk, __fadd2_rn(vs, hs));
      o[q] = __ffma2_rn(make_float2(k.dtG, k.dtG), lap, q ? wv_hi(st.hu) : wv_lo(st.hu));
    }
    out = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
  }
  st.pm = st.pc;
  st.pc = pn;
  st.hu = st.hc;
  st.hc = hn;
  st.qu = st.qc;
  st.qc = qn;
  return out;
}

// One strip segment of an Lx x Ly lattice whose u* planes are S values apart:
// lanes cover columns x0 .. x0 + 127 (x0 a multiple of 4, wrapped around the
// lattice as often as needed), output rows ys .. ys + NY - 1 (wrapped reads).
template <int SUB>
__device__ __forceinline__ void fd2d_wave_strip(const float *__restrict__ phi_in, const float *__restrict__ u,
                                                float *__restrict__ phi_out, const KParams<float> &p,
                                                const int Lx, const int Ly, const long long S, const int x0,
                                                const int ys, const int NY) {
  using G = Wave<SUB>;
  extern __shared__ __align__(16) float wv_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, c = 4 * lane;
  const int J = NY + 2 * G::HY;  // input rows of the segment
  const int T = G::ticks(NY);
  const WvConst k{p.dt, p.dtG, p.a, p.b, p.kappa, p.cubic_at_half != 0};
  // an output lane writes its float4 when the columns are inside the strip's
  // written range and the lattice (Lx % 4 == 0: a group never straddles Lx)
  const bool col_ok = c >= G::HX && c < G::HX + G::TX && x0 + c < Lx;
  float *coef = wv_smem + G::OFF_C + c;  // [3][CR][128], this lane's columns
  float *hand = wv_smem + G::OFF_H + c;  // [HR][128]
  auto ld_coef = [&](int r) {
    const int sc = (r & (G::CR - 1)) * WV_W;
    return WvCoef{wv_ld(coef + sc), wv_ld(coef + G::CR * WV_W + sc), wv_ld(coef + 2 * G::CR * WV_W + sc)};
  };
  pdl_wait();  // u*(t) comes from the collide kernel, phi(t) from the previous FD launch
  pdl_trigger();
  WvSub s1{}, s2{};
  if (warp == 0) {
    // ---- warp A: inputs, coefficients, substeps 1 and 2 ----
    float *rphi = wv_smem + G::OFF_PHI + c, *ru = wv_smem + G::OFF_U + c, *rv = wv_smem + G::OFF_V + c;
    const int gx = wrapi(x0 + c, Lx);
    int yi = wrapi(ys - G::HY, Ly);  // global row of the next input row to issue
    auto issue = [&](int j) {        // input row j of the segment into ring slot j % 8
      if (j < J) {
        const long long off = (long long)yi * Lx + gx;
        const int sl = (j & (WV_IR - 1)) * WV_W;
        wv_cp16(rphi + sl, phi_in + off);
        wv_cp16(ru + sl, u + off);
        wv_cp16(rv + sl, u + S + off);
        yi = yi + 1 == Ly ? 0 : yi + 1;
      }
      wv_commit();
    };
#pragma unroll 1
    for (int j = 0; j < WV_D; ++j) issue(j);
    float4 vm = make_float4(0.f, 0.f, 0.f, 0.f), vc = vm;  // v of rows t - 2, t - 1
    auto tick = [&](int t) {
      issue(t + WV_D);
      wv_wait_d();  // rows <= t have landed (this lane's copies)
      const int st = (t & (WV_IR - 1)) * WV_W, stm = ((t - 1) & (WV_IR - 1)) * WV_W;
      const float4 pn = wv_ld(rphi + st), vn = wv_ld(rv + st), uc = wv_ld(ru + stm);
      const WvCoef cf = wv_coef(uc, vm, vc, vn, k.dt);  // row a = t - 1
      vm = vc;
      vc = vn;
      {
        const int sc = ((t - 1) & (G::CR - 1)) * WV_W;
        wv_st(coef + sc, cf.c0);
        wv_st(coef + G::CR * WV_W + sc, cf.t1);
        wv_st(coef + 2 * G::CR * WV_W + sc, cf.t2);
      }
      const float4 o1 = wv_substep(s1, pn, cf, k);              // phi_1(a - 2)
      const float4 o2 = wv_substep(s2, o1, ld_coef(t - 4), k);  // phi_2(a - 5), coef(a - 3)
      if constexpr (SUB == 4) {
        wv_st(hand + ((t - 6) & (G::HR - 1)) * WV_W, o2);
      } else {
        const int r = t - 6;  // relative input row of the output
        if (r >= G::HY && r < G::HY + NY && ys + r - G::HY < Ly && col_ok)
          wv_st(phi_out + (long long)(ys + r - G::HY) * Lx + (x0 + c), o2);
      }
    };
    // two ticks per iteration: the second tick's early phases overlap the
    // first's late ones; warp B reads what both wrote after the barrier
#pragma unroll 1
    for (int t = 0; t < T; t += 2) {
      tick(t);
      tick(t + 1);
      if constexpr (SUB == 4) wv_bar<G::NT>();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if constexpr (SUB == 4) {
    // ---- warp B: substeps 3 and 4 of row b = t - 9 ----
    auto tick = [&](int t) {
      const float4 pn = wv_ld(hand + ((t - 8) & (G::HR - 1)) * WV_W);  // phi_2 of row b + 1
      const float4 o3 = wv_substep(s1, pn, ld_coef(t - 9), k);          // phi_3(b - 2)
      const float4 o4 = wv_substep(s2, o3, ld_coef(t - 12), k);         // phi_4(b - 5)
      const int r = t - 14;
      if (r >= G::HY && r < G::HY + NY && ys + r - G::HY < Ly && col_ok)
        wv_st(phi_out + (long long)(ys + r - G::HY) * Lx + (x0 + c), o4);
    };
#pragma unroll 1
    for (int t = 0; t < T; t += 2) {
      tick(t);
      tick(t + 1);
      wv_bar<G::NT>();
    }
  }
}

template <int SUB>
__global__ void __launch_bounds__(Wave<SUB>::NT)
    fd2d_wave_kernel(const float *__restrict__ phi_in, const float *__restrict__ u,
                     float *__restrict__ phi_out, KParams<float> p, int NY) {
  fd2d_wave_strip<SUB>(phi_in, u, phi_out, p, p.Lx, p.Ly, (long long)p.Lx * p.Ly,
                       blockIdx.x * Wave<SUB>::TX - Wave<SUB>::HX, blockIdx.y * NY, NY);
}

// The same update for many independent lattices packed end to end (one plane
// per field over all of them, u*_y ST values after u*_x): CTA b takes the
// item items[b] = (instance, strip, first output row, output rows).
template <int SUB>
__global__ void __launch_bounds__(Wave<SUB>::NT)
    fd2d_wave_batch_kernel(const float *__restrict__ phi_in, const float *__restrict__ u,
                           float *__restrict__ phi_out, long long ST, const TiledInst *__restrict__ inst,
                           const int4 *__restrict__ items, KParams<float> p) {
  const int4 it = items[blockIdx.x];
  const TiledInst I = inst[it.x];
  fd2d_wave_strip<SUB>(phi_in + I.off, u + I.off, phi_out + I.off, p, I.Lx, I.Ly, ST,
                       it.y * Wave<SUB>::TX - Wave<SUB>::HX, it.z, it.w);
}

template <int SUB>
cudaError_t fd2d_wave_one(lbm_handle *h, const KParams<float> &p, const float *src, float *dst, int NY) {
  using G = Wave<SUB>;
  dim3 grid((p.Lx + G::TX - 1) / G::TX, (p.Ly + NY - 1) / NY);
  return launch_pdl(fd2d_wave_kernel<SUB>, grid, dim3(G::NT), G::smem, h->stream, src,
                    static_cast<const float *>(h->u), dst, p, NY);
}

}  // namespace

bool fd2d_wave_eligible(const lbm_handle *h) {
  auto al = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  return h->dims == 2 && h->P.precision != LBM_F64 && h->P.adv_variant != LBM_ADV_FLUX &&
         h->P.Lx % 4 == 0 && h->m >= 2 && al(h->u) && al(h->phi[0]) && al(h->phi[1]) && al(h->phi[2]);
}

// CTAs of one wave (resident CTAs per SM x SMs) and strips of the lattice, for
// a segment height that makes the grid whole waves
int fd2d_wave_slots(int sub, int *strips, int Lx) {
  int dev = 0, sms = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  int tx;
  if (sub == 4) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fd2d_wave_kernel<4>, Wave<4>::NT, Wave<4>::smem);
    tx = Wave<4>::TX;
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fd2d_wave_kernel<2>, Wave<2>::NT, Wave<2>::smem);
    tx = Wave<2>::TX;
  }
  *strips = (Lx + tx - 1) / tx;
  return e == cudaSuccess ? nb * sms : 0;
}

// dynamic shared memory beyond the default 48 KB
cudaError_t fd2d_wave_configure() {
  cudaError_t e = cudaFuncSetAttribute(fd2d_wave_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Wave<4>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd2d_wave_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Wave<2>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd2d_wave_batch_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Wave<2>::smem);
  return e;
}

int fd2d_wave_batch_strip_columns() { return Wave<2>::TX; }

cudaError_t fd2d_wave_batch(const float *phi_in, const float *u, float *phi_out, long long ST,
                            const TiledInst *inst, const int4 *items, int nitems, const KParams<float> &p,
                            cudaStream_t s, bool pdl) {
  return launch_ex(pdl, fd2d_wave_batch_kernel<2>, dim3(nitems), dim3(Wave<2>::NT), Wave<2>::smem, s, phi_in, u,
                   phi_out, ST, inst, items, p);
}

// sub = 2 or 4 substeps in one launch; NY = output rows of a segment
cudaError_t fd2d_wave(lbm_handle *h, const KParams<float> &p, const float *src, float *dst, int sub,
                      int NY) {
  if (NY < 1) return cudaErrorInvalidValue;
  if (sub == 4) return fd2d_wave_one<4>(h, p, src, dst, NY);
  if (sub == 2) return fd2d_wave_one<2>(h, p, src, dst, NY);
  return cudaErrorInvalidValue;
}

}  // namespace hlbm
