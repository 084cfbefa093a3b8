// conv_tcgen05.cu -- periodic 3x3 convolution of the learned surrogate as an
// implicit GEMM on the tcgen05 tensor cores.
//
// One tile is 128 consecutive pixels of one image row (the MMA's M = 128); the
// output channels are N (16 or 32) and the reduction runs over the 9 taps x
// the input channels, K = 16 per instruction.  A CTA walks runs of tiles down
// a 128-pixel column strip and keeps the input rows it needs in a ring of
// shared-memory slots, each row 130 pixels wide (periodic halo of one); the A
// operand of tap (dy, dx) is a view of the slot of row y + dy shifted by dx
// pixels, so a tile stages one new row and the 9 taps need no copies.
//
// Shared-memory operand layout (K-major, no swizzle): a "core matrix" is 8
// rows x 16 bytes stored as 128 contiguous bytes.  Staged rows are kept as
// one plane per 8-channel chunk, [chunk][slot][pixel][8 channels], so 8
// consecutive pixels of one chunk form a core matrix, consecutive 8-pixel
// groups are 128 bytes apart (the stride-dimension offset) and the two chunks
// of one K = 16 step are one plane apart (the leading-dimension offset).  The
// weights use the same form, [K chunk][output channel][8].
//
// Roles per CTA (persistent): a loader warp stages rows with cp.async, an MMA
// warp issues the MMAs (one elected lane, warp-uniform operands) into FP32
// accumulators in tensor memory, four epilogue warps read them back with
// tcgen05.ld; they meet only on mbarriers, and every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "conv_tc.cuh"

namespace {

typedef __nv_bfloat16 bf16;
using hlbm::conv_act_index;
using hlbm::CONV_LINEAR_F32;
using hlbm::CONV_MASK;
using hlbm::CONV_RELU;

constexpr int TM = 128;        // pixels per tile (MMA M)
constexpr int RW = TM + 2;     // staged pixels per row
constexpr int NTHREADS = 192;  // epilogue warps 0-3 (32 accumulator lanes each), MMA warp 4, loader warp 5
constexpr int TMEM_COLS = 64;  // two accumulators of up to 32 FP32 columns

__device__ int g_conv_tc_err = 0;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, leading- and stride-
// dimension byte offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Issued by the whole warp in uniform control flow (so the operands can stay
// warp-uniform); elect.sync picks the one lane that issues the instruction.
__device__ __forceinline__ void mma_bf16_ss(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ uint64_t globaltimer();

// spin on a non-blocking test (the single-thread roles: no suspend quantum
// between the phase completing and the thread seeing it); bounded like mbar_wait
__device__ __forceinline__ bool mbar_poll(uint32_t addr, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer() - t0 > 500000000ull) return false;
  }
}

// bounded: gives up after half a second of global time and reports it
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer() - t0 > 500000000ull) return false;
  }
}

// 32 consecutive FP32 columns of this warp's 32 lanes (one pixel per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[32]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
#pragma unroll
  for (int j = 16; j < 32; ++j) v[j] = 0.f;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

template <int CIN, int NM>
struct TcGeom {
  static constexpr int CH = CIN / 8;       // 8-channel chunks per pixel
  static constexpr int SLOTS = 4;          // staged input rows
  static constexpr int NACC = 2;           // accumulators in tensor memory
  // +32 bytes: the chunk planes start in different shared-memory bank groups
  static constexpr int PLANE_A = SLOTS * RW * 16 + 32;
  static constexpr int ABYTES = CH * PLANE_A;
  static constexpr int KCH = 9 * CH;       // K chunks of a weight row
  static constexpr int PLANE_B = NM * 16;  // bytes of one weight chunk plane
  static constexpr int BBYTES = KCH * PLANE_B;
  static constexpr int NBAR = 2 * NACC + 2 * SLOTS;
  static constexpr int SMEM = ABYTES + BBYTES + NM * 4 + 8 * NBAR + 16;
  static_assert(PLANE_A % 16 == 0 && ABYTES % 16 == 0 && BBYTES % 16 == 0, "16-byte planes");
  static_assert(NACC * 32 <= TMEM_COLS, "accumulators fit the allocation");
};

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(addr)
               : "memory");
}

// Work item = a run of R tiles stacked in y (one 128-pixel column strip, rows
// y0 .. y0 + R - 1 of one image); CTAs take items round-robin and all roles
// walk the same sequence, numbering tiles g = 0, 1, ... and staged rows
// q = 0, 1, ... per CTA (row q in ring slot q % SLOTS; an item stages its
// rows y0 - 1 .. y0 + R).
//
// Loader (warp 5): copies each row's 130 staged pixels (periodic halo of one)
// into its slot with cp.async once the slot's previous row has been released
// on sfree[slot], and announces it on loaded[slot].
// MMA issuer (warp 4, one elected lane issues): per tile waits for its three rows and for its
// accumulator (aempty), issues the 9 x Cin/16 MMAs into accumulator g % NACC
// and commits them to full[g % NACC] and, for each row this tile reads last,
// to sfree[slot] (a commit arrives once all MMAs issued so far are complete).
// Epilogue (warps 0-3; warp w reads tensor-memory lanes 32w .. 32w + 31): wait
// full[g % NACC], load the accumulator, release it on aempty[g % NACC] (four
// arrivals), then bias/ReLU/mask, convert and store.
// Every barrier is refilled only by the side that waits on it, so a parity
// wait can never fall two phases behind; every wait is bounded.
template <int CIN, int NM, int COUTG, int EPI>
__global__ void __launch_bounds__(NTHREADS, 4)
    conv_tc_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ w, int ks,
                   const float *__restrict__ bias, const bf16 *__restrict__ mask, int N, int H,
                   int W, int R, bf16 *__restrict__ out_bf, float *__restrict__ out_f) {
  using G = TcGeom<CIN, NM>;
  constexpr int S = G::SLOTS, NACC = G::NACC, CH = G::CH, COCH = COUTG / 8;
  static_assert(CIN % 16 == 0 && (NM == 16 || NM == 32) && COUTG <= NM && COUTG % 8 == 0, "shape");
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *sB = smem + G::ABYTES;
  float *sbias = reinterpret_cast<float *>(sB + G::BBYTES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(sbias + NM);  // full, aempty, loaded, sfree
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + G::NBAR);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = W / TM, runs_y = (H + R - 1) / R;
  const long long nitems = (long long)N * runs_y * tiles_x;

  // weights -> [K chunk][co][8]; rows co >= COUTG are zero
  for (int k = tid; k < G::KCH * NM; k += NTHREADS) {
    const int co = k / G::KCH, kc = k - co * G::KCH;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (co < COUTG) v = __ldg(reinterpret_cast<const uint4 *>(w + (size_t)co * ks + kc * 8));
    *reinterpret_cast<uint4 *>(sB + kc * G::PLANE_B + co * 16) = v;
  }
  if (tid < NM) sbias[tid] = (EPI != CONV_MASK && tid < COUTG) ? bias[tid] : 0.f;
  const uint32_t full0 = smem_u32(bars), aempty0 = full0 + 8 * NACC, loaded0 = aempty0 + 8 * NACC,
                 sfree0 = loaded0 + 8 * S;
  if (tid == 0) {
    for (int k = 0; k < NACC; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * k), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(aempty0 + 8 * k), "r"(4) : "memory");
    }
    for (int k = 0; k < S; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(loaded0 + 8 * k), "r"(32) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sfree0 + 8 * k), "r"(1) : "memory");
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t abase = smem_u32(smem), bbase = smem_u32(sB);
  // a wait that also gives up once another role has given up
  auto wait = [&](uint32_t bar, uint32_t parity) { return !*abort_flag && mbar_wait(bar, parity); };
  auto poll = [&](uint32_t bar, uint32_t parity) { return !*abort_flag && mbar_poll(bar, parity); };

  if (warp == 5) {
    // ---------------- loader (warp 5) ----------------
    // lane l copies chunk l % CH of pixels l / CH + (32 / CH) i of a row with
    // cp.async (16 bytes each); each lane then waits for its own copies,
    // fences them towards the async proxy and arrives on loaded[slot]
    // (32 arrivals).  Rows are requested DEPTH ahead of their arrival; before
    // blocking on a slot, every requested row is completed and announced, so
    // the MMA issuer can always make progress.
    constexpr int DEPTH = 2;
    constexpr int PIX_STEP = 32 / CH;
    const int cl = lane % CH, jl = lane / CH;
    long long q = 0, qa = 0;  // next row to request; next row to announce
    bool ok = true;
    auto announce = [&](long long qq) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(loaded0 + 8 * (uint32_t)(qq % S));
    };
    auto flush = [&]() {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      for (; qa < q; ++qa) announce(qa);
    };
    for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int xt = (int)(item % tiles_x);
      const long long it = item / tiles_x;
      const int y0 = (int)(it % runs_y) * R;
      const long long row0 = (it / runs_y) * (long long)H;  // n H
      const int rows = min(R, H - y0);
      const int x0 = xt * TM;
      for (int r = 0; r < rows + 2; ++r, ++q) {
        const int slot = (int)(q % S);
        if (q >= S) {
          const uint32_t bar = sfree0 + 8 * slot, par = (uint32_t)(q / S - 1) & 1u;
          uint32_t done;
          asm volatile(
              "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
              "selp.u32 %0, 1, 0, p;\n\t}\n"
              : "=r"(done)
              : "r"(bar), "r"(par)
              : "memory");
          if (!done) {
            flush();
            if (!(ok = poll(bar, par))) break;
          }
        }
        int gy = y0 - 1 + r;
        gy = gy < 0 ? gy + H : (gy >= H ? gy - H : gy);
        const bf16 *plane = in + conv_act_index(row0 + gy, cl, 0, W, CH);
        const bf16 *src = plane + (long long)(x0 + jl - 1) * 8;
        uint32_t dst = abase + cl * G::PLANE_A + (slot * RW + jl) * 16;
#pragma unroll 4
        for (int j = jl; j < RW; j += PIX_STEP) {
          const bf16 *sp = src;
          if (j == 0 && x0 == 0) sp = plane + (long long)(W - 1) * 8;
          if (j == RW - 1 && x0 + TM == W) sp = plane;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(sp) : "memory");
          src += PIX_STEP * 8;
          dst += PIX_STEP * 16;
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (q + 1 - qa > DEPTH) {  // the oldest requested row has had DEPTH rows' time
          asm volatile("cp.async.wait_group %0;" ::"n"(DEPTH) : "memory");
          announce(qa++);
        }
      }
    }
    if (ok) flush();
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(&g_conv_tc_err, 1);
    }
  } else if (warp == 4) {
    // ---------------- MMA issuer (warp 4, one elected lane issues) ----------------
    constexpr uint32_t IDESC = instr_desc(TM, NM);
    // descriptors of slot 0 / weight chunk 0; start addresses advance in
    // 16-byte units and stay below 2^18 bytes, so they never carry out of
    // their 14-bit field
    const uint64_t a_desc0 = smem_desc(abase, G::PLANE_A, 128);
    const uint64_t b_desc0 = smem_desc(bbase, G::PLANE_B, 128);
    auto commit = [&](uint32_t bar) { mma_commit(bar); };
    int g = 0;
    long long qbase = 0;
    bool ok = true;
    for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const long long it = item / tiles_x;
      const int y0 = (int)(it % runs_y) * R;
      const int rows = min(R, H - y0);
      for (int t = 0; t < rows && ok; ++t, ++g) {
        const long long q0 = qbase + t;
        if (g >= NACC) ok = poll(aempty0 + 8 * (g % NACC), (uint32_t)(g / NACC - 1) & 1u);
        for (int d = 0; d < 3 && ok; ++d)
          ok = poll(loaded0 + 8 * (uint32_t)((q0 + d) % S), (uint32_t)((q0 + d) / S) & 1u);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = (uint32_t)(g % NACC);
        const int s0 = (int)(q0 % S);
        const int s1 = s0 + 1 == S ? 0 : s0 + 1, s2 = s1 + 1 == S ? 0 : s1 + 1;
        // descriptors differ only in the start address (bits 0..13)
        const uint64_t adesc[3] = {a_desc0 + (uint64_t)(s0 * RW), a_desc0 + (uint64_t)(s1 * RW),
                                   a_desc0 + (uint64_t)(s2 * RW)};
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3, dx = tap % 3;
#pragma unroll
          for (int kk = 0; kk < CIN / 16; ++kk) {
            const uint64_t da = adesc[dy] + (uint64_t)((2 * kk * G::PLANE_A) / 16 + dx);
            const uint64_t db = b_desc0 + (uint64_t)(((tap * CH + 2 * kk) * G::PLANE_B) / 16);
            mma_bf16_ss(tmem + acc * 32, da, db, IDESC, (tap | kk) != 0);
          }
        }
        commit(full0 + 8 * acc);
        // rows read for the last time by this tile
        commit(sfree0 + 8 * s0);
        if (t == rows - 1) {
          commit(sfree0 + 8 * s1);
          commit(sfree0 + 8 * s2);
        }
      }
      qbase += rows + 2;
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(&g_conv_tc_err, 1);
      if (g > 0) mbar_wait(full0 + 8 * ((g - 1) % NACC), (uint32_t)((g - 1) / NACC) & 1u);
    }
  } else if (warp < 4) {
    // ---------------- epilogue ----------------
    int g = 0;
    bool ok = true;
    for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int xt = (int)(item % tiles_x);
      const long long q = item / tiles_x;
      const int y0 = (int)(q % runs_y) * R;
      const long long row0 = (q / runs_y) * (long long)H;
      const int rows = min(R, H - y0);
      const int x = xt * TM + warp * 32 + lane;
      for (int t = 0; t < rows; ++t, ++g) {
        const uint32_t acc = (uint32_t)(g % NACC);
        if (!wait(full0 + 8 * acc, (uint32_t)(g / NACC) & 1u)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float v[32];
        const uint32_t taddr = tmem + acc * 32 + ((uint32_t)(warp * 32) << 16);
        if constexpr (NM == 32) tmem_ld32(taddr, v);
        else tmem_ld16(taddr, v);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(aempty0 + 8 * acc);
        const long long row = row0 + y0 + t;
        if constexpr (EPI == CONV_LINEAR_F32) {
          float4 *o = reinterpret_cast<float4 *>(out_f + (row * W + x) * COUTG);
#pragma unroll
          for (int c = 0; c < COUTG / 4; ++c)
            o[c] = make_float4(v[4 * c] + sbias[4 * c], v[4 * c + 1] + sbias[4 * c + 1],
                               v[4 * c + 2] + sbias[4 * c + 2], v[4 * c + 3] + sbias[4 * c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < COCH; ++c) {
            const long long o = conv_act_index(row, c, x, W, COCH);
            float e[8];
            if constexpr (EPI == CONV_RELU) {
#pragma unroll
              for (int j = 0; j < 8; ++j) e[j] = fmaxf(v[8 * c + j] + sbias[8 * c + j], 0.f);
            } else {
              const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(mask + o));
              const bf16 *mb = reinterpret_cast<const bf16 *>(&mk);
#pragma unroll
              for (int j = 0; j < 8; ++j) e[j] = __bfloat162float(mb[j]) > 0.f ? v[8 * c + j] : 0.f;
            }
            *reinterpret_cast<uint4 *>(out_bf + o) =
                make_uint4(pack_bf16(e[0], e[1]), pack_bf16(e[2], e[3]), pack_bf16(e[4], e[5]),
                           pack_bf16(e[6], e[7]));
          }
        }
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(&g_conv_tc_err, 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

template <int CIN, int NM, int COUTG, int EPI>
cudaError_t launch(const void *in, const void *w, int ks, const float *bias, const void *mask,
                   int N, int H, int W, void *out_bf, float *out_f, cudaStream_t s) {
  using G = TcGeom<CIN, NM>;
  auto *kern = conv_tc_kernel<CIN, NM, COUTG, EPI>;
  static int ctas_per_sm = -1;
  static int sms = 0;
  static std::once_flag once;
  static cudaError_t init_err = cudaSuccess;
  std::call_once(once, [&] {
    init_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (init_err == cudaSuccess)
      init_err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared);
    int dev = 0;
    if (init_err == cudaSuccess) init_err = cudaGetDevice(&dev);
    if (init_err == cudaSuccess)
      init_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // resident CTAs per SM from the shared memory (plus the driver's
    // reservation per CTA), the threads, and the 512 tensor-memory columns
    int smem_sm = 0, reserved = 0;
    if (init_err == cudaSuccess)
      init_err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (init_err == cudaSuccess)
      init_err = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa{};
    if (init_err == cudaSuccess) init_err = cudaFuncGetAttributes(&fa, kern);
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp
    const int by_regs = 65536 / std::max(1, warp_regs * (NTHREADS / 32));
    ctas_per_sm = std::min({smem_sm / (G::SMEM + reserved), 2048 / NTHREADS, 512 / TMEM_COLS, by_regs});
    if (std::getenv("HLBM_CONV_VERBOSE")) {
      int api = -1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&api, kern, NTHREADS, G::SMEM);
      std::fprintf(stderr, "hlbm conv_tc occupancy: %d CTAs/SM by resources, %d by the occupancy API\n",
                   ctas_per_sm, api);
    }
  });
  if (init_err != cudaSuccess) return init_err;
  if (ctas_per_sm < 1) return cudaErrorInvalidConfiguration;
  // runs of R tiles in y: about one run per resident CTA
  const long long ctas = (long long)ctas_per_sm * sms;
  const long long ntiles = (long long)N * H * (W / TM);
  const int R = (int)std::max<long long>(1, std::min<long long>(H, (ntiles + ctas - 1) / ctas));
  const long long nitems = (long long)N * ((H + R - 1) / R) * (W / TM);
  const long long grid = std::min(nitems, ctas);
  if (std::getenv("HLBM_CONV_VERBOSE"))
    std::fprintf(stderr,
                 "hlbm conv_tc cin=%d n=%d epi=%d %dx%dx%d: %d CTAs/SM x %d SMs, smem %d B, "
                 "runs of %d tiles, grid %lld\n",
                 CIN, NM, EPI, N, H, W, ctas_per_sm, sms, G::SMEM, R, grid);
  kern<<<(unsigned)grid, NTHREADS, G::SMEM, s>>>(
      static_cast<const bf16 *>(in), static_cast<const bf16 *>(w), ks, bias,
      static_cast<const bf16 *>(mask), N, H, W, R, static_cast<bf16 *>(out_bf), out_f);
  return cudaGetLastError();
}

}  // namespace

namespace hlbm {

bool conv_tc_supported(int cinp, int coutp, int W) {
  if (W < TM || W % TM) return false;
  return (cinp == 16 || cinp == 32) && (coutp == 8 || coutp == 16 || coutp == 32);
}

cudaError_t conv_tc(int cinp, int coutp, int epi, const void *in, const void *w, int ks,
                    const float *bias, const void *mask, int N, int H, int W, void *out_bf,
                    float *out_f, cudaStream_t s) {
  if (N < 1 || H < 1 || W < TM || W % TM || ks < 9 * cinp || ks % 8) return cudaErrorInvalidValue;
#define CASE(CI, NMM, CO, E)                                                   \
  if (cinp == CI && coutp == CO && epi == E)                                   \
    return launch<CI, NMM, CO, E>(in, w, ks, bias, mask, N, H, W, out_bf, out_f, s);
  CASE(16, 32, 32, CONV_RELU) CASE(32, 32, 32, CONV_RELU) CASE(16, 16, 16, CONV_RELU)
  CASE(32, 16, 8, CONV_LINEAR_F32) CASE(16, 16, 8, CONV_LINEAR_F32)
  CASE(32, 32, 32, CONV_MASK) CASE(16, 32, 32, CONV_MASK) CASE(16, 16, 16, CONV_MASK)
#undef CASE
  return cudaErrorInvalidValue;
}

int conv_tc_error(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_conv_tc_err, sizeof v) != cudaSuccess) return -1;
  if (reset && v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_conv_tc_err, &zero, sizeof zero);
  }
  return v;
}

}  // namespace hlbm
