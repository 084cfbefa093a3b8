// surrogate.cu -- the learned surrogate: a stack of periodic 3x3 convolutions
// (4 -> C -> ... -> C -> 4 channels, ReLU between layers) that maps the
// normalised state x_t = (phi, u*_x, u*_y, n - 1) of a 2D lattice to the
// normalised change x_{t+k} - x_t, with BF16 weights and activations and FP32
// accumulation on the tensor cores, its backward pass and Adam training, and
// the coupling to a lattice handle (pack the state, advance by the network,
// check a residual, fall back to the plain scheme).  The paper has no
// counterpart; the network is judged by the paper's observables.
//
// Layouts: activations (BF16) are stored row-chunk planar, [n][y][c / 8][x][8]:
// for each image row, the 8-channel chunks of all its pixels form contiguous
// planes, so one operand plane of a row is one contiguous copy (see
// conv_act_index); channel counts are padded (the 4-channel input to 16,
// hidden layers C = 32); the last layer's FP32 output is [p][8];
// weights [Cout_p][KS] with K = 9 Cin_p ordered (tap, ci), tap = (dy+1)*3 +
// (dx+1), KS = K + 8 (bank-conflict padding, always zero).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "conv_tc.cuh"
#include "lbm_common.cuh"

typedef __nv_bfloat16 bf16;

namespace {

using namespace hlbm;

constexpr int TILE_H = 8, TILE_W = 16;  // pixels per CTA (8 warps x one row of 16)

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned ld32(const bf16 *p) {
  return *reinterpret_cast<const unsigned *>(p);
}

constexpr int EPI_RELU = CONV_RELU, EPI_LINEAR_F32 = CONV_LINEAR_F32, EPI_MASK = CONV_MASK;

// out[p, co] = sum_{tap, ci} in[p + tap, ci] w[co][tap, ci] (periodic), then
//   EPI_RELU:       bf16 max(. + bias, 0)
//   EPI_LINEAR_F32: fp32 . + bias
//   EPI_MASK:       bf16 . * (mask[p, co] > 0)    (backward through a ReLU)
template <int CINP, int COUTP, int EPI>
__global__ void __launch_bounds__(256)
    conv_mma_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ w,
                    const float *__restrict__ bias, const bf16 *__restrict__ mask, int H, int W,
                    bf16 *__restrict__ out_bf, float *__restrict__ out_f) {
  constexpr int PS = CINP + 8;          // pixel stride in shared memory (bf16)
  constexpr int KS = 9 * CINP + 8;      // weight row stride (bf16)
  constexpr int RH = TILE_H + 2, RW = TILE_W + 2;
  __shared__ __align__(16) bf16 sin[RH * RW * PS];
  __shared__ __align__(16) bf16 sw[COUTP * KS];
  const int x0 = blockIdx.x * TILE_W, y0 = blockIdx.y * TILE_H, n = blockIdx.z;
  const int tid = threadIdx.x;
  const long long img = (long long)n * H * W;
  // input tile with a periodic halo of 1, 16-byte copies
  constexpr int VPP = CINP / 8;  // 16-byte vectors per pixel
  for (int k = tid; k < RH * RW * VPP; k += 256) {
    const int pix = k / VPP, v = k - pix * VPP;
    const int r = pix / RW, c = pix - r * RW;
    int gy = y0 + r - 1, gx = x0 + c - 1;
    gy = gy < 0 ? gy + H : (gy >= H ? gy - H : gy);
    gx = gx < 0 ? gx + W : (gx >= W ? gx - W : gx);
    const uint4 val = *reinterpret_cast<const uint4 *>(in + conv_act_index(img / W + gy, v, gx, W, VPP));
    *reinterpret_cast<uint4 *>(sin + pix * PS + v * 8) = val;
  }
  for (int k = tid; k < COUTP * KS / 8; k += 256)
    reinterpret_cast<uint4 *>(sw)[k] = reinterpret_cast<const uint4 *>(w)[k];
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  float acc[COUTP / 8][4];
#pragma unroll
  for (int j = 0; j < COUTP / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int ty = tap / 3, tx = tap % 3;
    const bf16 *pa0 = sin + ((warp + ty) * RW + g + tx) * PS + 2 * t;
    const bf16 *pa1 = pa0 + 8 * PS;
#pragma unroll
    for (int kb = 0; kb < CINP / 16; ++kb) {
      const unsigned a0 = ld32(pa0 + kb * 16), a1 = ld32(pa1 + kb * 16);
      const unsigned a2 = ld32(pa0 + kb * 16 + 8), a3 = ld32(pa1 + kb * 16 + 8);
#pragma unroll
      for (int j = 0; j < COUTP / 8; ++j) {
        const bf16 *pb = sw + (j * 8 + g) * KS + tap * CINP + kb * 16 + 2 * t;
        mma_bf16(acc[j], a0, a1, a2, a3, ld32(pb), ld32(pb + 8));
      }
    }
  }
  // rows g and g + 8 of the warp's 16 pixels; columns 2t, 2t + 1 of each n-tile
  const int y = y0 + warp;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const long long p = img + (long long)y * W + x0 + g + 8 * half;
    const long long row = img / W + y;
    const int x = x0 + g + 8 * half;
#pragma unroll
    for (int j = 0; j < COUTP / 8; ++j) {
      const int co = j * 8 + 2 * t;
      const long long q = conv_act_index(row, j, x, W, COUTP / 8) + 2 * t;
      float v0 = acc[j][2 * half], v1 = acc[j][2 * half + 1];
      if constexpr (EPI == EPI_LINEAR_F32) {
        *reinterpret_cast<float2 *>(out_f + p * COUTP + co) = make_float2(v0 + bias[co], v1 + bias[co + 1]);
      } else {
        if constexpr (EPI == EPI_RELU) {
          v0 = fmaxf(v0 + bias[co], 0.f);
          v1 = fmaxf(v1 + bias[co + 1], 0.f);
        } else {
          const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + q);
          v0 = __bfloat162float(mk.x) > 0.f ? v0 : 0.f;
          v1 = __bfloat162float(mk.y) > 0.f ? v1 : 0.f;
        }
        *reinterpret_cast<__nv_bfloat162 *>(out_bf + q) = __floats2bfloat162_rn(v0, v1);
      }
    }
  }
}

// Partial weight and bias gradients of one layer over a grid-stride set of
// pixel tiles: dW[co][tap, ci] += dz[p, co] x[p + tap, ci], db[co] += dz[p, co].
// Thread (co, ci4) owns 9 taps x 4 input channels; FP32 throughout.
template <int CINP, int COUTP, int DZS>
__global__ void __launch_bounds__(256)
    conv_wgrad_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ dz, int N, int H, int W,
                      float *__restrict__ partial) {
  // dz has DZS channels per pixel, of which the first COUTP are this layer's
  constexpr int RH = TILE_H + 2, RW = TILE_W + 2;
  constexpr int NT = COUTP * (CINP / 4);  // active threads
  static_assert(NT <= 256, "too many outputs");
  __shared__ float sx[RH * RW][CINP + 1];
  __shared__ float sd[TILE_H * TILE_W][COUTP + 1];
  const int tid = threadIdx.x;
  const int co = tid / (CINP / 4), c4 = (tid % (CINP / 4)) * 4;
  float acc[9][4];
  float accb = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.f;
  const int tiles_x = W / TILE_W, tiles_y = H / TILE_H;
  const long long ntiles = (long long)tiles_x * tiles_y * N;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = (int)(tile / ((long long)tiles_x * tiles_y));
    const int rem = (int)(tile - (long long)n * tiles_x * tiles_y);
    const int y0 = (rem / tiles_x) * TILE_H, x0 = (rem % tiles_x) * TILE_W;
    const long long img = (long long)n * H * W;
    __syncthreads();
    for (int k = tid; k < RH * RW * CINP; k += 256) {
      const int pix = k / CINP, c = k - pix * CINP;
      const int r = pix / RW, cc = pix - r * RW;
      int gy = y0 + r - 1, gx = x0 + cc - 1;
      gy = gy < 0 ? gy + H : (gy >= H ? gy - H : gy);
      gx = gx < 0 ? gx + W : (gx >= W ? gx - W : gx);
      sx[pix][c] = __bfloat162float(x[conv_act_index(img / W + gy, c / 8, gx, W, CINP / 8) + c % 8]);
    }
    for (int k = tid; k < TILE_H * TILE_W * COUTP; k += 256) {
      const int pix = k / COUTP, c = k - pix * COUTP;
      const int r = pix / TILE_W, cc = pix - r * TILE_W;
      sd[pix][c] = __bfloat162float(dz[conv_act_index(img / W + y0 + r, c / 8, x0 + cc, W, DZS / 8) + c % 8]);
    }
    __syncthreads();
    if (tid < NT) {
      for (int p = 0; p < TILE_H * TILE_W; ++p) {
        const int r = p / TILE_W, c = p - r * TILE_W;
        const float d = sd[p][co];
        accb += d;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const float *xr = sx[(r + tap / 3) * RW + c + tap % 3] + c4;
          acc[tap][0] += d * xr[0];
          acc[tap][1] += d * xr[1];
          acc[tap][2] += d * xr[2];
          acc[tap][3] += d * xr[3];
        }
      }
    }
  }
  if (tid < NT) {
    float *out = partial + (size_t)blockIdx.x * (COUTP * 9 * CINP + COUTP);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
      for (int k = 0; k < 4; ++k) out[(co * 9 + tap) * CINP + c4 + k] = acc[tap][k];
    if (c4 == 0) out[COUTP * 9 * CINP + co] = accb;
  }
}

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned &r0, unsigned &r1, unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}

// The same partial weight and bias gradients on the tensor cores.  Per pixel
// tile (TILE_H rows of TILE_W = 16 pixels) and per tile row r, the 16 pixels
// are one K step of
//   C[co][(tap, ci)] += sum_k dz[k, co] x[k + tap, ci]
// by mma.sync m16n8k16 (BF16 operands, FP32 accumulation): A = dz^T (16
// output channels x 16 pixels), B = the input shifted by the tap (16 pixels x
// 8 input channels).  Both are staged in shared memory as 16-byte rows of 8
// channels of one pixel ([chunk][row][x], as in global memory) and read with
// ldmatrix.trans, which turns the pixel-major rows into the row-major A and
// column-major B fragments.  Warp w owns the N tiles w, w + 8, ... of the
// 9 CINP / 8 (tap, 8 channels) tiles; warp 0 also multiplies A by a tile of
// ones, whose columns are the bias gradient sum_k dz[k, co].  COUTP = 8 fills
// the upper half of the 16-row A tile with a copy and drops those rows.
template <int CINP, int COUTP, int DZS>
__global__ void __launch_bounds__(256)
    conv_wgrad_mma_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ dz, int N, int H, int W,
                          float *__restrict__ partial) {
  constexpr int RH = TILE_H + 2, RW = TILE_W + 2;
  constexpr int CJ = CINP / 8, DJ = COUTP / 8;
  constexpr int MT = (COUTP + 15) / 16;  // 16-row tiles of output channels
  constexpr int NT = 9 * CJ;             // 8-column tiles of (tap, input channel)
  constexpr int NTW = (NT + 7) / 8;      // N tiles per warp
  static_assert(TILE_W == 16, "one K step of 16 pixels per tile row");
  __shared__ __align__(16) uint4 sx[CJ * RH * RW];
  __shared__ __align__(16) uint4 sd[DJ * TILE_H * TILE_W];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float acc[MT][NTW][4], accb[MT][4];
#pragma unroll
  for (int mi = 0; mi < MT; ++mi) {
#pragma unroll
    for (int t = 0; t < NTW; ++t) acc[mi][t][0] = acc[mi][t][1] = acc[mi][t][2] = acc[mi][t][3] = 0.f;
    accb[mi][0] = accb[mi][1] = accb[mi][2] = accb[mi][3] = 0.f;
  }
  const unsigned ONES = 0x3F803F80u;  // two BF16 ones
  const unsigned sx_base = static_cast<unsigned>(__cvta_generic_to_shared(sx));
  const unsigned sd_base = static_cast<unsigned>(__cvta_generic_to_shared(sd));
  const int tiles_x = W / TILE_W, tiles_y = H / TILE_H;
  const long long ntiles = (long long)tiles_x * tiles_y * N;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = (int)(tile / ((long long)tiles_x * tiles_y));
    const int rem = (int)(tile - (long long)n * tiles_x * tiles_y);
    const int y0 = (rem / tiles_x) * TILE_H, x0 = (rem % tiles_x) * TILE_W;
    const long long img = (long long)n * H * W;
    __syncthreads();
    for (int k = tid; k < CJ * RH * RW; k += 256) {
      const int j = k / (RH * RW), q = k - j * (RH * RW);
      const int r = q / RW, cc = q - r * RW;
      int gy = y0 + r - 1, gx = x0 + cc - 1;
      gy = gy < 0 ? gy + H : (gy >= H ? gy - H : gy);
      gx = gx < 0 ? gx + W : (gx >= W ? gx - W : gx);
      sx[k] = *reinterpret_cast<const uint4 *>(x + conv_act_index(img / W + gy, j, gx, W, CJ));
    }
    for (int k = tid; k < DJ * TILE_H * TILE_W; k += 256) {
      const int j = k / (TILE_H * TILE_W), q = k - j * (TILE_H * TILE_W);
      const int r = q / TILE_W, cc = q - r * TILE_W;
      sd[k] = *reinterpret_cast<const uint4 *>(dz + conv_act_index(img / W + y0 + r, j, x0 + cc, W, DZS / 8));
    }
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < TILE_H; ++r) {
      unsigned a[MT][4];
#pragma unroll
      for (int mi = 0; mi < MT; ++mi) {
        // lanes 8b .. 8b + 7 address the rows of 8 x 8 block b: blocks 0 / 1
        // are output channels 0-7 / 8-15 of pixels 0-7, blocks 2 / 3 of 8-15
        const int blk = lane >> 3;
        const int chunk = min(2 * mi + (blk & 1), DJ - 1);
        const int kk = (blk >> 1) * 8 + (lane & 7);
        ldsm_x4_t(a[mi], sd_base + 16u * (unsigned)((chunk * TILE_H + r) * TILE_W + kk));
      }
#pragma unroll
      for (int t = 0; t < NTW; ++t) {
        const int nt = warp + 8 * t;
        if (nt < NT) {
          const int tap = nt / CJ, j = nt - tap * CJ;
          // lanes 0-7: pixels 0-7 (block 0), lanes 8-15: pixels 8-15 (block 1)
          const int kk = lane & 15;
          unsigned b0, b1;
          ldsm_x2_t(b0, b1, sx_base + 16u * (unsigned)((j * RH + r + tap / 3) * RW + kk + tap % 3));
#pragma unroll
          for (int mi = 0; mi < MT; ++mi) mma_bf16(acc[mi][t], a[mi][0], a[mi][1], a[mi][2], a[mi][3], b0, b1);
        }
      }
      if (warp == 0) {
#pragma unroll
        for (int mi = 0; mi < MT; ++mi) mma_bf16(accb[mi], a[mi][0], a[mi][1], a[mi][2], a[mi][3], ONES, ONES);
      }
    }
  }
  // C fragment: rows g and g + 8, columns 2q and 2q + 1
  float *out = partial + (size_t)blockIdx.x * (COUTP * 9 * CINP + COUTP);
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int mi = 0; mi < MT; ++mi) {
#pragma unroll
    for (int t = 0; t < NTW; ++t) {
      const int nt = warp + 8 * t;
      if (nt >= NT) continue;
      const int tap = nt / CJ, j = nt - tap * CJ;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int co = 16 * mi + g + 8 * h;
        if (co < COUTP) {
          float *o = out + (co * 9 + tap) * CINP + 8 * j + 2 * q;
          o[0] = acc[mi][t][2 * h];
          o[1] = acc[mi][t][2 * h + 1];
        }
      }
    }
    if (warp == 0 && q == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int co = 16 * mi + g + 8 * h;
        if (co < COUTP) out[COUTP * 9 * CINP + co] = accb[mi][2 * h];
      }
    }
  }
}

// Sums the per-CTA partials in a fixed order into the padded weight (KS
// stride) and bias gradients.
__global__ void wgrad_reduce_kernel(const float *__restrict__ partial, int nparts, int cinp,
                                    int coutp, int ks, float *__restrict__ gw, float *__restrict__ gb) {
  const int per = coutp * 9 * cinp + coutp;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * per + i];
  if (i < coutp * 9 * cinp) {
    const int co = i / (9 * cinp), k = i - co * 9 * cinp;
    gw[co * ks + k] = (float)s;
  } else {
    gb[i - coutp * 9 * cinp] = (float)s;
  }
}

// raw FP32 state [p][4] -> normalised BF16 input, 16 channels (4..15 zero),
// row-chunk planar
__global__ void normalise_kernel(const float *__restrict__ x, long long P, int W,
                                 const float *__restrict__ nrm, bf16 *__restrict__ out) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  __align__(16) bf16 v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = __float2bfloat16(0.f);
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = __float2bfloat16((x[p * 4 + c] - nrm[c]) / nrm[4 + c]);
  const long long row = p / W;
  const int xx = (int)(p - row * W);
  *reinterpret_cast<uint4 *>(out + conv_act_index(row, 0, xx, W, 2)) = *reinterpret_cast<uint4 *>(v);
  *reinterpret_cast<uint4 *>(out + conv_act_index(row, 1, xx, W, 2)) = make_uint4(0u, 0u, 0u, 0u);
}

// MSE of the network output y [p][8] (4 used) against (x1 - x0) / out_std;
// writes the gradient dL/dy as BF16 [p][16] and per-block partial sums.
__global__ void __launch_bounds__(256)
    mse_kernel(const float *__restrict__ y, const float *__restrict__ x0, const float *__restrict__ x1,
               long long P, int W, const float *__restrict__ nrm, bf16 *__restrict__ dz,
               double *__restrict__ part) {
  __shared__ double red[256];
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const double inv = 1.0 / (4.0 * (double)P);
  double acc = 0.0;
  if (p < P) {
    __align__(16) bf16 v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = __float2bfloat16(0.f);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float target = (x1[p * 4 + c] - x0[p * 4 + c]) / nrm[8 + c];
      const float e = y[p * 8 + c] - target;
      acc += (double)e * e;
      v[c] = __float2bfloat16((float)(2.0 * inv) * e);
    }
    const long long row = p / W;
    const int xx = (int)(p - row * W);
    *reinterpret_cast<uint4 *>(dz + conv_act_index(row, 0, xx, W, 2)) = *reinterpret_cast<uint4 *>(v);
    *reinterpret_cast<uint4 *>(dz + conv_act_index(row, 1, xx, W, 2)) = make_uint4(0u, 0u, 0u, 0u);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0] * inv;
}

// x1 = x0 + y * out_std (prediction of the state after one window)
__global__ void predict_kernel(const float *__restrict__ y, const float *__restrict__ x0, long long P,
                               const float *__restrict__ nrm, float *__restrict__ x1) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
#pragma unroll
  for (int c = 0; c < 4; ++c) x1[p * 4 + c] = x0[p * 4 + c] + y[p * 8 + c] * nrm[8 + c];
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void cast_kernel(const float *__restrict__ a, bf16 *__restrict__ b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

// transposed, tap-flipped copy for the backward data pass:
// wt[ci][tap'][co] = w[co][tap][ci], tap' = 8 - tap, co padded to cinp_t
__global__ void transpose_kernel(const float *__restrict__ w, int cinp, int coutp, int ks, int cinp_t,
                                 int ks_t, bf16 *__restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cinp * ks_t) return;
  const int ci = i / ks_t, k = i - ci * ks_t;
  float v = 0.f;
  if (k < 9 * cinp_t) {
    const int tap = k / cinp_t, co = k - tap * cinp_t;
    if (co < coutp) v = w[co * ks + (8 - tap) * cinp + ci];
  }
  wt[i] = __float2bfloat16(v);
}

// n, phi, u* of a lattice (FP64 staging) -> state [p][4] = (phi, ux, uy, n - 1)
__global__ void state_from_staging_kernel(const double *__restrict__ stg, long long S,
                                          float *__restrict__ x) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= S) return;
  x[s * 4 + 0] = (float)stg[S + s];
  x[s * 4 + 1] = (float)stg[2 * S + s];
  x[s * 4 + 2] = (float)stg[3 * S + s];
  x[s * 4 + 3] = (float)(stg[s] - 1.0);
}

// predicted state -> FP64 staging (n, phi, ux, uy); optionally shifts phi so
// that sum phi equals `target_sum` (mass correction by a uniform shift)
__global__ void staging_from_state_kernel(const float *__restrict__ x, long long S, double shift,
                                          double *__restrict__ stg) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= S) return;
  stg[s] = 1.0 + (double)x[s * 4 + 3];
  stg[S + s] = (double)x[s * 4 + 0] - shift;
  stg[2 * S + s] = (double)x[s * 4 + 1];
  stg[3 * S + s] = (double)x[s * 4 + 2];
}

// Rebuild of a 2D FP32-deviation lattice (T = 1/3, body force off) from a
// network state, in FP32: mu = a phi + b phi^3 - kappa lap_D phi (Eqs. 5, 31)
// of the shifted phi on every site, then per site F = -phi d_D mu (Eqs. 28,
// 30), the velocity u = u* - F / 2n (Eq. 18) and f_i - w_i = f_i^eq(n, u) - w_i
// (Eq. 15) stored at r - e_i (pull layout), and phi.  The same construction
// as the library's initialisation, which runs in FP64.
__device__ __forceinline__ int wrap_1(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

__global__ void rebuild_mu_kernel(const float *__restrict__ x, hlbm::KParams<float> p, float shift,
                                  float *__restrict__ mu) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int Lx = p.Lx, Ly = p.Ly;
  if (s >= (long long)Lx * Ly) return;
  const int xx = (int)(s % Lx), yy = (int)(s / Lx);
  auto ph = [&](int dx, int dy) {
    return x[4 * ((long long)wrap_1(yy + dy, Ly) * Lx + wrap_1(xx + dx, Lx))] - shift;
  };
  const float c = ph(0, 0);
  float lap = p.R * ph(-1, -1);
  lap += p.Q * ph(0, -1);
  lap += p.R * ph(1, -1);
  lap += p.Q * ph(-1, 0);
  lap += p.C0 * c;
  lap += p.Q * ph(1, 0);
  lap += p.R * ph(-1, 1);
  lap += p.Q * ph(0, 1);
  lap += p.R * ph(1, 1);
  mu[s] = p.a * c + p.b * c * c * c - p.kappa * lap;
}

__global__ void rebuild_pop_kernel(const float *__restrict__ x, const float *__restrict__ mu,
                                   hlbm::KParams<float> p, float shift, float *__restrict__ hout,
                                   float *__restrict__ phiout) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int Lx = p.Lx, Ly = p.Ly;
  const long long S = (long long)Lx * Ly;
  if (s >= S) return;
  const int xx = (int)(s % Lx), yy = (int)(s / Lx);
  auto m = [&](int dx, int dy) { return mu[(long long)wrap_1(yy + dy, Ly) * Lx + wrap_1(xx + dx, Lx)]; };
  const float gmx = p.N * (m(1, 0) - m(-1, 0)) + p.M * ((m(1, -1) - m(-1, -1)) + (m(1, 1) - m(-1, 1)));
  const float gmy = p.N * (m(0, 1) - m(0, -1)) + p.M * ((m(-1, 1) - m(-1, -1)) + (m(1, 1) - m(1, -1)));
  const float ph = x[4 * s] - shift, n = 1.f + x[4 * s + 3];
  const float ux = x[4 * s + 1] + ph * gmx / (2.f * n), uy = x[4 * s + 2] + ph * gmy / (2.f * n);
  const float uu = ux * ux + uy * uy;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int ex = hlbm::q9_ex(i), ey = hlbm::q9_ey(i);
    const float eu = ex * ux + ey * uy;
    const float h = float(hlbm::q9_w(i)) * ((n - 1.f) + n * (3.f * eu + 4.5f * eu * eu - 1.5f * uu));
    hout[i * S + (long long)wrap_1(yy - ey, Ly) * Lx + wrap_1(xx - ex, Lx)] = h;
  }
  phiout[s] = ph;
}

// |phi| <= cap on the predicted state (the bulk value of the state the
// window starts from bounds phi under the Cahn-Hilliard dynamics)
__global__ void clamp_phi_kernel(float *__restrict__ x, long long S, float cap) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < S) x[s * 4] = fminf(fmaxf(x[s * 4], -cap), cap);
}

// per-block partials of sum phi, sum |phi|, max |phi|, max |u|, max |n - 1|
// over a state; a non-finite phi, u or n makes the maxima infinite
constexpr int NSTAT = 5;
__global__ void __launch_bounds__(256)
    state_stats_kernel(const float *__restrict__ x, long long S, double *__restrict__ part) {
  __shared__ double r[NSTAT][256];
  double sp = 0, sa = 0, mp = 0, mu = 0, mn = 0;
  for (long long s = blockIdx.x * 256LL + threadIdx.x; s < S; s += (long long)gridDim.x * 256) {
    const double ph = x[s * 4], ux = x[s * 4 + 1], uy = x[s * 4 + 2], dn = x[s * 4 + 3];
    sp += ph;
    sa += fabs(ph);
    mp = fmax(mp, fabs(ph));
    mu = fmax(mu, sqrt(ux * ux + uy * uy));
    mn = fmax(mn, fabs(dn));
    if (!isfinite(ph) || !isfinite(ux) || !isfinite(uy) || !isfinite(dn)) mp = mu = mn = INFINITY;
  }
  r[0][threadIdx.x] = sp;
  r[1][threadIdx.x] = sa;
  r[2][threadIdx.x] = mp;
  r[3][threadIdx.x] = mu;
  r[4][threadIdx.x] = mn;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      r[0][threadIdx.x] += r[0][threadIdx.x + k];
      r[1][threadIdx.x] += r[1][threadIdx.x + k];
      for (int q = 2; q < NSTAT; ++q) r[q][threadIdx.x] = fmax(r[q][threadIdx.x], r[q][threadIdx.x + k]);
    }
    __syncthreads();
  }
  if (threadIdx.x < NSTAT) part[blockIdx.x * NSTAT + threadIdx.x] = r[threadIdx.x][0];
}

struct Layer {
  int cin, cout, cinp, coutp, ks, cinp_t, ks_t;
  size_t woff, boff, wtoff;
};

unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace hlbm {
int queue_moments_for(lbm_handle *h);
}

struct lbm_net {
  int C = 32, layers = 6;
  std::vector<Layer> L;
  size_t nw = 0, nb = 0, nwt = 0;
  float *w32 = nullptr, *b32 = nullptr, *gw = nullptr, *gb = nullptr;
  float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
  bf16 *wbf = nullptr, *wtbf = nullptr;
  float *nrm = nullptr;  // in_mean[4], in_std[4], out_std[4]
  float hnrm[12];
  long long cap = 0;     // pixels the workspace holds
  bf16 *act[8] = {nullptr};
  float *yout = nullptr, *x0 = nullptr, *x1 = nullptr;
  void *bk = nullptr;     // a lattice's populations and phi (relaxed surrogate windows)
  size_t bk_cap = 0;
  bf16 *dz[2] = {nullptr, nullptr};
  float *partial = nullptr;
  double *dpart = nullptr;
  int wgrad_ctas = 0;
  long long adam_t = 0;
  std::string msg;
};

namespace {

thread_local std::string g_net_error;

int nfail(lbm_net *net, int code, const std::string &m) {
  if (net) net->msg = m;
  else g_net_error = m;
  return code;
}

#define NCK(net, call, what)                                                   \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return nfail(net, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, \
                   std::string(what) + ": " + cudaGetErrorString(e_));         \
  } while (0)

int ensure_workspace(lbm_net *net, long long P) {
  if (P <= net->cap) return LBM_OK;
  for (auto &a : net->act) if (a) cudaFree(a);
  for (auto &d : net->dz) if (d) cudaFree(d);
  cudaFree(net->yout);
  cudaFree(net->x0);
  cudaFree(net->x1);
  cudaFree(net->dpart);
  for (auto &a : net->act) a = nullptr;
  for (int l = 0; l < net->layers; l++) {
    const int ch = net->L[l].cinp;
    NCK(net, cudaMalloc(&net->act[l], sizeof(bf16) * ch * P), "cudaMalloc");
  }
  NCK(net, cudaMalloc(&net->yout, sizeof(float) * 8 * P), "cudaMalloc");
  NCK(net, cudaMalloc(&net->x0, sizeof(float) * 4 * P), "cudaMalloc");
  NCK(net, cudaMalloc(&net->x1, sizeof(float) * 4 * P), "cudaMalloc");
  for (auto &d : net->dz) NCK(net, cudaMalloc(&d, sizeof(bf16) * std::max(net->C, 16) * P), "cudaMalloc");
  NCK(net, cudaMalloc(&net->dpart, sizeof(double) * (nblk(P, 256) + 4096)), "cudaMalloc");
  net->cap = P;
  return LBM_OK;
}

template <int CINP, int COUTP, int EPI>
cudaError_t conv(const bf16 *in, const bf16 *w, const float *bias, const bf16 *mask, int N, int H,
                 int W, bf16 *ob, float *of, cudaStream_t s) {
  dim3 grid(W / TILE_W, H / TILE_H, N);
  conv_mma_kernel<CINP, COUTP, EPI><<<grid, 256, 0, s>>>(in, w, bias, mask, H, W, ob, of);
  return cudaGetLastError();
}

// the tcgen05 kernel unless the rows are not whole 128-pixel tiles or
// HLBM_CONV_PATH=mma asks for the mma.sync kernel
bool use_tc(int cinp, int coutp, int W) {
  const char *e = std::getenv("HLBM_CONV_PATH");
  if (e && std::strcmp(e, "mma") == 0) return false;
  return conv_tc_supported(cinp, coutp, W);
}

// dispatch on the padded channel counts used by the network (C = 32 or 16)
cudaError_t conv_any(int cinp, int coutp, int epi, const bf16 *in, const bf16 *w, const float *bias,
                     const bf16 *mask, int N, int H, int W, bf16 *ob, float *of, cudaStream_t s) {
  if (use_tc(cinp, coutp, W))
    return conv_tc(cinp, coutp, epi, in, w, 9 * cinp + 8, bias, mask, N, H, W, ob, of, s);
#define CASE(CI, CO, E)                                               \
  if (cinp == CI && coutp == CO && epi == E)                          \
    return conv<CI, CO, E>(in, w, bias, mask, N, H, W, ob, of, s);
  CASE(16, 32, EPI_RELU) CASE(32, 32, EPI_RELU) CASE(32, 8, EPI_LINEAR_F32)
  CASE(16, 16, EPI_RELU) CASE(16, 8, EPI_LINEAR_F32)
  CASE(16, 32, EPI_MASK) CASE(32, 32, EPI_MASK) CASE(16, 16, EPI_MASK)
#undef CASE
  return cudaErrorInvalidValue;
}

// HLBM_WGRAD_PATH=simt asks for the FP32 SIMT weight-gradient kernel (the
// tensor-core one is the default)
bool wgrad_simt() {
  const char *e = std::getenv("HLBM_WGRAD_PATH");  // read at each call (tests compare both paths)
  return e != nullptr && std::strcmp(e, "simt") == 0;
}

cudaError_t wgrad_any(int cinp, int coutp, int dzs, const bf16 *x, const bf16 *dz, int N, int H,
                      int W, float *partial, int ctas, cudaStream_t s) {
#define CASE(CI, CO, DS)                                                               \
  if (cinp == CI && coutp == CO && dzs == DS) {                                        \
    if (wgrad_simt())                                                                  \
      conv_wgrad_kernel<CI, CO, DS><<<ctas, 256, 0, s>>>(x, dz, N, H, W, partial);     \
    else                                                                               \
      conv_wgrad_mma_kernel<CI, CO, DS><<<ctas, 256, 0, s>>>(x, dz, N, H, W, partial); \
    return cudaGetLastError();                                                         \
  }
  CASE(16, 32, 32) CASE(32, 32, 32) CASE(32, 8, 16) CASE(16, 16, 16) CASE(16, 8, 16)
#undef CASE
  return cudaErrorInvalidValue;
}

int refresh_bf16(lbm_net *net, cudaStream_t s) {
  cast_kernel<<<nblk(net->nw, 256), 256, 0, s>>>(net->w32, net->wbf, (long long)net->nw);
  NCK(net, cudaGetLastError(), "cast kernel");
  for (const Layer &l : net->L) {
    if (l.wtoff == (size_t)-1) continue;
    transpose_kernel<<<nblk((long long)l.cinp * l.ks_t, 256), 256, 0, s>>>(
        net->w32 + l.woff, l.cinp, l.coutp, l.ks, l.cinp_t, l.ks_t, net->wtbf + l.wtoff);
    NCK(net, cudaGetLastError(), "transpose kernel");
  }
  return LBM_OK;
}

int check_shape(lbm_net *net, int N, int H, int W) {
  if (N < 1 || H < TILE_H || W < TILE_W || H % TILE_H || W % TILE_W)
    return nfail(net, LBM_EINVAL, "N >= 1, H a multiple of 8 and W a multiple of 16 are required");
  return LBM_OK;
}

// a failed (timed-out) completion wait inside a tensor-core convolution
// since the last check, seen after the stream has been synchronised
int check_conv(lbm_net *net) {
  if (conv_tc_error(true) != 0)
    return nfail(net, LBM_ETIMEOUT, "tensor-core convolution: an MMA completion wait timed out");
  return LBM_OK;
}

// forward pass on net->x0 (raw state, P pixels) -> net->yout; ev (optional)
// holds layers + 1 events recorded around the convolution launches
int forward_raw(lbm_net *net, int N, int H, int W, cudaStream_t s, cudaEvent_t *ev = nullptr) {
  const long long P = (long long)N * H * W;
  normalise_kernel<<<nblk(P, 256), 256, 0, s>>>(net->x0, P, W, net->nrm, net->act[0]);
  NCK(net, cudaGetLastError(), "normalise kernel");
  if (ev) NCK(net, cudaEventRecord(ev[0], s), "cudaEventRecord");
  for (int l = 0; l < net->layers; l++) {
    const Layer &Ly = net->L[l];
    const bool last = l == net->layers - 1;
    NCK(net, conv_any(Ly.cinp, Ly.coutp, last ? EPI_LINEAR_F32 : EPI_RELU, net->act[l],
                      net->wbf + Ly.woff, net->b32 + Ly.boff, nullptr, N, H, W,
                      last ? nullptr : net->act[l + 1], last ? net->yout : nullptr, s),
        "conv forward");
    if (ev) NCK(net, cudaEventRecord(ev[l + 1], s), "cudaEventRecord");
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_net_create(int channels, int layers, unsigned long long seed, lbm_net **out) {
  if (!out) return nfail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if ((channels != 16 && channels != 32) || layers < 2 || layers > 8)
    return nfail(nullptr, LBM_EINVAL, "channels must be 16 or 32 and layers 2..8");
  lbm_net *net = new lbm_net();
  net->C = channels;
  net->layers = layers;
  size_t wo = 0, bo = 0, wto = 0;
  for (int l = 0; l < layers; l++) {
    Layer Ly;
    Ly.cin = l == 0 ? 4 : channels;
    Ly.cout = l == layers - 1 ? 4 : channels;
    Ly.cinp = l == 0 ? 16 : channels;
    Ly.coutp = l == layers - 1 ? 8 : channels;
    Ly.ks = 9 * Ly.cinp + 8;
    Ly.cinp_t = std::max(16, Ly.coutp);
    Ly.ks_t = 9 * Ly.cinp_t + 8;
    Ly.woff = wo;
    Ly.boff = bo;
    Ly.wtoff = l == 0 ? (size_t)-1 : wto;  // the input needs no gradient
    wo += (size_t)Ly.coutp * Ly.ks;
    bo += Ly.coutp;
    if (l > 0) wto += (size_t)Ly.cinp * Ly.ks_t;
    net->L.push_back(Ly);
  }
  net->nw = wo;
  net->nb = bo;
  net->nwt = wto;
  auto bail = [&](int code) {
    g_net_error = net->msg;
    lbm_net_free(net);
    return code;
  };
  float **f32s[] = {&net->w32, &net->gw, &net->mw, &net->vw};
  for (float **p : f32s)
    if (cudaMalloc(p, sizeof(float) * wo) != cudaSuccess || cudaMemset(*p, 0, sizeof(float) * wo))
      return bail(nfail(net, LBM_ENOMEM, "cudaMalloc"));
  float **b32s[] = {&net->b32, &net->gb, &net->mb, &net->vb};
  for (float **p : b32s)
    if (cudaMalloc(p, sizeof(float) * bo) != cudaSuccess || cudaMemset(*p, 0, sizeof(float) * bo))
      return bail(nfail(net, LBM_ENOMEM, "cudaMalloc"));
  if (cudaMalloc(&net->wbf, sizeof(bf16) * wo) != cudaSuccess ||
      cudaMalloc(&net->wtbf, sizeof(bf16) * std::max<size_t>(wto, 8)) != cudaSuccess ||
      cudaMalloc(&net->nrm, sizeof(float) * 12) != cudaSuccess)
    return bail(nfail(net, LBM_ENOMEM, "cudaMalloc"));
  // He-normal initial weights (the last layer scaled by 0.1), zero biases
  std::vector<float> hw(wo, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < layers; l++) {
    const Layer &Ly = net->L[l];
    std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (9.f * Ly.cin)) * (l == layers - 1 ? 0.1f : 1.f));
    for (int co = 0; co < Ly.cout; co++)
      for (int tap = 0; tap < 9; tap++)
        for (int ci = 0; ci < Ly.cin; ci++) hw[Ly.woff + (size_t)co * Ly.ks + tap * Ly.cinp + ci] = nd(rng);
  }
  if (cudaMemcpy(net->w32, hw.data(), sizeof(float) * wo, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(nfail(net, LBM_ECUDA, "host-to-device copy"));
  const float unit[12] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1};
  std::memcpy(net->hnrm, unit, sizeof unit);
  if (cudaMemcpy(net->nrm, unit, sizeof unit, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(nfail(net, LBM_ECUDA, "host-to-device copy"));
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  net->wgrad_ctas = 2 * sms;
  const size_t per = (size_t)channels * 9 * channels + channels;
  if (cudaMalloc(&net->partial, sizeof(float) * per * net->wgrad_ctas) != cudaSuccess)
    return bail(nfail(net, LBM_ENOMEM, "cudaMalloc"));
  if (refresh_bf16(net, 0)) return bail(LBM_ECUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(nfail(net, LBM_ECUDA, "initialisation"));
  *out = net;
  return LBM_OK;
}

long long lbm_net_param_count(const lbm_net *net) {
  if (!net) return -1;
  long long n = 0;
  for (const Layer &l : net->L) n += (long long)l.cout * 9 * l.cin + l.cout;
  return n;
}

static int net_params_io(lbm_net *net, float *host, long long n, int set, bool grads) {
  if (!net || !host) return LBM_EINVAL;
  if (n != lbm_net_param_count(net)) return nfail(net, LBM_EINVAL, "wrong parameter count");
  std::vector<float> w(net->nw), b(net->nb);
  float *dw = grads ? net->gw : net->w32, *db = grads ? net->gb : net->b32;
  NCK(net, cudaDeviceSynchronize(), "synchronize");
  NCK(net, cudaMemcpy(w.data(), dw, sizeof(float) * net->nw, cudaMemcpyDeviceToHost), "copy");
  NCK(net, cudaMemcpy(b.data(), db, sizeof(float) * net->nb, cudaMemcpyDeviceToHost), "copy");
  long long k = 0;
  for (const Layer &l : net->L) {
    for (int co = 0; co < l.cout; co++)
      for (int tap = 0; tap < 9; tap++)
        for (int ci = 0; ci < l.cin; ci++) {
          float &slot = w[l.woff + (size_t)co * l.ks + tap * l.cinp + ci];
          if (set) slot = host[k]; else host[k] = slot;
          k++;
        }
    for (int co = 0; co < l.cout; co++) {
      float &slot = b[l.boff + co];
      if (set) slot = host[k]; else host[k] = slot;
      k++;
    }
  }
  if (set) {
    NCK(net, cudaMemcpy(dw, w.data(), sizeof(float) * net->nw, cudaMemcpyHostToDevice), "copy");
    NCK(net, cudaMemcpy(db, b.data(), sizeof(float) * net->nb, cudaMemcpyHostToDevice), "copy");
    if (!grads) {
      int rc = refresh_bf16(net, 0);
      if (rc) return rc;
      NCK(net, cudaDeviceSynchronize(), "synchronize");
    }
  }
  return LBM_OK;
}

int lbm_net_params(lbm_net *net, float *host, long long n, int set) {
  return net_params_io(net, host, n, set, false);
}

int lbm_net_grads(lbm_net *net, float *host, long long n) {
  return net_params_io(net, host, n, 0, true);
}

int lbm_net_set_normalisation(lbm_net *net, const float *in_mean, const float *in_std,
                              const float *out_std) {
  if (!net || !in_mean || !in_std || !out_std) return LBM_EINVAL;
  for (int c = 0; c < 4; c++) {
    if (!(in_std[c] > 0.f) || !(out_std[c] > 0.f)) return nfail(net, LBM_EINVAL, "std must be > 0");
    net->hnrm[c] = in_mean[c];
    net->hnrm[4 + c] = in_std[c];
    net->hnrm[8 + c] = out_std[c];
  }
  NCK(net, cudaMemcpy(net->nrm, net->hnrm, sizeof(float) * 12, cudaMemcpyHostToDevice), "copy");
  return LBM_OK;
}

int lbm_net_normalisation(const lbm_net *net, float *out12) {
  if (!net || !out12) return LBM_EINVAL;
  std::memcpy(out12, net->hnrm, sizeof(float) * 12);
  return LBM_OK;
}

int lbm_net_forward(lbm_net *net, const float *x0, int N, int H, int W, float *x1, void *cuda_stream) {
  if (!net || !x0 || !x1) return LBM_EINVAL;
  int rc = check_shape(net, N, H, W);
  if (rc) return rc;
  const long long P = (long long)N * H * W;
  rc = ensure_workspace(net, P);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  NCK(net, cudaMemcpyAsync(net->x0, x0, sizeof(float) * 4 * P, cudaMemcpyDeviceToDevice, s), "copy");
  rc = forward_raw(net, N, H, W, s);
  if (rc) return rc;
  predict_kernel<<<nblk(P, 256), 256, 0, s>>>(net->yout, net->x0, P, net->nrm, x1);
  NCK(net, cudaGetLastError(), "predict kernel");
  return LBM_OK;
}

int lbm_net_layer_times(lbm_net *net, const float *x0, int N, int H, int W, int reps, float *ms,
                        void *cuda_stream) {
  if (!net || !x0 || !ms || reps < 1) return LBM_EINVAL;
  int rc = check_shape(net, N, H, W);
  if (rc) return rc;
  const long long P = (long long)N * H * W;
  rc = ensure_workspace(net, P);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  NCK(net, cudaMemcpyAsync(net->x0, x0, sizeof(float) * 4 * P, cudaMemcpyDeviceToDevice, s), "copy");
  std::vector<cudaEvent_t> ev(net->layers + 1);
  for (auto &e : ev) NCK(net, cudaEventCreate(&e), "cudaEventCreate");
  std::vector<double> acc(net->layers, 0.0);
  for (int r = 0; r <= reps && rc == LBM_OK; r++) {  // r = 0: warm-up
    rc = forward_raw(net, N, H, W, s, ev.data());
    if (rc == LBM_OK && cudaStreamSynchronize(s) != cudaSuccess)
      rc = nfail(net, LBM_ECUDA, "synchronize");
    for (int l = 0; l < net->layers && rc == LBM_OK && r > 0; l++) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[l], ev[l + 1]);
      acc[l] += t;
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  for (int l = 0; l < net->layers; l++) ms[l] = (float)(acc[l] / reps);
  return check_conv(net);
}

int lbm_net_train_step(lbm_net *net, const float *x0, const float *x1, int N, int H, int W, float lr,
                       int update, double *loss, void *cuda_stream) {
  if (!net || !x0 || !x1) return LBM_EINVAL;
  int rc = check_shape(net, N, H, W);
  if (rc) return rc;
  const long long P = (long long)N * H * W;
  rc = ensure_workspace(net, P);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  NCK(net, cudaMemcpyAsync(net->x0, x0, sizeof(float) * 4 * P, cudaMemcpyDeviceToDevice, s), "copy");
  rc = forward_raw(net, N, H, W, s);
  if (rc) return rc;
  const unsigned nb = nblk(P, 256);
  mse_kernel<<<nb, 256, 0, s>>>(net->yout, net->x0, x1, P, W, net->nrm, net->dz[0], net->dpart);
  NCK(net, cudaGetLastError(), "mse kernel");
  // backward: dz holds dL/dz of layer l (BF16, cinp_t of layer l channels)
  int cur = 0;
  for (int l = net->layers - 1; l >= 0; l--) {
    const Layer &Ly = net->L[l];
    // weight and bias gradients of layer l
    NCK(net, wgrad_any(Ly.cinp, Ly.coutp, Ly.cinp_t, net->act[l], net->dz[cur], N, H, W,
                       net->partial, net->wgrad_ctas, s),
        "wgrad");
    const int per = Ly.coutp * 9 * Ly.cinp + Ly.coutp;
    wgrad_reduce_kernel<<<nblk(per, 256), 256, 0, s>>>(net->partial, net->wgrad_ctas, Ly.cinp, Ly.coutp,
                                                      Ly.ks, net->gw + Ly.woff, net->gb + Ly.boff);
    NCK(net, cudaGetLastError(), "wgrad reduce");
    if (l == 0) break;
    // dL/dz of layer l - 1 = (flipped, transposed conv of dz) * relu'(act[l])
    NCK(net, conv_any(Ly.cinp_t, Ly.cinp, EPI_MASK, net->dz[cur], net->wtbf + Ly.wtoff, nullptr,
                      net->act[l], N, H, W, net->dz[1 - cur], nullptr, s),
        "conv backward");
    cur = 1 - cur;
  }
  if (update) {
    net->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->adam_t), c2 = 1.f - std::pow(b2, (float)net->adam_t);
    adam_kernel<<<nblk(net->nw, 256), 256, 0, s>>>(net->w32, net->gw, net->mw, net->vw, net->nw, lr, b1,
                                                   b2, c1, c2, 1e-8f);
    adam_kernel<<<nblk(net->nb, 256), 256, 0, s>>>(net->b32, net->gb, net->mb, net->vb, net->nb, lr, b1,
                                                   b2, c1, c2, 1e-8f);
    NCK(net, cudaGetLastError(), "adam kernel");
    rc = refresh_bf16(net, s);
    if (rc) return rc;
  }
  if (loss) {
    std::vector<double> part(nb);
    NCK(net, cudaMemcpyAsync(part.data(), net->dpart, sizeof(double) * nb, cudaMemcpyDeviceToHost, s),
        "copy");
    NCK(net, cudaStreamSynchronize(s), "synchronize");
    double acc = 0.0;
    for (double v : part) acc += v;
    *loss = acc;
    return check_conv(net);
  }
  return LBM_OK;
}

// The network's state (FP32 [S][4]: phi, u*_x, u*_y, n - 1) of a 2D lattice
// at its current time; `out` is a device pointer.
int lbm_surrogate_state(lbm_handle *h, float *out) {
  if (!h || !out) return LBM_EINVAL;
  if (h->err) return h->err;
  if (!h->inited || h->dims != 2) return LBM_ESTATE;
  int rc = hlbm::queue_moments_for(h);
  if (rc) return rc;
  state_from_staging_kernel<<<nblk(h->S, 256), 256, 0, h->stream>>>(h->staging, h->S, out);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  return LBM_OK;
}

int lbm_surrogate_advance(lbm_handle *h, lbm_net *net, int windows, int window_steps,
                          double mass_tol, int conserve_mass, double phi_clamp, int *fallbacks) {
  return lbm_surrogate_advance_relaxed(h, net, windows, window_steps, 0, mass_tol, conserve_mass,
                                       phi_clamp, fallbacks);
}

int lbm_surrogate_advance_relaxed(lbm_handle *h, lbm_net *net, int windows, int window_steps,
                                  int relax_steps, double mass_tol, int conserve_mass, double phi_clamp,
                                  int *fallbacks) {
  if (!h || !net || windows < 0 || window_steps < 1 || relax_steps < 0) return LBM_EINVAL;
  if (h->err) return h->err;
  if (!h->inited || h->dims != 2) return LBM_ESTATE;
  if (h->P.force_steps > h->t) return nfail(net, LBM_EINVAL, "the surrogate needs the body force off");
  int rc = check_shape(net, 1, h->P.Ly, h->P.Lx);
  if (rc) return rc;
  const long long S = h->S;
  rc = ensure_workspace(net, S);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  const int sb = 512;
  int nfb = 0;
  if (relax_steps > 0 && net->bk_cap < h->hbytes + h->phibytes) {
    cudaFree(net->bk);
    net->bk = nullptr;
    NCK(net, cudaMalloc(&net->bk, h->hbytes + h->phibytes), "cudaMalloc");
    net->bk_cap = h->hbytes + h->phibytes;
  }
  // the predicted state net->x1 (phi shifted down by `shift`) becomes the
  // lattice's state at its current buffer parity
  auto rebuild = [&](double shift) -> int {
    if (h->P.precision == LBM_F32DEV && h->P.T == 1.0 / 3.0) {
      const KParams<float> kp = make_params<float>(h, 0);
      rebuild_mu_kernel<<<nblk(S, 256), 256, 0, s>>>(net->x1, kp, (float)shift, net->yout);
      rebuild_pop_kernel<<<nblk(S, 256), 256, 0, s>>>(net->x1, net->yout, kp, (float)shift,
                                                       static_cast<float *>(h->h[h->cur]),
                                                       static_cast<float *>(h->phi[h->cur]));
      NCK(net, cudaGetLastError(), "rebuild kernels");
      return LBM_OK;
    }
    staging_from_state_kernel<<<nblk(S, 256), 256, 0, s>>>(net->x1, S, shift, h->staging);
    NCK(net, cudaGetLastError(), "staging kernel");
    return launch_init(h, h->cur) == cudaSuccess ? LBM_OK : LBM_ECUDA;
  };
  // sums and maxima (NSTAT each) of a state array, reduced on the host
  std::vector<double> part(NSTAT * sb);
  auto stats_of = [&](const float *x, double (&out)[NSTAT]) -> int {
    state_stats_kernel<<<sb, 256, 0, s>>>(x, S, net->dpart);
    NCK(net, cudaGetLastError(), "surrogate kernels");
    NCK(net, cudaMemcpyAsync(part.data(), net->dpart, sizeof(double) * NSTAT * sb, cudaMemcpyDeviceToHost, s),
        "copy");
    NCK(net, cudaStreamSynchronize(s), "synchronize");
    for (int j = 0; j < NSTAT; j++) out[j] = 0.0;
    for (int b = 0; b < sb; b++) {
      const double *q = &part[b * NSTAT];
      out[0] += q[0];
      out[1] += q[1];
      for (int j = 2; j < NSTAT; j++) out[j] = std::max(out[j], q[j]);
    }
    return LBM_OK;
  };
  for (int w = 0; w < windows; w++) {
    rc = lbm_surrogate_state(h, net->x0);
    if (rc) return rc;
    rc = forward_raw(net, 1, h->P.Ly, h->P.Lx, s);
    if (rc) return rc;
    predict_kernel<<<nblk(S, 256), 256, 0, s>>>(net->yout, net->x0, S, net->nrm, net->x1);
    NCK(net, cudaGetLastError(), "surrogate kernels");
    double st[2][NSTAT];
    if ((rc = stats_of(net->x0, st[0]))) return rc;
    if (phi_clamp > 0.0) {
      clamp_phi_kernel<<<nblk(S, 256), 256, 0, s>>>(net->x1, S, (float)(phi_clamp * st[0][2]));
      NCK(net, cudaGetLastError(), "clamp kernel");
    }
    if ((rc = stats_of(net->x1, st[1]))) return rc;
    // relaxation: the prediction becomes the lattice state and relax_steps
    // plain steps damp its short-wavelength errors before the check (the
    // state of the window's start is kept to fall back to)
    const long long t_start = h->t;
    const int cur_start = h->cur;
    if (relax_steps > 0) {
      char *bk = static_cast<char *>(net->bk);
      NCK(net, cudaMemcpyAsync(bk, h->h[cur_start], h->hbytes, cudaMemcpyDeviceToDevice, s), "copy");
      NCK(net, cudaMemcpyAsync(bk + h->hbytes, h->phi[cur_start], h->phibytes, cudaMemcpyDeviceToDevice, s),
          "copy");
      if ((rc = rebuild(conserve_mass ? (st[1][0] - st[0][0]) / (double)S : 0.0))) return rc;
      h->t += window_steps;
      if ((rc = lbm_step(h, relax_steps))) return rc;
      if ((rc = lbm_surrogate_state(h, net->x1))) return rc;
      if ((rc = stats_of(net->x1, st[1]))) return rc;
    }
    // residual check: the mean change of phi per site, and bounds on |phi|,
    // |u*| and |n - 1| relative to the state the window starts from (an
    // unbounded, non-finite or runaway prediction fails them)
    const double drift = std::fabs(st[1][0] - st[0][0]) / (double)S;
    // (relative bounds, each under an absolute ceiling so that accepted
    // windows cannot compound them into a runaway: |phi| <= 1.5 phi0,
    // |u*| <= 0.5 c_s, |n - 1| <= 0.3; plain spinodal states with the
    // benchmark's parameters reach |u*| = 0.2 c_s and |n - 1| = 0.07)
    const double phi_cap = std::min(std::max(1.1 * h->phi0, 1.05 * st[0][2]), 1.5 * h->phi0);
    const double u_cap = std::min(std::max(1.5 * st[0][3], 0.01 / std::sqrt(3.0)), 0.5 / std::sqrt(3.0));
    const double n_cap = std::min(std::max(2.0 * st[0][4], 1e-3), 0.3);
    const bool ok = std::isfinite(st[1][2]) && std::isfinite(st[1][3]) && std::isfinite(st[1][4]) &&
                    drift <= mass_tol && st[1][2] <= phi_cap && st[1][3] <= u_cap && st[1][4] <= n_cap;
    if (std::getenv("HLBM_SURROGATE_VERBOSE"))
      std::fprintf(stderr,
                   "hlbm surrogate t=%lld mean dphi %.3e max|phi| %.4f (state %.4f) max|u| %.3e "
                   "(state %.3e) max|n-1| %.3e (state %.3e) -> %s\n",
                   h->t, drift, st[1][2], st[0][2], st[1][3], st[0][3], st[1][4], st[0][4],
                   ok ? "accepted" : "plain steps");
    if (relax_steps > 0) {
      if (!ok) {  // back to the window's start, then the plain steps
        nfb++;
        const char *bk = static_cast<const char *>(net->bk);
        h->cur = cur_start;
        h->t = t_start;
        NCK(net, cudaMemcpyAsync(h->h[cur_start], bk, h->hbytes, cudaMemcpyDeviceToDevice, s), "copy");
        NCK(net, cudaMemcpyAsync(h->phi[cur_start], bk + h->hbytes, h->phibytes, cudaMemcpyDeviceToDevice, s),
            "copy");
        if ((rc = lbm_step(h, window_steps + relax_steps))) return rc;
      }
    } else if (ok) {
      if ((rc = rebuild(conserve_mass ? (st[1][0] - st[0][0]) / (double)S : 0.0))) return rc;
      h->t += window_steps;
    } else {
      nfb++;
      rc = lbm_step(h, window_steps);
      if (rc) return rc;
    }
  }
  if (fallbacks) *fallbacks = nfb;
  NCK(net, cudaStreamSynchronize(s), "synchronize");
  return check_conv(net);
}

void lbm_net_free(lbm_net *net) {
  if (!net) return;
  cudaDeviceSynchronize();
  void *ptrs[] = {net->w32, net->b32, net->gw, net->gb, net->mw, net->vw, net->mb, net->vb, net->wbf,
                  net->wtbf, net->nrm, net->yout, net->x0, net->x1, net->dz[0], net->dz[1],
                  net->partial, net->dpart, net->bk};
  for (void *p : ptrs) if (p) cudaFree(p);
  for (auto &a : net->act) if (a) cudaFree(a);
  delete net;
}

const char *lbm_net_last_error(const lbm_net *net) {
  return net ? net->msg.c_str() : g_net_error.c_str();
}

}  // extern "C"
