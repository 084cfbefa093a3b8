// conv_tc.cuh -- the periodic 3x3 convolution of the learned surrogate on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory).
#pragma once
#include <cuda_runtime.h>

namespace hlbm {

// Activations are stored row-chunk planar: element (n, y, x, channel k) of a
// tensor with ch = C / 8 chunks sits at conv_act_index(n H + y, k / 8, x, W, ch)
// + k % 8, i.e. [n][y][k / 8][x][8].  One chunk of one image row is then a
// contiguous run of W x 16 bytes.
__host__ __device__ __forceinline__ long long conv_act_index(long long row, int c, int x, int W,
                                                             int ch) {
  return ((row * ch + c) * (long long)W + x) * 8;
}

// epilogues of a convolution layer
//   CONV_RELU:       bf16 max(conv + bias, 0)
//   CONV_LINEAR_F32: fp32 conv + bias
//   CONV_MASK:       bf16 conv * (mask > 0)   (backward through a ReLU)
enum ConvEpi { CONV_RELU = 0, CONV_LINEAR_F32 = 1, CONV_MASK = 2 };

// out[n, y, x, co] = epi(sum_{dy, dx, ci} in[n, y + dy, x + dx, ci] w[co][(dy+1)*3 + dx+1][ci])
// with periodic indices.  Activations bf16 row-chunk planar with `cinp`
// channels; the weights [coutp][ks] bf16 (K = 9 cinp ordered (tap, ci), ks >=
// 9 cinp, rows 16-byte aligned); bf16 outputs row-chunk planar with coutp
// channels, FP32 outputs [p][coutp].  W must be a multiple of 128 (one tile is
// 128 consecutive pixels of a row).  Returns cudaErrorInvalidValue for
// an unsupported shape or channel combination.  A timed-out completion wait
// inside the kernel is recorded and reported by conv_tc_error().
cudaError_t conv_tc(int cinp, int coutp, int epi, const void *in, const void *w, int ks,
                    const float *bias, const void *mask, int N, int H, int W, void *out_bf,
                    float *out_f, cudaStream_t s);

bool conv_tc_supported(int cinp, int coutp, int W);

// nonzero if a tensor-core convolution gave up waiting for its MMAs since
// the last call with reset = true
int conv_tc_error(bool reset);

}  // namespace hlbm
