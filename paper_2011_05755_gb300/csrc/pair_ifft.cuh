// Inverse angular DFT of one (row, reference) pair, computed by a group of
// T threads, plus the flat candidate index used by the argmax key.
//
// The pair's angular spectrum Z(f), f = 0..M-1, sits in shared memory at
// f ^ sw (an XOR swizzle with sw < T, so the T threads of a group read
// distinct banks).  With M = T x U, thread t transforms Z(t + T a),
// a = 0..U-1 (length U, in registers), multiplies by exp(2 pi i t k / M),
// writes its row of the transposed matrix [t][k] (row stride U + 1, which
// keeps both the row writes and the column reads conflict-free), and
// finishes the length-T transforms for k = t + T kk, giving
//     y[kk][jj] = c(k + U jj) = sum_f Z(f) exp(2 pi i f (k + U jj) / M).
// A pair's buffer therefore spans T (U + 1) float2 (IfftShape<M>::P).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dev_util.cuh"

namespace mra {

template <int M>
struct IfftShape {
  static constexpr int T = (M >= 256) ? 16 : M / 16;  // threads per pair
  static constexpr int U = M / T;                     // first-stage length
  static constexpr int KK = U / T;                    // second-stage transforms per thread
  static constexpr int P = T * (U + 1);               // float2 per pair buffer (>= M)
  static_assert(M >= 16 && M <= 512, "M out of range");
};

__device__ __forceinline__ float2 load_z(const float2 *p) { return *p; }
__device__ __forceinline__ float2 load_z(const __nv_bfloat162 *p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ float2 load_z(const __half2 *p) { return __half22float2(*p); }

// Every lane of the warp must call this (it contains __syncwarp).  `scratch`
// holds P float2 for this pair; it may alias `src` when src is float2.
// Requires sw < T.
template <int M, class SrcT>
__device__ __forceinline__ void pair_ifft(const SrcT *src, int sw, float2 *scratch, int t, bool write_ok,
                                          const float2 *tw, float2 (&y)[IfftShape<M>::KK][IfftShape<M>::T]) {
  constexpr int T = IfftShape<M>::T;
  constexpr int U = IfftShape<M>::U;
  float2 x[U];
  const SrcT *s0 = src + (t ^ sw);  // (t + T a) ^ sw = (t ^ sw) + T a
#pragma unroll
  for (int a = 0; a < U; ++a) x[a] = load_z(s0 + T * a);
  reg_fft<U, +1>(x);
  const float2 *twt = tw + t;
#pragma unroll
  for (int k = 1; k < U; ++k) x[k] = cmul(x[k], twt[k * T]);
  __syncwarp();
  if (write_ok) {
    float2 *row = scratch + t * (U + 1);
#pragma unroll
    for (int k = 0; k < U; ++k) row[k] = x[k];
  }
  __syncwarp();
#pragma unroll
  for (int kk = 0; kk < IfftShape<M>::KK; ++kk) {
    const float2 *col = scratch + t + T * kk;  // column k = t + T kk
#pragma unroll
    for (int tt = 0; tt < T; ++tt) y[kk][tt] = col[tt * (U + 1)];
    reg_fft<T, +1>(y[kk]);
  }
  __syncwarp();
}

// Angle index of output y[kk][jj] for thread t.
template <int M>
__device__ __forceinline__ int ifft_angle(int t, int kk, int jj) {
  return t + IfftShape<M>::T * kk + IfftShape<M>::U * jj;
}

}  // namespace mra
