// Per-ring pieces shared by the polar kernel and the FP32 rescore kernel:
// zero-padded bilinear sampling and a warp-cooperative in-place complex FFT.
#pragma once

#include "dev_util.cuh"

namespace mra {

// Bilinear sample of img[y][x] at (x, y): x0 = floor(x), fx = x - x0; every
// neighbour outside [0, L-1]^2 contributes zero.
__device__ __forceinline__ float bilinear(const float *__restrict__ img, int L, float x, float y) {
  const float xf = floorf(x), yf = floorf(y);
  const float fx = x - xf, fy = y - yf;
  const int x0 = static_cast<int>(xf), y0 = static_cast<int>(yf);
  const bool xa = static_cast<unsigned>(x0) < static_cast<unsigned>(L);
  const bool xb = static_cast<unsigned>(x0 + 1) < static_cast<unsigned>(L);
  const bool ya = static_cast<unsigned>(y0) < static_cast<unsigned>(L);
  const bool yb = static_cast<unsigned>(y0 + 1) < static_cast<unsigned>(L);
  float v00 = 0.f, v10 = 0.f, v01 = 0.f, v11 = 0.f;
  if (ya) {
    const float *p = img + static_cast<int64_t>(y0) * L;
    if (xa) v00 = __ldg(p + x0);
    if (xb) v10 = __ldg(p + x0 + 1);
  }
  if (yb) {
    const float *p = img + static_cast<int64_t>(y0 + 1) * L;
    if (xa) v01 = __ldg(p + x0);
    if (xb) v11 = __ldg(p + x0 + 1);
  }
  const float gx = 1.f - fx, gy = 1.f - fy;
  return gy * (gx * v00 + fx * v10) + fy * (gx * v01 + fx * v11);
}

// Same interpolation from an image staged in shared memory.
__device__ __forceinline__ float bilinear_smem(const float *img, int L, float x, float y) {
  const float xf = floorf(x), yf = floorf(y);
  const float fx = x - xf, fy = y - yf;
  const int x0 = static_cast<int>(xf), y0 = static_cast<int>(yf);
  const bool xa = static_cast<unsigned>(x0) < static_cast<unsigned>(L);
  const bool xb = static_cast<unsigned>(x0 + 1) < static_cast<unsigned>(L);
  const bool ya = static_cast<unsigned>(y0) < static_cast<unsigned>(L);
  const bool yb = static_cast<unsigned>(y0 + 1) < static_cast<unsigned>(L);
  const int o = y0 * L + x0;
  const float v00 = (ya && xa) ? img[o] : 0.f;
  const float v10 = (ya && xb) ? img[o + 1] : 0.f;
  const float v01 = (yb && xa) ? img[o + L] : 0.f;
  const float v11 = (yb && xb) ? img[o + L + 1] : 0.f;
  const float gx = 1.f - fx, gy = 1.f - fy;
  return gy * (gx * v00 + fx * v10) + fy * (gx * v01 + fx * v11);
}

// In-place forward FFT of H = 2^logH complex values in shared memory by one
// warp: bit-reversal permutation, then radix-2 stages with twiddles
// exp(-2 pi i p / span) = fwd_tw[p * M / span].
__device__ __forceinline__ void warp_fft_inplace(float2 *z, int H, int logH, int M, const float2 *fwd_tw,
                                                 int lane) {
  for (int u = lane; u < H; u += 32) {
    const int v = static_cast<int>(__brev(static_cast<unsigned>(u)) >> (32 - logH));
    if (u < v) {
      const float2 t = z[u];
      z[u] = z[v];
      z[v] = t;
    }
  }
  __syncwarp();
  for (int half = 1; half < H; half <<= 1) {
    const int span = half << 1;
    const int tstep = M / span;
    for (int b = lane; b < (H >> 1); b += 32) {
      const int p = b & (half - 1);
      const int u = (b - p) * 2 + p;  // (b / half) * span + p
      const int v = u + half;
      const float2 t = cmul(fwd_tw[p * tstep], z[v]);
      const float2 zu = z[u];
      z[v] = csub(zu, t);
      z[u] = cadd(zu, t);
    }
    __syncwarp();
  }
}

// Forward FFT of H complex points (power of two, 4..256) held in shared
// memory, by a group of T threads of one warp (T = H / 16 for H >= 32, else
// one thread): thread t transforms z(t + T a), a = 0..U-1, in registers,
// multiplies by exp(-2 pi i t k / H), the group transposes in place (XOR
// swizzle), finishes the length-T transforms, and writes X(k + U jj) back in
// natural order.  Every lane of the warp must call it (it uses __syncwarp);
// lanes with `active` false do no stores.  fwd_tw[q] = exp(-2 pi i q / M).
template <int H>
struct GroupFft {
  static constexpr int T = H >= 32 ? H / 16 : 1;
  static constexpr int U = H / T;
  static constexpr int KK = U / T;
};

template <int H>
__device__ __forceinline__ void group_fft(float2 *z, int t, bool active, const float2 *fwd_tw, int M) {
  constexpr int T = GroupFft<H>::T;
  constexpr int U = GroupFft<H>::U;
  float2 x[U];
#pragma unroll
  for (int a = 0; a < U; ++a) x[a] = z[t + T * a];
  reg_fft<U, -1>(x);
  if constexpr (T == 1) {
    __syncwarp();
    if (active) {
#pragma unroll
      for (int k = 0; k < U; ++k) z[k] = x[k];
    }
    __syncwarp();
  } else {
    const int tstep = (M / H) * t;
#pragma unroll
    for (int k = 1; k < U; ++k) x[k] = cmul(x[k], fwd_tw[(tstep * k) & (M - 1)]);
    __syncwarp();
    if (active) {
#pragma unroll
      for (int k = 0; k < U; ++k) z[k * T + (t ^ (k & (T - 1)))] = x[k];
    }
    __syncwarp();
    float2 y[GroupFft<H>::KK][T];
#pragma unroll
    for (int kk = 0; kk < GroupFft<H>::KK; ++kk) {
      const int k = t + T * kk;
#pragma unroll
      for (int tt = 0; tt < T; ++tt) y[kk][tt] = z[k * T + (tt ^ t)];
      reg_fft<T, -1>(y[kk]);
    }
    __syncwarp();
    if (active) {
#pragma unroll
      for (int kk = 0; kk < GroupFft<H>::KK; ++kk)
#pragma unroll
        for (int jj = 0; jj < T; ++jj) z[t + T * kk + U * jj] = y[kk][jj];
    }
    __syncwarp();
  }
}

// Bin k (0..H) of the real DFT of the N = 2H samples packed as
// z_q = x_{2q} + i x_{2q+1} and transformed by warp_fft_inplace:
// X(k) = E(k) + exp(-2 pi i k / N) O(k).
__device__ __forceinline__ float2 real_split(const float2 *z, int H, int k, float2 w) {
  const float2 zk = z[k & (H - 1)];
  const float2 zc = cconj(z[(H - k) & (H - 1)]);
  const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
  const float2 d = csub(zk, zc);
  const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);  // (zk - zc) / (2 i)
  return cadd(e, cmul(w, o));
}

// Bins k and H - k (0 <= k <= H / 2) of the same real DFT from one pair of
// spectrum loads and one twiddle: with E, O as in real_split,
// X(k) = E + w^k O and X(H - k) = conj(E - w^k O), since the odd part of
// bin H - k is conj(O) and w^(H - k) = -conj(w^k).  For k = H / 2 both
// entries are the same bin.
__device__ __forceinline__ void real_split_pair(const float2 *z, int H, int k, float2 w, float2 &xk, float2 &xhk) {
  const float2 zk = z[k & (H - 1)];
  const float2 zc = cconj(z[(H - k) & (H - 1)]);
  const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
  const float2 d = csub(zk, zc);
  const float2 wo = cmul(w, make_float2(0.5f * d.y, -0.5f * d.x));
  xk = cadd(e, wo);
  xhk = cconj(csub(e, wo));
}

}  // namespace mra
