// Device-side helpers shared by the MRA kernels: complex arithmetic,
// compile-time twiddle factors, register-resident radix-2 FFTs and the
// orderable 64-bit argmax key.
#pragma once

#include <cstdint>
#include <cstring>
#include <type_traits>
#include <cuda_runtime.h>

namespace mra {

// ---------------------------------------------------------------------------
// Compile-time cos / sin of 2 pi k / n.
// Quadrant reduction is exact in integers; the remaining angle (<= pi/4) is
// evaluated with the Taylor series of sin and cos about zero, which for
// |x| <= pi/4 converges below double rounding within 12 terms.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}
// cos and sin of theta = (pi/2) * r / n for 0 <= r < n (first quadrant).
__host__ __device__ constexpr double quad_cos(long r, long n) {
  constexpr double half_pi = 1.57079632679489661923;
  return (2 * r <= n) ? taylor_cos(half_pi * double(r) / double(n))
                      : taylor_sin(half_pi * double(n - r) / double(n));
}
__host__ __device__ constexpr double quad_sin(long r, long n) {
  constexpr double half_pi = 1.57079632679489661923;
  return (2 * r <= n) ? taylor_sin(half_pi * double(r) / double(n))
                      : taylor_cos(half_pi * double(n - r) / double(n));
}
__host__ __device__ constexpr double cos2pi(long k, long n) {
  k %= n;
  if (k < 0) k += n;
  long q = (4 * k) / n, r = (4 * k) % n;  // 2 pi k / n = q * pi/2 + (pi/2) r / n
  double c = quad_cos(r, n), s = quad_sin(r, n);
  return q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}
__host__ __device__ constexpr double sin2pi(long k, long n) {
  k %= n;
  if (k < 0) k += n;
  long q = (4 * k) / n, r = (4 * k) % n;
  double c = quad_cos(r, n), s = quad_sin(r, n);
  return q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
}

// ---------------------------------------------------------------------------
// Complex helpers on float2 (x = re, y = im).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Compile-time loop.
template <int B, int E, class F>
__device__ __forceinline__ void sfor(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(f);
  }
}

template <int N>
__host__ __device__ constexpr int ilog2() {
  int l = 0;
  while ((1 << l) < N) ++l;
  return l;
}
template <int N>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 0; b < ilog2<N>(); ++b) r |= ((i >> b) & 1) << (ilog2<N>() - 1 - b);
  return r;
}

// v * exp(SIGN * 2 pi i P / SPAN), with the trivial and 45-degree factors
// special-cased at compile time.
template <int P, int SPAN, int SIGN>
__device__ __forceinline__ float2 twiddle_mul(float2 v) {
  if constexpr (P == 0) {
    return v;
  } else if constexpr (4 * P == SPAN) {  // factor = SIGN * i
    return SIGN > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else if constexpr (8 * P == SPAN) {  // factor = (1 + SIGN i) / sqrt 2
    constexpr float h = float(cos2pi(1, 8));
    return SIGN > 0 ? make_float2(h * (v.x - v.y), h * (v.x + v.y))
                    : make_float2(h * (v.x + v.y), h * (v.y - v.x));
  } else if constexpr (8 * P == 3 * SPAN) {  // factor = (-1 + SIGN i) / sqrt 2
    constexpr float h = float(cos2pi(1, 8));
    return SIGN > 0 ? make_float2(-h * (v.x + v.y), h * (v.x - v.y))
                    : make_float2(h * (v.y - v.x), -h * (v.x + v.y));
  } else {
    constexpr float c = float(cos2pi(P, SPAN));
    constexpr float s = float(SIGN * sin2pi(P, SPAN));
    return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
  }
}

// In-register DFT of length N (power of two):
//   x[k] <- sum_n x[n] exp(SIGN * 2 pi i n k / N), natural order in and out.
// Radix-2 decimation in time after a compile-time bit-reversal permutation.
template <int N, int SIGN>
__device__ __forceinline__ void reg_fft(float2 (&x)[N]) {
  if constexpr (N > 1) {
    sfor<0, N>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      constexpr int j = bitrev<N>(i);
      if constexpr (i < j) {
        float2 t = x[i];
        x[i] = x[j];
        x[j] = t;
      }
    });
    sfor<0, ilog2<N>()>([&](auto ss) {
      constexpr int half = 1 << decltype(ss)::value;
      constexpr int span = 2 * half;
      sfor<0, N / 2>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        constexpr int p = b % half;
        constexpr int i = (b / half) * span + p;
        constexpr int j = i + half;
        float2 t = twiddle_mul<p, span, SIGN>(x[j]);
        x[j] = csub(x[i], t);
        x[i] = cadd(x[i], t);
      });
    });
  }
}

// ---------------------------------------------------------------------------
// Argmax key: order-preserving float bits in the high word, the inverted
// flat candidate index in the low word, so that atomicMax keeps the largest
// value and, among bit-equal values, the smallest index.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t float_to_ordered(float v) {
  uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ordered_to_float(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
__device__ __forceinline__ unsigned long long make_key(float v, uint32_t flat) {
  return (static_cast<unsigned long long>(float_to_ordered(v)) << 32) |
         static_cast<unsigned long long>(0xffffffffu - flat);
}

}  // namespace mra
