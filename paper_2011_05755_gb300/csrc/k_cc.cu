// Fused spectrum contraction, inverse angular FFT and argmax (FP32 path).
//
// Alg. 1, inner loop (CC step, inverse-FFT step, per-image reduction step):
// the ring spectra of every shifted particle are correlated with every
// reference, transformed back over the angle, and reduced to the best value
// per image.  The CC table of Sec. 2 is never
// materialised: each CTA owns a tile of 8 rows (image, shift) x KT
// references, holds the per-pair angular spectrum in shared memory, and
// reduces the correlation over angles on chip.
//
// For one (row, reference) pair and frequency f in [0, M/2] the products
//   P1 = sum_r ReA ReB, P2 = sum_r ImA ImB, P3 = sum_r ReA ImB, P4 = sum_r ImA ReB
// give the unmirrored spectrum C_u(f) = sum conj(A) B = (P1 + P2) + i (P3 - P4)
// and the spectrum of the particle's mirror (x -> -x about the centre, which
// maps X(f) to (-1)^f conj(X(f))) up to a half-turn, C'(f) = sum A B =
// (P1 - P2) + i (P3 + P4).  Both correlations are real, so one complex
// inverse DFT of Z(f) = C_u(f) + i C'(f) (Hermitian-extended to f = 0..M-1)
// returns c_u(j) in its real part and c'(j) in its imaginary part, with the
// mirrored correlation c_m(j) = c'((j + M/2) mod M).
//
// The length-M inverse DFT is split as M = T x U: thread t of the pair's T
// threads transforms Z(t + T a), a = 0..U-1 (length U), multiplies by
// exp(2 pi i t k / M), the group transposes through shared memory, and each
// thread finishes length-T transforms giving c(k + U jj).
#include "../../include/mra.h"
#include "dev_util.cuh"
#include "mra_internal.h"
#include "pair_ifft.cuh"
#include "smem_limit.cuh"
#include "tma.cuh"

namespace mra {

int cc_threads_per_pair(int M) { return M >= 256 ? 16 : M / 16; }

template <int M, int KT>
struct CCShape {
  static constexpr int RT = kTile;                         // rows per tile
  static constexpr int PAIRS = RT * KT;
  static constexpr int WARPS = (M >= 512) ? 8 : 16;        // 16 warps unless staging would not fit
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int LANES_PER_SLICE = (RT / 2) * (KT / 2);  // lane = 2 rows x 2 refs
  static constexpr int NSPLIT = 32 / LANES_PER_SLICE;          // bin slices per frequency
  static constexpr int P = IfftShape<M>::P;                    // float2 per pair buffer
  static constexpr size_t STATE = static_cast<size_t>(PAIRS) * P * sizeof(float2);
  static constexpr size_t TW = M * sizeof(float2);
  static constexpr size_t BARS = WARPS * sizeof(uint64_t);
  // staging per warp: one frequency segment of the 8-row A tile and the 8-ref B tile
  __host__ __device__ static size_t stage_bytes(int seg_max) { return 2 * static_cast<size_t>(seg_max) * kTile * sizeof(float2); }
  __host__ __device__ static size_t smem(int seg_max) { return STATE + TW + BARS + WARPS * stage_bytes(seg_max); }
};

// Bank swizzle of the per-pair spectrum buffers (an XOR below T, so the
// inverse DFT's reads stay one base plus constant offsets).
template <int M, int KT>
__device__ __forceinline__ int pair_swz(int p) {
  const int row = p / KT, ref = p % KT;
  return (row * (KT / 2) + (ref >> 1)) & (IfftShape<M>::T - 1);
}

template <int M, int KT>
__global__ void __launch_bounds__(CCShape<M, KT>::THREADS) cc_fp32_kernel(Geometry g, CCArgs a) {
  using Sh = CCShape<M, KT>;
  constexpr int T = IfftShape<M>::T;
  constexpr int U = IfftShape<M>::U;
  extern __shared__ float4 smem_f4[];
  unsigned char *sbase = reinterpret_cast<unsigned char *>(smem_f4);
  float2 *Zs = reinterpret_cast<float2 *>(sbase);                          // [PAIRS][P]
  float2 *tw = reinterpret_cast<float2 *>(sbase + Sh::STATE);              // [M] inverse twiddles, [k][t]
  uint64_t *bars = reinterpret_cast<uint64_t *>(sbase + Sh::STATE + Sh::TW);
  unsigned char *stage0 = sbase + Sh::STATE + Sh::TW + Sh::BARS;
  const size_t stage_bytes = Sh::stage_bytes(a.seg_max);

  const int kt = blockIdx.x;            // reference tile
  const int64_t rt = blockIdx.y;        // row tile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int i = threadIdx.x; i < M; i += Sh::THREADS) tw[i] = g.inv_tw[i];
  if (lane == 0) mbar_init(bars + warp, 1);
  mbar_init_fence();
  __syncwarp();

  // ---------------- Phase 1: contraction over rings, all f ----------------
  // Warp w handles f = w, w + WARPS, ...; each f's A segment (8 rows) and B
  // segment (8 references) arrive by two TMA bulk copies into the warp's
  // staging buffer.  Lane = (bin slice, ref pair kp, row pair rp); the bin
  // slices are summed with shuffles at the end of the frequency.
  bool failed = false;
  {
    const int slice = lane / Sh::LANES_PER_SLICE;
    const int li = lane % Sh::LANES_PER_SLICE;
    const int rp = li % (Sh::RT / 2);   // rows 2rp, 2rp+1
    const int kp = li / (Sh::RT / 2);   // refs 2kp, 2kp+1 of the tile
    const int ref0 = kt * KT;
    const float2 *Atile = a.A + rt * g.NB * kTile;
    const float2 *Btile = a.B + static_cast<int64_t>(ref0 / kTile) * g.NB * kTile;
    const int bsub = (ref0 % kTile) / 2 + kp;  // float4 index of this lane's 2 refs within a bin
    float4 *stA = reinterpret_cast<float4 *>(stage0 + warp * stage_bytes);
    float4 *stB = reinterpret_cast<float4 *>(stage0 + warp * stage_bytes + stage_bytes / 2);
    uint64_t *bar = bars + warp;
    uint32_t phase = 0;
    bool first_wait = true;
    for (int f = warp; f <= M / 2; f += Sh::WARPS) {
      const int2 seg = g.fseg[f];
      if (lane == 0) {
        const uint32_t bytes = static_cast<uint32_t>(seg.y) * kTile * sizeof(float2);
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, 2 * bytes);
        bulk_g2s(stA, Atile + static_cast<int64_t>(seg.x) * kTile, bytes, bar);
        bulk_g2s(stB, Btile + static_cast<int64_t>(seg.x) * kTile, bytes, bar);
      }
      const uint32_t limit = first_wait ? a.first_wait_limit : a.wait_limit;
      first_wait = false;
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, phase, limit))) {
        // give up: record the time-out, let the copies land (bounded), leave the loop
        if (lane == 0) atomicOr(a.err, 1);
        mbar_wait_bounded(bar, phase, a.wait_limit);
        failed = true;
        break;
      }
      phase ^= 1u;
      float p1[4] = {0.f, 0.f, 0.f, 0.f}, p2[4] = {0.f, 0.f, 0.f, 0.f};
      float p3[4] = {0.f, 0.f, 0.f, 0.f}, p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
      for (int b = slice; b < seg.y; b += Sh::NSPLIT) {
        const float4 av = stA[b * (kTile / 2) + rp];
        const float4 bv = stB[b * (kTile / 2) + bsub];
        const float ar[2] = {av.x, av.z}, ai[2] = {av.y, av.w};
        const float br[2] = {bv.x, bv.z}, bi[2] = {bv.y, bv.w};
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            p1[2 * i + j] = fmaf(ar[i], br[j], p1[2 * i + j]);
            p2[2 * i + j] = fmaf(ai[i], bi[j], p2[2 * i + j]);
            p3[2 * i + j] = fmaf(ar[i], bi[j], p3[2 * i + j]);
            p4[2 * i + j] = fmaf(ai[i], br[j], p4[2 * i + j]);
          }
      }
#pragma unroll
      for (int off = 16; off >= Sh::LANES_PER_SLICE; off >>= 1)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          p1[q] += __shfl_xor_sync(0xffffffffu, p1[q], off);
          p2[q] += __shfl_xor_sync(0xffffffffu, p2[q], off);
          p3[q] += __shfl_xor_sync(0xffffffffu, p3[q], off);
          p4[q] += __shfl_xor_sync(0xffffffffu, p4[q], off);
        }
      if (slice == 0) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int p = (2 * rp + i) * KT + 2 * kp + j;
            const int sw = pair_swz<M, KT>(p);
            const int q = 2 * i + j;
            float2 *zp = Zs + p * Sh::P;
            // Z(f) = C_u + i C'
            zp[f ^ sw] = make_float2((p1[q] + p2[q]) - (p3[q] + p4[q]), (p3[q] - p4[q]) + (p1[q] - p2[q]));
            if (f != 0 && f != M / 2)  // Z(M - f) = conj(C_u) + i conj(C')
              zp[(M - f) ^ sw] = make_float2((p1[q] + p2[q]) + (p3[q] + p4[q]),
                                             (p1[q] - p2[q]) - (p3[q] - p4[q]));
          }
      }
      __syncwarp();  // every lane is done with the staging buffer before it is refilled
    }
  }
  if (__syncthreads_or(failed)) return;

  // ---------------- Phase 2: inverse angular DFT + argmax ----------------
  constexpr int GROUPS = Sh::THREADS / T;  // pairs transformed concurrently
  const int t = threadIdx.x % T;
  const int S = g.S;
  for (int p0 = 0; p0 < Sh::PAIRS; p0 += GROUPS) {
    const int p = p0 + threadIdx.x / T;
    const bool in_tile = p < Sh::PAIRS;
    const int pc = in_tile ? p : 0;
    const int64_t row = rt * Sh::RT + pc / KT;
    const int ref = kt * KT + pc % KT;
    const bool valid = in_tile && row < a.rows && ref < a.K;
    float2 *zp = Zs + pc * Sh::P;
    const int sw = pair_swz<M, KT>(pc);

    float2 y[IfftShape<M>::KK][T];
    pair_ifft<M>(zp, sw, zp, t, in_tile, tw, y);
    float vmax = -INFINITY;
#pragma unroll
    for (int kk = 0; kk < U / T; ++kk)
#pragma unroll
      for (int jj = 0; jj < T; ++jj) {
        vmax = fmaxf(vmax, y[kk][jj].x);
        if (g.mirror) vmax = fmaxf(vmax, y[kk][jj].y);
      }

    const int64_t img = static_cast<uint32_t>(row) / static_cast<uint32_t>(S);  // rows < 2^31 per chunk
    const int s = static_cast<int>(row - img * S);
    if (a.dbg_cc && valid) {
      float *d = a.dbg_cc + ((img * a.K + ref) * S + s) * 2 * M;
#pragma unroll
      for (int kk = 0; kk < U / T; ++kk)
#pragma unroll
        for (int jj = 0; jj < T; ++jj) {
          const int j = t + T * kk + U * jj;
          d[j] = y[kk][jj].x;
          d[M + ((j + M / 2) & (M - 1))] = y[kk][jj].y;
        }
    }
    // pair maximum over the T threads
#pragma unroll
    for (int off = T / 2; off > 0; off >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off, T));
    bool cand = false;
    if (valid) {
      const unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(a.best + img);
      cand = float_to_ordered(vmax) >= static_cast<uint32_t>(cur >> 32);
    }
    // smallest flat index (k, s, m, j) holding the pair maximum
    uint32_t flat = 0xffffffffu;
    if (cand) {
      const uint32_t base = static_cast<uint32_t>((ref * S + s) * 2) * M;
#pragma unroll
      for (int kk = 0; kk < U / T; ++kk)
#pragma unroll
        for (int jj = 0; jj < T; ++jj) {
          const uint32_t j = t + T * kk + U * jj;
          if (y[kk][jj].x == vmax) flat = min(flat, base + j);
          if (g.mirror && y[kk][jj].y == vmax) flat = min(flat, base + M + ((j + M / 2) & (M - 1)));
        }
    }
#pragma unroll
    for (int off = T / 2; off > 0; off >>= 1) flat = min(flat, __shfl_xor_sync(0xffffffffu, flat, off, T));
    if (cand && t == 0) atomicMax(a.best + img, make_key(vmax, flat));
  }
}

template <int M, int KT>
static cudaError_t launch_cc_t(const Geometry &g, const CCArgs &a, cudaStream_t st) {
  using Sh = CCShape<M, KT>;
  const size_t smem = Sh::smem(a.seg_max);
  static size_t granted = 0;
  cudaError_t e = raise_smem_limit(cc_fp32_kernel<M, KT>, smem, granted);
  if (e != cudaSuccess) return e;
  const int64_t row_tiles = (a.rows + Sh::RT - 1) / Sh::RT;
  const int ref_tiles = (a.K + KT - 1) / KT;
  if (row_tiles <= 0) return cudaSuccess;
  dim3 grid(ref_tiles, static_cast<unsigned>(row_tiles));
  cc_fp32_kernel<M, KT><<<grid, Sh::THREADS, smem, st>>>(g, a);
  return cudaGetLastError();
}

size_t cc_fp32_smem(int M, int seg_max) {
  switch (M) {
    case 16: return CCShape<16, 8>::smem(seg_max);
    case 32: return CCShape<32, 8>::smem(seg_max);
    case 64: return CCShape<64, 8>::smem(seg_max);
    case 128: return CCShape<128, 8>::smem(seg_max);
    case 256: return CCShape<256, 8>::smem(seg_max);
    case 512: return CCShape<512, 4>::smem(seg_max);
    default: return 0;
  }
}

cudaError_t launch_cc_fp32(const Geometry &g, const CCArgs &a, cudaStream_t st) {
  switch (g.M) {
    case 16: return launch_cc_t<16, 8>(g, a, st);
    case 32: return launch_cc_t<32, 8>(g, a, st);
    case 64: return launch_cc_t<64, 8>(g, a, st);
    case 128: return launch_cc_t<128, 8>(g, a, st);
    case 256: return launch_cc_t<256, 8>(g, a, st);
    case 512: return launch_cc_t<512, 4>(g, a, st);
    default: return cudaErrorInvalidValue;
  }
}

// Pose decode (Alg. 1, parameter-lookup step: the argmax index becomes the
// reference, angle, shift and mirror of the image).
__global__ void decode_kernel(Geometry g, const unsigned long long *best, int64_t n, int K,
                              mra_pose_t *poses) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long key = best[i];
  const uint32_t flat = 0xffffffffu - static_cast<uint32_t>(key & 0xffffffffull);
  const float cc = ordered_to_float(static_cast<uint32_t>(key >> 32));
  const int M = g.M;
  const int j = static_cast<int>(flat % M);
  uint32_t rest = flat / M;
  const int m = static_cast<int>(rest & 1u);
  rest >>= 1;
  const int s = static_cast<int>(rest % g.S);
  const int k = static_cast<int>(rest / g.S);
  mra_pose_t p;
  p.k = k;
  p.ang_idx = j;
  p.mirror = m;
  p.shift_idx = s;
  p.angle_deg = static_cast<float>(360.0 * j / M);
  const float2 sh = g.shifts[s < g.S ? s : 0];
  p.sx = sh.x;
  p.sy = sh.y;
  p.cc = cc;
  poses[i] = p;
}

cudaError_t launch_decode(const Geometry &g, const unsigned long long *best, int64_t n, int K,
                          void *poses, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  decode_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(
      g, best, n, K, static_cast<mra_pose_t *>(poses));
  return cudaGetLastError();
}

}  // namespace mra
