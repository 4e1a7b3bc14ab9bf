// FP32 rescore of the precision-split path's candidate rows: the 8 rows
// (reference, shift, mirror) per image with the largest 16-bit row maxima
// are recomputed from the image in FP32, and the argmax over them is the
// answer (Algorithm 1's reduction restricted to those rows).
#include "../../include/mra.h"
#include "dev_util.cuh"
#include "mra_internal.h"
#include "pair_ifft.cuh"
#include "ring_fft.cuh"
#include "smem_limit.cuh"

namespace mra {

constexpr int kRescoreThreads = 256;  // 8 warps per CTA (one image)

// ---------------------------------------------------------------------------
// FP32 rescore: for each candidate row of an image, resample at its shift,
// ring-FFT, contract with its reference in FP32, inverse DFT; keep the best
// (value, smallest index) over the candidates' angles as the argmax key.
// One CTA per image.
// ---------------------------------------------------------------------------
// Registers are held to 64 per thread for M = 32..256, so that four CTAs
// (images) fit on an SM where their shared memory allows (the 76-pixel
// workload).
template <int M>
__global__ void __launch_bounds__(kRescoreThreads, (M >= 32 && M <= 256) ? 4 : 1)
    rescore_kernel(Geometry g, RescoreArgs a) {
  constexpr int T = IfftShape<M>::T;
  constexpr int U = IfftShape<M>::U;
  extern __shared__ float4 smem_f4[];
  const int L = g.L, NS = g.NS, S = g.S;
  const int LL = L * L;
  const int LLp = (LL + 3) & ~3;
  const int64_t img = blockIdx.x;
  float *im = reinterpret_cast<float *>(smem_f4);
  float2 *twf = reinterpret_cast<float2 *>(im + LLp);
  float2 *twi = twf + M;
  float2 *Z = twi + M;
  // ring samples, then (in place) each ring's spectrum: N real samples are
  // transformed as N/2 complex values and split into the bins X(0..N/2) in the
  // same N floats, with the two real bins packed as (X(0), X(N/2)) in slot 0
  float *samp = reinterpret_cast<float *>(Z + IfftShape<M>::P);
  int4 *s_rings = reinterpret_cast<int4 *>((reinterpret_cast<uintptr_t>(samp + g.NS) + 15) & ~uintptr_t(15));  // [NR]
  const float c0 = 0.5f * static_cast<float>(L);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NR = g.NR;

  {
    // the image, four 16-byte loads in flight per thread (when the rows allow)
    const float *src = a.imgs + img * LL;
    if ((LL & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
      const float4 *s4 = reinterpret_cast<const float4 *>(src);
      float4 *d4 = reinterpret_cast<float4 *>(im);
      for (int i0 = threadIdx.x; i0 < LL / 4; i0 += 4 * blockDim.x) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * blockDim.x;
          if (i < LL / 4) v[u] = __ldg(s4 + i);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * blockDim.x;
          if (i < LL / 4) d4[i] = v[u];
        }
      }
    } else {
      for (int i = threadIdx.x; i < LL; i += blockDim.x) im[i] = __ldg(src + i);
    }
  }
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    twf[i] = g.fwd_tw[i];
    twi[i] = g.inv_tw[i];
  }
  for (int i = threadIdx.x; i < NR; i += blockDim.x) s_rings[i] = g.rings[i];
  unsigned long long best = 0ull;
  __syncthreads();
  // Warp 0 runs each candidate's inverse DFT at the end of its iteration;
  // warps 1-7 resample the next candidate meanwhile (its samples are not
  // read by the inverse DFT, and warp 0 joins the barrier after resampling
  // only once its inverse DFT is done, before the spectrum buffer is
  // rewritten).
  for (int c = 0; c < kTopRows; ++c) {
    const int rowid = a.cand[img * kTopRows + c];
    if (rowid < 0) continue;  // uniform over the CTA
    const int m = rowid & 1;
    const int rs = rowid >> 1;
    const int s = rs % S;
    const int k = rs / S;
    if (warp > 0) {
      // the sample offsets of eight samples per thread in flight before they are used
      const float2 sh = g.shifts[s];
      const int nt = blockDim.x - 32;
      for (int q0 = threadIdx.x - 32; q0 < NS; q0 += 8 * nt) {
        float2 o[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = q0 + u * nt;
          if (q < NS) o[u] = __ldg(g.offs + q);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = q0 + u * nt;
          if (q < NS) samp[q] = bilinear_smem(im, L, c0 + sh.x + o[u].x, c0 + sh.y + o[u].y);
        }
      }
    }
    __syncthreads();
    for (int ring = NR - 1 - warp; ring >= 0; ring -= kRescoreThreads / 32) {
      const int4 rd = s_rings[ring];
      const int N = rd.x, H = N >> 1;
      float2 *z = reinterpret_cast<float2 *>(samp + rd.y);
      warp_fft_inplace(z, H, rd.w, M, twf, lane);
      __syncwarp();
      // in-place split: lane pair {kx, H - kx} reads and writes only its two slots
      const int wstep = M / N;
      for (int kx = lane; kx <= H / 2; kx += 32) {
        if (kx == 0) {
          const float2 x0 = real_split(z, H, 0, twf[0]), xh = real_split(z, H, H, twf[H * wstep]);
          z[0] = make_float2(x0.x, xh.x);  // both bins are real
        } else {
          const float2 xa = real_split(z, H, kx, twf[kx * wstep]);
          const float2 xb = real_split(z, H, H - kx, twf[(H - kx) * wstep]);
          z[kx] = xa;
          z[H - kx] = xb;
        }
      }
      __syncwarp();
    }
    __syncthreads();
    // FP32 contraction with reference k for every frequency: the lowest n2
    // frequencies (the most rings) by two threads each (alternate rings,
    // partial sums combined by a shuffle), the others by one thread, n2 as
    // large as fills the fewest whole passes of the CTA (M = 256: 129
    // frequencies in one pass; M = 512: 257 in two); the reference loads of
    // four rings in flight at a time
    constexpr int NF = M / 2 + 1;
    constexpr int kPasses = (NF + kRescoreThreads - 1) / kRescoreThreads;
    constexpr int n2 = NF < kPasses * kRescoreThreads - NF ? NF : kPasses * kRescoreThreads - NF;
    constexpr int NITEMS = NF + n2;
    const float2 *Bk = a.B + static_cast<int64_t>(k / kTile) * g.NB * kTile + (k % kTile);
    for (int it0 = 0; it0 < NITEMS; it0 += blockDim.x) {  // uniform trip count (shuffles below)
      const int it = it0 + threadIdx.x;
      const bool active = it < NITEMS;
      const bool split = it < 2 * n2;  // even count: the one-thread items start on an even lane
      const int f = !active ? 0 : (split ? it >> 1 : n2 + (it - 2 * n2));
      const int half = split ? (it & 1) : 0, step = split ? 2 : 1;
      float p1 = 0.f, p2 = 0.f, p3 = 0.f, p4 = 0.f;
      if (active) {
        // rings with N_r / 2 >= f are a suffix [lo, NR) of the (ascending) ring list
        int lo = 0, hi = NR;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (s_rings[mid].x / 2 < f) lo = mid + 1;
          else hi = mid;
        }
        const float2 *Bf = Bk + static_cast<int64_t>(g.kpos[f]) * kTile;  // bin (ring, f) at kpos[f] + ring
#pragma unroll 4
        for (int ring = NR - 1 - half; ring >= lo; ring -= step) {
          const int4 rd = s_rings[ring];
          const float2 *zr = reinterpret_cast<const float2 *>(samp + rd.y);
          const float2 z0 = zr[0];
          const float2 A = f == 0 ? make_float2(z0.x, 0.f) : (2 * f == rd.x ? make_float2(z0.y, 0.f) : zr[f]);
          const float2 Bv = __ldg(Bf + static_cast<int64_t>(ring) * kTile);
          p1 = fmaf(A.x, Bv.x, p1);
          p2 = fmaf(A.y, Bv.y, p2);
          p3 = fmaf(A.x, Bv.y, p3);
          p4 = fmaf(A.y, Bv.x, p4);
        }
      }
      // the two items of a split frequency are neighbouring lanes of one warp
      const float q1 = __shfl_xor_sync(0xffffffffu, p1, 1), q2 = __shfl_xor_sync(0xffffffffu, p2, 1);
      const float q3 = __shfl_xor_sync(0xffffffffu, p3, 1), q4 = __shfl_xor_sync(0xffffffffu, p4, 1);
      if (split) {
        p1 += q1;
        p2 += q2;
        p3 += q3;
        p4 += q4;
      }
      if (active && half == 0) {
        Z[f] = make_float2((p1 + p2) - (p3 + p4), (p3 - p4) + (p1 - p2));
        if (f != 0 && f != M / 2) Z[M - f] = make_float2((p1 + p2) + (p3 + p4), (p1 - p2) - (p3 - p4));
      }
    }
    __syncthreads();
    if (warp == 0) {
      const int tt = lane % T;
      const bool owner = lane < T;
      float2 y[IfftShape<M>::KK][T];
      pair_ifft<M>(Z, 0, Z, tt, owner, twi, y);
      float v = -INFINITY;
      uint32_t ang = 0xffffffffu;
#pragma unroll
      for (int kk = 0; kk < U / T; ++kk)
#pragma unroll
        for (int jj = 0; jj < T; ++jj) {
          const int j = ifft_angle<M>(tt, kk, jj);
          const float x = m ? y[kk][jj].y : y[kk][jj].x;
          const uint32_t aj = m ? static_cast<uint32_t>((j + M / 2) & (M - 1)) : static_cast<uint32_t>(j);
          if (x > v || (x == v && aj < ang)) {
            v = x;
            ang = aj;
          }
        }
      unsigned long long key = owner ? make_key(v, static_cast<uint32_t>(rowid) * M + ang) : 0ull;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, off);
        key = o > key ? o : key;
      }
      if (lane == 0 && key > best) best = key;
    }
  }
  if (threadIdx.x == 0) a.best[img] = best;
}

size_t rescore_smem(const Geometry &g) {
  const int T = g.M >= 256 ? 16 : g.M / 16;
  const int P = T * (g.M / T + 1);
  return static_cast<size_t>((g.L * g.L + 3) & ~3) * sizeof(float) + (2 * g.M + P) * sizeof(float2) +
         static_cast<size_t>(g.NS) * sizeof(float) + 16 + static_cast<size_t>(g.NR) * sizeof(int4);
}

// The kernel's dynamic shared-memory limit only ever grows (handles of
// several geometries share the kernel).
template <int M>
static cudaError_t rescore_smem_attr(size_t smem) {
  static size_t granted = 0;
  return raise_smem_limit(rescore_kernel<M>, smem, granted);
}

template <int M>
static cudaError_t launch_rescore_t(const Geometry &g, const RescoreArgs &a, cudaStream_t st) {
  const size_t smem = rescore_smem(g);
  cudaError_t e = rescore_smem_attr<M>(smem);
  if (e != cudaSuccess) return e;
  rescore_kernel<M><<<static_cast<unsigned>(a.n), kRescoreThreads, smem, st>>>(g, a);
  return cudaGetLastError();
}

template <int M>
static int rescore_occupancy_t(const Geometry &g) {
  const size_t smem = rescore_smem(g);
  int n = 0;
  if (rescore_smem_attr<M>(smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rescore_kernel<M>, kRescoreThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int rescore_ctas_per_sm(const Geometry &g) {
  switch (g.M) {
    case 16: return rescore_occupancy_t<16>(g);
    case 32: return rescore_occupancy_t<32>(g);
    case 64: return rescore_occupancy_t<64>(g);
    case 128: return rescore_occupancy_t<128>(g);
    case 256: return rescore_occupancy_t<256>(g);
    case 512: return rescore_occupancy_t<512>(g);
    default: return 0;
  }
}

cudaError_t launch_rescore(const Geometry &g, const RescoreArgs &a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  switch (g.M) {
    case 16: return launch_rescore_t<16>(g, a, st);
    case 32: return launch_rescore_t<32>(g, a, st);
    case 64: return launch_rescore_t<64>(g, a, st);
    case 128: return launch_rescore_t<128>(g, a, st);
    case 256: return launch_rescore_t<256>(g, a, st);
    case 512: return launch_rescore_t<512>(g, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mra
