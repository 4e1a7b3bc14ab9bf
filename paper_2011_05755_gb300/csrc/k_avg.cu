// Class averaging (Alg. 1, class-average step: the new references Y' are
// built from the aligned particles; the paper runs this step in CuPy, Sec. 3).
//
// For class k: avg_k(c0 + w) = (1/n_k) sum_{i: k_i = k} I_i(c0 + s_i + Mm_i R(-phi_i) w)
// on the integer grid w, bilinear with zero outside the box.
//
// Determinism without floating-point atomics:
//  1. a stable counting sort groups image indices by class (per-block
//     histograms, one exclusive scan, per-block stable ranks);
//  2. each class is cut into chunks of kAvgChunk consecutive images; a CTA
//     sums one chunk over a block of pixels in image order with Neumaier
//     compensation (running sum s and correction c, value = s + c);
//  3. the chunk partials of a class are combined in chunk order.
// The order of every floating-point addition is fixed by the image indices,
// so repeated calls give bit-identical results.
#include "../../include/mra.h"
#include "dev_util.cuh"
#include "mra_internal.h"

namespace mra {

// Neumaier's compensated addition: s + v into (s, c), with c gathering the
// rounding error of every addition (the total is s + c).
__device__ __forceinline__ void neumaier_add(float &s, float &c, float v) {
  const float t = s + v;
  if (fabsf(s) >= fabsf(v))
    c += (s - t) + v;
  else
    c += (v - t) + s;
  s = t;
}

__device__ __forceinline__ float bilinear_avg(const float *__restrict__ img, int L, float x, float y) {
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

// 1a. per-block class histogram, stored class-major: hist[k * nblk + b]
__global__ void avg_hist_kernel(const mra_pose_t *poses, int64_t n, int K, int nblk, int *hist) {
  extern __shared__ int sh_hist[];
  for (int k = threadIdx.x; k < K; k += blockDim.x) sh_hist[k] = 0;
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kAvgBlock + threadIdx.x;
  if (i < n) {
    const int k = poses[i].k;
    if (k >= 0 && k < K) atomicAdd(&sh_hist[k], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) hist[static_cast<int64_t>(k) * nblk + blockIdx.x] = sh_hist[k];
}

// 1b. exclusive scan of hist (one CTA) in class-major order, so class k
//     starts at scan[k * nblk]; per-class counts and the chunk directory
//     (class k owns chunks [first[k], first[k+1])).
__global__ void avg_scan_kernel(const int *hist, int *scan, int K, int nblk, int *counts,
                                int *class_first_chunk, int *n_chunks) {
  __shared__ int part[1024];
  __shared__ int total;
  const int64_t len = static_cast<int64_t>(K) * nblk;
  const int64_t per = (len + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = min(len, static_cast<int64_t>(threadIdx.x) * per);
  const int64_t b1 = min(len, b0 + per);
  int s = 0;
  for (int64_t i = b0; i < b1; ++i) s += hist[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int i = 0; i < static_cast<int>(blockDim.x); ++i) {
      const int v = part[i];
      part[i] = run;
      run += v;
    }
    total = run;
  }
  __syncthreads();
  int run = part[threadIdx.x];
  for (int64_t i = b0; i < b1; ++i) {
    const int v = hist[i];
    scan[i] = run;
    run += v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const int start = scan[static_cast<int64_t>(k) * nblk];
    const int end = (k + 1 < K) ? scan[static_cast<int64_t>(k + 1) * nblk] : total;
    counts[k] = end - start;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int chunks = 0;
    for (int k = 0; k < K; ++k) {
      class_first_chunk[k] = chunks;
      chunks += (counts[k] + kAvgChunk - 1) / kAvgChunk;
    }
    class_first_chunk[K] = chunks;
    *n_chunks = chunks;
  }
}

// 1c. stable scatter of image indices into class order.
__global__ void avg_scatter_kernel(const mra_pose_t *poses, int64_t n, int K, int nblk, const int *scan,
                                   int *perm) {
  __shared__ int ks[kAvgBlock];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kAvgBlock + threadIdx.x;
  int k = -1;
  if (i < n) {
    k = poses[i].k;
    if (k < 0 || k >= K) k = -1;
  }
  ks[threadIdx.x] = k;
  __syncthreads();
  if (k >= 0) {
    int rank = 0;
    for (int j = 0; j < static_cast<int>(threadIdx.x); ++j) rank += (ks[j] == k);
    perm[scan[static_cast<int64_t>(k) * nblk + blockIdx.x] + rank] = static_cast<int>(i);
  }
}

// 1d. chunk directory entries (class, first image slot, count).
__global__ void avg_chunks_kernel(int K, const int *counts, const int *class_first_chunk, const int *scan,
                                  int nblk, int *chunk_class, int *chunk_begin, int *chunk_count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int c = counts[k];
  const int start = scan[static_cast<int64_t>(k) * nblk];
  const int f0 = class_first_chunk[k];
  for (int j = 0; j * kAvgChunk < c; ++j) {
    chunk_class[f0 + j] = k;
    chunk_begin[f0 + j] = start + j * kAvgChunk;
    chunk_count[f0 + j] = min(kAvgChunk, c - j * kAvgChunk);
  }
}

// 2. partial compensated sums of one chunk over 1024 pixels (4 per thread).
constexpr int kPixPerThread = 4;
__global__ void __launch_bounds__(256) avg_chunk_sum_kernel(Geometry g, const float *imgs,
                                                            const mra_pose_t *poses, const int *perm,
                                                            const int *n_chunks, const int *chunk_begin,
                                                            const int *chunk_count, float *part_sum,
                                                            float *part_comp) {
  const int ch = blockIdx.x;
  if (ch >= *n_chunks) return;
  const int L = g.L;
  const int LL = L * L;
  const float c0 = 0.5f * static_cast<float>(L);
  float s[kPixPerThread], c[kPixPerThread], wx[kPixPerThread], wy[kPixPerThread];
  int px[kPixPerThread];
#pragma unroll
  for (int u = 0; u < kPixPerThread; ++u) {
    px[u] = blockIdx.y * (256 * kPixPerThread) + u * 256 + threadIdx.x;
    s[u] = 0.f;
    c[u] = 0.f;
    const int y = px[u] / L, x = px[u] - (px[u] / L) * L;
    wx[u] = static_cast<float>(x) - c0;
    wy[u] = static_cast<float>(y) - c0;
  }
  const int b = chunk_begin[ch], cnt = chunk_count[ch];
  for (int e = 0; e < cnt; ++e) {
    const int i = perm[b + e];
    const mra_pose_t p = poses[i];
    int j = p.ang_idx % g.M;
    if (j < 0) j += g.M;
    const float2 cs = g.angles[j];
    const float *img = imgs + static_cast<int64_t>(i) * LL;
    const float sgn = p.mirror ? -1.f : 1.f;
#pragma unroll
    for (int u = 0; u < kPixPerThread; ++u) {
      if (px[u] < LL) {
        // R(-phi) w, then the mirror on x, then the shift
        const float rx = fmaf(cs.x, wx[u], cs.y * wy[u]);
        const float ry = fmaf(-cs.y, wx[u], cs.x * wy[u]);
        const float v = bilinear_avg(img, L, c0 + p.sx + sgn * rx, c0 + p.sy + ry);
        neumaier_add(s[u], c[u], v);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kPixPerThread; ++u)
    if (px[u] < LL) {
      part_sum[static_cast<int64_t>(ch) * LL + px[u]] = s[u];
      part_comp[static_cast<int64_t>(ch) * LL + px[u]] = c[u];
    }
}

// 3. ordered combination of a class's chunk partials; optionally added into
//    existing (sum, comp, counts) for sharded use.
__global__ void avg_class_combine_kernel(Geometry g, int K, const int *class_first_chunk,
                                         const float *part_sum, const float *part_comp, const int *cnt_in,
                                         float *sum, float *comp, int *counts, bool accumulate) {
  const int k = blockIdx.x;
  const int LL = g.L * g.L;
  const int px = blockIdx.y * blockDim.x + threadIdx.x;
  if (px < LL) {
    float s = 0.f, c = 0.f;
    if (accumulate) {
      s = sum[static_cast<int64_t>(k) * LL + px];
      c = comp[static_cast<int64_t>(k) * LL + px];
    }
    for (int ch = class_first_chunk[k]; ch < class_first_chunk[k + 1]; ++ch) {
      neumaier_add(s, c, part_sum[static_cast<int64_t>(ch) * LL + px]);
      c += part_comp[static_cast<int64_t>(ch) * LL + px];
    }
    sum[static_cast<int64_t>(k) * LL + px] = s;
    comp[static_cast<int64_t>(k) * LL + px] = c;
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) counts[k] = (accumulate ? counts[k] : 0) + cnt_in[k];
}

__global__ void avg_finalize_kernel(int LL, const float *sum, const float *comp, const int *counts, float *avg) {
  const int k = blockIdx.x;
  const int cnt = counts[k];
  if (cnt <= 0) return;  // empty class: leave avg untouched
  const float inv = 1.0f / static_cast<float>(cnt);
  for (int px = blockIdx.y * blockDim.x + threadIdx.x; px < LL; px += gridDim.y * blockDim.x) {
    const int64_t o = static_cast<int64_t>(k) * LL + px;
    avg[o] = (sum[o] + comp[o]) * inv;
  }
}

// Compensated sum over the CTA of each thread's (s, c), in a fixed tree
// order (deterministic); returns s + c to every thread.
__device__ __forceinline__ float cta_sum_compensated(float s, float c, float *rs, float *rc) {
  rs[threadIdx.x] = s;
  rc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      float a = rs[threadIdx.x], ca = rc[threadIdx.x] + rc[threadIdx.x + w];
      neumaier_add(a, ca, rs[threadIdx.x + w]);
      rs[threadIdx.x] = a;
      rc[threadIdx.x] = ca;
    }
    __syncthreads();
  }
  const float total = rs[0] + rc[0];
  __syncthreads();
  return total;
}

// Requires n >= 1 (the C-ABI layer handles n == 0).
// Reference refresh: reseed empty classes from a chosen image, then
// normalise every populated (or reseeded) class to zero mean and unit
// standard deviation over the box.  One CTA per class; two passes (the
// mean, then the centred second moment), each summed in FP32 with Neumaier
// compensation in a fixed reduction order; 1 / sqrt(var) from correctly
// rounded square root and division.
__global__ void __launch_bounds__(256) refresh_refs_kernel(int L, float *refs, const int *counts, const int *reseed,
                                                           const float *imgs, int64_t n) {
  const int k = blockIdx.x;
  const int LL = L * L;
  float *r = refs + static_cast<int64_t>(k) * LL;
  int src = -1;
  if (counts[k] <= 0) {
    src = reseed ? reseed[k] : -1;
    if (src < 0 || src >= n || !imgs) return;  // leave the class as it is
    const float *im = imgs + static_cast<int64_t>(src) * LL;
    for (int i = threadIdx.x; i < LL; i += blockDim.x) r[i] = im[i];
    __syncthreads();
  }
  __shared__ float rs[256], rc[256];
  float s = 0.f, c = 0.f;
  for (int i = threadIdx.x; i < LL; i += blockDim.x) neumaier_add(s, c, r[i]);
  const float mean = cta_sum_compensated(s, c, rs, rc) / static_cast<float>(LL);
  s = 0.f;
  c = 0.f;
  for (int i = threadIdx.x; i < LL; i += blockDim.x) {
    const float d = r[i] - mean;
    neumaier_add(s, c, d * d);
  }
  const float var = cta_sum_compensated(s, c, rs, rc) / static_cast<float>(LL);
  const float inv = var > 0.f ? __fdiv_rn(1.0f, __fsqrt_rn(var)) : 0.f;
  for (int i = threadIdx.x; i < LL; i += blockDim.x) r[i] = (r[i] - mean) * inv;
}

cudaError_t launch_refresh_refs(int L, float *refs, const int *counts, int K, const int *reseed, const float *imgs,
                                int64_t n, cudaStream_t st) {
  refresh_refs_kernel<<<K, 256, 0, st>>>(L, refs, counts, reseed, imgs, n);
  return cudaGetLastError();
}

cudaError_t launch_class_sums(const Geometry &g, const float *imgs, const void *poses_v, int64_t n, int K,
                              const AvgWork &w, float *sum, float *comp, int *counts, bool accumulate,
                              cudaStream_t st) {
  const mra_pose_t *poses = static_cast<const mra_pose_t *>(poses_v);
  const int nblk = static_cast<int>((n + kAvgBlock - 1) / kAvgBlock);
  const int LL = g.L * g.L;
  avg_hist_kernel<<<nblk, kAvgBlock, K * sizeof(int), st>>>(poses, n, K, nblk, w.hist);
  avg_scan_kernel<<<1, 1024, 0, st>>>(w.hist, w.scan, K, nblk, w.class_counts, w.class_first_chunk, w.n_chunks);
  avg_scatter_kernel<<<nblk, kAvgBlock, 0, st>>>(poses, n, K, nblk, w.scan, w.perm);
  avg_chunks_kernel<<<(K + 255) / 256, 256, 0, st>>>(K, w.class_counts, w.class_first_chunk, w.scan, nblk,
                                                     w.chunk_class, w.chunk_begin, w.chunk_count);
  dim3 grid(w.max_chunks, (LL + 256 * kPixPerThread - 1) / (256 * kPixPerThread));
  avg_chunk_sum_kernel<<<grid, 256, 0, st>>>(g, imgs, poses, w.perm, w.n_chunks, w.chunk_begin, w.chunk_count,
                                             w.part_sum, w.part_comp);
  dim3 g2(K, (LL + 255) / 256);
  avg_class_combine_kernel<<<g2, 256, 0, st>>>(g, K, w.class_first_chunk, w.part_sum, w.part_comp,
                                               w.class_counts, sum, comp, counts, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_average_finalize(const Geometry &g, int K, const float *sum, const float *comp,
                                    const int *counts, float *avg, cudaStream_t st) {
  const int LL = g.L * g.L;
  dim3 grid(K, (LL + 255) / 256 < 64 ? (LL + 255) / 256 : 64);
  avg_finalize_kernel<<<grid, 256, 0, st>>>(LL, sum, comp, counts, avg);
  return cudaGetLastError();
}

}  // namespace mra
