// Polar resampling and ring FFT (Alg. 1, shift-loop conversion step: each
// particle is resampled on the rings about its shifted centre and every ring
// is Fourier transformed; the references get the same with no shift,
// followed by the ring weights of the Sec. 2 quadrature).
//
// A CTA stages one image in shared memory and walks groups of R consecutive
// rows (row = image * rows_per_img + shift): the groups blockIdx.x,
// blockIdx.x + gridDim.x, ...  Per group, phase 1 writes the bilinear
// samples of its rows into shared memory; phase 2
// gives each warp one (row, ring) job: an in-place N/2-point complex FFT of
// the ring's real samples packed as z_q = x_{2q} + i x_{2q+1}, then the
// split into the N/2 + 1 real-input bins X(f), written straight into the
// frequency-major tiled layout [row / 8][bin][row % 8] (FP32 path), or, for
// the 16-bit tensor-core paths, into the mma.sync A-fragment order: per tile
// of 8 rows and k-step of 16 rings of one frequency, lane 4g + t of a warp
// holds {q[g][2t..2t+1], p[g][2t..2t+1], q[g][2t+8..9], p[g][2t+8..9]} with
// q = Re X - Im X and p = Re X + Im X (rows 0-7 of the MMA are the q values of
// the 8 tile rows, rows 8-15 their p values).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dev_util.cuh"
#include "mra_internal.h"
#include "ring_fft.cuh"
#include "smem_limit.cuh"
#include "tma.cuh"

namespace mra {

// Row stride of the sample buffer: >= NS and 16 floats off a multiple of 32,
// so the ring-FFT jobs of consecutive rows start in opposite halves of the
// shared-memory banks.
__host__ __device__ inline int sample_stride(int NS) { return NS + ((16 - NS) & 31); }

// Output layouts of the polar kernel: FP32 frequency-major tiles, or the
// 16-bit q / p planes (BF16 or FP16) that phase 3 turns into mma.sync
// fragments (kOutBF16, kOutF16) or into the k-step tiles of the tcgen05
// path (kOutUBF16, kOutUF16: per tile of 16 rows and MMA k-step u a
// 128 x 16 operand in the canonical K-major layout, row = frequency slot * 32
// + (q|p) * 16 + row in tile; see k_umma256.cu).
enum PolarOut { kOutF32 = 0, kOutBF16 = 1, kOutF16 = 2, kOutUBF16 = 3, kOutUF16 = 4 };
__host__ __device__ constexpr bool out_is_fp16(int out) { return out == kOutF16 || out == kOutUF16; }
__host__ __device__ constexpr bool out_is_umma(int out) { return out == kOutUBF16 || out == kOutUF16; }

// (q, p) of one bin packed as a 16-bit pair word: q low, p high.
template <int OUT>
__device__ __forceinline__ uint32_t pack_qp(float q, float p) {
  if constexpr (out_is_fp16(OUT)) {
    const __half2 h = __floats2half2_rn(q, p);  // .x (low half) = q
    return *reinterpret_cast<const uint32_t *>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(q, p);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
}

// Position of word w (k-step w / 16, word w % 16) in a row of the (q, p)
// planes: the word index inside the k-step is XORed with (k-step & 14), so
// that the stores of one ring's consecutive frequencies (k-steps 1, 2 or 3
// apart, same word) fall in different banks.  The XOR keeps word pairs
// (2j, 2j + 1) adjacent.
__device__ __forceinline__ int plane_swz(int w) { return w ^ ((w >> 4) & 14); }

// One bin of a particle or reference row into the path's output layout
// (weights for references, the debug copy, FP32 tiles or 16-bit words).
template <int OUT>
__device__ __forceinline__ void put_bin(const Geometry &g, const PolarArgs &a, uint32_t *planes_row, const int *s_kpos,
                                        int ring, int bin0, int64_t row, int k, float2 X) {
  if (a.weighted) {
    const float w = g.bweight[bin0 + k];
    X.x *= w;
    X.y *= w;
  }
  if (a.dbg_spec) a.dbg_spec[row * g.NBIN + bin0 + k] = X;
  if constexpr (OUT == kOutF32) {
    if (a.out) a.out[((row >> 3) * g.NB + s_kpos[k] + ring) * kTile + (row & 7)] = X;
  } else {
    const int w = s_kpos[k] + ring;  // k-step w / 16, word w % 16 of it
    planes_row[plane_swz(w)] = pack_qp<OUT>(X.x - X.y, X.x + X.y);
  }
}

// All (ring, row) jobs of one ring-length class [i0, i1) of a CTA: forward
// FFT of the packed samples, real split, weights, and the spectrum written in
// the layout the path needs (FP32 tiled, 16-bit q/p words, debug).  s_kpos
// holds the per-frequency base of the output layout: bin (ring, k) goes to
// s_kpos[k] + ring.
template <int H, int R, int OUT>
__device__ __forceinline__ int ring_class(const Geometry &g, const PolarArgs &a, float *smem, uint32_t *planes,
                                          int NB16, const float2 *tws, const int *s_kpos, int i0, int i1, int nrows,
                                          int64_t row0, int warp, int lane, int nwarps, int first_warp) {
  constexpr int T = GroupFft<H>::T;
  constexpr int JPW = 32 / T;  // jobs per warp pass
  const int njobs = (i1 - i0) * nrows;
  const int t = lane % T;
  // warp passes of this class start after the previous class's last pass
  const int wslot = (warp - first_warp + nwarps) % nwarps;
  for (int j0 = wslot * JPW; j0 < njobs; j0 += nwarps * JPW) {
    const int job = j0 + lane / T;
    const bool active = job < njobs;
    const int jc = active ? job : j0;
    // (ring, row) of the job; nrows is R except in an image's last group
    const int ring = i0 + (nrows == R ? jc / R : jc / nrows);
    const int i = nrows == R ? jc % R : jc % nrows;
    const int4 rd = g.rings[ring];  // {N, sample offset, natural-bin offset, log2(N/2)}
    float2 *z = reinterpret_cast<float2 *>(smem + i * sample_stride(g.NS) + rd.y);
    group_fft<H>(z, t, active, tws, g.M);
    if (active) {
      const int wstep = g.M / (2 * H);
      const int64_t row = row0 + i;
      uint32_t *prow = planes + i * NB16;
      // bins k and H - k from one pair of loads and one twiddle
      for (int k = t; 2 * k <= H; k += T) {
        float2 xk, xhk;
        real_split_pair(z, H, k, tws[k * wstep], xk, xhk);
        put_bin<OUT>(g, a, prow, s_kpos, ring, rd.z, row, k, xk);
        if (2 * k != H) put_bin<OUT>(g, a, prow, s_kpos, ring, rd.z, row, H - k, xhk);
      }
    }
    __syncwarp();
  }
  return (first_warp + (njobs + JPW - 1) / JPW) % nwarps;  // first warp of the next class
}

// Shared-memory image floats: the image, or (TAPS) the image inside a zero
// border of g.pad pixels.
__host__ __device__ inline int image_floats(const Geometry &g, bool taps) {
  const int Lp = taps ? g.L + 2 * g.pad : g.L;
  return (Lp * Lp + 3) & ~3;
}

template <int R, bool TAPS, int OUT>
__global__ void __launch_bounds__(256, 2) polar_fft_kernel(Geometry g, const __grid_constant__ PolarArgs a) {
  extern __shared__ float4 smem_f4[];
  const int L = g.L, NS = g.NS, M = g.M;
  const int NSp = sample_stride(NS);
  const int LL = L * L;
  const int64_t img = blockIdx.y;
  float *im = reinterpret_cast<float *>(smem_f4);       // the image (with its zero border if TAPS)
  uint64_t *ibar = reinterpret_cast<uint64_t *>(im + image_floats(g, TAPS));  // image copy barrier (16 B)
  float2 *tws = reinterpret_cast<float2 *>(im + image_floats(g, TAPS) + 4);  // [M] forward twiddles
  int *s_kpos = reinterpret_cast<int *>(tws + M);       // [M/2 + 1] output bases (padded to even)
  float *smem = reinterpret_cast<float *>(s_kpos + ((M / 2 + 2) & ~1));  // [R][NSp] samples, then ring FFTs
  const float c0 = 0.5f * static_cast<float>(L);
  // 16-bit paths: (q, p) words [row][NB16] after the samples; the padding
  // words are zeroed once, every group rewrites the same non-padding words
  const int NB16 = g.KS * 16;
  uint32_t *planes = reinterpret_cast<uint32_t *>(smem + R * NSp);
  if constexpr (OUT != kOutF32)
    for (int idx = threadIdx.x; idx < R * NB16; idx += blockDim.x) planes[idx] = 0u;
  {
    const int *kp = OUT == kOutF32 ? g.kpos : g.kpos16;
    for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) s_kpos[k] = kp[k];
  }
  const float *src = a.imgs + img * LL;
  const bool vec = (L & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
  // TMA staging: one tensor copy of the image (and, with TAPS, its zero
  // border from the map's out-of-bounds fill), issued by thread 0 while the
  // CTA loads its tables; the destination must be 128-byte aligned
  const bool tma = a.tma && (smem_u32(im) & 127u) == 0;
  if (tma) {
    if (threadIdx.x == 0) {
      mbar_init(ibar, 1);
      mbar_init_fence();
      const int pad = TAPS ? g.pad : 0;
      const int Lp = L + 2 * pad;
      mbar_arrive_expect_tx(ibar, static_cast<uint32_t>(Lp * Lp) * 4u);
      tma_load_3d(im, &a.tmap, -pad, -pad, static_cast<int>(img), ibar);
    }
  } else if constexpr (TAPS) {
    // zero the bordered buffer, then copy the interior (pad is a multiple of 4)
    const int Lp = L + 2 * g.pad;
    for (int i = threadIdx.x; i < image_floats(g, true) / 4; i += blockDim.x)
      reinterpret_cast<float4 *>(im)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    float *dst = im + g.pad * Lp + g.pad;
    if (vec) {
      const int W = L / 4;
      for (int i = threadIdx.x; i < L * W; i += blockDim.x) {
        const int y = i / W, x4 = i - y * W;
        reinterpret_cast<float4 *>(dst + y * Lp)[x4] = __ldg(reinterpret_cast<const float4 *>(src + y * L) + x4);
      }
    } else {
      for (int i = threadIdx.x; i < LL; i += blockDim.x) {
        const int y = i / L, x = i - y * L;
        dst[y * Lp + x] = __ldg(src + i);
      }
    }
  } else {
    if (vec) {
      const float4 *s4 = reinterpret_cast<const float4 *>(src);
      for (int i = threadIdx.x; i < LL / 4; i += blockDim.x) reinterpret_cast<float4 *>(im)[i] = __ldg(s4 + i);
    } else {
      for (int i = threadIdx.x; i < LL; i += blockDim.x) im[i] = __ldg(src + i);
    }
  }
  for (int i = threadIdx.x; i < M; i += blockDim.x) tws[i] = g.fwd_tw[i];
  if (tma) {
    __syncthreads();  // the barrier's initialisation is visible to every thread
    const bool ok = mbar_wait_bounded(ibar, 0, a.wait_limit);
    if (__syncthreads_or(!ok)) {  // uniform: every thread leaves
      if (threadIdx.x == 0) {
        atomicOr(a.err, 1);
        mbar_wait_bounded(ibar, 0, a.wait_limit);  // the copy must land before the CTA's memory goes
      }
      return;
    }
  }
  __syncthreads();

  for (int s0 = blockIdx.x * R; s0 < a.rows_per_img; s0 += gridDim.x * R) {
    const int nrows = min(R, a.rows_per_img - s0);
    const int64_t row0 = img * a.rows_per_img + s0;
    // Phase 1: samples x_r(theta_q) = I(c0 + s + r (cos theta_q, sin theta_q)).
    if constexpr (TAPS) {
      // integer shifts: the bilinear weights of a sample do not depend on the
      // shift, which only moves the neighbourhood inside the bordered image
      const int Lp = L + 2 * g.pad;
      int soff[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        soff[i] = 0;
        if (a.use_shifts && i < nrows) {
          const float2 sh = g.shifts[s0 + i];
          soff[i] = static_cast<int>(sh.y) * Lp + static_cast<int>(sh.x);
        }
      }
      // eight samples per thread and pass, their tap loads issued together
      constexpr int QU = 8;
      for (int q0 = threadIdx.x; q0 < NS; q0 += QU * blockDim.x) {
        float4 tp[QU];
#pragma unroll
        for (int u = 0; u < QU; ++u) {
          const int q = q0 + u * blockDim.x;
          tp[u] = q < NS ? __ldg(g.taps + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < QU; ++u) {
          const int q = q0 + u * blockDim.x;
          if (q < NS) {
            const int base = __float_as_int(tp[u].x);
            const float fx = tp[u].y, fy = tp[u].z, gx = 1.f - fx, gy = 1.f - fy;
#pragma unroll
            for (int i = 0; i < R; ++i) {
              if (i < nrows) {
                const float *p = im + base + soff[i];
                const float v = gy * (gx * p[0] + fx * p[1]) + fy * (gx * p[Lp] + fx * p[Lp + 1]);
                smem[i * NSp + q] = v;
                if (a.dbg_samples) a.dbg_samples[(row0 + i) * NS + q] = v;
              }
            }
          }
        }
      }
    } else {
      float cx[R], cy[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        cx[i] = c0;
        cy[i] = c0;
        if (a.use_shifts && i < nrows) {
          const float2 sh = g.shifts[s0 + i];
          cx[i] += sh.x;
          cy[i] += sh.y;
        }
      }
      for (int q = threadIdx.x; q < NS; q += blockDim.x) {
        const float2 o = g.offs[q];
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (i < nrows) {
            const float v = bilinear_smem(im, L, cx[i] + o.x, cy[i] + o.y);
            smem[i * NSp + q] = v;
            if (a.dbg_samples) a.dbg_samples[(row0 + i) * NS + q] = v;
          }
        }
      }
    }
    __syncthreads();

    // Phase 2: ring FFTs.  Rings of equal length form a contiguous class; the
    // (ring, row) jobs of a class are spread over the warps, 32 / T jobs per
    // warp, each transformed by a group of T threads (group_fft).
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    int fw = 0;  // warp that takes the first pass of the next class
    for (int i1 = g.NR; i1 > 0;) {
      const int H = g.rings[i1 - 1].x >> 1;
      int i0 = i1 - 1;
      while (i0 > 0 && (g.rings[i0 - 1].x >> 1) == H) --i0;
#define MRA_RING_CLASS(HH) \
    fw = ring_class<HH, R, OUT>(g, a, smem, planes, NB16, tws, s_kpos, i0, i1, nrows, row0, warp, lane, nwarps, fw)
      switch (H) {
        case 4: MRA_RING_CLASS(4); break;
        case 8: MRA_RING_CLASS(8); break;
        case 16: MRA_RING_CLASS(16); break;
        case 32: MRA_RING_CLASS(32); break;
        case 64: MRA_RING_CLASS(64); break;
        case 128: MRA_RING_CLASS(128); break;
        default: MRA_RING_CLASS(256); break;
      }
#undef MRA_RING_CLASS
      i1 = i0;
    }

    // Phase 3 (16-bit paths): copy-out in the layout of the tensor-core
    // kernel, 16 bytes per store.
    if constexpr (out_is_umma(OUT)) {
      __syncthreads();
      // job (row i, old k-step kk, half hh): 8 rings of one k-step; its q and
      // p halves go to rows slot * 32 + row % 16 and slot * 32 + 16 + row % 16
      // of MMA k-step tile u = umap[kk] / 4 (slot = umap[kk] % 4)
      unsigned char *out = reinterpret_cast<unsigned char *>(a.out16);
      for (int idx = threadIdx.x; idx < g.KS * 2 * nrows; idx += blockDim.x) {
        const int i = nrows == R ? idx % R : idx % nrows, rem = nrows == R ? idx / R : idx / nrows;
        const int hh = rem & 1, kk = rem >> 1;
        const int64_t row = row0 + i;
        const int um = __ldg(g.umap + kk);
        const int u = um >> 2, slot = um & 3;
        const uint32_t *w = planes + i * NB16 + kk * 16;
        const int swz = kk & 14;
        uint32_t wq[4], wp[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const uint2 v = *reinterpret_cast<const uint2 *>(w + ((8 * hh + 2 * jj) ^ swz));
          wq[jj] = __byte_perm(v.x, v.y, 0x5410);  // q of rings 2jj, 2jj + 1
          wp[jj] = __byte_perm(v.x, v.y, 0x7632);  // p of the same rings
        }
        unsigned char *blk = out + ((row >> 4) * g.NU + u) * 4096 + hh * 128;
        const int mq = slot * 32 + static_cast<int>(row & 15), mp = mq + 16;
        *reinterpret_cast<uint4 *>(blk + (mq >> 3) * 256 + (mq & 7) * 16) = make_uint4(wq[0], wq[1], wq[2], wq[3]);
        *reinterpret_cast<uint4 *>(blk + (mp >> 3) * 256 + (mp & 7) * 16) = make_uint4(wp[0], wp[1], wp[2], wp[3]);
      }
    } else if constexpr (OUT != kOutF32) {
      __syncthreads();
      const int per_k = nrows * 4;
      for (int idx = threadIdx.x; idx < g.KS * per_k; idx += blockDim.x) {
        const int kk = nrows == R ? idx / (4 * R) : idx / per_k;
        const int rem = idx - kk * per_k;
        const int i = rem >> 2, t = rem & 3;
        const int64_t row = row0 + i;
        const int lane16 = 4 * static_cast<int>(row & 7) + t;
        const uint32_t *w = planes + i * NB16 + kk * 16;
        const uint2 w01 = *reinterpret_cast<const uint2 *>(w + ((2 * t) ^ (kk & 14)));
        const uint2 w89 = *reinterpret_cast<const uint2 *>(w + ((2 * t + 8) ^ (kk & 14)));
        const uint32_t w0 = w01.x, w1 = w01.y, w8 = w89.x, w9 = w89.y;
        // {q[2t], q[2t+1]}, {p[2t], p[2t+1]}, {q[2t+8], q[2t+9]}, {p[2t+8], p[2t+9]}
        a.out16[((row >> 3) * g.KS + kk) * 32 + lane16] =
            make_uint4(__byte_perm(w0, w1, 0x5410), __byte_perm(w0, w1, 0x7632), __byte_perm(w8, w9, 0x5410),
                       __byte_perm(w8, w9, 0x7632));
      }
      // the next group's phase 2 rewrites the planes only after the barrier
      // that follows its phase 1
    } else {
      __syncthreads();  // the next group's phase 1 overwrites the samples
    }
  }
}

template <int R, bool TAPS, int OUT>
static cudaError_t launch_polar_r(const Geometry &g, const PolarArgs &a, size_t smem, cudaStream_t st) {
  static size_t granted = 0;
  cudaError_t e = raise_smem_limit(polar_fft_kernel<R, TAPS, OUT>, smem, granted);
  if (e != cudaSuccess) return e;
  // CTAs per image (each walks its share of the image's shift groups and
  // stages the image once): four when two or more CTAs fit on an SM, so
  // that the CTAs stay short and the last wave small; one when a CTA fills
  // an SM, where the image staging would not overlap other work; more when
  // the images are too few for about four waves of two CTAs per SM.
  // (Measured on GB300: L = 76, 2 CTAs per SM: 1 / 2 / 4 per image 22.8 /
  // 21.4 / 20.7 ms per 8192 images; L = 128, 1 CTA per SM: 1 / 2 per image
  // 51.7 / 57.3 ms per 2048 images.)
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int64_t groups = (a.rows_per_img + R - 1) / R;
  const int64_t want = (static_cast<int64_t>(8) * sms + a.n_imgs - 1) / a.n_imgs;
  int64_t per_img = smem + 1024 <= 232448 / 2 ? 4 : 1;
  if (per_img < want) per_img = want;
  if (per_img > groups) per_img = groups;
  dim3 grid(static_cast<unsigned>(per_img), static_cast<unsigned>(a.n_imgs));
  polar_fft_kernel<R, TAPS, OUT><<<grid, 256, smem, st>>>(g, a);
  return cudaGetLastError();
}

// Shared memory of a CTA with R rows: the staged image, its copy barrier,
// the twiddles, the output bases, then per row the samples and (16-bit
// output) the planes.
inline size_t polar_smem_bytes(const Geometry &g, bool taps, bool out16, int R) {
  const size_t fixed = static_cast<size_t>(image_floats(g, taps)) * sizeof(float) + 16 + g.M * sizeof(float2) +
                       static_cast<size_t>((g.M / 2 + 2) & ~1) * sizeof(int);
  size_t per_row = static_cast<size_t>(sample_stride(g.NS)) * sizeof(float);
  if (out16) per_row += static_cast<size_t>(g.KS) * 16 * sizeof(uint32_t);
  return fixed + per_row * R;
}

template <bool TAPS, int OUT>
static cudaError_t launch_polar_t(const Geometry &g, const PolarArgs &a, cudaStream_t st) {
  const size_t fixed = polar_smem_bytes(g, TAPS, OUT != kOutF32, 0);
  const size_t per_row = polar_smem_bytes(g, TAPS, OUT != kOutF32, 1) - fixed;
  // two CTAs per SM when the rows fit in ~110 KB, else as many rows as fit in 200 KB
  int R = static_cast<int>((112640 > fixed ? 112640 - fixed : 0) / per_row);
  if (R < 1) R = static_cast<int>((204800 > fixed ? 204800 - fixed : 0) / per_row);
  R = R < 1 ? 1 : (R > 4 ? 4 : R);
  if (R > a.rows_per_img) R = a.rows_per_img;
  const size_t smem = fixed + per_row * R;
  switch (R) {
    case 1: return launch_polar_r<1, TAPS, OUT>(g, a, smem, st);
    case 2: return launch_polar_r<2, TAPS, OUT>(g, a, smem, st);
    case 3: return launch_polar_r<3, TAPS, OUT>(g, a, smem, st);
    default: return launch_polar_r<4, TAPS, OUT>(g, a, smem, st);
  }
}

}  // namespace mra
