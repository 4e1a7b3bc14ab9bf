// Internal declarations shared by the C-ABI layer (mra_api.cpp) and the
// kernel translation units.  Not part of the public interface.
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only: the library does not link libcuda)
#include <cuda_runtime.h>

#include "../../include/mra.h"

namespace mra {

// Rows of the particle-spectrum layout and columns of the reference-spectrum
// layout are grouped in tiles of this many; within a tile the 8 values of one
// bin are contiguous (float2 each), so one bin of a tile is 64 bytes.
constexpr int kTile = 8;

// Geometry tables on the device (built in FP64 on the host, stored FP32).
struct Geometry {
  int L;            // box size
  int M;            // angles = largest ring length
  int NR;           // rings
  int NS;           // samples = sum N_r
  int NBIN;         // natural bins = sum (N_r/2 + 1)
  int NB;           // bins in the padded frequency-major layout
  int S;            // shifts
  int mirror;       // 0/1
  const float2 *offs;     // [NS]  r (cos theta_q, sin theta_q)
  // Integer shift grids: bilinear taps of the unshifted sample positions in
  // a copy of the image with a zero border of `pad` pixels (row length
  // L + 2 pad); tap q = {index of the top-left neighbour (int bits), fx, fy}.
  // Null when the shift grid is not integer or the border would exceed 8.
  const float4 *taps;     // [NS] or null
  int pad;
  const int4 *rings;      // [NR]  {N_r, sample offset, natural-bin offset, log2(N_r/2)}
  const int *binpos;      // [NBIN] padded position of (ring, f), ring-major natural order
  const float *bweight;   // [NBIN] reference-side weight of (ring, f)
  const float2 *fwd_tw;   // [M]   exp(-2 pi i q / M)
  const float2 *inv_tw;   // [M]   exp(+2 pi i t k / M) at [k * T + t] (T threads per pair)
  const float2 *shifts;   // [S]   (sx, sy)
  const float2 *angles;   // [M]   (cos phi_j, sin phi_j)
  const int2 *fseg;       // [M/2 + 1] {segment offset, padded segment length} per frequency
  // 16-bit tensor-core layouts: frequency f owns k-steps [kso[f], kso[f+1]) of
  // 16 rings each; ksinfo[kk] = {f, k-step index within f}.
  int KS;                 // total k-steps
  const int *kso;         // [M/2 + 2]
  const int2 *ksinfo;     // [KS]
  const int *binpos16;    // [NBIN] position kso[f] * 16 + (ring - first ring of f)
  const int *kpos;        // [M/2 + 1] binpos of (ring i, f) = kpos[f] + i
  const int *kpos16;      // [M/2 + 1] binpos16 of (ring i, f) = kpos16[f] + i
  // BF16 mma fragments of the two 16-point DFT stages of the tensor-core
  // inverse angular DFT (M = 256): [0, 512) stage-1 A, [512, 1024) stage-2 B,
  // each [32 lanes][16 words].
  const uint32_t *dft16;
  // Staging chunks of the M = 256 and M = 512 tensor-core kernels: chunk c
  // holds the whole frequencies [chunk_f[c], chunk_f[c + 1]), at most
  // kTc256ChunkKs (M = 256) or kTc512ChunkKs (M = 512) k-steps.
  int NCH;
  const int *chunk_f;     // [NCH + 1]
  // tcgen05 path (M = 256): frequencies packed four to an MMA.  A group holds
  // up to four frequencies with the same number of 16-ring k-steps (fewer
  // are padded with zero k-steps); MMA k-step u runs over (group, k-step).
  int NU;                 // MMA k-steps per tile
  int NG;                 // groups
  const int *umap;        // [KS] k-step kso[f] + j of frequency f -> u * 4 + slot
  const int *uinfo;       // [NU] group | (k-step in group) << 8 | (last k-step of the group) << 10
  const int *gfreq;       // [NG * 4] frequency in each slot of a group, -1 if empty
  const uint32_t *idft_w; // [1024] BF16 16-point DFT matrices W1, W2 (32 x 32, canonical K-major layout)
  const float2 *idft_tw;  // [256] w256^(t k) = exp(2 pi i t k / 256) at [t * 16 + k]
};

// Tile of the tcgen05 M = 256 kernel and its table bounds.
constexpr int kUmmaRows = 16;   // particle rows per tile
constexpr int kUmmaRefs = 8;    // references per tile
constexpr int kUmmaMaxU = 128;  // MMA k-steps per tile
constexpr int kUmmaMaxG = 64;   // frequency groups
constexpr int kUmmaUPerStage = 5;  // MMA k-steps per TMA box (one load of each operand per stage)

constexpr int kTc256ChunkKs = 22;
constexpr int kTc512ChunkKs = 44;
constexpr int kTc512MaxKsPerF = 6;  // rings with N_r <= 512 have r <= 81: at most 6 k-steps of 16 per frequency

struct PolarArgs {
  const float *imgs;   // [n][L][L]
  int64_t n_imgs;
  int rows_per_img;    // S for particles, 1 for references
  bool use_shifts;     // false for references (s = 0)
  bool weighted;       // multiply bins by bweight (references)
  float2 *out;         // tiled spectra [ceil(rows/8)][NB][8] (may be null in debug)
  uint4 *out16;        // 16-bit A fragments [ceil(rows/8)][KS][32 lanes], or (umma) k-step tiles
                       // [ceil(rows/16)][NU][4096 B], or null
  bool fp16;           // out16 element type: FP16 (true) or BF16 (false)
  bool umma;           // out16 in the tcgen05 k-step tile layout
  float *dbg_samples;  // [rows][NS] or null
  float2 *dbg_spec;    // [rows][NBIN] or null
  // Image staging by one TMA tensor copy per CTA (tma true): a 3-D map over
  // imgs ({L, L, n_imgs} FP32) whose box is the image in its zero border
  // ({L + 2 pad, L + 2 pad, 1}, loaded from (-pad, -pad, image); the border
  // is the map's zero fill) or the bare image (pad 0) of the path's layout.
  // tma false: plain loads.
  CUtensorMap tmap;
  bool tma;
  int *err;              // device flag: bit 0 = the staging wait timed out
  uint32_t wait_limit;   // polls before that wait gives up
};

struct CCArgs {
  const float2 *A;               // tiled particle spectra [row tiles][NB][8]
  const float2 *B;               // tiled weighted reference spectra [ref tiles][NB][8]
  int64_t rows;                  // images_in_chunk * S
  int K;                         // references
  unsigned long long *best;      // [images_in_chunk] argmax keys (pre-set to 0)
  float *dbg_cc;                 // [n][K][S][2][M] full table, or null
  int seg_max;                   // longest padded frequency segment (bins)
  int *err;                      // device flag: bit 0 = a bounded wait timed out
  uint32_t wait_limit;           // polls before a barrier wait gives up
  uint32_t first_wait_limit;     // same for each warp's first wait (tests shorten it)
};

// Precision-split path (16-bit tensor-core contraction + FP32 rescore).
constexpr int kTopRows = 8;  // candidate rows per image rescored in FP32

struct TcArgs {
  const uint4 *A16;              // [row tiles][KS][32 lanes] A fragments
  const uint2 *B16;              // [ref tiles of 8][2 N-blocks][KS][32 lanes] B fragments
  int64_t rows;                  // images_in_chunk * S
  int K;
  float *rowmax;                 // [images_in_chunk][K][S][2] row maxima over angles
  float *dbg_cc;                 // [n][K][S][2][M] full (16-bit-contraction) table, or null
  int ks_max;                    // most k-steps of any frequency
  int *err;
  uint32_t wait_limit, first_wait_limit;
};

struct RescoreArgs {
  const float *imgs;             // [n][L][L] images of the chunk
  int64_t n;
  const int *cand;               // [n][kTopRows] row ids (k * S + s) * 2 + m, or -1
  const float2 *B;               // FP32 weighted reference spectra, tiled
  unsigned long long *best;      // [n] argmax keys (written)
};

cudaError_t launch_refs16(const Geometry &g, const float2 *B, int ktiles, uint2 *B16, bool fp16, cudaStream_t st);
// tcgen05 path (M = 256): reference k-step tiles [ktiles][NU][2048 B], and the
// contraction / inverse-DFT / row-maxima kernel.  tmA and tmB point to the
// CUtensorMap of the particle and reference k-step tiles (2-D, 16-bit
// elements, rows of 256 bytes; boxes of 16 and 8 rows).
cudaError_t launch_refs16u(const Geometry &g, const float2 *B, int ktiles, void *B16u, bool fp16, cudaStream_t st);
cudaError_t launch_cc_umma256(const void *tmA, const void *tmB, const Geometry &g, const TcArgs &a, bool fp16,
                              cudaStream_t st);
cudaError_t launch_cc_tc(const Geometry &g, const TcArgs &a, bool fp16, cudaStream_t st);
cudaError_t launch_top8(const float *rowmax, int64_t n, int nrows, int *cand, cudaStream_t st);
cudaError_t launch_rescore(const Geometry &g, const RescoreArgs &a, cudaStream_t st);
size_t rescore_smem(const Geometry &g);
int rescore_ctas_per_sm(const Geometry &g);  // resident rescore CTAs per SM (0 if unknown)
// Shared memory of one CTA of the polar kernel with one row, of the FP32
// contraction kernel, and the per-CTA opt-in limit of the device.
size_t polar_smem_one_row(const Geometry &g, bool taps, bool out16);
size_t cc_fp32_smem(int M, int seg_max);
constexpr size_t kMaxSmemPerBlock = 232448;  // 227 KB
// Every check mra_create makes on a configuration, without CUDA calls or heap
// use: MRA_OK, MRA_EINVAL or MRA_EUNSUPPORTED with a message in why.
int check_config(const mra_config_t *c, char *why, size_t why_len);

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_polar(const Geometry &g, const PolarArgs &a, cudaStream_t st);
cudaError_t launch_cc_fp32(const Geometry &g, const CCArgs &a, cudaStream_t st);
cudaError_t launch_decode(const Geometry &g, const unsigned long long *best, int64_t n, int K,
                          void *poses, cudaStream_t st);
int cc_threads_per_pair(int M);

// Class averaging.
struct AvgWork {
  int *hist;          // [K * nblk]
  int *scan;          // [K * nblk]
  int *perm;          // [n]
  int *chunk_class;   // [max_chunks]
  int *chunk_begin;   // [max_chunks]
  int *chunk_count;   // [max_chunks]
  int *n_chunks;      // [1]
  int *class_counts;  // [K]
  int *class_first_chunk; // [K + 1]
  float *part_sum;    // [max_chunks][L*L]
  float *part_comp;   // [max_chunks][L*L]
  int max_chunks;
};
constexpr int kClassSumLaunches = 6;  // kernels launched by launch_class_sums
constexpr int kAvgBlock = 256;   // images per histogram block
constexpr int kAvgChunk = 64;    // images per partial-sum chunk
cudaError_t launch_class_sums(const Geometry &g, const float *imgs, const void *poses, int64_t n,
                              int K, const AvgWork &w, float *sum, float *comp, int *counts,
                              bool accumulate, cudaStream_t st);
cudaError_t launch_refresh_refs(int L, float *refs, const int *counts, int K, const int *reseed, const float *imgs,
                                int64_t n, cudaStream_t st);
cudaError_t launch_average_finalize(const Geometry &g, int K, const float *sum, const float *comp,
                                    const int *counts, float *avg, cudaStream_t st);

}  // namespace mra
