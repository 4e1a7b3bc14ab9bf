// Precision-split path, M = 256 angles (rings up to 40): spectrum
// contraction and inverse angular DFT on the 5th-generation tensor cores
// (tcgen05.mma, FP32 accumulation in tensor memory), operands staged by TMA.
//
// Contraction (Alg. 1, CC step).  With q = Re X - Im X, p = Re X + Im X for
// a particle ring bin and v = Re Y - Im Y, u = Re Y + Im Y for a weighted
// reference bin, the angular spectrum of a (row, reference) pair is
//     Z(f) = sum_r q (v + i u),   Z(-f) = sum_r p (u + i v),
// i.e. Z = C_u + i C' (unmirrored plus i times mirrored correlation).  A
// tile is 16 particle rows x 8 references = 128 pairs.  One MMA
// (M = 128, N = 64, K = 16 rings) serves four frequencies at once: A holds,
// for each of the four frequency slots, the q and p rows of the 16 particle
// rows (32 rows per slot), B the v and u rows of the 8 references (16 per
// slot); only the four diagonal 32 x 16 blocks of the 128 x 64 product are
// used.  (A tcgen05.mma costs at least ~45 cycles whatever its size below
// N = 64 on GB300, so four narrow per-frequency products in one instruction
// cost what one does; the unused blocks are free.)  Frequencies with the
// same number of 16-ring k-steps share an MMA group; a group's k-steps
// accumulate in one 64-column TMEM slot.
//
// Corner turn.  Slot s of the accumulator sits in TMEM lanes 32 s .. 32 s + 31
// (lane = (q/p, row)), which warp s % 4 of a warpgroup reads; each such
// drain thread holds Z of one (row, +-f) for the 8 references and writes
// them as BF16 into the stage-1 operand in shared memory, where a row is a
// pair (pair = ref * 16 + row).
//
// Inverse angular DFT (Alg. 1, inverse-FFT step), 256 = 16 x 16, f = t + 16 a,
// angle index n = k + 16 j:
//     Y(k, t)    = sum_a w16^(a k) Z(t + 16 a)          stage 1: per t, M = 128 pairs, N = 32, K = 32
//     c(k + 16j) = sum_t w16^(t j) w256^(t k) Y(k, t)    twiddle in FP32, stage 2: per k
// with BF16 operands (the spectrum, the two 16-point DFT matrices, the
// twiddled intermediate) and FP32 accumulation; c = c_u + i c' gives the
// unmirrored correlation (real part) and the mirrored one (imaginary part,
// at the half-turn shifted angle).  The drain of stage 2 reduces each pair
// to its two row maxima over the 256 angles (Alg. 1 reduction step, Fig. 2)
// for the FP32 rescore of the top rows.
//
// Roles (18 warps, one persistent CTA per SM, tiles walked with stride
// gridDim.x): warp 0 streams each tile's A and B k-step tiles with TMA
// tensor-map loads into a ring of shared-memory stages; warp 1 owns the
// 512 TMEM columns and issues every MMA from one thread; warps 2-17 drain
// TMEM, in four quads of four warps (one per TMEM lane quarter): quad d
// drains the contraction groups g = d mod 4, the stage-1 columns of
// t = 4 d .. 4 d + 3 and the stage-2 columns of k = 4 d .. 4 d + 3.  All waits are bounded; a wait that gives up raises a CTA abort
// flag and the device error flag, every role leaves its loop, the producer
// waits for its copies still in flight and the MMA issuer for its MMAs, and
// the TMEM is released.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/mra.h"
#include "dev_util.cuh"
#include "mra_internal.h"
#include "umma.cuh"

namespace mra {

namespace u256 {
constexpr int kDrainWarps = 16;                             // 4 quads x the 4 TMEM lane quarters
constexpr int kThreads = 64 + 32 * kDrainWarps;
// Registers per thread: the warps of a CTA are spread over the SM's four
// sub-partitions, each with 16384 registers, so the sub-partition holding
// the most warps bounds the per-thread count.
constexpr int kMaxRegs = 96;
static_assert((kThreads / 32 + 3) / 4 * 32 * kMaxRegs <= 16384, "register file of a sub-partition exceeded");
constexpr int kUPerStage = kUmmaUPerStage;                  // k-steps per TMA stage (one box per operand)
constexpr int kStages = 3;
constexpr uint32_t kABytes = 4096, kBBytes = 2048;          // one k-step: A 128 x 16, B 64 x 16 (BF16/FP16)
constexpr uint32_t kStageBytes = kUPerStage * (kABytes + kBBytes);
constexpr int kAcc = 8;                                     // 64-column accumulator slots (all 512 columns)
constexpr int kCommits = 16;                                // ring of stage-commit barriers
constexpr uint32_t kTileBytes = 8192;                        // a 128 x 32 operand tile of the inverse DFT
constexpr uint32_t kOffZ = 0;                                // Z_t tiles (stage 1), then Y_k tiles (stage 2)
constexpr uint32_t kOffStage = kOffZ + 16 * kTileBytes;
constexpr uint32_t kOffW = kOffStage + kStages * kStageBytes;  // W1, W2: 32 x 32 BF16 each
constexpr uint32_t kOffTw = kOffW + 2 * 2048;                // w256^(t k), [t][k]
// partial row maxima [3 quads][128 pairs]: in the Y_k tiles, which are dead
// once the stage-2 MMAs have completed
constexpr uint32_t kOffMax = kOffZ;
constexpr uint32_t kOffUinfo = kOffTw + 256 * sizeof(float2);
constexpr uint32_t kOffGfreq = kOffUinfo + kUmmaMaxU * sizeof(int);
constexpr uint32_t kOffGlast = kOffGfreq + kUmmaMaxG * 4 * sizeof(int);
constexpr uint32_t kOffBar = kOffGlast + kUmmaMaxG * sizeof(int);
// barriers: full[S], done[16], acce[8], zs_done, d1_full[4], y_done, d2_full[4], tm_free, fin, mx_full
constexpr int kNumBars = kStages + kCommits + kAcc + 13;
constexpr uint32_t kOffMisc = kOffBar + kNumBars * 8;        // TMEM base, abort flag
constexpr uint32_t kSmem = kOffMisc + 16;
static_assert(kSmem <= 232448, "tcgen05 M = 256 kernel exceeds 227 KB of shared memory");
static_assert(kOffStage % 1024 == 0 && kStageBytes % 1024 == 0, "TMA stages must stay 1 KB aligned");
static_assert(3 * 128 * 8 <= 16 * kTileBytes, "partial maxima must fit the Y_k tiles");
}  // namespace u256

__device__ __forceinline__ uint32_t pack_bf2u(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

template <bool FP16>
__global__ void __maxnreg__(u256::kMaxRegs)
    cc_umma256_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Geometry g,
                      TcArgs a, int ref_tiles, int64_t ntiles) {
  using namespace u256;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);
  uint64_t *full = bars, *done = bars + kStages, *acce = done + kCommits;
  uint64_t *zs_done = acce + kAcc, *d1_full = zs_done + 1, *y_done = d1_full + 4, *d2_full = y_done + 1,
           *tm_free = d2_full + 4, *fin = tm_free + 1, *mx_full = fin + 1;
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kOffMisc);
  volatile int *abort = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);
  int *s_uinfo = reinterpret_cast<int *>(smem + kOffUinfo);
  int *s_gfreq = reinterpret_cast<int *>(smem + kOffGfreq);
  int *s_glast = reinterpret_cast<int *>(smem + kOffGlast);  // k-step of each group's last MMA
  float2 *s_tw = reinterpret_cast<float2 *>(smem + kOffTw);
  float2 *s_max = reinterpret_cast<float2 *>(smem + kOffMax);
  const int NU = g.NU, NG = g.NG;
  const int SPT = (NU + kUPerStage - 1) / kUPerStage;  // TMA stages (and stage commits) per tile

  // ---- set-up: tables, DFT matrices, barriers, TMEM ----
  for (int i = tid; i < NU; i += kThreads) {
    const int info = g.uinfo[i];
    s_uinfo[i] = info;
    if ((info >> 10) & 1) s_glast[info & 255] = i;
  }
  for (int i = tid; i < NG * 4; i += kThreads) s_gfreq[i] = g.gfreq[i];
  for (int i = tid; i < 256; i += kThreads) s_tw[i] = g.idft_tw[i];
  for (int i = tid; i < 1024; i += kThreads)
    reinterpret_cast<uint32_t *>(smem + kOffW)[i] = g.idft_w[i];
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(full + s, 1);
    for (int s = 0; s < kCommits; ++s) mbar_init(done + s, 1);
    for (int s = 0; s < kAcc; ++s) mbar_init(acce + s, 4);  // the four drain warps of one quad
    mbar_init(zs_done, kDrainWarps);
    for (int d = 0; d < 4; ++d) mbar_init(d1_full + d, 1);
    mbar_init(y_done, kDrainWarps);
    for (int d = 0; d < 4; ++d) mbar_init(d2_full + d, 1);
    mbar_init(tm_free, kDrainWarps);
    mbar_init(fin, 1);
    mbar_init(mx_full, kDrainWarps - 4);
    *abort = (smem_u32(smem) & 1023u) ? 1 : 0;  // TMA stages and descriptors assume a 1 KB aligned base
    if (*abort) atomicOr(a.err, 2);
  }
  if (warp == 1) tmem_alloc(s_tmem, 512);
  mbar_init_fence();
  fence_proxy_async();  // the DFT matrices written above are read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t sbase = smem_u32(smem);

  if (warp == 0) {
    // ---------------- producer: TMA tensor loads of the k-step tiles ----------------
    // Stage use c (counted over the CTA's tiles) fills ring slot c % kStages
    // once the MMAs of use c - kStages have completed (their stage commit).
    if (lane == 0 && !*abort) {
      int c = 0;
      bool ok = true;
      for (int64_t tau = blockIdx.x; tau < ntiles && ok; tau += gridDim.x) {
        const int rt = static_cast<int>(tau / ref_tiles), kt = static_cast<int>(tau - static_cast<int64_t>(rt) * ref_tiles);
        int ya = rt * NU * 16, yb = kt * NU * 8;  // tensor-map rows of the tile's first k-step
        // the next tile's particle k-step tiles (contiguous, NU * 4 KB) into L2 while this one runs
        if (tau + gridDim.x < ntiles) {
          const int64_t rn = (tau + gridDim.x) / ref_tiles;
          if (rn != rt) prefetch_l2(reinterpret_cast<const unsigned char *>(a.A16) + rn * NU * kABytes, NU * kABytes);
        }
        for (int u0 = 0; u0 < NU; u0 += kUPerStage, ++c) {
          if (c >= kStages) {
            const int cp = c - kStages;
            if (!spin_or_abort(done + (cp & (kCommits - 1)), static_cast<uint32_t>((cp / kCommits) & 1), a.wait_limit,
                               abort, a.err)) {
              ok = false;
              break;
            }
          }
          // one box of kUPerStage k-steps per operand; a tile's last stage may
          // read k-steps of the next tile (or zeros past the end), never used
          const int rs = c % kStages;
          unsigned char *dst = smem + kOffStage + rs * kStageBytes;
          mbar_arrive_expect_tx(full + rs, kStageBytes);
          tma_load_2d(dst, &tmA, 0, ya, full + rs);
          tma_load_2d(dst + kUPerStage * kABytes, &tmB, 0, yb, full + rs);
          ya += kUPerStage * 16;
          yb += kUPerStage * 8;
        }
      }
      // let every copy still in flight land before the CTA's shared memory goes
      for (int cp = c - kStages < 0 ? 0 : c - kStages; cp < c; ++cp)
        mbar_wait_bounded(full + cp % kStages, static_cast<uint32_t>((cp / kStages) & 1), a.wait_limit);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && !*abort) {
      const uint32_t idc = umma_idesc(128, 64, !FP16);
      const uint32_t idi = umma_idesc(128, 32, true);
      int c = 0;  // stage uses so far
      bool first = true, ok = true;
      int64_t tile_iter = 0;
      const uint64_t wdesc1 = umma_sdesc(sbase + kOffW, 128, 512), wdesc2 = umma_sdesc(sbase + kOffW + 2048, 128, 512);
      for (int64_t tau = blockIdx.x; tau < ntiles && ok; tau += gridDim.x, ++tile_iter) {
        if (tile_iter > 0 &&
            !spin_or_abort(tm_free, static_cast<uint32_t>((tile_iter - 1) & 1), a.wait_limit, abort, a.err))
          break;
        tc_fence_after();
        const int64_t gbase = tile_iter * NG;
        // contraction: stage use c holds k-steps [4 s, 4 s + 4) of the tile; one commit per stage
        // (to done[c % 16]) frees the stage for the producer and tells the drain warps that the
        // groups ending in it are complete
        for (int sp = 0; sp < SPT && ok; ++sp, ++c) {
          const int rs = c % kStages;
          if (!spin_or_abort(full + rs, static_cast<uint32_t>((c / kStages) & 1),
                             first ? a.first_wait_limit : a.wait_limit, abort, a.err)) {
            ok = false;
            break;
          }
          first = false;
          tc_fence_after();
          const uint32_t st = sbase + kOffStage + rs * kStageBytes;
          const uint64_t adesc = umma_sdesc(st, 128, 256), bdesc = umma_sdesc(st + kUPerStage * kABytes, 128, 256);
#pragma unroll
          for (int ui = 0; ui < kUPerStage; ++ui) {
            const int u = sp * kUPerStage + ui;
            if (u < NU) {
              const int info = s_uinfo[u];
              const int grp = info & 255, j = (info >> 8) & 3;
              const int64_t G = gbase + grp;
              const int slot = static_cast<int>(G & (kAcc - 1));
              if (j == 0 && G >= kAcc) {
                if (!spin_or_abort(acce + slot, static_cast<uint32_t>(((G >> 3) - 1) & 1), a.wait_limit, abort,
                                   a.err)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
              umma_ss(tmem + slot * 64, adesc + static_cast<uint64_t>(ui * (kABytes >> 4)),
                      bdesc + static_cast<uint64_t>(ui * (kBBytes >> 4)), idc, j > 0);
            }
          }
          umma_commit(done + (c & (kCommits - 1)));
        }
        if (!ok) break;
        // stage 1 of the inverse DFT: D1_t = Z_t W1 for every t
        if (!spin_or_abort(zs_done, static_cast<uint32_t>(tile_iter & 1), a.wait_limit, abort, a.err)) break;
        tc_fence_after();
        // in four batches of four t, each committed for the drain quad that owns it
        for (int d = 0; d < 4; ++d) {
          for (int t = 4 * d; t < 4 * d + 4; ++t)
            for (int h = 0; h < 2; ++h)
              umma_ss(tmem + t * 32, umma_sdesc(sbase + kOffZ + t * kTileBytes + h * 256, 128, 512),
                      wdesc1 + static_cast<uint64_t>(h * 16), idi, h);
          umma_commit(d1_full + d);
        }
        // stage 2: D2_k = Y'_k W2 for every k
        if (!spin_or_abort(y_done, static_cast<uint32_t>(tile_iter & 1), a.wait_limit, abort, a.err)) break;
        tc_fence_after();
        for (int d = 0; d < 4; ++d) {
          for (int k = 4 * d; k < 4 * d + 4; ++k)
            for (int h = 0; h < 2; ++h)
              umma_ss(tmem + k * 32, umma_sdesc(sbase + kOffZ + 2 * h * 32768 + k * 2048, 32768, 128),
                      wdesc2 + static_cast<uint64_t>(h * 16), idi, h);
          umma_commit(d2_full + d);
        }
      }
      // every MMA issued has completed before the TMEM and the stages are released
      umma_commit(fin);
      mbar_wait_bounded(fin, 0, a.wait_limit);
    }
  } else {
    // ---------------- drain warps ----------------
    const int dw = warp - 2, q = warp & 3, quad = dw >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    const int pair = q * 32 + lane;              // TMEM lane of the inverse-DFT stages
    const int qp = lane >> 4, ri = lane & 15;    // contraction: q or p row, particle row in the tile
    // this thread's corner-turn target: pair ref * 16 + ri of tile t at K = 2 a (+1): rows of 8 pairs
    // are 512 bytes apart, so reference ref adds 1024 bytes
    unsigned char *zrow = smem + kOffZ + (ri >> 3) * 512 + (ri & 7) * 16;
    const int S = g.S;
    int64_t tile_iter = 0;
    for (int64_t tau = blockIdx.x; tau < ntiles && !*abort; tau += gridDim.x, ++tile_iter) {
      const int rt = static_cast<int>(tau / ref_tiles), kt = static_cast<int>(tau - static_cast<int64_t>(rt) * ref_tiles);
      const int64_t gbase = tile_iter * NG;
      bool ok = true;
      // contraction drains: the pairs of consecutive groups (2 p, 2 p + 1) with p = quad mod 4,
      // whose stage commits are usually one and the same: both TMEM loads in flight per wait
      for (int pg = quad; 2 * pg < NG; pg += 4) {
        const int g0 = 2 * pg, ng = (2 * pg + 1 < NG) ? 2 : 1;
        const int cg = static_cast<int>(tile_iter) * SPT + s_glast[g0 + ng - 1] / kUPerStage;  // the later commit
        if (!wait_or_abort(done + (cg & (kCommits - 1)), static_cast<uint32_t>((cg / kCommits) & 1), a.wait_limit,
                           abort, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        int fg[2], slots[2];
        uint32_t r[2][16];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int64_t G = gbase + g0 + e;
          slots[e] = static_cast<int>(G & (kAcc - 1));
          fg[e] = e < ng ? s_gfreq[(g0 + e) * 4 + q] : -1;
          if (fg[e] >= 0) tmem_ld16(tmem + lane_base + slots[e] * 64 + q * 16, r[e]);
        }
        tmem_ld_wait();
        tc_fence_before();  // the slots are free as soon as their columns are in registers
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(acce + slots[0]);
          if (ng > 1) mbar_arrive(acce + slots[1]);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int f = fg[e];
          // q rows: Z(f) = (sum q v, sum q u); p rows: Z(256 - f) = (sum p u, sum p v)
          if (f >= 0 && !(qp && (f == 0 || f == 128))) {
            const int fp = qp ? ((256 - f) & 255) : f;
            unsigned char *z = zrow + (fp & 15) * kTileBytes + ((fp >> 4) >> 2) * 128 + ((fp >> 4) & 3) * 4;
#pragma unroll
            for (int ref = 0; ref < 8; ++ref) {
              const float v = __uint_as_float(r[e][ref]), uu = __uint_as_float(r[e][8 + ref]);
              *reinterpret_cast<uint32_t *>(z + ref * 1024) = qp ? pack_bf2u(uu, v) : pack_bf2u(v, uu);
            }
          }
        }
      }
      if (!ok) break;
      fence_proxy_async();  // the Z_t tiles are read by the tensor cores next
      __syncwarp();
      if (lane == 0) mbar_arrive(zs_done);
      // stage-1 drain: Y'(k, t) = w256^(t k) Y(k, t), t = 4 quad .. 4 quad + 3, into the Y_k tiles
      // (core column `quad` of each; the Z_t tiles are consumed)
      if (!wait_or_abort(d1_full + quad, static_cast<uint32_t>(tile_iter & 1), a.wait_limit, abort, a.err)) break;
      tc_fence_after();
      {
        // Y_k tiles: core column d (t = 4 d .. 4 d + 3) of every k in region d of the buffer, the
        // 32 KB that held Z_t for those t (consumed by stage-1 batch d, which this quad waited for;
        // the other batches read only their own regions): k-th 2 KB block, rows of 8 pairs 128 B apart
        unsigned char *y = smem + kOffZ + quad * 32768 + (pair >> 3) * 128 + (pair & 7) * 16;
        // two t and half of the 16 k per pass (8-byte stores of (t, t + 1)): the
        // real and imaginary columns of both t in flight at once, 48 live values
#pragma unroll
        for (int tt = 0; tt < 4; tt += 2) {
#pragma unroll
          for (int kh = 0; kh < 16; kh += 8) {
            const int t0 = quad * 4 + tt;
            uint32_t r[4][8];
            tmem_ld8(tmem + lane_base + t0 * 32 + kh, r[0]);
            tmem_ld8(tmem + lane_base + t0 * 32 + 16 + kh, r[1]);
            tmem_ld8(tmem + lane_base + (t0 + 1) * 32 + kh, r[2]);
            tmem_ld8(tmem + lane_base + (t0 + 1) * 32 + 16 + kh, r[3]);
            tmem_ld_wait();
#pragma unroll
            for (int k8 = 0; k8 < 8; ++k8) {
              uint32_t o[2];
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const float2 w = s_tw[(t0 + e) * 16 + kh + k8];
                const float yr = __uint_as_float(r[2 * e][k8]), yi = __uint_as_float(r[2 * e + 1][k8]);
                o[e] = pack_bf2u(fmaf(yr, w.x, -yi * w.y), fmaf(yr, w.y, yi * w.x));
              }
              *reinterpret_cast<uint2 *>(y + (kh + k8) * 2048 + tt * 4) = make_uint2(o[0], o[1]);
            }
          }
        }
      }
      tc_fence_before();
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(y_done);
      // stage-2 drain: row maxima over the 256 angles (and the full table in debug mode)
      if (!wait_or_abort(d2_full + quad, static_cast<uint32_t>(tile_iter & 1), a.wait_limit, abort, a.err)) break;
      tc_fence_after();
      const int ref = pair >> 4, prow = pair & 15;
      const int64_t row = static_cast<int64_t>(rt) * 16 + prow;
      const int refg = kt * 8 + ref;
      const bool valid = row < a.rows && refg < a.K;
      int64_t rbase = 0;
      if (valid) {
        const int64_t img = row / S;
        rbase = (img * a.K + refg) * S + (row - img * S);
      }
      float vu = -INFINITY, vm = -INFINITY;
      for (int kk = 0; kk < 4; ++kk) {
        const int k = quad * 4 + kk;
        uint32_t r[32];
        tmem_ld32(tmem + lane_base + k * 32, r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          vu = fmaxf(vu, __uint_as_float(r[j]));
          vm = fmaxf(vm, __uint_as_float(r[16 + j]));
        }
        if (a.dbg_cc && valid) {
          float *d = a.dbg_cc + rbase * 512;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = k + 16 * j;
            d[n] = __uint_as_float(r[j]);
            d[256 + ((n + 128) & 255)] = __uint_as_float(r[16 + j]);
          }
        }
      }
      tc_fence_before();
      // quads 1-3 hand their maxima to quad 0 (bounded wait: an abort
      // elsewhere cannot leave a warp stuck here)
      bool have = true;
      if (quad) {
        // the maxima go into the Y_k tiles: wait until the last stage-2 batch has read them
        have = wait_or_abort(d2_full + 3, static_cast<uint32_t>(tile_iter & 1), a.wait_limit, abort, a.err);
        if (have) s_max[(quad - 1) * 128 + pair] = make_float2(vu, vm);
        __syncwarp();
        if (lane == 0) mbar_arrive(mx_full);
      } else {
        have = wait_or_abort(mx_full, static_cast<uint32_t>(tile_iter & 1), a.wait_limit, abort, a.err);
      }
      if (!quad && have && valid) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float2 o = s_max[d * 128 + pair];
          vu = fmaxf(vu, o.x);
          vm = fmaxf(vm, o.y);
        }
        a.rowmax[rbase * 2] = vu;
        a.rowmax[rbase * 2 + 1] = g.mirror ? vm : -INFINITY;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(tm_free);
      if (!have) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// Reference k-step tiles of the tcgen05 path: for reference tile kt (8
// references) and MMA k-step u, the 64 x 16 B operand (row n = slot * 16 +
// (v|u) * 8 + ref, K = ring within the k-step) in the canonical K-major
// layout; zero for empty slots, padding k-steps and rings beyond R_f.
__global__ void refs16u_kernel(Geometry g, const float2 *__restrict__ B, int ktiles, uint4 *B16u, bool fp16) {
  const int64_t total = static_cast<int64_t>(ktiles) * g.NU * 128;
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int hh = static_cast<int>(idx & 1), n = static_cast<int>((idx >> 1) & 63);
    const int64_t ku = idx >> 7;
    const int u = static_cast<int>(ku % g.NU), kt = static_cast<int>(ku / g.NU);
    const int info = g.uinfo[u];
    const int grp = info & 255, j = (info >> 8) & 3;
    const int s = n >> 4, vu = (n >> 3) & 1, ref = n & 7;
    const int f = g.gfreq[grp * 4 + s];
    uint16_t v16[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      float val = 0.f;
      if (f >= 0 && j < g.kso[f + 1] - g.kso[f]) {
        const int2 seg = g.fseg[f];
        const int rr = 16 * j + 8 * hh + e;
        if (rr < seg.y) {
          const float2 X = B[(static_cast<int64_t>(kt) * g.NB + seg.x + rr) * kTile + ref];
          val = vu ? (X.x + X.y) : (X.x - X.y);
        }
      }
      v16[e] = fp16 ? __half_as_ushort(__float2half_rn(val)) : __bfloat16_as_ushort(__float2bfloat16_rn(val));
    }
    uint4 o;
    o.x = v16[0] | (static_cast<uint32_t>(v16[1]) << 16);
    o.y = v16[2] | (static_cast<uint32_t>(v16[3]) << 16);
    o.z = v16[4] | (static_cast<uint32_t>(v16[5]) << 16);
    o.w = v16[6] | (static_cast<uint32_t>(v16[7]) << 16);
    B16u[(ku * 2048 + (n >> 3) * 256 + hh * 128 + (n & 7) * 16) / 16] = o;
  }
}

cudaError_t launch_refs16u(const Geometry &g, const float2 *B, int ktiles, void *B16u, bool fp16, cudaStream_t st) {
  const int64_t total = static_cast<int64_t>(ktiles) * g.NU * 128;
  const int blocks = static_cast<int>((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  refs16u_kernel<<<blocks, 256, 0, st>>>(g, B, ktiles, static_cast<uint4 *>(B16u), fp16);
  return cudaGetLastError();
}

template <bool FP16>
static cudaError_t launch_u256_t(const CUtensorMap &tmA, const CUtensorMap &tmB, const Geometry &g, const TcArgs &a,
                                 cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(cc_umma256_kernel<FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(u256::kSmem));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int64_t row_tiles = (a.rows + kUmmaRows - 1) / kUmmaRows;
  const int ref_tiles = (a.K + kUmmaRefs - 1) / kUmmaRefs;
  const int64_t ntiles = row_tiles * ref_tiles;
  if (ntiles <= 0) return cudaSuccess;
  const int grid = static_cast<int>(ntiles < sms ? ntiles : sms);
  cc_umma256_kernel<FP16><<<grid, u256::kThreads, u256::kSmem, st>>>(tmA, tmB, g, a, ref_tiles, ntiles);
  return cudaGetLastError();
}

cudaError_t launch_cc_umma256(const void *tmA, const void *tmB, const Geometry &g, const TcArgs &a, bool fp16,
                              cudaStream_t st) {
  if (g.M != 256 || g.NU <= 0 || g.NU > kUmmaMaxU || g.NG > kUmmaMaxG) return cudaErrorInvalidValue;
  const CUtensorMap &A = *static_cast<const CUtensorMap *>(tmA);
  const CUtensorMap &B = *static_cast<const CUtensorMap *>(tmB);
  return fp16 ? launch_u256_t<true>(A, B, g, a, st) : launch_u256_t<false>(A, B, g, a, st);
}

}  // namespace mra
