// Precision-split path: 16-bit tensor-core spectrum contraction, top-8 row
// selection, FP32 rescoring of the candidate rows.
//
// Contraction on tensor cores.  With q = Re A - Im A, p = Re A + Im A for a
// particle bin and v = Re B - Im B, u = Re B + Im B for a weighted reference
// bin, the angular spectrum of a (row, reference) pair at frequency f is
//     Z(f)     = sum_r q (v + i u),        Z(M - f) = sum_r p (u + i v),
// i.e. Z = C_u + i C' with C_u = sum conj(A) B and C' = sum A B (the mirror
// identity).  One mma.sync.m16n8k16 per k-step of 16 rings therefore takes
// an A operand whose rows 0-7 are the q values of the tile's 8 rows and rows
// 8-15 their p values, and a B operand whose 8 columns are (v, u) of 4
// references: the accumulator holds Re/Im Z(f) (q rows) and Im/Re Z(M - f)
// (p rows) for 8 rows x 4 references.  A tile of 8 rows x 8 references is
// two such MMAs per k-step.  Operands are BF16 (or FP16), accumulation FP32.
//
// For M = 256 (rings up to 40) the per-pair angular state is kept as BF16 in
// shared memory and the inverse angular DFT runs on tensor cores too
// (cc_tc256_kernel); for M = 512 the state is BF16 and the inverse DFT runs
// in FP32 (cc_tc512_kernel); for M <= 128 the state stays FP32
// (cc_tc_kernel).  Either way the row maxima select the 8 rows
// (reference, shift, mirror) per image that the rescore kernel recomputes
// from scratch in FP32; its argmax is the answer.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/mra.h"
#include "dev_util.cuh"
#include "mra_internal.h"
#include "pair_ifft.cuh"
#include "ring_fft.cuh"
#include "smem_limit.cuh"
#include "tma.cuh"

namespace mra {

__device__ __forceinline__ uint16_t to16(float v, bool fp16) {
  return fp16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ uint32_t pack16x2(uint16_t lo, uint16_t hi) {
  return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

// ---------------------------------------------------------------------------
// Reference B fragments: [ref tile of 8][N-block 2][KS][lane 32] x uint2.
// Lane 4g + t of N-block nb holds column g = (reference 4 nb + g/2, value
// v if g even else u) at k = 2t, 2t+1 (first word) and 2t+8, 2t+9 (second).
// ---------------------------------------------------------------------------
__global__ void refs16_kernel(Geometry g, const float2 *__restrict__ B, int ktiles, uint2 *B16, bool fp16) {
  const int64_t total = static_cast<int64_t>(ktiles) * g.KS * 64;
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int lane = static_cast<int>(idx & 31);
    const int64_t r = idx >> 5;
    const int kk = static_cast<int>(r % g.KS);
    const int nb = static_cast<int>((r / g.KS) & 1);
    const int kt = static_cast<int>(r / g.KS / 2);
    const int2 ki = g.ksinfo[kk];
    const int2 seg = g.fseg[ki.x];
    const int gi = lane >> 2, t = lane & 3;
    const int refl = 4 * nb + (gi >> 1), c = gi & 1;
    const int ks[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
    uint16_t v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int rr = 16 * ki.y + ks[e];
      float val = 0.f;
      if (rr < seg.y) {
        const float2 X = B[(static_cast<int64_t>(kt) * g.NB + seg.x + rr) * kTile + refl];
        val = c ? (X.x + X.y) : (X.x - X.y);
      }
      v[e] = to16(val, fp16);
    }
    B16[idx] = make_uint2(pack16x2(v[0], v[1]), pack16x2(v[2], v[3]));
  }
}

template <bool FP16>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint4 &a, const uint2 &b) {
  if constexpr (FP16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
  }
}

template <int M, int KT_>
struct TcShape {
  static constexpr int RT = kTile, KT = KT_, PAIRS = RT * KT;
  static constexpr int NBLK = KT / 4;  // MMAs (N-blocks of 4 references) per k-step
  static constexpr int WARPS = 16, THREADS = 32 * WARPS;
  static constexpr int P = IfftShape<M>::P;  // float2 per pair buffer
  static constexpr size_t STATE = static_cast<size_t>(PAIRS) * P * sizeof(float2);
  static constexpr size_t TW = M * sizeof(float2);
  static constexpr size_t BARS = WARPS * sizeof(uint64_t);
  // A: ks_max k-steps x 512 B, then B: NBLK x ks_max x 256 B
  __host__ __device__ static size_t stage_bytes(int ks_max) {
    return static_cast<size_t>(ks_max) * 512 + static_cast<size_t>(NBLK) * ks_max * 256;
  }
  __host__ __device__ static size_t smem(int ks_max) { return STATE + TW + BARS + WARPS * stage_bytes(ks_max); }
};

// XOR swizzle (below T) matching the epilogue's store pattern
// (lane 4g + t -> row g, ref t or t + 4).
template <int M, int KT>
__device__ __forceinline__ int tc_swz(int p) {
  return (((p % KT) & 3) + 4 * ((p / KT) & 3)) & (IfftShape<M>::T - 1);
}

// ---------------------------------------------------------------------------
// M = 256: contraction and inverse angular DFT both on tensor cores.
//
// The angular spectrum of a pair is kept in shared memory as BF16 (Re, Im)
// words, 1 KB per pair: BF16 has the FP32 exponent range, so no scaling is
// needed, and its rounding (2^-9) is of the same order as that of the BF16
// contraction operands; the FP32 rescore of the top rows restores full
// accuracy.  Word position of Z(f) in a pair's buffer:
//     f ^ sw ^ (((f >> 5) & 3) << 3),   sw = 4 (pair / 8) + (pair % 4),
// which makes both the contraction's stores (32 lanes, 32 pairs, one f) and
// the inverse DFT's fragment loads (one pair, lanes 4g + t4 reading
// f = 8 nb + g + 16 a) bank-conflict free.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int z256_fold(int f) { return f ^ (((f >> 5) & 3) << 3); }
__device__ __forceinline__ int z256_swz(int pair) { return 4 * (pair >> 3) + (pair & 3); }

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// Lane-invariant parts of the inverse DFT, computed once per kernel: the
// folded positions of the 8 spectrum words a lane loads, and the 8 stage
// twiddles it applies.
struct TcLane {
  int zoff[8];    // z256_fold(f) for f = 8 nb + g + 16 a, a in {2 t4, 2 t4 + 1, 2 t4 + 8, 2 t4 + 9}
  float2 tw[8];   // w256^(t k) for fragment (nb, q)
};

__device__ __forceinline__ void tc_lane_init(TcLane &L, const float2 *tw, int lane) {
  const int g = lane >> 2, t4 = lane & 3;
  const int aa[4] = {2 * t4, 2 * t4 + 1, 2 * t4 + 8, 2 * t4 + 9};
#pragma unroll
  for (int nb = 0; nb < 2; ++nb)
#pragma unroll
    for (int e = 0; e < 4; ++e) L.zoff[nb * 4 + e] = z256_fold(8 * nb + g + 16 * aa[e]);
#pragma unroll
  for (int nb = 0; nb < 2; ++nb)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = g + 8 * (q >> 1), t = 8 * nb + 2 * t4 + (q & 1);
      L.tw[nb * 4 + q] = tw[k * 16 + t];
    }
}

// 256-point inverse DFT of one pair on tensor cores by one warp (16 x 16):
// Y(k, t) = sum_a w16^(a k) Z(t + 16 a) as a 32 x 32 x 16 real GEMM (A = the
// DFT matrix [[C, -S], [S, C]], B = Z), twiddle w256^(t k) in FP32, then
// c(k + 16 j) = sum_t w16^(t j) Y'(k, t) as a 16 x 32 x 32 real GEMM whose A
// fragments are exactly the stage-1 accumulators.  BF16 operands, FP32
// accumulation.  z[nb * 4 + i] is the spectrum word (Re, Im) of
// f = 8 nb + g + 16 a_i, a_i in {2 t4, 2 t4 + 1, 2 t4 + 8, 2 t4 + 9}, and
// tw[nb * 4 + q] the stage twiddle w256^(t k) of fragment q of t block nb.
// On return d2[b][q] (b = 0, 1: real part, b = 2, 3: imaginary part) is c at
// angle k + 16 j with k = g + 8 (q >> 1), j = 8 (b & 1) + 2 t4 + (q & 1).
__device__ __forceinline__ void idft256_core(const uint32_t (&z)[8], const float2 (&tw)[8],
                                             const uint32_t (&a1)[16], const uint32_t (&b2)[16],
                                             float (&d2)[4][4]) {
  // B fragments: [re/im k-step][t block]; word halves are (Re, Im) of one f
  uint2 b1[2][2];
#pragma unroll
  for (int nb = 0; nb < 2; ++nb) {
    b1[0][nb] = make_uint2(__byte_perm(z[4 * nb], z[4 * nb + 1], 0x5410), __byte_perm(z[4 * nb + 2], z[4 * nb + 3], 0x5410));
    b1[1][nb] = make_uint2(__byte_perm(z[4 * nb], z[4 * nb + 1], 0x7632), __byte_perm(z[4 * nb + 2], z[4 * nb + 3], 0x7632));
  }
  float d1[2][2][4];  // [re/im of Y][t block][fragment]
#pragma unroll
  for (int mb = 0; mb < 2; ++mb)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      d1[mb][nb][0] = d1[mb][nb][1] = d1[mb][nb][2] = d1[mb][nb][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint4 af = make_uint4(a1[(mb * 2 + ks) * 4 + 0], a1[(mb * 2 + ks) * 4 + 1], a1[(mb * 2 + ks) * 4 + 2],
                                    a1[(mb * 2 + ks) * 4 + 3]);
        mma16816<false>(d1[mb][nb], af, b1[ks][nb]);
      }
    }
  // twiddle w256^(t k): fragment q of block nb holds k = g + 8 (q >> 1), t = 8 nb + 2 t4 + (q & 1)
  float yr[2][4], yi[2][4];
#pragma unroll
  for (int nb = 0; nb < 2; ++nb)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 w = tw[nb * 4 + q];
      const float r = d1[0][nb][q], im = d1[1][nb][q];
      yr[nb][q] = fmaf(r, w.x, -im * w.y);
      yi[nb][q] = fmaf(r, w.y, im * w.x);
    }
  uint4 a2[2];  // [re/im k-step]
  a2[0] = make_uint4(pack_bf2(yr[0][0], yr[0][1]), pack_bf2(yr[0][2], yr[0][3]), pack_bf2(yr[1][0], yr[1][1]),
                     pack_bf2(yr[1][2], yr[1][3]));
  a2[1] = make_uint4(pack_bf2(yi[0][0], yi[0][1]), pack_bf2(yi[0][2], yi[0][3]), pack_bf2(yi[1][0], yi[1][1]),
                     pack_bf2(yi[1][2], yi[1][3]));
#pragma unroll
  for (int nb = 0; nb < 4; ++nb) {
    d2[nb][0] = d2[nb][1] = d2[nb][2] = d2[nb][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
      mma16816<false>(d2[nb], a2[ks], make_uint2(b2[(ks * 4 + nb) * 2], b2[(ks * 4 + nb) * 2 + 1]));
  }
}

// Inverse angular DFT of one pair (M = 256) by one warp (idft256_core).
// Returns this lane's maxima of the real (unmirrored) and imaginary
// (mirrored) parts (the caller reduces over the warp); `dbg` (or null)
// receives every value: dbg[j] = Re c(j), dbg[M + (j + M/2) mod M] = Im c(j).
__device__ __forceinline__ void pair_idft_tc256(const uint32_t *zp, int sw, const TcLane &L,
                                                const uint32_t (&a1)[16], const uint32_t (&b2)[16], int lane,
                                                float &vu, float &vm, float *dbg) {
  const int g = lane >> 2, t4 = lane & 3;
  uint32_t z[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) z[e] = zp[L.zoff[e] ^ sw];
  float d2[4][4];  // [(re/im of c, j block)][fragment]
  idft256_core(z, L.tw, a1, b2, d2);
  vu = fmaxf(fmaxf(fmaxf(d2[0][0], d2[0][1]), fmaxf(d2[0][2], d2[0][3])),
             fmaxf(fmaxf(d2[1][0], d2[1][1]), fmaxf(d2[1][2], d2[1][3])));
  vm = fmaxf(fmaxf(fmaxf(d2[2][0], d2[2][1]), fmaxf(d2[2][2], d2[2][3])),
             fmaxf(fmaxf(d2[3][0], d2[3][1]), fmaxf(d2[3][2], d2[3][3])));
  if (dbg) {
#pragma unroll
    for (int nb = 0; nb < 4; ++nb)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = g + 8 * (q >> 1), j = 8 * (nb & 1) + 2 * t4 + (q & 1);
        const int ang = k + 16 * j;
        if (nb < 2)
          dbg[ang] = d2[nb][q];
        else
          dbg[256 + ((ang + 128) & 255)] = d2[nb][q];
      }
  }
}

// Maxima over the 32 lanes of two values per lane in 5 shuffles: at the
// first butterfly step lanes 0-15 keep `u` and lanes 16-31 keep `m`, so
// afterwards lanes 0-15 hold max(u) and lanes 16-31 max(m).
__device__ __forceinline__ float warp_max2(float u, float m, int lane) {
  const bool hi = (lane & 16) != 0;
  float v = fmaxf(hi ? m : u, __shfl_xor_sync(0xffffffffu, hi ? u : m, 16));
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Maxima over the 32 lanes of four values per lane, the (u, m) maxima of
// two pairs A and B, in 6 shuffles: afterwards lanes 0-7 hold max(uA), 8-15
// max(mA), 16-23 max(uB) and 24-31 max(mB).
__device__ __forceinline__ float warp_max4(float uA, float mA, float uB, float mB, int lane) {
  const bool hb = (lane & 16) != 0;  // this half keeps pair B and sends pair A
  float x = fmaxf(hb ? uB : uA, __shfl_xor_sync(0xffffffffu, hb ? uA : uB, 16));
  float y = fmaxf(hb ? mB : mA, __shfl_xor_sync(0xffffffffu, hb ? mA : mB, 16));
  const bool hm = (lane & 8) != 0;   // this quarter keeps m and sends u
  float v = fmaxf(hm ? y : x, __shfl_xor_sync(0xffffffffu, hm ? x : y, 8));
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// M = 256 kernel: one CTA per tile of 8 rows, looping over the reference
// tiles of 8 (64 pairs each), 8 warps, two CTAs per SM.  Phase 1 streams a
// tile's A and B fragments in chunks of whole frequencies (at most
// kTc256ChunkKs k-steps, 1 KB each) through two shared-memory buffers with
// TMA bulk copies issued by thread 0, one mbarrier per buffer; the copy of
// chunk q + 2 (of this tile or the first two of the next one) starts as soon
// as chunk q has been consumed, so the next tile's first chunks load while
// this tile's inverse DFTs run.  Warp w contracts frequencies f0 + w,
// f0 + w + 8, ... of each chunk (two MMAs per k-step, one per 4-reference
// block) and stores Z(f), Z(M - f) of its 32 lanes' pairs as BF16 words.
// Phase 2: warp w takes reference w of the tile and its 8 rows, one
// tensor-core inverse DFT and one warp reduction of the two row maxima each.  Every wait is bounded; the CTA agrees on a failed wait at the
// per-chunk barrier, thread 0 records it, waits (bounded) for the copies
// still in flight, and the CTA leaves.
constexpr int kTc256Warps = 8;
constexpr int kTc256Threads = 32 * kTc256Warps;
constexpr int kTc256MaxChunks = 32;
constexpr size_t kTc256Stage = static_cast<size_t>(kTc256ChunkKs) * 1024;
constexpr size_t kTc256Smem = 2 * kTc256Stage + 64 * 256 * sizeof(uint32_t) + 256 * sizeof(float2) +
                              2 * sizeof(uint64_t) + 8 * sizeof(int2) + (130 + kTc256MaxChunks + 2) * sizeof(int);

template <bool FP16>
__global__ void __launch_bounds__(kTc256Threads, 2) cc_tc256_kernel(Geometry g, TcArgs a, int ref_tiles) {
  constexpr int M = 256, PAIRS = 64, NF = M / 2 + 1;
  extern __shared__ float4 smem_f4[];
  unsigned char *stage = reinterpret_cast<unsigned char *>(smem_f4);
  uint32_t *Zw = reinterpret_cast<uint32_t *>(stage + 2 * kTc256Stage);  // [64 pairs][256 words]
  float2 *tw = reinterpret_cast<float2 *>(Zw + PAIRS * M);
  uint64_t *full = reinterpret_cast<uint64_t *>(tw + M);
  int2 *rinfo = reinterpret_cast<int2 *>(full + 2);  // {image, shift} of the tile's rows
  int *s_kso = reinterpret_cast<int *>(rinfo + 8);   // [NF + 1]
  int *s_cf = s_kso + NF + 1;                        // [NCH + 1]

  const int64_t rt = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = g.NCH;
  const int total = ref_tiles * nch;  // chunks over the whole reference loop
  for (int i = tid; i < M; i += kTc256Threads) tw[i] = g.inv_tw[i];
  for (int i = tid; i <= NF; i += kTc256Threads) s_kso[i] = g.kso[i];
  for (int i = tid; i <= nch; i += kTc256Threads) s_cf[i] = g.chunk_f[i];
  if (tid < 8) {
    const int64_t row = rt * 8 + tid;
    const int img = static_cast<int>(static_cast<uint32_t>(row) / static_cast<uint32_t>(g.S));  // rows < 2^31
    rinfo[tid] = make_int2(img, static_cast<int>(row - static_cast<int64_t>(img) * g.S));
  }
  if (tid == 0) {
    mbar_init(full, 1);
    mbar_init(full + 1, 1);
  }
  mbar_init_fence();
  __syncthreads();

  auto issue = [&](int q) {  // thread 0: stage chunk q % nch of reference tile q / nch into buffer q & 1
    const int kt = q / nch, c = q - kt * nch;
    const int k0 = s_kso[s_cf[c]];
    const uint32_t nks = static_cast<uint32_t>(s_kso[s_cf[c + 1]] - k0);
    unsigned char *dst = stage + (q & 1) * kTc256Stage;
    fence_proxy_async();
    mbar_arrive_expect_tx(full + (q & 1), nks * 1024u);
    bulk_g2s(dst, a.A16 + (rt * g.KS + k0) * 32, nks * 512u, full + (q & 1));
    bulk_g2s(dst + nks * 512u, a.B16 + ((static_cast<int64_t>(kt) * 2) * g.KS + k0) * 32, nks * 256u, full + (q & 1));
    bulk_g2s(dst + nks * 768u, a.B16 + ((static_cast<int64_t>(kt) * 2 + 1) * g.KS + k0) * 32, nks * 256u,
             full + (q & 1));
  };
  if (tid == 0) {
    issue(0);
    if (total > 1) issue(1);
  }

  // lane constants of phase 2
  uint32_t a1[16], b2[16];
  {
    const uint4 *fa = reinterpret_cast<const uint4 *>(g.dft16) + lane * 4;
    const uint4 *fb = reinterpret_cast<const uint4 *>(g.dft16 + 512) + lane * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint4 va = __ldg(fa + i), vb = __ldg(fb + i);
      a1[4 * i] = va.x;
      a1[4 * i + 1] = va.y;
      a1[4 * i + 2] = va.z;
      a1[4 * i + 3] = va.w;
      b2[4 * i] = vb.x;
      b2[4 * i + 1] = vb.y;
      b2[4 * i + 2] = vb.z;
      b2[4 * i + 3] = vb.w;
    }
  }
  TcLane Ln;
  tc_lane_init(Ln, tw, lane);
  const int g8 = lane >> 2, t4 = lane & 3;
  const int sw = 4 * g8 + t4;                 // z256_swz of both of this lane's phase-1 pairs
  uint32_t *z0 = Zw + (8 * g8 + t4) * M;      // pair (row g8, reference t4)
  uint32_t *z1 = z0 + 4 * M;                  // pair (row g8, reference 4 + t4)
  const int S = g.S;

  int q = 0;  // global chunk index
  for (int kt = 0; kt < ref_tiles; ++kt) {
    // ---------------- Phase 1: tensor-core contraction ----------------
    for (int c = 0; c < nch; ++c, ++q) {
      const int buf = q & 1;
      const bool ok = mbar_wait_bounded(full + buf, static_cast<uint32_t>((q >> 1) & 1),
                                        q == 0 ? a.first_wait_limit : a.wait_limit);
      if (ok) {
        const int f0 = s_cf[c], f1 = s_cf[c + 1];
        const int kbase = s_kso[f0];
        const int nks_c = s_kso[f1] - kbase;
        const uint4 *stA = reinterpret_cast<const uint4 *>(stage + buf * kTc256Stage) + lane;
        const uint2 *stB0 = reinterpret_cast<const uint2 *>(stage + buf * kTc256Stage + static_cast<size_t>(nks_c) * 512) + lane;
        const uint2 *stB1 = stB0 + nks_c * 32;
        for (int f = f0 + warp; f < f1; f += kTc256Warps) {
          const int jb = s_kso[f] - kbase, nj = s_kso[f + 1] - s_kso[f];  // 1..3 k-steps
          float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) {
            if (jj < nj) {
              const int j = (jb + jj) * 32;
              const uint4 af = stA[j];
              mma16816<FP16>(d0, af, stB0[j]);
              mma16816<FP16>(d1, af, stB1[j]);
            }
          }
          // lane (g8, t4): d[0..1] = Re/Im Z(f), d[2..3] = Im/Re Z(M - f)
          const int pf = z256_fold(f) ^ sw;
          z0[pf] = pack_bf2(d0[0], d0[1]);
          z1[pf] = pack_bf2(d1[0], d1[1]);
          if (f != 0 && f != M / 2) {
            const int pm = z256_fold(M - f) ^ sw;
            z0[pm] = pack_bf2(d0[3], d0[2]);
            z1[pm] = pack_bf2(d1[3], d1[2]);
          }
        }
      }
      if (__syncthreads_or(!ok)) {  // uniform: every thread leaves
        if (tid == 0) {
          atomicOr(a.err, 1);
          // let the copies still in flight land before the CTA's memory goes
          mbar_wait_bounded(full + (q & 1), static_cast<uint32_t>((q >> 1) & 1), a.wait_limit);
          if (q + 1 < total)
            mbar_wait_bounded(full + ((q + 1) & 1), static_cast<uint32_t>(((q + 1) >> 1) & 1), a.wait_limit);
        }
        return;
      }
      if (tid == 0 && q + 2 < total) issue(q + 2);
    }

    // ---------------- Phase 2: tensor-core inverse DFT, row maxima ----------------
    const int ref = kt * 8 + warp;  // pairs warp + 8 i: reference `warp` of the tile, row i
    const int nvalid = ref < a.K ? static_cast<int>(min(static_cast<int64_t>(8), a.rows - rt * 8)) : 0;
    // the row maxima of two consecutive pairs are reduced over the warp together
    float su = -INFINITY, sm = -INFINITY;  // the even pair's lane maxima
    int64_t sbase = 0;
#pragma unroll 1
    for (int i = 0; i < nvalid; ++i) {  // padding pairs are skipped (warp-uniform)
      const int pc = 8 * i + warp;
      const int2 ri = rinfo[i];
      const int64_t rbase = (static_cast<int64_t>(ri.x) * a.K + ref) * S + ri.y;
      float *dbg = a.dbg_cc ? a.dbg_cc + rbase * 2 * M : nullptr;
      float vu, vm;
      pair_idft_tc256(Zw + pc * M, z256_swz(pc), Ln, a1, b2, lane, vu, vm, dbg);
      if ((i & 1) == 0 && i + 1 < nvalid) {
        su = vu;
        sm = vm;
        sbase = rbase;
        continue;
      }
      if (i & 1) {
        const float v = warp_max4(su, sm, vu, vm, lane);
        if ((lane & 7) == 0) {
          const bool mrow = (lane & 8) != 0;
          a.rowmax[((lane & 16) ? rbase : sbase) * 2 + mrow] = (mrow && !g.mirror) ? -INFINITY : v;
        }
      } else {  // the last pair of an odd count
        const float best = warp_max2(vu, vm, lane);
        if ((lane & 15) == 0) a.rowmax[rbase * 2 + (lane >> 4)] = (lane && !g.mirror) ? -INFINITY : best;
      }
    }
    __syncthreads();  // the next tile's contraction overwrites the pair buffers
  }
}

// M = 512 kernel (rings up to 81): the tile walk and chunked staging of the
// M = 256 kernel with one CTA of 16 warps per SM (the BF16 spectra of the
// 64 pairs take 128 KB) and chunks of up to kTc512ChunkKs k-steps.
// Spectrum word of Z(f) in a pair's 512-word buffer: z512_fold(f) ^ s with
// s = 4 (pair / 8) + (pair % 4) < 32, so the contraction's stores (32 lanes,
// 32 pairs, one f) hit distinct banks.  Phase 2: the inverse DFT on tensor
// cores by an even / odd split (decimation in frequency index):
//     c(n)       = E(n) + w512^n O(n),    c(n + 256) = E(n) - w512^n O(n),
//     E(n) = sum_m Z(2 m) w256^(m n),     O(n) = sum_m Z(2 m + 1) w256^(m n),
// n = 0..255: two 256-point inverse DFTs per pair (idft256_core) and a
// radix-2 combine in FP32, one warp per pair.  z512_fold places the words
// those 256-point DFTs load (f = 2 (8 nb + g + 16 a) (+1)) in 32 distinct
// banks for every load of the warp.
__device__ __forceinline__ int z512_fold(int f) { return f ^ ((f >> 6) & 1) ^ (((f >> 7) & 1) << 4); }

constexpr int kTc512Warps = 16;
constexpr int kTc512Threads = 32 * kTc512Warps;
constexpr int kTc512MaxChunks = 48;
constexpr size_t kTc512Stage = static_cast<size_t>(kTc512ChunkKs) * 1024;
constexpr size_t kTc512Smem = 2 * kTc512Stage + 64 * 512 * sizeof(uint32_t) + 2 * sizeof(uint64_t) + 8 * sizeof(int2) +
                              (258 + kTc512MaxChunks + 2) * sizeof(int);
static_assert(kTc512Smem <= 232448, "M = 512 kernel exceeds 227 KB of shared memory");

template <bool FP16>
__global__ void __launch_bounds__(kTc512Threads, 1) cc_tc512_kernel(Geometry g, TcArgs a, int ref_tiles) {
  constexpr int M = 512, PAIRS = 64, NF = M / 2 + 1;
  extern __shared__ float4 smem_f4[];
  unsigned char *stage = reinterpret_cast<unsigned char *>(smem_f4);
  uint32_t *Zw = reinterpret_cast<uint32_t *>(stage + 2 * kTc512Stage);  // [64 pairs][512 words]
  uint64_t *full = reinterpret_cast<uint64_t *>(Zw + PAIRS * M);
  int2 *rinfo = reinterpret_cast<int2 *>(full + 2);  // {image, shift} of the tile's rows
  int *s_kso = reinterpret_cast<int *>(rinfo + 8);   // [NF + 1]
  int *s_cf = s_kso + NF + 1;                        // [NCH + 1]

  const int64_t rt = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = g.NCH;
  const int total = ref_tiles * nch;
  for (int i = tid; i <= NF; i += kTc512Threads) s_kso[i] = g.kso[i];
  for (int i = tid; i <= nch; i += kTc512Threads) s_cf[i] = g.chunk_f[i];
  if (tid < 8) {
    const int64_t row = rt * 8 + tid;
    const int img = static_cast<int>(static_cast<uint32_t>(row) / static_cast<uint32_t>(g.S));  // rows < 2^31
    rinfo[tid] = make_int2(img, static_cast<int>(row - static_cast<int64_t>(img) * g.S));
  }
  if (tid == 0) {
    mbar_init(full, 1);
    mbar_init(full + 1, 1);
  }
  mbar_init_fence();
  __syncthreads();

  auto issue = [&](int q) {  // thread 0: stage chunk q % nch of reference tile q / nch into buffer q & 1
    const int kt = q / nch, c = q - kt * nch;
    const int k0 = s_kso[s_cf[c]];
    const uint32_t nks = static_cast<uint32_t>(s_kso[s_cf[c + 1]] - k0);
    unsigned char *dst = stage + (q & 1) * kTc512Stage;
    fence_proxy_async();
    mbar_arrive_expect_tx(full + (q & 1), nks * 1024u);
    bulk_g2s(dst, a.A16 + (rt * g.KS + k0) * 32, nks * 512u, full + (q & 1));
    bulk_g2s(dst + nks * 512u, a.B16 + ((static_cast<int64_t>(kt) * 2) * g.KS + k0) * 32, nks * 256u, full + (q & 1));
    bulk_g2s(dst + nks * 768u, a.B16 + ((static_cast<int64_t>(kt) * 2 + 1) * g.KS + k0) * 32, nks * 256u,
             full + (q & 1));
  };
  if (tid == 0) {
    issue(0);
    if (total > 1) issue(1);
  }

  const int g8 = lane >> 2, t4 = lane & 3;
  const int sw = 4 * g8 + t4;              // spectrum swizzle of both of this lane's phase-1 pairs
  uint32_t *z0 = Zw + (8 * g8 + t4) * M;   // pair (row g8, reference t4)
  uint32_t *z1 = z0 + 4 * M;               // pair (row g8, reference 4 + t4)
  const int S = g.S;

  // lane constants of phase 2: the 16-point DFT fragments, the folded word
  // positions of the even spectrum words this lane loads (the odd word of
  // each sits at the position XOR 1), the 256-point stage twiddles
  // w256^(t k) = w512^(2 t k) and the combine twiddles w512^n of its angles
  // (g.angles[q] = exp(2 pi i q / M))
  uint32_t a1[16], b2[16];
  {
    const uint4 *fa = reinterpret_cast<const uint4 *>(g.dft16) + lane * 4;
    const uint4 *fb = reinterpret_cast<const uint4 *>(g.dft16 + 512) + lane * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint4 va = __ldg(fa + i), vb = __ldg(fb + i);
      a1[4 * i] = va.x;
      a1[4 * i + 1] = va.y;
      a1[4 * i + 2] = va.z;
      a1[4 * i + 3] = va.w;
      b2[4 * i] = vb.x;
      b2[4 * i + 1] = vb.y;
      b2[4 * i + 2] = vb.z;
      b2[4 * i + 3] = vb.w;
    }
  }
  int zoff[8];
  float2 tws[8], wn[8];
  {
    const int aa[4] = {2 * t4, 2 * t4 + 1, 2 * t4 + 8, 2 * t4 + 9};
#pragma unroll
    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
      for (int e = 0; e < 4; ++e) zoff[nb * 4 + e] = z512_fold(2 * (8 * nb + g8 + 16 * aa[e]));
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = g8 + 8 * (q >> 1);
        tws[b * 4 + q] = __ldg(g.angles + ((2 * (8 * b + 2 * t4 + (q & 1)) * k) & (M - 1)));
        wn[b * 4 + q] = __ldg(g.angles + k + 16 * (8 * b + 2 * t4 + (q & 1)));
      }
  }

  int q = 0;  // global chunk index
  for (int kt = 0; kt < ref_tiles; ++kt) {
    // ---------------- Phase 1: tensor-core contraction ----------------
    for (int c = 0; c < nch; ++c, ++q) {
      const int buf = q & 1;
      const bool ok = mbar_wait_bounded(full + buf, static_cast<uint32_t>((q >> 1) & 1),
                                        q == 0 ? a.first_wait_limit : a.wait_limit);
      if (ok) {
        const int f0 = s_cf[c], f1 = s_cf[c + 1];
        const int kbase = s_kso[f0];
        const int nks_c = s_kso[f1] - kbase;
        const uint4 *stA = reinterpret_cast<const uint4 *>(stage + buf * kTc512Stage) + lane;
        const uint2 *stB0 =
            reinterpret_cast<const uint2 *>(stage + buf * kTc512Stage + static_cast<size_t>(nks_c) * 512) + lane;
        const uint2 *stB1 = stB0 + nks_c * 32;
        for (int f = f0 + warp; f < f1; f += kTc512Warps) {
          const int jb = s_kso[f] - kbase, nj = s_kso[f + 1] - s_kso[f];  // 1..6 k-steps
          float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int jj = 0; jj < kTc512MaxKsPerF; ++jj) {
            if (jj < nj) {
              const int j = (jb + jj) * 32;
              const uint4 af = stA[j];
              mma16816<FP16>(d0, af, stB0[j]);
              mma16816<FP16>(d1, af, stB1[j]);
            }
          }
          // lane (g8, t4): d[0..1] = Re/Im Z(f), d[2..3] = Im/Re Z(M - f)
          const int pf = z512_fold(f) ^ sw;
          z0[pf] = pack_bf2(d0[0], d0[1]);
          z1[pf] = pack_bf2(d1[0], d1[1]);
          if (f != 0 && f != M / 2) {
            const int pm = z512_fold(M - f) ^ sw;
            z0[pm] = pack_bf2(d0[3], d0[2]);
            z1[pm] = pack_bf2(d1[3], d1[2]);
          }
        }
      }
      if (__syncthreads_or(!ok)) {  // uniform: every thread leaves
        if (tid == 0) {
          atomicOr(a.err, 1);
          // let the copies still in flight land before the CTA's memory goes
          mbar_wait_bounded(full + (q & 1), static_cast<uint32_t>((q >> 1) & 1), a.wait_limit);
          if (q + 1 < total)
            mbar_wait_bounded(full + ((q + 1) & 1), static_cast<uint32_t>(((q + 1) >> 1) & 1), a.wait_limit);
        }
        return;
      }
      if (tid == 0 && q + 2 < total) issue(q + 2);
    }

    // ---------------- Phase 2: tensor-core inverse DFT (even / odd split), row maxima ----------------
    // warp w: reference w % 8 of the tile, rows 4 (w / 8) .. 4 (w / 8) + 3
    const int refl = warp & 7;
    const int ref = kt * 8 + refl;
    const int i0 = 4 * (warp >> 3);
    const int64_t left = a.rows - rt * 8 - i0;
    const int nvalid = ref < a.K ? (left >= 4 ? 4 : (left > 0 ? static_cast<int>(left) : 0)) : 0;
#pragma unroll 1
    for (int r = 0; r < nvalid; ++r) {  // padding pairs are skipped (warp-uniform)
      const int i = i0 + r, pc = 8 * i + refl;
      const uint32_t *zp = Zw + pc * M;
      const int swp = 4 * (pc >> 3) + (pc & 3);
      float de[4][4], dd[4][4];  // E and O at this lane's angles (idft256_core's fragment order)
      {
        uint32_t z[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) z[e] = zp[zoff[e] ^ swp];
        idft256_core(z, tws, a1, b2, de);
      }
      {
        uint32_t z[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) z[e] = zp[zoff[e] ^ 1 ^ swp];
        idft256_core(z, tws, a1, b2, dd);
      }
      const int2 ri = rinfo[i];
      const int64_t rbase = (static_cast<int64_t>(ri.x) * a.K + ref) * S + ri.y;
      float *dbg = a.dbg_cc ? a.dbg_cc + rbase * 2 * M : nullptr;
      float vu = -INFINITY, vm = -INFINITY;
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 w = wn[b * 4 + q];
          const float orr = dd[b][q], oi = dd[b + 2][q];
          const float wr = fmaf(w.x, orr, -w.y * oi), wi = fmaf(w.x, oi, w.y * orr);
          const float c1r = de[b][q] + wr, c1i = de[b + 2][q] + wi;  // angle n
          const float c2r = de[b][q] - wr, c2i = de[b + 2][q] - wi;  // angle n + 256
          vu = fmaxf(vu, fmaxf(c1r, c2r));
          vm = fmaxf(vm, fmaxf(c1i, c2i));
          if (dbg) {
            const int n = g8 + 8 * (q >> 1) + 16 * (8 * b + 2 * t4 + (q & 1));
            dbg[n] = c1r;
            dbg[n + 256] = c2r;
            dbg[M + n + 256] = c1i;  // Im c(n) at (n + M / 2) mod M
            dbg[M + n] = c2i;        // Im c(n + 256) at n
          }
        }
      // (reducing two pairs together as the M = 256 kernel does needs registers this kernel does not have)
      const float best = warp_max2(vu, vm, lane);
      if ((lane & 15) == 0) a.rowmax[rbase * 2 + (lane >> 4)] = (lane && !g.mirror) ? -INFINITY : best;
    }
    __syncthreads();  // the next tile's contraction overwrites the pair buffers
  }
}

template <int M, int KT, bool FP16>
__global__ void __launch_bounds__(TcShape<M, KT>::THREADS) cc_tc_kernel(Geometry g, TcArgs a) {
  using Sh = TcShape<M, KT>;
  constexpr int T = IfftShape<M>::T;
  constexpr int U = IfftShape<M>::U;
  extern __shared__ float4 smem_f4[];
  unsigned char *sbase = reinterpret_cast<unsigned char *>(smem_f4);
  float2 *Zs = reinterpret_cast<float2 *>(sbase);
  float2 *tw = reinterpret_cast<float2 *>(sbase + Sh::STATE);
  uint64_t *bars = reinterpret_cast<uint64_t *>(sbase + Sh::STATE + Sh::TW);
  unsigned char *stage0 = sbase + Sh::STATE + Sh::TW + Sh::BARS;
  const size_t stage_bytes = Sh::stage_bytes(a.ks_max);

  const int kt = blockIdx.x;
  const int64_t rt = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < M; i += Sh::THREADS) tw[i] = g.inv_tw[i];
  if (lane == 0) mbar_init(bars + warp, 1);
  mbar_init_fence();
  __syncwarp();

  // ---------------- Phase 1: tensor-core contraction ----------------
  bool failed = false;
  {
    uint4 *stA = reinterpret_cast<uint4 *>(stage0 + warp * stage_bytes);
    uint2 *stB = reinterpret_cast<uint2 *>(stage0 + warp * stage_bytes + static_cast<size_t>(a.ks_max) * 512);
    uint64_t *bar = bars + warp;
    uint32_t phase = 0;
    bool first_wait = true;
    const int g8 = lane >> 2, t4 = lane & 3;
    for (int f = warp; f <= M / 2; f += Sh::WARPS) {
      const int kb = g.kso[f];
      const int nks = g.kso[f + 1] - kb;
      if (lane == 0) {
        const uint32_t abytes = static_cast<uint32_t>(nks) * 512u;
        const uint32_t bbytes = static_cast<uint32_t>(nks) * 256u;
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, abytes + Sh::NBLK * bbytes);
        bulk_g2s(stA, a.A16 + (rt * g.KS + kb) * 32, abytes, bar);
        const int ref0 = kt * KT;
#pragma unroll
        for (int nb = 0; nb < Sh::NBLK; ++nb) {
          const int64_t blk = static_cast<int64_t>(ref0 / kTile) * 2 + (ref0 % kTile) / 4 + nb;
          bulk_g2s(stB + nb * nks * 32, a.B16 + (blk * g.KS + kb) * 32, bbytes, bar);
        }
      }
      const uint32_t limit = first_wait ? a.first_wait_limit : a.wait_limit;
      first_wait = false;
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, phase, limit))) {
        if (lane == 0) atomicOr(a.err, 1);
        mbar_wait_bounded(bar, phase, a.wait_limit);
        failed = true;
        break;
      }
      phase ^= 1u;
      float d[Sh::NBLK][4];
#pragma unroll
      for (int nb = 0; nb < Sh::NBLK; ++nb) d[nb][0] = d[nb][1] = d[nb][2] = d[nb][3] = 0.f;
      for (int j = 0; j < nks; ++j) {
        const uint4 af = stA[j * 32 + lane];
#pragma unroll
        for (int nb = 0; nb < Sh::NBLK; ++nb) mma16816<FP16>(d[nb], af, stB[(nb * nks + j) * 32 + lane]);
      }
      // lane (g8, t4): pair (row g8, ref 4 nb + t4) in d[nb]
#pragma unroll
      for (int nb = 0; nb < Sh::NBLK; ++nb) {
        const int pa = g8 * KT + 4 * nb + t4;
        float2 *za = Zs + pa * Sh::P;
        const int sa = tc_swz<M, KT>(pa);
        za[f ^ sa] = make_float2(d[nb][0], d[nb][1]);
        if (f != 0 && f != M / 2) za[(M - f) ^ sa] = make_float2(d[nb][3], d[nb][2]);
      }
      __syncwarp();
    }
  }
  if (__syncthreads_or(failed)) return;

  // ---------------- Phase 2: inverse angular DFT, row maxima ----------------
  constexpr int GROUPS = Sh::THREADS / T;
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
    float2 y[IfftShape<M>::KK][T];
    pair_ifft<M>(zp, tc_swz<M, KT>(pc), zp, t, in_tile, tw, y);
    float vu = -INFINITY, vm = -INFINITY;
#pragma unroll
    for (int kk = 0; kk < U / T; ++kk)
#pragma unroll
      for (int jj = 0; jj < T; ++jj) {
        vu = fmaxf(vu, y[kk][jj].x);
        vm = fmaxf(vm, y[kk][jj].y);
      }
#pragma unroll
    for (int off = T / 2; off > 0; off >>= 1) {
      vu = fmaxf(vu, __shfl_xor_sync(0xffffffffu, vu, off, T));
      vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, off, T));
    }
    const int64_t img = row / S;
    const int s = static_cast<int>(row - img * S);
    if (valid && t == 0) {
      float *rm = a.rowmax + (img * a.K + ref) * static_cast<int64_t>(S) * 2 + 2 * s;
      rm[0] = vu;
      rm[1] = g.mirror ? vm : -INFINITY;
    }
    if (a.dbg_cc && valid) {
      float *d = a.dbg_cc + ((img * a.K + ref) * S + s) * 2 * M;
#pragma unroll
      for (int kk = 0; kk < U / T; ++kk)
#pragma unroll
        for (int jj = 0; jj < T; ++jj) {
          const int j = ifft_angle<M>(t, kk, jj);
          d[j] = y[kk][jj].x;
          d[M + ((j + M / 2) & (M - 1))] = y[kk][jj].y;
        }
    }
  }
}

// ---------------------------------------------------------------------------
// Top-8 rows (reference, shift, mirror) per image by row maximum; ties keep
// the smaller row index.  One warp per image.
// ---------------------------------------------------------------------------
__global__ void top8_kernel(const float *__restrict__ rowmax, int64_t n, int nrows, int *cand) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t img = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  if (img >= n) return;
  float v[kTopRows];
  int id[kTopRows];
#pragma unroll
  for (int e = 0; e < kTopRows; ++e) {
    v[e] = -INFINITY;
    id[e] = 0x7fffffff;
  }
  const float *rm = rowmax + img * nrows;
  for (int j = lane; j < nrows; j += 32) {
    const float x = rm[j];
    if (x > v[kTopRows - 1]) {
      v[kTopRows - 1] = x;
      id[kTopRows - 1] = j;
#pragma unroll
      for (int e = kTopRows - 1; e > 0; --e)
        if (v[e] > v[e - 1]) {
          const float tv = v[e];
          v[e] = v[e - 1];
          v[e - 1] = tv;
          const int ti = id[e];
          id[e] = id[e - 1];
          id[e - 1] = ti;
        }
    }
  }
  for (int round = 0; round < kTopRows; ++round) {
    unsigned long long key = (v[0] == -INFINITY) ? 0ull : make_key(v[0], static_cast<uint32_t>(id[0]));
    unsigned long long best = key;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
      best = o > best ? o : best;
    }
    if (lane == 0) cand[img * kTopRows + round] = best ? static_cast<int>(0xffffffffu - static_cast<uint32_t>(best)) : -1;
    const unsigned win = __ballot_sync(0xffffffffu, best != 0 && key == best);
    if (best != 0 && lane == __ffs(win) - 1) {
#pragma unroll
      for (int e = 0; e < kTopRows - 1; ++e) {
        v[e] = v[e + 1];
        id[e] = id[e + 1];
      }
      v[kTopRows - 1] = -INFINITY;
      id[kTopRows - 1] = 0x7fffffff;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers (the FP32 rescore kernel is in k_rescore.cu)
// ---------------------------------------------------------------------------
cudaError_t launch_refs16(const Geometry &g, const float2 *B, int ktiles, uint2 *B16, bool fp16, cudaStream_t st) {
  const int64_t total = static_cast<int64_t>(ktiles) * g.KS * 64;
  const int blocks = static_cast<int>((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  refs16_kernel<<<blocks, 256, 0, st>>>(g, B, ktiles, B16, fp16);
  return cudaGetLastError();
}

template <int M, int KT, bool FP16>
static cudaError_t launch_tc_t(const Geometry &g, const TcArgs &a, cudaStream_t st) {
  using Sh = TcShape<M, KT>;
  const size_t smem = Sh::smem(a.ks_max);
  static size_t granted = 0;
  cudaError_t e = raise_smem_limit(cc_tc_kernel<M, KT, FP16>, smem, granted);
  if (e != cudaSuccess) return e;
  const int64_t row_tiles = (a.rows + Sh::RT - 1) / Sh::RT;
  if (row_tiles <= 0) return cudaSuccess;
  dim3 grid((a.K + KT - 1) / KT, static_cast<unsigned>(row_tiles));
  cc_tc_kernel<M, KT, FP16><<<grid, Sh::THREADS, smem, st>>>(g, a);
  return cudaGetLastError();
}

template <bool FP16>
static cudaError_t launch_tc256(const Geometry &g, const TcArgs &a, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(cc_tc256_kernel<FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kTc256Smem));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t row_tiles = (a.rows + kTile - 1) / kTile;
  if (row_tiles <= 0) return cudaSuccess;
  if (g.NCH > kTc256MaxChunks) return cudaErrorInvalidValue;
  cc_tc256_kernel<FP16><<<static_cast<unsigned>(row_tiles), kTc256Threads, kTc256Smem, st>>>(
      g, a, (a.K + kTile - 1) / kTile);
  return cudaGetLastError();
}

template <bool FP16>
static cudaError_t launch_tc512(const Geometry &g, const TcArgs &a, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(cc_tc512_kernel<FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kTc512Smem));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t row_tiles = (a.rows + kTile - 1) / kTile;
  if (row_tiles <= 0) return cudaSuccess;
  if (g.NCH > kTc512MaxChunks) return cudaErrorInvalidValue;
  cc_tc512_kernel<FP16><<<static_cast<unsigned>(row_tiles), kTc512Threads, kTc512Smem, st>>>(
      g, a, (a.K + kTile - 1) / kTile);
  return cudaGetLastError();
}

cudaError_t launch_cc_tc(const Geometry &g, const TcArgs &a, bool fp16, cudaStream_t st) {
  if (g.M == 256) return fp16 ? launch_tc256<true>(g, a, st) : launch_tc256<false>(g, a, st);
  if (g.M == 512) return fp16 ? launch_tc512<true>(g, a, st) : launch_tc512<false>(g, a, st);
#define MRA_TC_CASE(MM, KK) \
  case MM: return fp16 ? launch_tc_t<MM, KK, true>(g, a, st) : launch_tc_t<MM, KK, false>(g, a, st);
  switch (g.M) {
    MRA_TC_CASE(16, 8)
    MRA_TC_CASE(32, 8)
    MRA_TC_CASE(64, 8)
    MRA_TC_CASE(128, 8)
    default: return cudaErrorInvalidValue;
  }
#undef MRA_TC_CASE
}

cudaError_t launch_top8(const float *rowmax, int64_t n, int nrows, int *cand, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  top8_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, st>>>(rowmax, n, nrows, cand);
  return cudaGetLastError();
}

}  // namespace mra
