// C-ABI of the MRA library (declared in include/mra.h): argument checks,
// geometry tables (computed in FP64 on the host, stored FP32 on the device),
// workspace ownership and the chunked launch sequence of Algorithm 1.
#include "../../include/mra.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_fp16.h>

#include "mra_internal.h"

namespace {

thread_local std::string g_create_error;

// Host-side fault injection for tests of error propagation: the environment
// variable MRA_FAULT = alloc | launch | timeout makes the next device
// allocation / kernel launch / alignment report ENOMEM / ECUDA / ETIMEOUT
// without touching the GPU.
bool fault(const char *what) {
  const char *f = std::getenv("MRA_FAULT");
  return f && std::strcmp(f, what) == 0;
}

constexpr double kTwoPi = 6.283185307179586476925286766559;

}  // namespace

struct mra_handle {
  mra_config_t cfg{};
  int device = 0;
  mra::Geometry g{};
  int NBIN = 0, NB = 0;
  int seg_max = 0;             // longest padded frequency segment
  int ks_max = 0;              // most 16-ring k-steps of any frequency (16-bit paths)
  bool half = false;           // precision-split path (BF16/FP16 contraction + FP32 rescore)
  bool fp16 = false;           // FP16 rather than BF16 operands
  uint2 *B16 = nullptr;        // reference B fragments
  int B16_refs = 0;            // references (padded) the fragment buffer holds
  uint4 *A16 = nullptr;        // particle A fragments for one chunk (mma.sync kernels), or
                               // the k-step tiles of the tcgen05 kernel (umma)
  bool umma = false;           // M = 256 precision split on tcgen05 (k_umma256.cu)
  void *B16u = nullptr;        // reference k-step tiles of the tcgen05 kernel
  int B16u_refs = 0;           // references (padded to tiles) the tiles hold
  CUtensorMap tmA{}, tmB{};    // TMA descriptors of the particle / reference k-step tiles
  size_t A16_bytes = 0;
  float *rowmax = nullptr;     // [chunk][K][S][2]
  int64_t rowmax_cap = 0;      // floats
  int *cand = nullptr;         // [chunk][8]
  int *d_err = nullptr;        // device failure flags (bit 0: a bounded wait timed out)
  std::vector<void *> tables;  // device geometry tables
  // references
  int K = 0, Kpad = 0;
  float2 *B = nullptr;
  // per-chunk workspace
  int chunk = 0;
  float2 *A = nullptr;
  size_t A_bytes = 0;
  unsigned long long *best = nullptr;
  // averaging workspace
  mra::AvgWork avg{};
  int64_t avg_n_cap = 0;
  int avg_K_cap = 0;
  float *avg_sum = nullptr, *avg_comp = nullptr;
  int *avg_cnt = nullptr;
  // host-path staging
  float *h_stage_imgs = nullptr, *h_stage_refs = nullptr, *h_stage_avg = nullptr;
  mra_pose_t *h_stage_poses = nullptr;
  int *h_stage_counts = nullptr;
  int64_t h_stage_n = 0;
  int h_stage_K = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t workspace = 0;
  std::string err;
  // whole-pass CUDA graph (mra_run_graph): the buffers and sizes it was captured for
  struct GraphKey {
    const void *refs, *imgs, *poses, *avg, *counts;
    int64_t n;
    int K;
    bool operator==(const GraphKey &o) const {
      return refs == o.refs && imgs == o.imgs && poses == o.poses && avg == o.avg && counts == o.counts && n == o.n &&
             K == o.K;
    }
  };
  GraphKey graph_key{};
  int graph_seen = 0;               // calls with graph_key so far (the graph is captured on the second)
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  bool capturing = false;           // stage timing records are not taken inside a capture
  // per-stage event timing (mra_profile)
  bool prof_on = false;
  struct ProfRec {
    int stage;
    int launches;
    cudaEvent_t start, stop;
  };
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  int64_t prof_launches[MRA_STAGE_COUNT] = {};
  double prof_ms[MRA_STAGE_COUNT] = {};
};

namespace {

int set_err(mra_handle *h, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return code;
}

int cuda_err(mra_handle *h, cudaError_t e, const char *where) {
  return set_err(h, MRA_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

cudaEvent_t prof_event(mra_handle *h) {
  if (!h->prof_pool.empty()) {
    cudaEvent_t e = h->prof_pool.back();
    h->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Open a timed stage on stream st; returns a record index or -1 when off.
int prof_begin(mra_handle *h, int stage, cudaStream_t st) {
  if (!h->prof_on || h->capturing) return -1;
  cudaEvent_t a = prof_event(h), b = prof_event(h);
  if (!a || !b) return -1;
  cudaEventRecord(a, st);
  h->prof_recs.push_back({stage, 0, a, b});
  return static_cast<int>(h->prof_recs.size()) - 1;
}

void prof_end(mra_handle *h, int rec, int launches, cudaStream_t st) {
  if (rec < 0) return;
  h->prof_recs[rec].launches = launches;
  cudaEventRecord(h->prof_recs[rec].stop, st);
}

// Fold finished records into the per-stage totals.
void prof_collect(mra_handle *h) {
  for (auto &r : h->prof_recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.stop);
    if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      h->prof_ms[r.stage] += ms;
      h->prof_launches[r.stage] += r.launches;
    } else {
      cudaGetLastError();
    }
    h->prof_pool.push_back(r.start);
    h->prof_pool.push_back(r.stop);
  }
  h->prof_recs.clear();
}

template <class T>
int dev_alloc(mra_handle *h, T **p, size_t bytes, const char *what) {
  *p = nullptr;
  if (fault("alloc")) return set_err(h, MRA_ENOMEM, "injected allocation failure (%s)", what);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_err(h, MRA_ENOMEM, "cudaMalloc(%zu bytes) for %s failed: %s", bytes, what, cudaGetErrorString(e));
  }
  h->workspace += bytes;
  return MRA_OK;
}

void dev_free(mra_handle *h, void *p, size_t bytes) {
  if (p) {
    cudaFree(p);
    h->workspace -= (bytes == 0 ? 16 : bytes);
  }
}

int check_launch(mra_handle *h, cudaError_t e, const char *what) {
  if (fault("launch")) return set_err(h, MRA_ECUDA, "injected launch failure (%s)", what);
  if (e != cudaSuccess) return cuda_err(h, e, what);
  return MRA_OK;
}

template <class T>
int upload(mra_handle *h, const std::vector<T> &v, const T **out, const char *what) {
  T *d = nullptr;
  int rc = dev_alloc(h, &d, v.size() * sizeof(T), what);
  if (rc) return rc;
  h->tables.push_back(d);
  cudaError_t e = cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_err(h, e, what);
  *out = d;
  return MRA_OK;
}

}  // namespace

namespace mra {

// Whether every kernel the configuration launches fits the per-CTA shared
// memory limit (host arithmetic only, before any CUDA call; no heap use, so
// the allocation-free entry point can call it too).  The sizes follow the
// table construction in build_tables; the staged image is counted with the
// widest zero border (8 pixels) whenever the shift grid is integral.
// MRA_EUNSUPPORTED names the kernel that does not fit.  Expects a
// configuration whose rings give 16 <= M <= 512 (at most 81 rings).
static int fits_shared_memory(const mra_config_t &c, char *why, size_t why_len) {
  constexpr int kMaxRingsChecked = 96;
  int NN[kMaxRingsChecked];
  int NR = 0;
  for (int r = c.first_ring; r <= c.last_ring && NR < kMaxRingsChecked; r += c.ring_step) {
    int n = 1;
    while (n < kTwoPi * r) n *= 2;
    NN[NR++] = n;
  }
  int M = 0;
  for (int i = 0; i < NR; ++i) M = NN[i] > M ? NN[i] : M;
  Geometry g{};
  g.L = c.L;
  g.M = M;
  g.NR = NR;
  for (int i = 0; i < NR; ++i) {
    g.NS += NN[i];
    g.NBIN += NN[i] / 2 + 1;
  }
  int seg_max = 0;
  for (int f = 0; f <= M / 2; ++f) {
    int R = 0;
    for (int i = 0; i < NR; ++i) R += NN[i] / 2 >= f;
    g.KS += (R + 15) / 16;
    seg_max = std::max(seg_max, (R + 1) & ~1);
  }
  const double nx = std::round(2.0 * double(c.shift_range) / double(c.shift_step)) + 1.0;
  bool integral = true;
  for (int i = 0; i < static_cast<int>(nx); ++i) {
    const float v = static_cast<float>(-double(c.shift_range) + i * double(c.shift_step));  // as build_tables
    integral = integral && v == std::floor(v);
  }
  g.pad = 8;
  const bool half = c.precision != MRA_FP32;
  struct Need {
    const char *kernel;
    size_t bytes;
  };
  const Need needs[2] = {{"polar resampling / ring FFT", polar_smem_one_row(g, integral, half)},
                         half ? Need{"FP32 rescore", rescore_smem(g)} : Need{"FP32 contraction", cc_fp32_smem(M, seg_max)}};
  for (const Need &n : needs)
    if (n.bytes > kMaxSmemPerBlock) {
      std::snprintf(why, why_len,
                    "the %s kernel would need %zu bytes of shared memory per CTA for this configuration; at most "
                    "%zu are available (smaller box, fewer rings, or MRA_FP32)",
                    n.kernel, n.bytes, kMaxSmemPerBlock);
      return MRA_EUNSUPPORTED;
    }
  return MRA_OK;
}

int check_config(const mra_config_t *c, char *why, size_t why_len) {
  auto bad = [&](const char *m) {
    std::snprintf(why, why_len, "%s", m);
    return MRA_EINVAL;
  };
  if (!c) return bad("config is NULL");
  if (c->L < 8 || c->L > 1024 || (c->L & 1)) return bad("L must be even and in [8, 1024]");
  if (c->first_ring < 1) return bad("first_ring must be >= 1");
  if (c->last_ring < c->first_ring) return bad("last_ring must be >= first_ring");
  if (c->ring_step < 1) return bad("ring_step must be >= 1");
  if (!(c->shift_range >= 0.f) || !std::isfinite(c->shift_range)) return bad("shift_range must be finite and >= 0");
  if (!(c->shift_step > 0.f) || !std::isfinite(c->shift_step)) return bad("shift_step must be finite and > 0");
  const double q = 2.0 * double(c->shift_range) / double(c->shift_step);
  if (!std::isfinite(q) || std::fabs(q - std::round(q)) > 1e-6) return bad("2*shift_range/shift_step must be an integer");
  const double nx = std::round(q) + 1.0;
  if (nx * nx > 4096.0) {  // in double: no overflow for any finite grid
    std::snprintf(why, why_len, "shift grid has %.0f points; at most 4096 are supported", nx * nx);
    return MRA_EINVAL;
  }
  if (c->mirror != 0 && c->mirror != 1) return bad("mirror must be 0 or 1");
  if (c->precision != MRA_FP32 && c->precision != MRA_BF16_RESCORE && c->precision != MRA_FP16_RESCORE)
    return bad("precision must be MRA_FP32, MRA_BF16_RESCORE or MRA_FP16_RESCORE");
  if (c->chunk_images < 0) return bad("chunk_images must be >= 0");
  if (c->kernel != MRA_KERNEL_AUTO && c->kernel != MRA_KERNEL_MMA_SYNC && c->kernel != MRA_KERNEL_TCGEN05)
    return bad("kernel must be MRA_KERNEL_AUTO, MRA_KERNEL_MMA_SYNC or MRA_KERNEL_TCGEN05");
  // the largest ring sets M = its ring length
  const long long r_max = c->first_ring + (static_cast<long long>(c->last_ring - c->first_ring) / c->ring_step) *
                                              c->ring_step;
  long long M = 1;
  while (M < kTwoPi * static_cast<double>(r_max) && M <= 1024) M *= 2;
  if (M < 16 || M > 512) {
    std::snprintf(why, why_len, "largest ring length M = %lld; supported range is 16..512 (last ring 3..81)", M);
    return MRA_EINVAL;
  }
  return fits_shared_memory(*c, why, why_len);
}

}  // namespace mra

namespace {

int validate(const mra_config_t *c, std::string *why) {
  char buf[320];
  buf[0] = '\0';
  const int rc = mra::check_config(c, buf, sizeof(buf));
  *why = buf;
  return rc;
}

// Build every geometry table of the configuration (FP64 on the host).
int build_tables(mra_handle *h) {
  const mra_config_t &c = h->cfg;
  std::vector<int> rr, NN;
  for (int r = c.first_ring; r <= c.last_ring; r += c.ring_step) {
    int n = 1;
    while (n < kTwoPi * r) n *= 2;
    rr.push_back(r);
    NN.push_back(n);
  }
  const int NR = static_cast<int>(rr.size());
  int M = 0;
  for (int n : NN) M = n > M ? n : M;
  if (M < 16 || M > 512)
    return set_err(h, MRA_EINVAL, "largest ring length M = %d; supported range is 16..512 (last ring 3..81)", M);
  const int H = M / 2;
  // per-ring offsets
  std::vector<int4> rings(NR);
  int NS = 0, NBIN = 0;
  for (int i = 0; i < NR; ++i) {
    int lg = 0;
    while ((1 << lg) < NN[i] / 2) ++lg;
    rings[i] = make_int4(NN[i], NS, NBIN, lg);
    NS += NN[i];
    NBIN += NN[i] / 2 + 1;
  }
  // frequency-major padded layout: frequency f holds rings [first_f, NR)
  std::vector<int> first(H + 1);
  std::vector<int2> fseg(H + 1);
  int NB = 0;
  h->seg_max = 0;
  for (int f = 0; f <= H; ++f) {
    int i0 = 0;
    while (i0 < NR && NN[i0] / 2 < f) ++i0;
    first[f] = i0;
    const int R = NR - i0;
    const int Rp = (R + 1) & ~1;
    fseg[f] = make_int2(NB, Rp);
    NB += Rp;
    if (Rp > h->seg_max) h->seg_max = Rp;
  }
  // 16-bit tensor-core layout: frequency f owns ceil(R_f / 16) k-steps
  std::vector<int> kso(H + 2, 0);
  std::vector<int2> ksinfo;
  h->ks_max = 0;
  for (int f = 0; f <= H; ++f) {
    const int nks = (NR - first[f] + 15) / 16;
    kso[f] = static_cast<int>(ksinfo.size());
    for (int j = 0; j < nks; ++j) ksinfo.push_back(make_int2(f, j));
    if (nks > h->ks_max) h->ks_max = nks;
  }
  kso[H + 1] = static_cast<int>(ksinfo.size());
  std::vector<int> binpos16(NBIN);
  std::vector<int> binpos(NBIN);
  std::vector<float> bweight(NBIN);
  std::vector<float2> offs(NS);
  for (int i = 0; i < NR; ++i) {
    const int N = NN[i];
    for (int f = 0; f <= N / 2; ++f) {
      binpos[rings[i].z + f] = fseg[f].x + (i - first[f]);
      binpos16[rings[i].z + f] = kso[f] * 16 + (i - first[f]);
      double w = kTwoPi * rr[i] * c.ring_step / (double(N) * double(N));
      if (f == N / 2 && N < M) w *= 0.5;  // Nyquist split of an inner ring
      bweight[rings[i].z + f] = static_cast<float>(w);
    }
    for (int q = 0; q < N; ++q) {
      const double th = kTwoPi * q / N;
      offs[rings[i].y + q] = make_float2(static_cast<float>(rr[i] * std::cos(th)),
                                         static_cast<float>(rr[i] * std::sin(th)));
    }
  }
  std::vector<float2> fwd(M), ang(M), inv(M);
  for (int q = 0; q < M; ++q) {
    const double th = kTwoPi * q / M;
    fwd[q] = make_float2(static_cast<float>(std::cos(th)), static_cast<float>(-std::sin(th)));
    ang[q] = make_float2(static_cast<float>(std::cos(th)), static_cast<float>(std::sin(th)));
  }
  const int T = mra::cc_threads_per_pair(M), U = M / T;
  for (int k = 0; k < U; ++k)
    for (int t = 0; t < T; ++t) {
      const double th = kTwoPi * double(t) * double(k) / M;
      inv[k * T + t] = make_float2(static_cast<float>(std::cos(th)), static_cast<float>(std::sin(th)));
    }
  const int nx = static_cast<int>(std::lround(2.0 * double(c.shift_range) / double(c.shift_step))) + 1;
  std::vector<float2> shifts(static_cast<size_t>(nx) * nx);
  for (int iy = 0; iy < nx; ++iy)
    for (int ix = 0; ix < nx; ++ix)
      shifts[iy * nx + ix] = make_float2(static_cast<float>(-double(c.shift_range) + ix * double(c.shift_step)),
                                         static_cast<float>(-double(c.shift_range) + iy * double(c.shift_step)));

  // Taps for integer shift grids (the sample position c0 + o in FP32, as the
  // kernel would form it; an integer shift moves only the tap index).
  std::vector<float4> taps;
  int pad = -1;
  {
    bool integral = true;
    for (const float2 &sv : shifts) integral = integral && sv.x == std::floor(sv.x) && sv.y == std::floor(sv.y);
    int smax = 0;
    for (const float2 &sv : shifts)
      smax = std::max(smax, static_cast<int>(std::max(std::fabs(sv.x), std::fabs(sv.y))));
    if (integral) {
      const float c0 = 0.5f * static_cast<float>(c.L);
      int lo = 0, hi = 0;
      std::vector<int2> base(NS);
      std::vector<float2> frac(NS);
      for (int q = 0; q < NS; ++q) {
        const float x = c0 + offs[q].x, y = c0 + offs[q].y;
        const float xf = std::floor(x), yf = std::floor(y);
        base[q] = make_int2(static_cast<int>(xf), static_cast<int>(yf));
        frac[q] = make_float2(x - xf, y - yf);
        lo = std::min(lo, std::min(base[q].x, base[q].y) - smax);
        hi = std::max(hi, std::max(base[q].x, base[q].y) + 1 + smax - (c.L - 1));
      }
      const int need = std::max(-lo, hi);
      if (need <= 8) {
        pad = need <= 4 ? 4 : 8;  // a multiple of 4 keeps the interior float4-aligned
        const int Lp = c.L + 2 * pad;
        taps.resize(NS);
        for (int q = 0; q < NS; ++q) {
          const int idx = (base[q].y + pad) * Lp + (base[q].x + pad);
          float fidx;
          std::memcpy(&fidx, &idx, 4);
          taps[q] = make_float4(fidx, frac[q].x, frac[q].y, 0.f);
        }
      }
    }
  }

  mra::Geometry &g = h->g;
  g.L = c.L;
  g.M = M;
  g.NR = NR;
  g.NS = NS;
  g.NBIN = NBIN;
  g.NB = NB;
  g.S = nx * nx;
  g.mirror = c.mirror;
  h->NBIN = NBIN;
  h->NB = NB;
  int rc;
  if ((rc = upload(h, offs, &g.offs, "ring offsets"))) return rc;
  g.taps = nullptr;
  g.pad = 0;
  if (pad >= 0) {
    if ((rc = upload(h, taps, &g.taps, "bilinear taps"))) return rc;
    g.pad = pad;
  }
  if ((rc = upload(h, rings, &g.rings, "ring table"))) return rc;
  if ((rc = upload(h, binpos, &g.binpos, "bin positions"))) return rc;
  if ((rc = upload(h, bweight, &g.bweight, "ring weights"))) return rc;
  if ((rc = upload(h, fwd, &g.fwd_tw, "forward twiddles"))) return rc;
  if ((rc = upload(h, inv, &g.inv_tw, "inverse twiddles"))) return rc;
  if ((rc = upload(h, shifts, &g.shifts, "shift grid"))) return rc;
  if ((rc = upload(h, ang, &g.angles, "angle table"))) return rc;
  if ((rc = upload(h, fseg, &g.fseg, "frequency segments"))) return rc;
  g.KS = static_cast<int>(ksinfo.size());
  if ((rc = upload(h, kso, &g.kso, "k-step offsets"))) return rc;
  if ((rc = upload(h, ksinfo, &g.ksinfo, "k-step table"))) return rc;
  if ((rc = upload(h, binpos16, &g.binpos16, "16-bit bin positions"))) return rc;
  {
    // per-frequency bases: position of (ring i, f) = base[f] + i in both layouts
    std::vector<int> kpos(H + 1), kpos16(H + 1);
    for (int f = 0; f <= H; ++f) {
      kpos[f] = fseg[f].x - first[f];
      kpos16[f] = kso[f] * 16 - first[f];
    }
    if ((rc = upload(h, kpos, &g.kpos, "frequency bases"))) return rc;
    if ((rc = upload(h, kpos16, &g.kpos16, "16-bit frequency bases"))) return rc;
  }
  {
    // whole frequencies per staging chunk of the M = 256 / M = 512 kernels, greedily
    const int cap = g.M == 512 ? mra::kTc512ChunkKs : mra::kTc256ChunkKs;
    std::vector<int> chunk_f(1, 0);
    for (int f = 0; f <= H; ++f) {
      const int start = kso[chunk_f.back()];
      if (f > chunk_f.back() && kso[f + 1] - start > cap) chunk_f.push_back(f);
      if (g.M == 512 && kso[f + 1] - kso[f] > mra::kTc512MaxKsPerF)
        return set_err(h, MRA_EINVAL, "more than %d k-steps at frequency %d", mra::kTc512MaxKsPerF, f);
    }
    chunk_f.push_back(H + 1);
    g.NCH = static_cast<int>(chunk_f.size()) - 1;
    if ((rc = upload(h, chunk_f, &g.chunk_f, "staging chunks"))) return rc;
  }
  h->half = c.precision != MRA_FP32;
  h->fp16 = c.precision == MRA_FP16_RESCORE;
  // BF16 fragments of the 16-point DFT matrices for the tensor-core inverse DFT.
  // Stage 1 (A, rows (re/im, k), cols (re/im, a)): [[C, -S], [S, C]];
  // stage 2 (B, rows (re/im, t), cols (re/im, j)): [[C, S], [-S, C]];
  // C = cos(2 pi x y / 16), S = sin(2 pi x y / 16).  Lane 4g + t4 of a warp.
  {
    std::vector<uint32_t> frag(1024);
    auto h16 = [](double v) {  // BF16, round to nearest even (|v| <= 1)
      const float x = static_cast<float>(v);
      uint32_t u;
      std::memcpy(&u, &x, 4);
      return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
    };
    auto F = [](int blk_r, int blk_c, int x, int y, bool stage2) {
      const double th = kTwoPi * x * y / 16.0;
      const double C = std::cos(th), Sn = std::sin(th);
      if (blk_r == blk_c) return C;
      if (!stage2) return blk_r == 0 ? -Sn : Sn;   // stage 1: [[C,-S],[S,C]] (row block, col block)
      return blk_r == 0 ? Sn : -Sn;                 // stage 2: [[C,S],[-S,C]] (K block, N block)
    };
    for (int lane = 0; lane < 32; ++lane) {
      const int gg = lane >> 2, t4 = lane & 3;
      // stage-1 A fragments: index (mb * 2 + ks) * 4 + reg
      for (int mb = 0; mb < 2; ++mb)
        for (int ks = 0; ks < 2; ++ks) {
          const int rows[4] = {gg, gg + 8, gg, gg + 8};
          const int cols[4] = {2 * t4, 2 * t4, 2 * t4 + 8, 2 * t4 + 8};
          for (int r = 0; r < 4; ++r) {
            const double lo = F(mb, ks, rows[r], cols[r], false), hi = F(mb, ks, rows[r], cols[r] + 1, false);
            frag[lane * 16 + (mb * 2 + ks) * 4 + r] = h16(lo) | (h16(hi) << 16);
          }
        }
      // stage-2 B fragments: index (ks * 4 + nb) * 2 + reg; column j = 8 (nb % 2) + gg, out block nb / 2
      for (int ks = 0; ks < 2; ++ks)
        for (int nb = 0; nb < 4; ++nb) {
          const int j = 8 * (nb % 2) + gg, ob = nb / 2;
          for (int r = 0; r < 2; ++r) {
            const int t0 = 2 * t4 + 8 * r;
            const double lo = F(ks, ob, t0, j, true), hi = F(ks, ob, t0 + 1, j, true);
            frag[512 + lane * 16 + (ks * 4 + nb) * 2 + r] = h16(lo) | (h16(hi) << 16);
          }
        }
    }
    if ((rc = upload(h, frag, &g.dft16, "DFT fragments"))) return rc;
  }
  // tcgen05 path (M = 256): frequencies four to an MMA.  Greedy in f order:
  // a group takes the next frequencies while it has fewer than four; its
  // k-step count is that of its first (lowest) frequency, the largest, as
  // R_f does not grow with f; the others are padded with zero k-steps.
  h->umma = h->half && M == 256 && c.kernel == MRA_KERNEL_TCGEN05;
  if (M == 256) {
    std::vector<int> gfreq, uinfo, umap(kso[H + 1], -1);
    int NG = 0, NU = 0;
    for (int f = 0; f <= H;) {
      const int nks = kso[f + 1] - kso[f];
      int members[4] = {-1, -1, -1, -1};
      for (int sl = 0; sl < 4 && f <= H; ++sl, ++f) {
        members[sl] = f;
        for (int j = 0; j < kso[f + 1] - kso[f]; ++j) umap[kso[f] + j] = (NU + j) * 4 + sl;
      }
      for (int sl = 0; sl < 4; ++sl) gfreq.push_back(members[sl]);
      for (int j = 0; j < nks; ++j) uinfo.push_back(NG | (j << 8) | ((j == nks - 1 ? 1 : 0) << 10));
      NU += nks;
      ++NG;
    }
    if (NU > mra::kUmmaMaxU || NG > mra::kUmmaMaxG)
      return set_err(h, MRA_EINVAL, "%d MMA k-steps in %d groups exceed the tcgen05 tables", NU, NG);
    h->g.NU = NU;
    h->g.NG = NG;
    if ((rc = upload(h, umap, &h->g.umap, "k-step map"))) return rc;
    if ((rc = upload(h, uinfo, &h->g.uinfo, "k-step groups"))) return rc;
    if ((rc = upload(h, gfreq, &h->g.gfreq, "group frequencies"))) return rc;
    // BF16 16-point DFT matrices in the canonical K-major layout (B operands,
    // 32 N-rows x 32 K): W1[(c', k)][(a, c)] and W2[(c'', j)][(t, c')] with
    // K = 2 a + c: [[cos, -sin], [sin, cos]] of 2 pi a k / 16 (resp. t j).
    auto bf16 = [](double v) {  // round to nearest even (|v| <= 1)
      const float x = static_cast<float>(v);
      uint32_t u;
      std::memcpy(&u, &x, 4);
      return static_cast<uint16_t>((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
    };
    std::vector<uint16_t> w16(2048, 0);
    for (int m = 0; m < 2; ++m)
      for (int n = 0; n < 32; ++n)
        for (int K = 0; K < 32; ++K) {
          const int co = n >> 4, x = n & 15, ci = K & 1, y = K >> 1;
          const double th = kTwoPi * x * y / 16.0;
          const double v = co == ci ? std::cos(th) : (co == 0 ? -std::sin(th) : std::sin(th));
          w16[m * 1024 + ((n >> 3) * 512 + (K >> 3) * 128 + (n & 7) * 16 + (K & 7) * 2) / 2] = bf16(v);
        }
    std::vector<uint32_t> wpk(1024);
    for (int i = 0; i < 1024; ++i) wpk[i] = w16[2 * i] | (static_cast<uint32_t>(w16[2 * i + 1]) << 16);
    if ((rc = upload(h, wpk, &h->g.idft_w, "inverse-DFT matrices"))) return rc;
    std::vector<float2> tw(256);
    for (int t = 0; t < 16; ++t)
      for (int k = 0; k < 16; ++k) {
        const double th = kTwoPi * t * k / 256.0;
        tw[t * 16 + k] = make_float2(static_cast<float>(std::cos(th)), static_cast<float>(std::sin(th)));
      }
    if ((rc = upload(h, tw, &h->g.idft_tw, "inverse-DFT twiddles"))) return rc;
  }
  if ((rc = dev_alloc(h, &h->d_err, sizeof(int), "failure flags"))) return rc;
  h->tables.push_back(h->d_err);
  cudaError_t e = cudaMemset(h->d_err, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_err(h, e, "cudaMemset(failure flags)");
  return MRA_OK;
}

// TMA descriptor of a buffer of k-step tiles seen as a 2-D tensor of 16-bit
// elements with rows of 256 bytes (128 elements); one load box is box_rows
// rows, the kUmmaUPerStage consecutive k-step tiles of one pipeline stage
// (4 KB particle tiles: 16 rows each; 2 KB reference tiles: 8).  Rows past
// the end read as zero.
// cuTensorMapEncodeTiled comes from the driver through the runtime's entry
// point query, so the library needs no link to libcuda.
using TensorMapEncode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                     const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TensorMapEncode tensor_map_encoder() {
  static TensorMapEncode encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    encode = reinterpret_cast<TensorMapEncode>(fn);
  }
  return encode;
}

int make_tile_map(mra_handle *h, CUtensorMap *tm, void *base, uint64_t rows, uint32_t box_rows, const char *what) {
  const TensorMapEncode encode = tensor_map_encoder();
  if (!encode) return set_err(h, MRA_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {128, rows};
  const cuuint64_t strides[1] = {256};
  const cuuint32_t box[2] = {128, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_err(h, MRA_ECUDA, "cuTensorMapEncodeTiled(%s) failed with %d", what, int(r));
  return MRA_OK;
}

// Particle-spectrum workspace for one chunk of images (FP32 tiled spectra,
// or 16-bit fragments plus row maxima and candidates for the split path).
int ensure_chunk_workspace(mra_handle *h) {
  const int64_t S = h->g.S;
  if (!h->best) {
    size_t per_img = h->half ? static_cast<size_t>(S) * h->g.KS * 64 + static_cast<size_t>(h->K) * S * 8
                             : static_cast<size_t>(S) * h->NB * sizeof(float2);
    if (h->umma) per_img = static_cast<size_t>(S) * h->g.NU * 256 + static_cast<size_t>(h->K) * S * 8;
    int chunk = h->cfg.chunk_images;
    if (chunk <= 0) {
      const size_t budget = size_t(2) << 30;
      chunk = static_cast<int>(budget / per_img);
      if (chunk < 1) chunk = 1;
    }
    // images of one chunk index the polar kernel's grid.y, its row tiles the
    // contraction kernels' grid.y (both <= 65535)
    if (chunk > 65535) chunk = 65535;
    const int64_t max_chunk = (int64_t(65535) * mra::kTile) / S;
    if (chunk > max_chunk) chunk = static_cast<int>(max_chunk < 1 ? 1 : max_chunk);
    if (h->cfg.chunk_images <= 0 && h->half) {
      // the default chunk in whole waves of the FP32 rescore (one CTA per
      // image) when that costs at most a tenth of it: a chunk that ends with
      // a nearly empty wave leaves most SMs idle for one rescore CTA's time
      // (the polar kernel's waves, four CTAs per image at two per SM, divide
      // the same count at L = 76)
      int dev = 0, sms = 0;
      const int occ = mra::rescore_ctas_per_sm(h->g);
      if (occ > 0 && cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
        const int wave = occ * sms;
        const int whole = chunk / wave * wave;
        if (whole > 0 && 10 * static_cast<int64_t>(whole) >= 9 * static_cast<int64_t>(chunk)) chunk = whole;
      } else {
        cudaGetLastError();
      }
    }
    h->chunk = chunk;
    const int64_t tiles = (int64_t(chunk) * S + mra::kTile - 1) / mra::kTile;
    int rc;
    if (h->umma) {
      // k-step tiles of 16 rows; slots and k-steps no frequency fills are
      // never written and must read as zero
      const int64_t utiles = (int64_t(chunk) * S + mra::kUmmaRows - 1) / mra::kUmmaRows;
      h->A16_bytes = static_cast<size_t>(utiles) * h->g.NU * 4096;
      if ((rc = dev_alloc(h, &h->A16, h->A16_bytes, "particle k-step tiles"))) return rc;
      cudaError_t e = cudaMemset(h->A16, 0, h->A16_bytes);
      if (e != cudaSuccess) return cuda_err(h, e, "cudaMemset(particle k-step tiles)");
      if ((rc = make_tile_map(h, &h->tmA, h->A16, static_cast<uint64_t>(utiles) * h->g.NU * 16, 16 * mra::kUmmaUPerStage,
                              "particle k-step tiles")))
        return rc;
      if ((rc = dev_alloc(h, &h->cand, sizeof(int) * mra::kTopRows * chunk, "candidate rows"))) return rc;
    } else if (h->half) {
      h->A16_bytes = static_cast<size_t>(tiles) * h->g.KS * 512;
      if ((rc = dev_alloc(h, &h->A16, h->A16_bytes, "particle fragments"))) return rc;
      if ((rc = dev_alloc(h, &h->cand, sizeof(int) * mra::kTopRows * chunk, "candidate rows"))) return rc;
    } else {
      h->A_bytes = static_cast<size_t>(tiles) * h->NB * mra::kTile * sizeof(float2);
      if ((rc = dev_alloc(h, &h->A, h->A_bytes, "particle spectra"))) return rc;
      // padding bins of the layout are never written and must read as zero
      cudaError_t e = cudaMemset(h->A, 0, h->A_bytes);
      if (e != cudaSuccess) return cuda_err(h, e, "cudaMemset(particle spectra)");
    }
    if ((rc = dev_alloc(h, &h->best, sizeof(unsigned long long) * chunk, "argmax keys"))) return rc;
  }
  if (h->half) {
    const int64_t need = int64_t(h->chunk) * h->K * S * 2;
    if (need > h->rowmax_cap) {
      dev_free(h, h->rowmax, sizeof(float) * h->rowmax_cap);
      h->rowmax = nullptr;
      h->rowmax_cap = 0;
      if (int rc = dev_alloc(h, &h->rowmax, sizeof(float) * need, "row maxima")) return rc;
      h->rowmax_cap = need;
    }
  }
  return MRA_OK;
}

int ensure_avg_workspace(mra_handle *h, int64_t n) {
  if (h->avg_n_cap >= n && h->avg_K_cap >= h->K) return MRA_OK;
  mra::AvgWork &w = h->avg;
  const int64_t LL = int64_t(h->cfg.L) * h->cfg.L;
  // free the old buffers
  const int64_t old_nblk = (h->avg_n_cap + mra::kAvgBlock - 1) / mra::kAvgBlock;
  dev_free(h, w.hist, sizeof(int) * h->avg_K_cap * old_nblk);
  dev_free(h, w.scan, sizeof(int) * h->avg_K_cap * old_nblk);
  dev_free(h, w.perm, sizeof(int) * h->avg_n_cap);
  dev_free(h, w.chunk_class, sizeof(int) * w.max_chunks);
  dev_free(h, w.chunk_begin, sizeof(int) * w.max_chunks);
  dev_free(h, w.chunk_count, sizeof(int) * w.max_chunks);
  dev_free(h, w.n_chunks, sizeof(int));
  dev_free(h, w.class_counts, sizeof(int) * h->avg_K_cap);
  dev_free(h, w.class_first_chunk, sizeof(int) * (h->avg_K_cap + 1));
  dev_free(h, w.part_sum, sizeof(float) * w.max_chunks * LL);
  dev_free(h, w.part_comp, sizeof(float) * w.max_chunks * LL);
  dev_free(h, h->avg_sum, sizeof(float) * h->avg_K_cap * LL);
  dev_free(h, h->avg_comp, sizeof(float) * h->avg_K_cap * LL);
  dev_free(h, h->avg_cnt, sizeof(int) * h->avg_K_cap);
  w = mra::AvgWork{};
  h->avg_sum = h->avg_comp = nullptr;
  h->avg_cnt = nullptr;
  h->avg_n_cap = 0;
  h->avg_K_cap = 0;
  const int64_t ncap = n < 1024 ? 1024 : n;
  const int K = h->K;
  const int64_t nblk = (ncap + mra::kAvgBlock - 1) / mra::kAvgBlock;
  const int64_t maxc = ncap / mra::kAvgChunk + K + 1;
  w.max_chunks = static_cast<int>(maxc);
  int rc;
  if ((rc = dev_alloc(h, &w.hist, sizeof(int) * K * nblk, "class histogram"))) return rc;
  if ((rc = dev_alloc(h, &w.scan, sizeof(int) * K * nblk, "class scan"))) return rc;
  if ((rc = dev_alloc(h, &w.perm, sizeof(int) * ncap, "class order"))) return rc;
  if ((rc = dev_alloc(h, &w.chunk_class, sizeof(int) * maxc, "chunk classes"))) return rc;
  if ((rc = dev_alloc(h, &w.chunk_begin, sizeof(int) * maxc, "chunk starts"))) return rc;
  if ((rc = dev_alloc(h, &w.chunk_count, sizeof(int) * maxc, "chunk sizes"))) return rc;
  if ((rc = dev_alloc(h, &w.n_chunks, sizeof(int), "chunk count"))) return rc;
  if ((rc = dev_alloc(h, &w.class_counts, sizeof(int) * K, "class counts"))) return rc;
  if ((rc = dev_alloc(h, &w.class_first_chunk, sizeof(int) * (K + 1), "class chunk index"))) return rc;
  if ((rc = dev_alloc(h, &w.part_sum, sizeof(float) * maxc * LL, "chunk partial sums"))) return rc;
  if ((rc = dev_alloc(h, &w.part_comp, sizeof(float) * maxc * LL, "chunk partial corrections"))) return rc;
  if ((rc = dev_alloc(h, &h->avg_sum, sizeof(float) * K * LL, "class sums"))) return rc;
  if ((rc = dev_alloc(h, &h->avg_comp, sizeof(float) * K * LL, "class corrections"))) return rc;
  if ((rc = dev_alloc(h, &h->avg_cnt, sizeof(int) * K, "class counts out"))) return rc;
  h->avg_n_cap = ncap;
  h->avg_K_cap = K;
  return MRA_OK;
}

void free_all(mra_handle *h) {
  for (void *p : h->tables) cudaFree(p);
  h->tables.clear();
  auto fr = [](void *p) {
    if (p) cudaFree(p);
  };
  fr(h->B);
  fr(h->A);
  fr(h->best);
  fr(h->B16);
  fr(h->A16);
  fr(h->B16u);
  fr(h->rowmax);
  fr(h->cand);
  mra::AvgWork &w = h->avg;
  fr(w.hist);
  fr(w.scan);
  fr(w.perm);
  fr(w.chunk_class);
  fr(w.chunk_begin);
  fr(w.chunk_count);
  fr(w.n_chunks);
  fr(w.class_counts);
  fr(w.class_first_chunk);
  fr(w.part_sum);
  fr(w.part_comp);
  fr(h->avg_sum);
  fr(h->avg_comp);
  fr(h->avg_cnt);
  fr(h->h_stage_imgs);
  fr(h->h_stage_refs);
  fr(h->h_stage_avg);
  fr(h->h_stage_poses);
  fr(h->h_stage_counts);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (auto &r : h->prof_recs) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  for (auto e : h->prof_pool) cudaEventDestroy(e);
}

// Polls of an mbarrier before a kernel gives up waiting for its own bulk
// copies (each poll sleeps until the copies land or at most 0.5 ms; ~1 s in
// total).
constexpr uint32_t kWaitLimit = 2000;

// Tests of the time-out path shorten each warp's first wait with
// MRA_DEBUG_FIRST_WAIT_LIMIT (e.g. 0: give up at once, then drain normally).
uint32_t first_wait_limit() {
  const char *v = std::getenv("MRA_DEBUG_FIRST_WAIT_LIMIT");
  if (!v || !*v) return kWaitLimit;
  return static_cast<uint32_t>(std::strtoul(v, nullptr, 10));
}

int run_polar(mra_handle *h, const float *imgs, int64_t n, int rows_per_img, bool use_shifts, bool weighted,
              float2 *out, float *dbg_samples, float2 *dbg_spec, cudaStream_t st, uint4 *out16 = nullptr) {
  const int rec = prof_begin(h, weighted ? MRA_STAGE_REFS : MRA_STAGE_POLAR, st);
  mra::PolarArgs a{};
  a.imgs = imgs;
  a.n_imgs = n;
  a.rows_per_img = rows_per_img;
  a.use_shifts = use_shifts;
  a.weighted = weighted;
  a.out = out;
  a.dbg_samples = dbg_samples;
  a.dbg_spec = dbg_spec;
  a.out16 = out16;
  a.fp16 = h->fp16;
  a.umma = h->umma && out16 != nullptr;
  a.err = h->d_err;
  a.wait_limit = kWaitLimit;
  // image staging by a TMA tensor copy: a 3-D map over this call's stack
  // (rows of L * 4 bytes must be a multiple of 16, the base 16-byte
  // aligned, the bordered box at most 256 wide); else plain loads
  {
    const int L = h->g.L, pad = h->g.taps ? h->g.pad : 0, Lp = L + 2 * pad;
    const TensorMapEncode encode = (L % 4 == 0 && Lp <= 256 && (reinterpret_cast<uintptr_t>(imgs) & 15) == 0)
                                       ? tensor_map_encoder() : nullptr;
    if (encode) {
      const cuuint64_t dims[3] = {static_cast<cuuint64_t>(L), static_cast<cuuint64_t>(L), static_cast<cuuint64_t>(n)};
      const cuuint64_t strides[2] = {static_cast<cuuint64_t>(L) * 4, static_cast<cuuint64_t>(L) * L * 4};
      const cuuint32_t box[3] = {static_cast<cuuint32_t>(Lp), static_cast<cuuint32_t>(Lp), 1};
      const cuuint32_t estr[3] = {1, 1, 1};
      a.tma = encode(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(imgs), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
  }
  const int rc = check_launch(h, mra::launch_polar(h->g, a, st), "polar/ring-FFT kernel");
  prof_end(h, rec, 1, st);
  return rc;
}

// Precision-split chunk: 16-bit fragments, tensor-core contraction with row
// maxima, top-8 rows per image, FP32 rescore into the argmax keys.
int align_chunk_half(mra_handle *h, const float *imgs, int64_t cnt, mra_pose_t *poses, float *dbg_cc,
                     cudaStream_t st) {
  int rc = run_polar(h, imgs, cnt, h->g.S, true, false, nullptr, nullptr, nullptr, st, h->A16);
  if (rc) return rc;
  mra::TcArgs t{};
  t.A16 = h->A16;
  t.B16 = h->B16;
  t.rows = cnt * h->g.S;
  t.K = h->K;
  t.rowmax = h->rowmax;
  t.dbg_cc = dbg_cc;
  t.ks_max = h->ks_max;
  t.err = h->d_err;
  t.wait_limit = kWaitLimit;
  t.first_wait_limit = first_wait_limit();
  int rec = prof_begin(h, MRA_STAGE_CC, st);
  if (h->umma) {
    t.B16 = static_cast<const uint2 *>(h->B16u);
    rc = check_launch(h, mra::launch_cc_umma256(&h->tmA, &h->tmB, h->g, t, h->fp16, st),
                      "tcgen05 contraction/IFFT kernel");
  } else {
    rc = check_launch(h, mra::launch_cc_tc(h->g, t, h->fp16, st), "tensor-core contraction/IFFT kernel");
  }
  prof_end(h, rec, 1, st);
  if (rc) return rc;
  rec = prof_begin(h, MRA_STAGE_RESCORE, st);
  rc = check_launch(h, mra::launch_top8(h->rowmax, cnt, h->K * h->g.S * 2, h->cand, st), "top-8 kernel");
  if (!rc) {
    mra::RescoreArgs r{};
    r.imgs = imgs;
    r.n = cnt;
    r.cand = h->cand;
    r.B = h->B;
    r.best = h->best;
    rc = check_launch(h, mra::launch_rescore(h->g, r, st), "FP32 rescore kernel");
  }
  prof_end(h, rec, 2, st);
  if (rc) return rc;
  if (poses) {
    rec = prof_begin(h, MRA_STAGE_DECODE, st);
    rc = check_launch(h, mra::launch_decode(h->g, h->best, cnt, h->K, poses, st), "pose decode kernel");
    prof_end(h, rec, 1, st);
  }
  return rc;
}

// Align images [c0, c0 + cnt) of the stack (one chunk); optional full CC table.
int align_chunk(mra_handle *h, const float *imgs, int64_t cnt, mra_pose_t *poses, float *dbg_cc, cudaStream_t st) {
  if (h->half) return align_chunk_half(h, imgs, cnt, poses, dbg_cc, st);
  int rc = run_polar(h, imgs, cnt, h->g.S, true, false, h->A, nullptr, nullptr, st);
  if (rc) return rc;
  cudaError_t e = cudaMemsetAsync(h->best, 0, sizeof(unsigned long long) * cnt, st);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaMemsetAsync(keys)");
  mra::CCArgs a{};
  a.A = h->A;
  a.B = h->B;
  a.rows = cnt * h->g.S;
  a.K = h->K;
  a.best = h->best;
  a.dbg_cc = dbg_cc;
  a.seg_max = h->seg_max;
  a.err = h->d_err;
  a.wait_limit = kWaitLimit;
  a.first_wait_limit = first_wait_limit();
  int rec = prof_begin(h, MRA_STAGE_CC, st);
  rc = check_launch(h, mra::launch_cc_fp32(h->g, a, st), "contraction/IFFT/argmax kernel");
  prof_end(h, rec, 1, st);
  if (rc) return rc;
  if (poses) {
    rec = prof_begin(h, MRA_STAGE_DECODE, st);
    rc = check_launch(h, mra::launch_decode(h->g, h->best, cnt, h->K, poses, st), "pose decode kernel");
    prof_end(h, rec, 1, st);
  }
  return rc;
}

int need_handle(mra_handle *h) { return h ? MRA_OK : set_err(nullptr, MRA_EINVAL, "handle is NULL"); }

int select_device(mra_handle *h) {
  cudaError_t e = cudaSetDevice(h->device);
  return e == cudaSuccess ? MRA_OK : cuda_err(h, e, "cudaSetDevice");
}

}  // namespace

extern "C" {

int mra_create(const mra_config_t *cfg, mra_t *out) {
  g_create_error.clear();
  if (!out) return set_err(nullptr, MRA_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  if (int rc = validate(cfg, &why)) return set_err(nullptr, rc, "%s", why.c_str());
  auto *h = new mra_handle();
  h->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return set_err(nullptr, MRA_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  int rc = build_tables(h);
  if (rc) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return MRA_OK;
}

int mra_destroy(mra_t h) {
  if (!h) return MRA_OK;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return MRA_OK;
}

const char *mra_last_error(mra_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int mra_get_info(mra_t h, mra_info_t *info) {
  if (int rc = need_handle(h)) return rc;
  if (!info) return set_err(h, MRA_EINVAL, "info is NULL");
  info->M = h->g.M;
  info->n_rings = h->g.NR;
  info->n_samples = h->g.NS;
  info->n_bins = h->NBIN;
  info->n_bins_padded = h->NB;
  info->S = h->g.S;
  info->K = h->K;
  info->chunk_images = h->chunk;
  info->workspace_bytes = static_cast<int64_t>(h->workspace);
  return MRA_OK;
}

int mra_set_refs(mra_t h, const float *d_refs, int32_t K, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (K < 1) return set_err(h, MRA_EINVAL, "K must be >= 1 (got %d)", K);
  if (!d_refs) return set_err(h, MRA_EINVAL, "d_refs is NULL");
  const double flat_max = double(K) * h->g.S * 2.0 * h->g.M;
  if (flat_max >= 4294967295.0)
    return set_err(h, MRA_EINVAL, "K * S * 2 * M = %.0f exceeds the 32-bit candidate index", flat_max);
  if (int rc = select_device(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int Kpad = (K + mra::kTile - 1) / mra::kTile * mra::kTile;
  if (Kpad != h->Kpad) {
    dev_free(h, h->B, static_cast<size_t>(h->Kpad) * h->NB * sizeof(float2));
    h->B = nullptr;
    h->Kpad = 0;
    h->K = 0;
    if (int rc = dev_alloc(h, &h->B, static_cast<size_t>(Kpad) * h->NB * sizeof(float2), "reference spectra"))
      return rc;
    h->Kpad = Kpad;
  }
  cudaError_t e = cudaMemsetAsync(h->B, 0, static_cast<size_t>(Kpad) * h->NB * sizeof(float2), st);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaMemsetAsync(reference spectra)");
  if (int rc = run_polar(h, d_refs, K, 1, false, true, h->B, nullptr, nullptr, st)) return rc;
  if (h->umma) {
    const int ktiles = Kpad / mra::kUmmaRefs;
    if (!h->B16u || Kpad > h->B16u_refs) {
      dev_free(h, h->B16u, static_cast<size_t>(h->B16u_refs / mra::kUmmaRefs) * h->g.NU * 2048);
      h->B16u = nullptr;
      h->B16u_refs = 0;
      if (int rc = dev_alloc(h, &h->B16u, static_cast<size_t>(ktiles) * h->g.NU * 2048, "reference k-step tiles"))
        return rc;
      h->B16u_refs = Kpad;
      if (int rc = make_tile_map(h, &h->tmB, h->B16u, static_cast<uint64_t>(ktiles) * h->g.NU * 8, 8 * mra::kUmmaUPerStage,
                                 "reference k-step tiles"))
        return rc;
    }
    const int rec = prof_begin(h, MRA_STAGE_CONVERT, st);
    const int rc = check_launch(h, mra::launch_refs16u(h->g, h->B, ktiles, h->B16u, h->fp16, st),
                                "reference k-step tile kernel");
    prof_end(h, rec, 1, st);
    if (rc) return rc;
  } else if (h->half) {
    const size_t b16 = static_cast<size_t>(Kpad / mra::kTile) * 2 * h->g.KS * 32 * sizeof(uint2);
    if (!h->B16 || Kpad > h->B16_refs) {
      dev_free(h, h->B16, static_cast<size_t>(h->B16_refs / mra::kTile) * 2 * h->g.KS * 32 * sizeof(uint2));
      h->B16 = nullptr;
      h->B16_refs = 0;
      if (int rc = dev_alloc(h, &h->B16, b16, "reference fragments")) return rc;
      h->B16_refs = Kpad;
    }
    const int rec = prof_begin(h, MRA_STAGE_CONVERT, st);
    const int rc = check_launch(h, mra::launch_refs16(h->g, h->B, Kpad / mra::kTile, h->B16, h->fp16, st),
                                "reference fragment kernel");
    prof_end(h, rec, 1, st);
    if (rc) return rc;
  }
  h->K = K;
  return MRA_OK;
}

int mra_copy_refs(mra_t dst, mra_t src, mra_stream_t stream) {
  if (int rc = need_handle(dst)) return rc;
  if (!src) return set_err(dst, MRA_EINVAL, "source handle is NULL");
  if (src == dst) return MRA_OK;
  if (src->K == 0) return set_err(dst, MRA_ESTATE, "source handle holds no references");
  const mra_config_t &a = dst->cfg, &b = src->cfg;
  if (a.L != b.L || a.first_ring != b.first_ring || a.last_ring != b.last_ring || a.ring_step != b.ring_step ||
      a.shift_range != b.shift_range || a.shift_step != b.shift_step || a.mirror != b.mirror ||
      a.precision != b.precision || dst->umma != src->umma)
    return set_err(dst, MRA_EINVAL,
                   "source and destination configurations differ (chunk_images may differ, the kernel may not)");
  if (src->device != dst->device) return set_err(dst, MRA_EINVAL, "source handle lives on another device");
  if (int rc = select_device(dst)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int Kpad = src->Kpad;
  if (Kpad != dst->Kpad) {
    dev_free(dst, dst->B, static_cast<size_t>(dst->Kpad) * dst->NB * sizeof(float2));
    dst->B = nullptr;
    dst->Kpad = 0;
    dst->K = 0;
    if (int rc = dev_alloc(dst, &dst->B, static_cast<size_t>(Kpad) * dst->NB * sizeof(float2), "reference spectra"))
      return rc;
    dst->Kpad = Kpad;
  }
  dst->K = 0;
  cudaError_t e = cudaMemcpyAsync(dst->B, src->B, static_cast<size_t>(Kpad) * dst->NB * sizeof(float2),
                                  cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_err(dst, e, "cudaMemcpyAsync(reference spectra)");
  if (dst->umma) {
    const int ktiles = Kpad / mra::kUmmaRefs;
    if (!dst->B16u || Kpad > dst->B16u_refs) {
      dev_free(dst, dst->B16u, static_cast<size_t>(dst->B16u_refs / mra::kUmmaRefs) * dst->g.NU * 2048);
      dst->B16u = nullptr;
      dst->B16u_refs = 0;
      if (int rc = dev_alloc(dst, &dst->B16u, static_cast<size_t>(ktiles) * dst->g.NU * 2048, "reference k-step tiles"))
        return rc;
      dst->B16u_refs = Kpad;
      if (int rc = make_tile_map(dst, &dst->tmB, dst->B16u, static_cast<uint64_t>(ktiles) * dst->g.NU * 8, 8 * mra::kUmmaUPerStage,
                                 "reference k-step tiles"))
        return rc;
    }
    e = cudaMemcpyAsync(dst->B16u, src->B16u, static_cast<size_t>(ktiles) * dst->g.NU * 2048,
                        cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_err(dst, e, "cudaMemcpyAsync(reference k-step tiles)");
  } else if (dst->half) {
    const size_t b16 = static_cast<size_t>(Kpad / mra::kTile) * 2 * dst->g.KS * 32 * sizeof(uint2);
    if (!dst->B16 || Kpad > dst->B16_refs) {
      dev_free(dst, dst->B16, static_cast<size_t>(dst->B16_refs / mra::kTile) * 2 * dst->g.KS * 32 * sizeof(uint2));
      dst->B16 = nullptr;
      dst->B16_refs = 0;
      if (int rc = dev_alloc(dst, &dst->B16, b16, "reference fragments")) return rc;
      dst->B16_refs = Kpad;
    }
    e = cudaMemcpyAsync(dst->B16, src->B16, b16, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_err(dst, e, "cudaMemcpyAsync(reference fragments)");
  }
  dst->K = src->K;
  return MRA_OK;
}

int mra_align(mra_t h, const float *d_imgs, int64_t n, mra_pose_t *d_poses, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (n < 0) return set_err(h, MRA_EINVAL, "n must be >= 0");
  if (h->K == 0) return set_err(h, MRA_ESTATE, "mra_align before mra_set_refs");
  if (n == 0) return MRA_OK;
  if (!d_imgs || !d_poses) return set_err(h, MRA_EINVAL, "d_imgs / d_poses is NULL");
  if (fault("timeout")) return set_err(h, MRA_ETIMEOUT, "injected timeout");
  if (int rc = select_device(h)) return rc;
  if (int rc = ensure_chunk_workspace(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t LL = int64_t(h->cfg.L) * h->cfg.L;
  for (int64_t c0 = 0; c0 < n; c0 += h->chunk) {
    const int64_t cnt = (n - c0 < h->chunk) ? n - c0 : h->chunk;
    if (int rc = align_chunk(h, d_imgs + c0 * LL, cnt, d_poses + c0, nullptr, st)) return rc;
  }
  return MRA_OK;
}

int mra_class_sums(mra_t h, const float *d_imgs, const mra_pose_t *d_poses, int64_t n, float *d_sum, float *d_comp,
                   int32_t *d_counts, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (n < 0) return set_err(h, MRA_EINVAL, "n must be >= 0");
  if (h->K == 0) return set_err(h, MRA_ESTATE, "class sums need the reference count: call mra_set_refs first");
  if (n == 0) return MRA_OK;
  if (!d_imgs || !d_poses || !d_sum || !d_comp || !d_counts) return set_err(h, MRA_EINVAL, "NULL buffer");
  if (n > 2147483647LL) return set_err(h, MRA_EINVAL, "n too large for averaging (max 2^31-1)");
  if (int rc = select_device(h)) return rc;
  if (int rc = ensure_avg_workspace(h, n)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int rec = prof_begin(h, MRA_STAGE_AVERAGE, st);
  const int rc = check_launch(h, mra::launch_class_sums(h->g, d_imgs, d_poses, n, h->K, h->avg, d_sum, d_comp,
                                                        d_counts, true, st),
                              "class-sum kernels");
  prof_end(h, rec, mra::kClassSumLaunches, st);
  return rc;
}

int mra_average_finalize(mra_t h, const float *d_sum, const float *d_comp, const int32_t *d_counts, float *d_avg,
                         mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (h->K == 0) return set_err(h, MRA_ESTATE, "finalize needs the reference count: call mra_set_refs first");
  if (!d_sum || !d_comp || !d_counts || !d_avg) return set_err(h, MRA_EINVAL, "NULL buffer");
  if (int rc = select_device(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int rec = prof_begin(h, MRA_STAGE_AVERAGE, st);
  const int rc = check_launch(h, mra::launch_average_finalize(h->g, h->K, d_sum, d_comp, d_counts, d_avg, st),
                              "average finalize kernel");
  prof_end(h, rec, 1, st);
  return rc;
}

int mra_average(mra_t h, const float *d_imgs, const mra_pose_t *d_poses, int64_t n, float *d_avg, int32_t *d_counts,
                mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (n < 0) return set_err(h, MRA_EINVAL, "n must be >= 0");
  if (h->K == 0) return set_err(h, MRA_ESTATE, "mra_average before mra_set_refs");
  if (!d_avg || !d_counts) return set_err(h, MRA_EINVAL, "d_avg / d_counts is NULL");
  if (int rc = select_device(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(int) * h->K, st);
    return e == cudaSuccess ? MRA_OK : cuda_err(h, e, "cudaMemsetAsync(counts)");
  }
  if (!d_imgs || !d_poses) return set_err(h, MRA_EINVAL, "d_imgs / d_poses is NULL");
  if (n > 2147483647LL) return set_err(h, MRA_EINVAL, "n too large for averaging (max 2^31-1)");
  if (int rc = ensure_avg_workspace(h, n)) return rc;
  const int rec = prof_begin(h, MRA_STAGE_AVERAGE, st);
  int rc = check_launch(h, mra::launch_class_sums(h->g, d_imgs, d_poses, n, h->K, h->avg, h->avg_sum, h->avg_comp,
                                                  d_counts, false, st),
                        "class-sum kernels");
  if (!rc)
    rc = check_launch(h, mra::launch_average_finalize(h->g, h->K, h->avg_sum, h->avg_comp, d_counts, d_avg, st),
                      "average finalize kernel");
  prof_end(h, rec, mra::kClassSumLaunches + 1, st);
  return rc;
}

int mra_refresh_refs(mra_t h, float *d_refs, const int32_t *d_counts, int32_t K, const int32_t *d_reseed,
                     const float *d_imgs, int64_t n, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (K < 1 || !d_refs || !d_counts) return set_err(h, MRA_EINVAL, "need K >= 1, d_refs and d_counts");
  if (d_reseed && (!d_imgs || n < 1)) return set_err(h, MRA_EINVAL, "reseeding needs d_imgs and n >= 1");
  if (int rc = select_device(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int rec = prof_begin(h, MRA_STAGE_AVERAGE, st);
  const int rc = check_launch(h, mra::launch_refresh_refs(h->cfg.L, d_refs, d_counts, K, d_reseed, d_imgs, n, st),
                              "reference refresh kernel");
  prof_end(h, rec, 1, st);
  return rc;
}

int mra_run_host(mra_t h, const float *h_refs, int32_t K, const float *h_imgs, int64_t n, mra_pose_t *h_poses,
                 float *h_avg, int32_t *h_counts, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (K < 1 || n < 0) return set_err(h, MRA_EINVAL, "need K >= 1 and n >= 0");
  if (!h_refs || (n > 0 && (!h_imgs || !h_poses)) || !h_avg || !h_counts)
    return set_err(h, MRA_EINVAL, "NULL host buffer");
  if (int rc = select_device(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t LL = int64_t(h->cfg.L) * h->cfg.L;
  cudaError_t e;
  if (!h->copy_stream) {
    if ((e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_err(h, e, "cudaStreamCreate");
    for (auto &ev : h->ev)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_err(h, e, "cudaEventCreate");
  }
  if (n > h->h_stage_n) {
    dev_free(h, h->h_stage_imgs, sizeof(float) * h->h_stage_n * LL);
    dev_free(h, h->h_stage_poses, sizeof(mra_pose_t) * h->h_stage_n);
    h->h_stage_imgs = nullptr;
    h->h_stage_poses = nullptr;
    h->h_stage_n = 0;
    if (int rc = dev_alloc(h, &h->h_stage_imgs, sizeof(float) * n * LL, "device image stack")) return rc;
    if (int rc = dev_alloc(h, &h->h_stage_poses, sizeof(mra_pose_t) * n, "device poses")) return rc;
    h->h_stage_n = n;
  }
  if (K > h->h_stage_K) {
    dev_free(h, h->h_stage_refs, sizeof(float) * h->h_stage_K * LL);
    dev_free(h, h->h_stage_avg, sizeof(float) * h->h_stage_K * LL);
    dev_free(h, h->h_stage_counts, sizeof(int) * h->h_stage_K);
    h->h_stage_refs = h->h_stage_avg = nullptr;
    h->h_stage_counts = nullptr;
    h->h_stage_K = 0;
    if (int rc = dev_alloc(h, &h->h_stage_refs, sizeof(float) * K * LL, "device references")) return rc;
    if (int rc = dev_alloc(h, &h->h_stage_avg, sizeof(float) * K * LL, "device averages")) return rc;
    if (int rc = dev_alloc(h, &h->h_stage_counts, sizeof(int) * K, "device counts")) return rc;
    h->h_stage_K = K;
  }
  if ((e = cudaMemcpyAsync(h->h_stage_refs, h_refs, sizeof(float) * K * LL, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return cuda_err(h, e, "copy references in");
  if (int rc = mra_set_refs(h, h->h_stage_refs, K, stream)) return rc;
  // The averages of empty classes stay untouched: start them from the caller's values.
  if ((e = cudaMemcpyAsync(h->h_stage_avg, h_avg, sizeof(float) * K * LL, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return cuda_err(h, e, "copy averages in");
  if (n > 0) {
    if (int rc = ensure_chunk_workspace(h)) return rc;
    // copy chunk c on the copy stream while chunk c-1 is aligned on `st`
    if ((e = cudaEventRecord(h->ev[2], st)) != cudaSuccess) return cuda_err(h, e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(h->copy_stream, h->ev[2], 0)) != cudaSuccess)
      return cuda_err(h, e, "cudaStreamWaitEvent");
    int slot = 0;
    for (int64_t c0 = 0; c0 < n; c0 += h->chunk, slot ^= 1) {
      const int64_t cnt = (n - c0 < h->chunk) ? n - c0 : h->chunk;
      e = cudaMemcpyAsync(h->h_stage_imgs + c0 * LL, h_imgs + c0 * LL, sizeof(float) * cnt * LL,
                          cudaMemcpyHostToDevice, h->copy_stream);
      if (e != cudaSuccess) return cuda_err(h, e, "copy images in");
      if ((e = cudaEventRecord(h->ev[slot], h->copy_stream)) != cudaSuccess) return cuda_err(h, e, "cudaEventRecord");
      if ((e = cudaStreamWaitEvent(st, h->ev[slot], 0)) != cudaSuccess) return cuda_err(h, e, "cudaStreamWaitEvent");
      if (int rc = align_chunk(h, h->h_stage_imgs + c0 * LL, cnt, h->h_stage_poses + c0, nullptr, st)) return rc;
    }
    if (int rc = mra_average(h, h->h_stage_imgs, h->h_stage_poses, n, h->h_stage_avg, h->h_stage_counts, stream))
      return rc;
    if ((e = cudaMemcpyAsync(h_poses, h->h_stage_poses, sizeof(mra_pose_t) * n, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return cuda_err(h, e, "copy poses out");
  } else {
    if ((e = cudaMemsetAsync(h->h_stage_counts, 0, sizeof(int) * K, st)) != cudaSuccess)
      return cuda_err(h, e, "cudaMemsetAsync(counts)");
  }
  if ((e = cudaMemcpyAsync(h_avg, h->h_stage_avg, sizeof(float) * K * LL, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_err(h, e, "copy averages out");
  if ((e = cudaMemcpyAsync(h_counts, h->h_stage_counts, sizeof(int) * K, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_err(h, e, "copy counts out");
  return mra_sync(h, stream);
}

int mra_run_graph(mra_t h, const float *d_refs, int32_t K, const float *d_imgs, int64_t n, mra_pose_t *d_poses,
                  float *d_avg, int32_t *d_counts, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (K < 1 || n < 1) return set_err(h, MRA_EINVAL, "need K >= 1 and n >= 1");
  if (!d_refs || !d_imgs || !d_poses || !d_avg || !d_counts) return set_err(h, MRA_EINVAL, "NULL buffer");
  if (int rc = select_device(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const mra_handle::GraphKey key{d_refs, d_imgs, d_poses, d_avg, d_counts, n, K};
  auto eager = [&]() -> int {
    if (int rc = mra_set_refs(h, d_refs, K, stream)) return rc;
    if (int rc = mra_align(h, d_imgs, n, d_poses, stream)) return rc;
    return mra_average(h, d_imgs, d_poses, n, d_avg, d_counts, stream);
  };
  if (!(key == h->graph_key)) {  // new buffers or sizes: drop the old graph, run eagerly
    if (h->graph_exec) {
      cudaGraphExecDestroy(h->graph_exec);
      h->graph_exec = nullptr;
    }
    h->graph_key = key;
    h->graph_seen = 0;
  }
  // the first call with these buffers runs eagerly: it sizes and allocates every workspace and sets
  // every kernel attribute, none of which may happen inside a capture
  if (!h->graph_exec && h->graph_seen++ == 0) return eager();
  if (!h->graph_exec) {
    cudaError_t e;
    if (!h->capture_stream &&
        (e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_err(h, e, "cudaStreamCreate(capture)");
    if ((e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_err(h, e, "cudaStreamBeginCapture");
    h->capturing = true;
    const mra_stream_t cs = reinterpret_cast<mra_stream_t>(h->capture_stream);
    int rc = mra_set_refs(h, d_refs, K, cs);
    if (!rc) rc = mra_align(h, d_imgs, n, d_poses, cs);
    if (!rc) rc = mra_average(h, d_imgs, d_poses, n, d_avg, d_counts, cs);
    h->capturing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->capture_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc;
    }
    if (e != cudaSuccess) return cuda_err(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->graph_exec = nullptr;
      return cuda_err(h, e, "cudaGraphInstantiate");
    }
  }
  cudaError_t e = cudaGraphLaunch(h->graph_exec, st);
  return e == cudaSuccess ? MRA_OK : cuda_err(h, e, "cudaGraphLaunch");
}

int mra_graph_info(mra_t h, int32_t *captured) {
  if (int rc = need_handle(h)) return rc;
  if (!captured) return set_err(h, MRA_EINVAL, "captured is NULL");
  *captured = h->graph_exec ? 1 : 0;
  return MRA_OK;
}

int mra_sync(mra_t h, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (int rc = select_device(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaStreamSynchronize");
  int flags = 0;
  if ((e = cudaMemcpy(&flags, h->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_err(h, e, "read failure flags");
  if (flags) {
    if ((e = cudaMemset(h->d_err, 0, sizeof(int))) != cudaSuccess) return cuda_err(h, e, "clear failure flags");
    return set_err(h, MRA_ETIMEOUT, "a kernel gave up waiting for its bulk copies; the last results are invalid");
  }
  return MRA_OK;
}

int mra_profile(mra_t h, int enable) {
  if (int rc = need_handle(h)) return rc;
  prof_collect(h);
  for (int i = 0; i < MRA_STAGE_COUNT; ++i) {
    h->prof_ms[i] = 0.0;
    h->prof_launches[i] = 0;
  }
  h->prof_on = enable != 0;
  return MRA_OK;
}

int mra_profile_read(mra_t h, mra_stage_time_t *out) {
  if (int rc = need_handle(h)) return rc;
  if (!out) return set_err(h, MRA_EINVAL, "out is NULL");
  prof_collect(h);
  for (int i = 0; i < MRA_STAGE_COUNT; ++i) {
    out[i].launches = h->prof_launches[i];
    out[i].ms = h->prof_ms[i];
  }
  return MRA_OK;
}

int mra_debug_polar(mra_t h, const float *d_imgs, int64_t n, float *d_out, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (n < 0 || (n > 0 && (!d_imgs || !d_out))) return set_err(h, MRA_EINVAL, "bad arguments");
  if (n == 0) return MRA_OK;
  if (int rc = select_device(h)) return rc;
  return run_polar(h, d_imgs, n, h->g.S, true, false, nullptr, d_out, nullptr,
                   reinterpret_cast<cudaStream_t>(stream));
}

int mra_debug_spectra(mra_t h, const float *d_imgs, int64_t n, float *d_out, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (n < 0 || (n > 0 && (!d_imgs || !d_out))) return set_err(h, MRA_EINVAL, "bad arguments");
  if (n == 0) return MRA_OK;
  if (int rc = select_device(h)) return rc;
  return run_polar(h, d_imgs, n, h->g.S, true, false, nullptr, nullptr, reinterpret_cast<float2 *>(d_out),
                   reinterpret_cast<cudaStream_t>(stream));
}

int mra_debug_cc(mra_t h, const float *d_imgs, int64_t n, float *d_out, mra_stream_t stream) {
  if (int rc = need_handle(h)) return rc;
  if (h->K == 0) return set_err(h, MRA_ESTATE, "mra_debug_cc before mra_set_refs");
  if (n < 0 || (n > 0 && (!d_imgs || !d_out))) return set_err(h, MRA_EINVAL, "bad arguments");
  if (n == 0) return MRA_OK;
  if (int rc = select_device(h)) return rc;
  if (int rc = ensure_chunk_workspace(h)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t LL = int64_t(h->cfg.L) * h->cfg.L;
  const int64_t per_img = int64_t(h->K) * h->g.S * 2 * h->g.M;
  for (int64_t c0 = 0; c0 < n; c0 += h->chunk) {
    const int64_t cnt = (n - c0 < h->chunk) ? n - c0 : h->chunk;
    if (int rc = align_chunk(h, d_imgs + c0 * LL, cnt, nullptr, d_out + c0 * per_img, st)) return rc;
  }
  return MRA_OK;
}

}  // extern "C"
