// mra_align_static: the FP32 alignment of mra_align for callers that must
// not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted: inside a framework that owns every device allocation through its
// own pool, in a real-time loop where an allocation could stall or fail, or
// in a process that has handed all free device memory to someone else.  Such
// a caller cannot create an mra_t handle (mra_create allocates its geometry
// tables and workspaces), so this entry point takes the configuration
// directly and keeps every intermediate (geometry tables, reference
// spectra, particle spectra of one chunk, argmax keys) in a single
// fixed-size file-scope device array (MRA_STATIC_SCRATCH_BYTES).  Under
// CUDA's lazy module loading the array is committed on a device by the first
// call there (its cudaGetSymbolAddress) and then held until the process
// exits.
//
// The array is shared by every call in the process: the last call's data
// stays in it and whatever must start at zero is cleared by each call.  Two
// calls whose GPU work overlapped would corrupt each other, so a call holds
// a process-wide lock from its first enqueue until its GPU work has finished
// (error returns after an enqueue synchronise the stream first).  The
// kernels are the ones mra_align uses.
#include "../../include/mra.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mra_internal.h"

namespace {

constexpr size_t kScratchBytes = MRA_STATIC_SCRATCH_BYTES;

// The reserved device array.  In host code this name is only a stand-in:
// kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_mu;  // guards the address cache and the host table staging below

// Host staging of the geometry tables (no heap use); bounds follow from
// M <= 512 and the 4096-shift limit of the configuration.
constexpr int kMaxRings = 1024;
constexpr int kMaxSamples = 65536;
constexpr int kMaxBins = 65536;
constexpr int kMaxM = 512;
constexpr int kMaxShifts = 4096;
float2 h_offs[kMaxSamples];
int4 h_rings[kMaxRings];
int h_binpos[kMaxBins];
float h_bweight[kMaxBins];
float2 h_fwd[kMaxM], h_inv[kMaxM], h_ang[kMaxM];
float2 h_shifts[kMaxShifts];
int2 h_fseg[kMaxM / 2 + 1];
int h_kpos[kMaxM / 2 + 1];

// Error text goes to the caller's buffer (msg, msg_len), if one was given.
thread_local char *g_msg = nullptr;
thread_local int32_t g_msg_len = 0;

int fail(int code, const char *fmt, ...) {
  if (g_msg && g_msg_len > 0) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_msg, static_cast<size_t>(g_msg_len), fmt, ap);
    va_end(ap);
  }
  return code;
}

// The same after work has been enqueued on `st`: wait for that work first,
// so that the next call (which may take the lock as soon as this one drops
// it) cannot overwrite the array while this call's copies or kernels still
// use it.
int fail_sync(cudaStream_t st, int code, const char *fmt, ...) {
  cudaStreamSynchronize(st);
  cudaGetLastError();
  if (g_msg && g_msg_len > 0) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_msg, static_cast<size_t>(g_msg_len), fmt, ap);
    va_end(ap);
  }
  return code;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

constexpr double kTwoPi = 6.283185307179586476925286766559;

}  // namespace

extern "C" {

int mra_align_static(const mra_config_t *cfg, const float *d_refs, int32_t K, const float *d_imgs, int64_t n,
                     mra_pose_t *d_poses, mra_stream_t stream, char *msg, int32_t msg_len) {
  g_msg = msg;
  g_msg_len = msg_len;
  if (msg && msg_len > 0) msg[0] = '\0';
  // The checks of mra_create (shift grid in double with finiteness, ring
  // range, shared memory per CTA), before any table is built or CUDA call made.
  {
    char why[320];
    why[0] = '\0';
    if (int rc = mra::check_config(cfg, why, sizeof(why))) return fail(rc, "%s", why);
  }
  const mra_config_t &c = *cfg;
  const double qd = 2.0 * double(c.shift_range) / double(c.shift_step);
  const int nx = static_cast<int>(std::lround(qd)) + 1;  // check_config bounded nx * nx by 4096
  const int S = nx * nx;
  if (c.precision != MRA_FP32) return fail(MRA_EUNSUPPORTED, "mra_align_static runs the FP32 path only");
  if (K < 1) return fail(MRA_EINVAL, "K must be >= 1");
  if (n < 0) return fail(MRA_EINVAL, "n must be >= 0");
  if (n > 0 && (!d_imgs || !d_poses)) return fail(MRA_EINVAL, "NULL image or pose buffer");
  if (!d_refs) return fail(MRA_EINVAL, "d_refs is NULL");

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MRA_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(MRA_EUNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
  // First call on this device (with it current): look up the array's device address.
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return fail(MRA_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  unsigned char *base = g_scratch_ptr[dev];

  // ---- geometry tables (FP64 on the host, the same construction as mra_create) ----
  int NR = 0, M = 0;
  int rr[kMaxRings];
  for (int r = c.first_ring; r <= c.last_ring; r += c.ring_step) {
    if (NR >= kMaxRings) return fail(MRA_EINVAL, "more than %d rings", kMaxRings);
    int nn = 1;
    while (nn < kTwoPi * r) nn *= 2;
    rr[NR] = r;
    h_rings[NR].x = nn;
    M = nn > M ? nn : M;
    ++NR;
  }
  if (M < 16 || M > 512) return fail(MRA_EINVAL, "largest ring length M = %d; supported range is 16..512", M);
  const int H = M / 2;
  int NS = 0, NBIN = 0;
  for (int i = 0; i < NR; ++i) {
    const int nn = h_rings[i].x;
    int lg = 0;
    while ((1 << lg) < nn / 2) ++lg;
    h_rings[i] = make_int4(nn, NS, NBIN, lg);
    NS += nn;
    NBIN += nn / 2 + 1;
  }
  if (NS > kMaxSamples || NBIN > kMaxBins) return fail(MRA_EINVAL, "too many ring samples for the static tables");
  int first[kMaxM / 2 + 1];
  int NB = 0, seg_max = 0;
  for (int f = 0; f <= H; ++f) {
    int i0 = 0;
    while (i0 < NR && h_rings[i0].x / 2 < f) ++i0;
    first[f] = i0;
    const int Rp = (NR - i0 + 1) & ~1;
    h_fseg[f] = make_int2(NB, Rp);
    h_kpos[f] = NB - i0;  // bin (ring i, f) sits at h_kpos[f] + i
    NB += Rp;
    seg_max = Rp > seg_max ? Rp : seg_max;
  }
  for (int i = 0; i < NR; ++i) {
    const int nn = h_rings[i].x;
    for (int f = 0; f <= nn / 2; ++f) {
      h_binpos[h_rings[i].z + f] = h_fseg[f].x + (i - first[f]);
      double w = kTwoPi * rr[i] * c.ring_step / (double(nn) * double(nn));
      if (f == nn / 2 && nn < M) w *= 0.5;
      h_bweight[h_rings[i].z + f] = static_cast<float>(w);
    }
    for (int q = 0; q < nn; ++q) {
      const double th = kTwoPi * q / nn;
      h_offs[h_rings[i].y + q] =
          make_float2(static_cast<float>(rr[i] * std::cos(th)), static_cast<float>(rr[i] * std::sin(th)));
    }
  }
  for (int q = 0; q < M; ++q) {
    const double th = kTwoPi * q / M;
    h_fwd[q] = make_float2(static_cast<float>(std::cos(th)), static_cast<float>(-std::sin(th)));
    h_ang[q] = make_float2(static_cast<float>(std::cos(th)), static_cast<float>(std::sin(th)));
  }
  const int T = mra::cc_threads_per_pair(M), U = M / T;
  for (int k = 0; k < U; ++k)
    for (int t = 0; t < T; ++t) {
      const double th = kTwoPi * double(t) * double(k) / M;
      h_inv[k * T + t] = make_float2(static_cast<float>(std::cos(th)), static_cast<float>(std::sin(th)));
    }
  for (int iy = 0; iy < nx; ++iy)
    for (int ix = 0; ix < nx; ++ix)
      h_shifts[iy * nx + ix] = make_float2(static_cast<float>(-double(c.shift_range) + ix * double(c.shift_step)),
                                           static_cast<float>(-double(c.shift_range) + iy * double(c.shift_step)));
  if (double(K) * S * 2.0 * M >= 4294967295.0) return fail(MRA_EINVAL, "K * S * 2 * M exceeds 32 bits");

  // ---- carve the array: tables, failure flag, reference spectra, keys, particle spectra ----
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base + off;
    off = align256(off + bytes);
    return p;
  };
  mra::Geometry g{};
  g.L = c.L;
  g.M = M;
  g.NR = NR;
  g.NS = NS;
  g.NBIN = NBIN;
  g.NB = NB;
  g.S = S;
  g.mirror = c.mirror;
  float2 *d_offs = reinterpret_cast<float2 *>(take(sizeof(float2) * NS));
  int4 *d_rings = reinterpret_cast<int4 *>(take(sizeof(int4) * NR));
  int *d_binpos = reinterpret_cast<int *>(take(sizeof(int) * NBIN));
  float *d_bweight = reinterpret_cast<float *>(take(sizeof(float) * NBIN));
  float2 *d_fwd = reinterpret_cast<float2 *>(take(sizeof(float2) * M));
  float2 *d_inv = reinterpret_cast<float2 *>(take(sizeof(float2) * M));
  float2 *d_shifts = reinterpret_cast<float2 *>(take(sizeof(float2) * S));
  float2 *d_ang = reinterpret_cast<float2 *>(take(sizeof(float2) * M));
  int2 *d_fseg = reinterpret_cast<int2 *>(take(sizeof(int2) * (H + 1)));
  int *d_kpos = reinterpret_cast<int *>(take(sizeof(int) * (H + 1)));
  int *d_err = reinterpret_cast<int *>(take(sizeof(int)));
  const int Kpad = (K + mra::kTile - 1) / mra::kTile * mra::kTile;
  const size_t b_bytes = static_cast<size_t>(Kpad) * NB * sizeof(float2);
  float2 *d_B = reinterpret_cast<float2 *>(take(b_bytes));
  const size_t fixed = off;
  // Bytes of the argmax keys and the tiled particle spectra of a chunk of
  // `ch` images (rows padded to whole tiles of 8, each piece 256-aligned).
  auto chunk_bytes = [&](int64_t ch) {
    const int64_t tiles = (ch * S + mra::kTile - 1) / mra::kTile;
    return align256(sizeof(unsigned long long) * ch) + static_cast<size_t>(tiles) * NB * mra::kTile * sizeof(float2);
  };
  if (fixed + chunk_bytes(1) > kScratchBytes)
    return fail(MRA_EINVAL,
                "this configuration needs at least %zu bytes of scratch for one image; the reserved array holds %zu",
                fixed + chunk_bytes(1), kScratchBytes);
  const size_t per_img = static_cast<size_t>(S) * NB * sizeof(float2) + sizeof(unsigned long long);
  int64_t chunk = static_cast<int64_t>((kScratchBytes - fixed) / per_img);
  // images of a chunk index the polar kernel's grid.y and its row tiles the
  // contraction kernel's grid.y (both <= 65535)
  if (chunk > 65535) chunk = 65535;
  if (chunk > int64_t(65535) * mra::kTile / S) chunk = int64_t(65535) * mra::kTile / S;
  if (chunk < 1) chunk = 1;
  while (chunk > 1 && fixed + chunk_bytes(chunk) > kScratchBytes) --chunk;  // tile padding and alignment
  unsigned long long *d_best = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long) * chunk));
  float2 *d_A = reinterpret_cast<float2 *>(base + off);
  const int64_t a_tiles = (chunk * S + mra::kTile - 1) / mra::kTile;
  const size_t a_bytes = static_cast<size_t>(a_tiles) * NB * mra::kTile * sizeof(float2);

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
#define MRA_COPY(dst, src, bytes)                                                               \
  do {                                                                                          \
    cudaError_t ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);              \
    if (ce != cudaSuccess) return fail_sync(st, MRA_ECUDA, "table copy: %s", cudaGetErrorString(ce));    \
  } while (0)
  MRA_COPY(d_offs, h_offs, sizeof(float2) * NS);
  MRA_COPY(d_rings, h_rings, sizeof(int4) * NR);
  MRA_COPY(d_binpos, h_binpos, sizeof(int) * NBIN);
  MRA_COPY(d_bweight, h_bweight, sizeof(float) * NBIN);
  MRA_COPY(d_fwd, h_fwd, sizeof(float2) * M);
  MRA_COPY(d_inv, h_inv, sizeof(float2) * M);
  MRA_COPY(d_shifts, h_shifts, sizeof(float2) * S);
  MRA_COPY(d_ang, h_ang, sizeof(float2) * M);
  MRA_COPY(d_fseg, h_fseg, sizeof(int2) * (H + 1));
  MRA_COPY(d_kpos, h_kpos, sizeof(int) * (H + 1));
#undef MRA_COPY
  g.offs = d_offs;
  g.rings = d_rings;
  g.binpos = d_binpos;
  g.bweight = d_bweight;
  g.fwd_tw = d_fwd;
  g.inv_tw = d_inv;
  g.shifts = d_shifts;
  g.angles = d_ang;
  g.fseg = d_fseg;
  g.kpos = d_kpos;

  // The array keeps the previous call's data: padding bins of both spectra
  // layouts and the failure flag must read as zero.
  if ((e = cudaMemsetAsync(d_err, 0, sizeof(int), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_B, 0, b_bytes, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_A, 0, a_bytes, st)) != cudaSuccess)
    return fail_sync(st, MRA_ECUDA, "cudaMemsetAsync(scratch): %s", cudaGetErrorString(e));

  // reference spectra (weighted), then the chunks of particles
  mra::PolarArgs pr{};
  pr.imgs = d_refs;
  pr.n_imgs = K;
  pr.rows_per_img = 1;
  pr.use_shifts = false;
  pr.weighted = true;
  pr.out = d_B;
  if ((e = mra::launch_polar(g, pr, st)) != cudaSuccess)
    return fail_sync(st, MRA_ECUDA, "reference polar kernel: %s", cudaGetErrorString(e));
  const int64_t LL = int64_t(c.L) * c.L;
  for (int64_t c0 = 0; c0 < n; c0 += chunk) {
    const int64_t cnt = (n - c0 < chunk) ? n - c0 : chunk;
    mra::PolarArgs pa{};
    pa.imgs = d_imgs + c0 * LL;
    pa.n_imgs = cnt;
    pa.rows_per_img = S;
    pa.use_shifts = true;
    pa.weighted = false;
    pa.out = d_A;
    if ((e = mra::launch_polar(g, pa, st)) != cudaSuccess)
      return fail_sync(st, MRA_ECUDA, "particle polar kernel: %s", cudaGetErrorString(e));
    if ((e = cudaMemsetAsync(d_best, 0, sizeof(unsigned long long) * cnt, st)) != cudaSuccess)
      return fail_sync(st, MRA_ECUDA, "cudaMemsetAsync(keys): %s", cudaGetErrorString(e));
    mra::CCArgs ca{};
    ca.A = d_A;
    ca.B = d_B;
    ca.rows = cnt * S;
    ca.K = K;
    ca.best = d_best;
    ca.seg_max = seg_max;
    ca.err = d_err;
    ca.wait_limit = 2000;  // ~1 s of 0.5 ms polls
    ca.first_wait_limit = 2000;
    if ((e = mra::launch_cc_fp32(g, ca, st)) != cudaSuccess)
      return fail_sync(st, MRA_ECUDA, "contraction kernel: %s", cudaGetErrorString(e));
    if ((e = mra::launch_decode(g, d_best, cnt, K, d_poses + c0, st)) != cudaSuccess)
      return fail_sync(st, MRA_ECUDA, "decode kernel: %s", cudaGetErrorString(e));
  }
  // Host-synchronous: the next call reuses the array, and a kernel that gave
  // up a bounded wait is reported here.
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail_sync(st, MRA_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
  int flag = 0;
  if ((e = cudaMemcpy(&flag, d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return fail_sync(st, MRA_ECUDA, "read failure flag: %s", cudaGetErrorString(e));
  if (flag) return fail(MRA_ETIMEOUT, "a kernel gave up waiting for its bulk copies; the poses are invalid");
  return MRA_OK;
}

}  // extern "C"
