/*
 * mra.h - C ABI of a GB300 (sm_103a) library for multi-reference alignment
 * (MRA) of 2D particle images by resampling to polar coordinates.
 *
 * Method: Cryo-RALib (arXiv 2011.05755).  Sec. 2 defines the rotational
 * cross-correlation of a particle x and a reference y,
 *     c(phi) = int_{r1}^{r2} int_0^{2pi} x(r, theta) y(r, theta + phi) |r| dtheta dr,
 * and Algorithm 1 (Sec. 3) evaluates it for every reference, every shift on
 * the search grid and both mirror states, keeps the maximum per image (the
 * reduction of Fig. 2) and rebuilds the class averages from the aligned
 * images.  The calls below are that algorithm's inputs and outputs: a set of
 * particle images X, a set of references Y, per-image alignment parameters
 * and the new class averages Y'.
 *
 * Discretisation (a reading of the integral, fixed here and in the oracle):
 *   rings r = first_ring, first_ring + ring_step, ..., <= last_ring;
 *   N_r   = smallest power of two >= 2 pi r samples at theta_q = 2 pi q / N_r;
 *   M     = max_r N_r in-plane angles phi_j = 2 pi j / M are searched;
 *   c(phi_j) = sum_r (2 pi r dr / N_r^2) sum_{f=-N_r/2}^{N_r/2} eps_f
 *              conj(X_r(f)) Y_r(f) e^{i f phi_j},  eps_{+-N_r/2} = 1/2,
 *   X_r(f) = sum_q x_r(theta_q) e^{-2 pi i f q / N_r}.
 * Geometry: box centre c0 = (L/2, L/2); images row-major [y][x], x fast;
 * bilinear sampling with every neighbour outside [0, L-1]^2 read as 0.
 * Particle samples at c0 + s + Mm r (cos theta, sin theta), Mm = diag(-1,1)^m.
 * The shift grid has S = (2R/d + 1)^2 points (sx, sy) in [-R, R] step d,
 * indexed sy-major (index = iy * nx + ix).
 *
 * Pose meaning: the aligned image is a(c0 + w) = I(c0 + s + Mm R(-phi) w),
 * i.e. shift by -s, mirror, then rotate counter-clockwise by phi.  Among
 * bit-equal CC values the smallest (k, shift_idx, mirror, ang_idx) in
 * lexicographic order wins.
 *
 * Conventions for every call:
 *   - All buffers belong to the caller; pointers named d_* are CUDA device
 *     pointers, h_* host pointers.  All calls are asynchronous on `stream`
 *     (a cudaStream_t; NULL = legacy default stream) except where noted, and
 *     buffers must stay valid until the stream reaches the call's work.
 *   - Return value: MRA_OK (0) or an MRA_E* status; mra_last_error() gives a
 *     message.  A failed call leaves the handle usable.
 *   - One handle must not be used from two host threads at once.
 */
#ifndef MRA_H
#define MRA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without the CUDA headers (same underlying type). */
typedef struct CUstream_st *mra_stream_t;

typedef struct mra_handle *mra_t;

enum mra_status {
    MRA_OK = 0,
    MRA_EINVAL = 1,      /* bad argument or configuration                        */
    MRA_ESTATE = 2,      /* e.g. mra_align before mra_set_refs                    */
    MRA_ENOMEM = 3,      /* device or host allocation failed                      */
    MRA_ECUDA = 4,       /* a CUDA runtime call or kernel launch failed           */
    MRA_ETIMEOUT = 5,    /* a bounded device-side wait gave up                    */
    MRA_EUNSUPPORTED = 6 /* valid request the library does not implement          */
};

enum mra_precision {
    MRA_FP32 = 0,          /* contraction on FP32 FFMA, exact argmax in FP32               */
    MRA_BF16_RESCORE = 1,  /* BF16 tensor-core contraction, top-8 rows rescored in FP32    */
    MRA_FP16_RESCORE = 2   /* FP16 tensor-core contraction, top-8 rows rescored in FP32    */
};

/* Tensor-core kernel of the 16-bit paths when M = 256 (rings up to 40); the
 * two compute the same table and differ only in speed.  Other M and the
 * FP32 path ignore the choice. */
enum mra_kernel {
    MRA_KERNEL_AUTO = 0,     /* the library's default (MRA_KERNEL_MMA_SYNC)                    */
    MRA_KERNEL_MMA_SYNC = 1, /* warp-level mma.sync, tiles of 8 rows x 8 references            */
    MRA_KERNEL_TCGEN05 = 2   /* tcgen05.mma with TMEM accumulators and TMA tensor-map staging,
                                tiles of 16 rows x 8 references (k_umma256.cu)                  */
};

/* Search configuration.  Validated by mra_create:
 *   L even, 8 <= L <= 1024; 1 <= first_ring <= last_ring; ring_step >= 1;
 *   16 <= M <= 512 (so 3 <= last ring radius <= 81);
 *   shift_range >= 0, shift_step > 0, 2*shift_range/shift_step an integer
 *   (to 1e-6), S <= 4096; mirror 0 or 1; precision one of mra_precision.
 *   Rings may reach outside the box; samples there read as zero.
 *   chunk_images: images per internal chunk (0 = sized from a 2 GiB
 *   workspace budget).  kernel: one of mra_kernel (0 = default); the
 *   autotuner of the Python package picks it (and chunk_images) per
 *   configuration by measurement. */
typedef struct {
    int32_t L, first_ring, last_ring, ring_step;
    float shift_range, shift_step;
    int32_t mirror;
    int32_t precision;
    int32_t chunk_images;
    int32_t kernel;
} mra_config_t;

/* Per-image result (Alg. 1, parameter-lookup step: the alignment
 * parameters of the best CC value).  32 bytes, naturally aligned. */
typedef struct {
    int32_t k;          /* best reference (class)                          */
    int32_t ang_idx;    /* j: angle phi_j = 2 pi j / M                       */
    int32_t mirror;     /* m in {0, 1}                                       */
    int32_t shift_idx;  /* index into the sy-major shift grid                */
    float angle_deg;    /* 360 j / M                                         */
    float sx, sy;       /* the shift s = (sx, sy) in pixels                  */
    float cc;           /* c at the argmax (raw, unnormalised)               */
} mra_pose_t;

/* Derived sizes of a handle's configuration. */
typedef struct {
    int32_t M;            /* angles searched = largest ring length            */
    int32_t n_rings;      /* number of rings                                  */
    int32_t n_samples;    /* sum_r N_r                                        */
    int32_t n_bins;       /* sum_r (N_r/2 + 1) complex ring-spectrum bins     */
    int32_t n_bins_padded;/* bins in the device layout (frequency-major, padded) */
    int32_t S;            /* shifts on the grid                               */
    int32_t K;            /* references currently set (0 before mra_set_refs)  */
    int32_t chunk_images; /* images per internal chunk                        */
    int64_t workspace_bytes; /* device memory held by the handle             */
} mra_info_t;

/* Create a handle for one configuration.  Host-synchronous; allocates the
 * geometry tables on the current device.  *out is set only on MRA_OK.
 * Errors: MRA_EINVAL for a malformed configuration (see mra_config_t);
 * MRA_EUNSUPPORTED, before any CUDA call, when a kernel the configuration
 * launches would need more than 227 KB of shared memory per CTA (the
 * message names it; e.g. on the 16-bit paths the polar kernel's CTA holds
 * the image in a zero border, one row's ring samples and its 16-bit
 * spectrum words, which exceeds the limit from L = 146 with rings up to
 * 65, or from L = 100 with rings up to 81); MRA_ECUDA if a CUDA call
 * fails. */
int mra_create(const mra_config_t *cfg, mra_t *out);

/* Release the handle and all device memory it owns (synchronises the device
 * work it issued).  NULL is accepted. */
int mra_destroy(mra_t h);

/* Message for the last non-OK status returned on this handle (or, for
 * h == NULL, by mra_create in this thread).  Valid until the next call. */
const char *mra_last_error(mra_t h);

int mra_get_info(mra_t h, mra_info_t *info);

/* Alg. 1, reference-preparation step (polar conversion and FFT of every
 * reference before the particle loop): resample
 * the K references d_refs [K][L][L] (float32, device) on the rings with no
 * shift, take each ring's real DFT, scale bin f of ring r by
 * 2 pi r dr / N_r^2 (halved at f = N_r/2 when N_r < M) and keep the result
 * (FP32, plus FP16/BF16 copies for the precision-split paths) resident in
 * the handle.  K >= 1.  d_refs may be freed once the stream passes this call. */
int mra_set_refs(mra_t h, const float *d_refs, int32_t K, mra_stream_t stream);

/* Give handle dst the resident reference spectra of handle src (the output
 * of mra_set_refs, all precisions the configuration uses) by a device-to-
 * device copy on `stream`, so that several handles with the same
 * configuration, each with its own chunk workspace and stream, can align
 * against one reference set that was transformed once (Algorithm 1's
 * reference preparation is done per set, not per handle).  The two
 * configurations must agree in every field but chunk_images (else
 * MRA_EINVAL); src must hold references (else MRA_ESTATE).  The copy reads
 * src's buffers: the caller orders it after src's mra_set_refs (same stream,
 * or an event) and keeps src alive and its references unchanged until the
 * copy has run.  No paper counterpart: this is serving plumbing. */
int mra_copy_refs(mra_t dst, mra_t src, mra_stream_t stream);

/* Algorithm 1 per batch: for each image of d_imgs [n][L][L] (float32,
 * device), resample at every shift, ring-FFT, correlate with every reference
 * with and without mirror, inverse angular DFT, and write the argmax pose to
 * d_poses [n] (device).  n == 0 is a no-op.  MRA_ESTATE before mra_set_refs. */
int mra_align(mra_t h, const float *d_imgs, int64_t n, mra_pose_t *d_poses,
              mra_stream_t stream);

/* Alg. 1, class-average step (new references Y' from the aligned
 * particles): for every class k,
 * avg_k = (1/n_k) sum_{i: k_i = k} a_i with a_i(c0 + w) = I_i(c0 + s_i +
 * Mm_i R(-phi_i) w) on the integer grid (bilinear, zero outside), summed in
 * FP32 with Neumaier compensation in a fixed order (deterministic).
 * d_avg [K][L][L] and d_counts [K] (device) are written; a class with no
 * image keeps its d_avg slice untouched and gets count 0.  Poses with k
 * outside [0, K) are MRA_EINVAL only if detected on the host; on the device
 * they are skipped and not counted. */
int mra_average(mra_t h, const float *d_imgs, const mra_pose_t *d_poses, int64_t n,
                float *d_avg, int32_t *d_counts, mra_stream_t stream);

/* Sharded form of mra_average (one exchange step for several GPUs): ADD this
 * shard's per-class compensated sums into d_sum / d_comp [K][L][L] and its
 * counts into d_counts [K] (all device, caller-initialised, e.g. to zero).
 * After summing every shard's (sum, comp, counts) element-wise (e.g. by an
 * all-reduce), mra_average_finalize gives the same result as mra_average on
 * the whole stack. */
int mra_class_sums(mra_t h, const float *d_imgs, const mra_pose_t *d_poses, int64_t n,
                   float *d_sum, float *d_comp, int32_t *d_counts, mra_stream_t stream);
int mra_average_finalize(mra_t h, const float *d_sum, const float *d_comp,
                         const int32_t *d_counts, float *d_avg, mra_stream_t stream);

/* Reference refresh for iterative classification (the outer "repeat until
 * convergence" loop of Algorithm 1): for every class k with d_counts[k] > 0,
 * d_refs[k] <- (d_refs[k] - mean) / std over the L x L box (std computed
 * with 1/L^2; a constant image becomes all zero); for a class with count 0
 * and d_reseed[k] >= 0, d_refs[k] is first replaced by image d_reseed[k] of
 * d_imgs (then normalised); count 0 and d_reseed[k] < 0 leaves it as is.
 * d_refs [K][L][L], d_counts [K], d_reseed [K] (device, may be NULL: no
 * reseeding), d_imgs [n][L][L] (device; may be NULL without reseeding).
 * Uses the handle's L; K >= 1. */
int mra_refresh_refs(mra_t h, float *d_refs, const int32_t *d_counts, int32_t K, const int32_t *d_reseed,
                     const float *d_imgs, int64_t n, mra_stream_t stream);

/* The whole pass from HOST memory, for callers whose data is not on the
 * device: copies h_refs [K][L][L] and h_imgs [n][L][L] in (chunked and
 * overlapped with compute), runs mra_set_refs, mra_align and mra_average,
 * and copies h_poses [n], h_avg [K][L][L] and h_counts [K] back.  Uses
 * device staging owned by the handle.  Host-synchronous: returns when the
 * outputs are in host memory.  Pinned host buffers copy fastest. */
int mra_run_host(mra_t h, const float *h_refs, int32_t K, const float *h_imgs, int64_t n,
                 mra_pose_t *h_poses, float *h_avg, int32_t *h_counts, mra_stream_t stream);

/* The whole pass of Algorithm 1 on device buffers (the batch pattern: one
 * launch per pass): mra_set_refs(d_refs, K), mra_align(d_imgs, n, d_poses)
 * and mra_average(d_imgs, d_poses, n, d_avg, d_counts), run as ONE CUDA graph
 * launch on `stream`.  The first call with a given set of buffers and sizes
 * runs the three calls one after the other (sizing and allocating every
 * workspace); the second captures them into a graph (on a stream of the
 * handle; nothing runs during the capture) and launches it, and every
 * later call with the same buffers and sizes replays it.  A call with
 * other buffers or sizes drops the graph and starts again.  The buffers'
 * contents may change between calls; their addresses and sizes must not
 * while a graph is cached (the graph holds them, and the TMA descriptor of
 * the image stack).
 * Stage timing (mra_profile) records only the eager calls.  Same errors as
 * the three calls; MRA_ECUDA if capture or instantiation fails.  No
 * counterpart in the paper: this is launch plumbing. */
int mra_run_graph(mra_t h, const float *d_refs, int32_t K, const float *d_imgs, int64_t n, mra_pose_t *d_poses,
                  float *d_avg, int32_t *d_counts, mra_stream_t stream);
/* *captured = 1 once mra_run_graph holds an instantiated graph, else 0. */
int mra_graph_info(mra_t h, int32_t *captured);

/* Wait for the handle's work on `stream`, then report device-side failures:
 * MRA_ETIMEOUT if a kernel gave up a bounded wait for its own asynchronous
 * copies since the last mra_sync (the outputs of that work are invalid; the
 * flag is cleared and the handle stays usable).  Host-synchronous. */
int mra_sync(mra_t h, mra_stream_t stream);

/* ---- Per-stage timing (tracing) ----
 * mra_profile(h, 1) makes every later call record a CUDA event pair on its
 * stream around each stage's kernel launches (off by default; enabling or
 * disabling clears the counters).  mra_profile_read waits for the recorded
 * events and returns, per stage, the number of kernel launches and the
 * summed device time in milliseconds.  out must hold MRA_STAGE_COUNT entries. */
enum mra_stage {
    MRA_STAGE_POLAR = 0,    /* particle polar resampling + ring FFT            */
    MRA_STAGE_REFS = 1,     /* reference polar resampling + ring FFT + weights */
    MRA_STAGE_CC = 2,       /* contraction + inverse angular FFT + argmax       */
    MRA_STAGE_DECODE = 3,   /* pose decode                                       */
    MRA_STAGE_AVERAGE = 4,  /* class sums + finalize                             */
    MRA_STAGE_RESCORE = 5,  /* FP32 rescoring of candidate rows                  */
    MRA_STAGE_CONVERT = 6,  /* 16-bit copies of spectra                          */
    MRA_STAGE_COUNT = 8
};
typedef struct {
    int64_t launches;
    double ms;
} mra_stage_time_t;
int mra_profile(mra_t h, int enable);
int mra_profile_read(mra_t h, mra_stage_time_t *out);

/* ---- Alignment without device allocation ----
 * (No counterpart in the paper: this serves callers rather than the method.)
 * For code that may not call cudaMalloc at all: a framework that owns every
 * device allocation through its own pool, a latency-critical loop where an
 * allocation could stall or fail, a process whose free device memory is
 * promised elsewhere.  Such a caller cannot create a handle (mra_create
 * allocates), so this call takes the configuration directly and runs the
 * FP32 alignment of mra_align (precision must be MRA_FP32) with every
 * intermediate (geometry tables, reference spectra, one chunk of particle
 * spectra, argmax keys) inside one fixed device array of
 * MRA_STATIC_SCRATCH_BYTES, a file-scope __device__ array of the library.
 * It calls no allocating routine.
 *   d_refs [K][L][L], d_imgs [n][L][L] float32 and d_poses [n] are the
 *   caller's device buffers (same meaning as mra_set_refs / mra_align);
 *   msg (may be NULL) receives an error text of at most msg_len bytes.
 *   The configuration gets every check of mra_create (MRA_EINVAL,
 *   MRA_EUNSUPPORTED) before any CUDA call.  Images are processed in chunks
 *   that fit the array; a configuration whose tables and reference spectra
 *   plus one image (its rows padded to whole tiles) do not fit is rejected
 *   with MRA_EINVAL and a message giving the bytes it would need.
 *   With CUDA's default lazy module loading the array is committed on a
 *   device at the first use there: the first call on each device, with that
 *   device current, looks up the array's device address
 *   (cudaGetSymbolAddress), and that first call can return MRA_ECUDA (out of
 *   memory) if the device has no room for the array.  The first call on
 *   each device should come before any stream capture.  Once committed, the
 *   array stays until the process exits.
 *   Host-synchronous: before returning, the call synchronises `stream` and
 *   reads a device failure flag with a blocking copy (MRA_ETIMEOUT if a
 *   kernel gave up a bounded wait).  Every call uses the same array, which
 *   keeps the previous call's contents (each call clears what must start at
 *   zero).  Calls whose GPU work overlapped would race on the array; the
 *   library prevents that with a process-wide lock held from the first
 *   enqueue until the call's GPU work has finished (also on error returns),
 *   so calls from several host threads run one after another. */
#define MRA_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int mra_align_static(const mra_config_t *cfg, const float *d_refs, int32_t K, const float *d_imgs, int64_t n,
                     mra_pose_t *d_poses, mra_stream_t stream, char *msg, int32_t msg_len);

/* ---- Stage-level entry points (for parity tests; same kernels as above) ----
 * mra_debug_polar: d_out [n][S][n_samples] float32, ring samples of every
 *   image at every shift (unmirrored), rings in order, q in order.
 * mra_debug_spectra: d_out [n][S][n_bins][2] float32 (re, im), the ring DFT
 *   bins X_r(f), f = 0..N_r/2, rings in order.
 * mra_debug_cc: d_out [n][K][S][2][M] float32, the full CC table c(k,s,m,j)
 *   computed by the path selected by `precision` (for the split paths, the
 *   16-bit contraction before rescoring).  Only for small n. */
int mra_debug_polar(mra_t h, const float *d_imgs, int64_t n, float *d_out, mra_stream_t stream);
int mra_debug_spectra(mra_t h, const float *d_imgs, int64_t n, float *d_out, mra_stream_t stream);
int mra_debug_cc(mra_t h, const float *d_imgs, int64_t n, float *d_out, mra_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MRA_H */
