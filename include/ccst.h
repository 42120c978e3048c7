/*
 * ccst.h -- C ABI of libccst: cross-correlation sub-pixel tracking on one GPU.
 *
 * Method (arXiv 2310.08770):
 *   - Sec. II, Eqs. (1)-(4): uniform-weight cross-correlation (CC-U). The
 *     displacement maximises c(s) = sum_r I(r+s) E(r) = F^-1[F[I] conj F[E]](s)
 *     between a frame I and the reference image E (periodic boundaries).
 *   - Sec. II, Eqs. (5)-(7): shot-noise-weighted cross-correlation (CC-SN).
 *     The frame is offset by eps, I' = I + eps, the reference becomes
 *     E_SN = E + eps, and the surface is c(s) = sum_r I'(r+s)^2 / E_SN(r).
 *     The chi^2 of Eq. (6) is smallest where this surface is smallest, so CC-SN
 *     takes the minimum.
 *   - Sec. III: the integer extremum of c is refined on a grid of
 *     M = ceil(1.5 u) x M points, spaced 1/u pixel, centred on it. The product
 *     spectrum of Eq. (4) / (7) is inverse-DFT'd onto that grid (the
 *     matrix-multiply DFT of the paper's ref. [27]), and the extremum of that
 *     upsampled surface is the sub-pixel displacement.
 *
 * Conventions:
 *   - Images are H rows x W columns, row-major; x is the column (contiguous) index.
 *   - The reported displacement d = (dx, dy) is the motion of the frame content
 *     relative to the reference: frame(r) ~ ref(r - d).
 *   - Integer peaks are wrapped to (-ceil(N/2), floor(N/2)] per axis.
 *   - Grid offsets are (j - floor(M/2))/u, j = 0..M-1.
 *   - Ties go to the lowest row-major index, as in the FP64 oracle.
 *   - `peak` is the surface value at the reported point, in the units of the
 *     direct sum above. It equals c(p) at offset 0.
 *
 * Errors: every call returns an int. 0 is CCST_OK; negative values are errors.
 *   - No exception or abort crosses the ABI.
 *   - A CUDA error inside a call marks the context unusable (sticky). Later calls
 *     return CCST_E_CUDA, and ccst_last_error() gives the message.
 *
 * Threading: one context must not be used from two host threads at once.
 * Separate contexts are independent.
 */
#ifndef CCST_H
#define CCST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCST_VERSION 10000 /* 1.0.0 */

/* return codes */
#define CCST_OK             0
#define CCST_E_INVALID     -1  /* null pointer, bad enum, n < 0, ... */
#define CCST_E_SHAPE       -2  /* H, W outside the supported set, or frames larger than create() allowed */
#define CCST_E_UNSUPPORTED -3  /* a valid request this build does not implement */
#define CCST_E_NOMEM       -4  /* device or pinned host allocation failed */
#define CCST_E_CUDA        -5  /* a CUDA runtime error; the context is now unusable */
#define CCST_E_TIMEOUT     -6  /* ccst_poll: not finished within the timeout */
#define CCST_E_BUSY        -7  /* ccst_submit: all in-flight slots are taken */

/* methods (Sec. II) */
#define CCST_CC_U  0  /* uniform weight, Eq. (4): maximum of sum I E        */
#define CCST_CC_SN 1  /* shot-noise weight, Eq. (7): minimum of sum I'^2/E_SN */

/* frame element types */
#define CCST_U16 0
#define CCST_F32 1

/* ccst_params.flags */
/* TIE_GUARD, GRAPHS and PROFILE concern power-of-two contexts; a general-shape context
 * (see ccst_create) runs its own guard levels always, launches directly, and has no
 * profiling. */
#define CCST_FLAG_TIE_GUARD 0x1u  /* resolve near-ties of the FP32 surfaces in higher precision (default on) */
#define CCST_FLAG_GRAPHS    0x2u  /* ccst_track replays one captured CUDA graph per (stream, frames, n,
                                      pitch, out); each graph owns its frame counter, so graphs of
                                      different batches may run at once on different streams
                                      (ccst_set_stream) */
#define CCST_FLAG_PROFILE   0x4u  /* record CUDA events around each launch of the tracking kernel */
#define CCST_FLAG_EXHAUSTIVE 0x8u /* general-shape contexts (ccst_create): every frame on the
                                     double-float kernel, evaluating the whole upsampled grid in
                                     double-float (no FP32 general-size kernel, no FP32 grid with
                                     a rounding bound). Decisions are the same; this is for
                                     verification. */

/* ccst_result.flags (per frame) */
#define CCST_R_INT_GUARD   0x01u /* integer peak re-decided in higher precision (FP64 direct sums; the
                                    FP32 general-size kernel: its double-float spectrum) */
#define CCST_R_SUB_GUARD   0x02u /* sub-pixel peak re-decided by exact FP32 grid differences */
#define CCST_R_DF64        0x04u /* sub-pixel peak decided from a double-float (~48-bit) product spectrum */
#define CCST_R_OVERFLOW    0x08u /* too many near-tied points to certify: the FP32 choice is reported */
#define CCST_R_NONFINITE   0x10u /* the surface held no finite value (non-finite input) */
#define CCST_R_TIMEOUT     0x20u /* a bounded wait inside the kernel gave up (the staged stage tables never
                                    arrived); this frame and the rest of its CTA's frames are not tracked */
#define CCST_R_GENERIC     0x80u /* tracked by the double-float general-size kernel (ccst_track_rois,
                                    sides other than 16, 32, 64, 128): direct DFTs in double-float,
                                    no near-tie levels */
#define CCST_R_FP32_GENERAL 0x100u /* tracked by the FP32 general-size kernel (48, 96, 192 and 256
                                    square, 256 x 128 either way, u <= 256): mixed-radix (2, 3) FFTs and the
                                    upsampled contraction in FP32, with the integer and sub-pixel
                                    guard levels; a frame they cannot certify is tracked again by
                                    the double-float kernel and its record carries CCST_R_GENERIC */
#define CCST_R_RT_STALE    0x40u /* real-time mode: the reference update after this frame did not complete
                                    (a bounded wait gave up, now or earlier); the reference stays stale
                                    until the next ccst_rt_begin */

typedef struct ccst_params {
    int32_t  upsample;   /* u >= 1, default 100 (Sec. III)                          */
    int32_t  method;     /* CCST_CC_U or CCST_CC_SN                                 */
    float    eps;        /* CC-SN offset, default 200 = 200 x noise gain 1 (Sec. IV) */
    int32_t  in_dtype;   /* CCST_U16 or CCST_F32                                    */
    int32_t  max_batch;  /* largest n one ccst_track call may pass; > 0            */
    int32_t  max_H;      /* reserved: 0                                             */
    int32_t  max_W;      /* reserved: 0                                             */
    void*    stream;     /* cudaStream_t the context works on; NULL = legacy default */
    uint32_t flags;      /* CCST_FLAG_*                                             */
} ccst_params;

/* Per-frame result: 24 bytes, naturally aligned. */
typedef struct ccst_result {
    float    dx, dy;     /* sub-pixel displacement (px), frame(r) ~ ref(r - d)      */
    float    peak;       /* surface value at d, direct-sum units                    */
    int32_t  ipy, ipx;   /* wrapped integer peak                                    */
    uint32_t flags;      /* CCST_R_*                                                */
} ccst_result;

/* One region of interest of an uneven batch (ccst_track_rois): 32 bytes. */
typedef struct ccst_roi {
    const void* frame;      /* device memory: H rows pitch_elems apart, the context's in_dtype */
    int32_t  H, W;          /* must equal the size of reference ref_id                        */
    int64_t  pitch_elems;   /* 0 means W                                                       */
    int32_t  ref_id;        /* 0: the context's reference; others from ccst_add_reference      */
    int32_t  reserved;      /* 0                                                               */
} ccst_roi;

typedef struct ccst_ctx ccst_ctx;

/* Library version, CCST_VERSION. */
int ccst_version(void);

/* Fill *p with the defaults: u = 100, CC-U, eps = 200, uint16 frames,
 * max_batch = 256, stream NULL, flags = CCST_FLAG_TIE_GUARD. */
int ccst_default_params(ccst_params* p);

/* Create a tracking context for H x W frames against the reference image `ref`.
 *
 * Arguments:
 *   ref   H*W float32, row-major, host or device memory (detected). It is copied;
 *         the caller keeps ownership.
 *   H, W  8 <= H, W <= 256, any factors (H != W allowed). Other sizes return
 *         CCST_E_SHAPE.
 *         - Powers of two up to 128 (8, 16, 32, 64, 128 per axis) make a power-of-two
 *           context: FP32 FFTs, the upsampled contraction on tensor cores, the near-tie
 *           levels, and every entry point below.
 *         - Every other shape makes a general-shape context.
 *           48 x 48, 96 x 96, 192 x 192, 256 x 256, and 256 x 128 either way round
 *           (u <= 256) run on the FP32
 *           general-size kernel: mixed-radix (2, 3) FFTs and the upsampled contraction
 *           in FP32 in shared memory (one to four CTAs per frame), with the integer,
 *           sub-pixel, pair-difference and double-float guard levels; records carry
 *           CCST_R_FP32_GENERAL. A frame those levels cannot certify (a tie within
 *           2^-36 sum|X|) is tracked again by the double-float kernel.
 *           Every other shape (192 x 64, 100 x 60, ...), and those frames, run on the
 *           double-float kernel: direct DFTs over the Hermitian half and the full-grid
 *           upsampled sum, in double-float (about 2^-46 per term, so no near-tie levels
 *           are needed); records carry CCST_R_GENERIC.
 *           ccst_track, ccst_track_host, ccst_submit, ccst_submit_host, ccst_poll,
 *           ccst_set_reference_frame, ccst_add_reference, ccst_track_rois and the server
 *           work on a general-shape context; so do ccst_debug_surfaces and
 *           ccst_debug_pairs when it has the FP32 general-size kernel. The real-time and
 *           offline reference, the continuous peak, the adjoint and profiling return
 *           CCST_E_UNSUPPORTED.
 *   p     parameters; NULL means the defaults.
 *   out   receives the context.
 *
 * The context owns the reference spectrum (power-of-two: FP32 and FP64; general: double-
 * float; Eq. (4)/(7) right-hand side), the upsampling tables and all device workspace.
 * Synchronous.
 * Errors: CCST_E_INVALID, CCST_E_SHAPE, CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_create(const float* ref, int H, int W, const ccst_params* p, ccst_ctx** out);

/* Track n frames (Sec. II-III) on the context's stream. Stream-ordered and
 * asynchronous.
 *
 * Arguments:
 *   frames_dev   caller-owned device memory holding n frames of H rows, each row
 *                `pitch_elems` elements apart (0 means W), frames H*pitch
 *                apart, element type params.in_dtype.
 *   out_dev      caller-owned device memory for n ccst_result records.
 *
 * The results are valid once the stream reaches this point (synchronise the
 * stream or call ccst_sync). 0 <= n <= max_batch; n = 0 is a no-op.
 * Errors: CCST_E_INVALID (null pointers, n out of range, pitch < W),
 *         CCST_E_CUDA. */
int ccst_track(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
               ccst_result* out_dev);

/* Same computation for host memory. Copies the n frames host -> device, tracks
 * them, copies the results back, and returns after the results are in out_host.
 * Pageable or pinned host memory are both accepted; pinned is faster.
 * Errors: as ccst_track. */
int ccst_track_host(ccst_ctx* ctx, const void* frames_host, int64_t n, int64_t pitch_elems,
                    ccst_result* out_host);

/* Pipelined host form for streaming from host memory (not in the paper: the serving side
 * of a camera link). It enqueues, without waiting: the copy of n frames host -> device,
 * the tracking, and the copy of the results to out_host. It returns a ticket for
 * ccst_poll, and the results are in out_host once that ticket is done.
 *   Submissions rotate over four device staging slots on two internal streams. The
 *   copies of one batch therefore overlap the tracking of the previous one.
 *   Submitting into a slot whose previous batch is still running blocks until it ends.
 *   The internal streams start after the work already issued on the context's stream.
 *   They are not ordered against later work on it: use the tickets.
 *   frames_host and out_host must stay valid until the ticket is done. They must be
 *   pinned host memory for the copies to be asynchronous.
 * Errors: as ccst_track, plus CCST_E_BUSY when all tickets are in flight and CCST_E_NOMEM
 * when the staging slots (4 x max_batch frames) cannot be allocated on first use. */
int ccst_submit_host(ccst_ctx* ctx, const void* frames_host, int64_t n, int64_t pitch_elems,
                     ccst_result* out_host, uint64_t* ticket);

/* Work on `stream` (a cudaStream_t) from now on. The caller orders this
 * against earlier work. Cached graphs (CCST_FLAG_GRAPHS) are keyed by stream as well as
 * by batch, so switching streams drops none of them: each (stream, batch) pair is
 * captured once and then replayed. Every cached graph owns a frame counter that no other
 * graph or launch uses, and direct launches wait for the previous user of their counter,
 * so batches in flight at once on different streams never share a frame counter.
 * Calls that use the context's shared buffers (ccst_track_rois; ccst_track on a
 * general-shape context) are ordered after the previous such call, on any stream. */
int ccst_set_stream(ccst_ctx* ctx, void* stream);

/* Graph-cache statistics of a context (CCST_FLAG_GRAPHS):
 *   instantiations  graphs captured and instantiated so far;
 *   replays         graph launches so far;
 *   cached          graphs held now (at most 512; when full, the cache waits for the
 *                   cached graphs' last replays, destroys them and starts again).
 * Not in the paper: a measure of the batching machinery (Sec. III makes frames
 * independent under a fixed reference, so batches may run on several streams at once).
 * Errors: CCST_E_INVALID (null context or output). */
int ccst_graph_stats(ccst_ctx* ctx, int64_t* instantiations, int64_t* replays, int64_t* cached);

/* Block until all work issued on the context's stream has finished. */
int ccst_sync(ccst_ctx* ctx);

/* Asynchronous serving form of ccst_track: enqueue and return a ticket.
 * At most 64 submissions may be in flight per context; more return CCST_E_BUSY. */
int ccst_submit(ccst_ctx* ctx, const void* frames_dev, int64_t n, ccst_result* out_dev,
                uint64_t* ticket);

/* Ask whether a ticket has finished. Waits at most timeout_us microseconds.
 *   CCST_OK          *done = 1 and the slot is released.
 *   CCST_E_TIMEOUT   *done = 0; poll again later.
 *   CCST_E_INVALID   unknown ticket. */
int ccst_poll(ccst_ctx* ctx, uint64_t ticket, int timeout_us, int* done);

/* Add a reference for uneven-ROI batches (ccst_track_rois) and return its id in *ref_id.
 *   ref      H*W float32, row-major, host or device memory; copied.
 *   H, W     square, 8 to 256 pixels a side; others return CCST_E_SHAPE.
 *            16, 32, 64 and 128 run on the power-of-two ROI kernel (FP32 surfaces with the
 *            near-tie levels, as ccst_track). 48, 96, 192 and 256 run on the FP32
 *            general-size kernel and every other side (8, 24, odd sides, ...) on the
 *            double-float kernel, as in general-shape contexts (see ccst_create).
 * The first reference of a new size also creates that size's plan (geometry, FFT
 * twiddles, upsampling tables) with the context's parameters (u, method, eps); for the
 * general path u * N must not exceed 2^22. Each power-of-two reference keeps its spectra
 * resident (FP32, FP64 and double-float) and its FP64 operand, about 26 H*W bytes; a
 * general-size reference keeps its half spectrum in double-float, 16 N (N/2 + 1) bytes.
 * All of it is owned by the context. The context's own reference is id 0, usable unless
 * it is a power-of-two context of a non-square or 8 x 8 shape. Synchronous.
 * Errors: CCST_E_INVALID (null pointers), CCST_E_SHAPE, CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_add_reference(ccst_ctx* ctx, const float* ref, int H, int W, int* ref_id);

/* Track an uneven batch: n ROIs of mixed sizes, each against its own reference (Secs. II-III
 * per ROI, as ccst_track), in one call of persistent launches.
 *   rois      host memory, n descriptors (read during the call).
 *   out_dev   device memory, n records; record i belongs to rois[i].
 * Work items run largest ROI first; each CTA takes the next item from a counter. The
 * power-of-two ROIs run on the context's stream, one launch per side present (128, 64,
 * 32, 16 px), each compiled for its own side. Their records are identical to those of ccst_track on a context made for that ROI's
 * reference. ROIs of general sizes run on an internal stream beside them: one persistent
 * launch of the FP32 general-size kernel per side it takes (48, 96, 192, 256). On each
 * stream a launch may start in the last wave of the one before it (programmatic dependent
 * launch). After both, one launch of the double-float kernel takes the other general sides
 * and the frames the FP32 kernel handed on; the call's work is complete when the context's
 * stream reaches it.
 * With CCST_FLAG_GRAPHS (and a non-default stream), the launches are captured once as
 * one CUDA graph per (stream, out_dev, work list), with the work items uploaded to memory
 * the graph owns, and replayed by later calls with the same list (compared byte by byte).
 * A graph's frame counters and items are its own. The general-size scratch is one area
 * per stream, and graphs on one stream run in order. Adding a reference or running
 * ccst_autotune drops the captured graphs, after their last replays have finished.
 * At most 64 are kept; beyond that the cache is emptied and starts again.
 * Without the flag every call uploads its items and launches directly.
 * Stream-ordered and asynchronous.
 * Errors: CCST_E_INVALID (null pointers, n < 0, unknown ref_id, pitch < W), CCST_E_SHAPE (a
 * ROI whose size differs from its reference's), CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_track_rois(ccst_ctx* ctx, const ccst_roi* rois, int64_t n, ccst_result* out_dev);

/* One tuned general-size plan (ccst_autotune): 32 bytes. */
typedef struct ccst_tune_result {
    int32_t H, W;           /* the plan's frame shape                                        */
    int32_t H1, W1;         /* chosen two-level splits: H = H1 (H / H1), W = W1 (W / W1)     */
    int32_t threads;        /* chosen CTA size of the general-size kernel (the context's)    */
    int32_t timed;          /* configurations timed in the call                              */
    double   us_per_frame;  /* the chosen splits' time per frame (512 threads, two grid waves) */
} ccst_tune_result;

/* Autotune the double-float general-size kernel (NEXT-2: the size-dependent choices of the
 * uneven-ROI path; the FP32 general-size kernel has one compiled schedule per side and
 * nothing to tune, and is bypassed while this call times, so that every plan's frames
 * exercise the double-float kernel, which also takes the FP32 kernel's fallback frames).
 * For every general-size plan of the context (shapes added by ccst_create or
 * ccst_add_reference outside the power-of-two kernel) it times, on synthetic frames of the
 * plan's shape and one of its references, each two-level split of the row and column DFTs
 * (the default: the largest divisor of N not above sqrt(N); its cofactor; the next divisor
 * below) as the best of `reps` launches of two grid waves after a warm-up, and keeps the
 * fastest. Then it times both CTA sizes (512 and 256 threads, one per launch) and keeps the
 * faster: on the caller's ROI batch `rois` (n_rois > 0; run through ccst_track_rois, all
 * its kernels, as the caller will run it), else on a work list of every plan's frames, largest
 * first. Later launches of the context (ccst_track, ccst_track_rois, the server) use them.
 *   rois     host, n_rois descriptors as for ccst_track_rois, or NULL with n_rois = 0. The splits change only the rounding order of the double-float DFTs: records
 * keep the parity bar and stay the same alone and in a batch. Power-of-two shapes have
 * nothing to tune (one compiled schedule per size).
 *   out      host, max_out records (may be NULL when max_out is 0), one per general plan.
 *   n_out    receives the number of records written (may be NULL).
 * Synchronous; the context must not be in use by a server or other calls meanwhile.
 * Errors: CCST_E_INVALID, CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_autotune(ccst_ctx* ctx, int reps, const ccst_roi* rois, int64_t n_rois, ccst_tune_result* out,
                  int max_out, int* n_out);

/* ---- Serving: continuous batching of single frames from several cameras.
 * Not in the paper, which tracks one camera; frames are independent under a fixed
 * reference (Sec. III), so frames of several cameras can share a launch.
 *
 * A server runs a worker thread over a context. Each camera is a reference of the
 * context (id 0 or from ccst_add_reference): its frames have that reference's size.
 * Admission is by memory: a submitted frame is copied into an arena of budget_bytes
 * (pinned host memory mapped into the device's address space, so the kernels read each
 * frame in place with no per-frame copy), taking its own size rounded up to 256 bytes.
 * A submit that does not fit in what admitted frames leave free is refused with
 * CCST_E_BUSY. So small cameras are not charged the largest camera's size. The device
 * memory of the in-flight batches (records, work items, general-size scratch) is
 * allocated at creation, so the budget bounds what admitted frames add.
 * The worker takes everything pending (up to max_batch frames, any cameras and sizes) as
 * one batch on its own stream, launched as ccst_track_rois launches a batch: the
 * power-of-two ROI kernels for cameras of 16, 32, 64 or 128 px and, beside them, the
 * general-size kernels for the others (each ring entry has its own lane and second
 * stream for them). Up to max_in_flight (at most 4) batches are in flight. Frames that
 * arrive while others run are admitted as memory frees up, and their work overlaps on
 * the device. With max_batch = 1 and max_in_flight = 1 the server is the plain form:
 * one launch per frame, each after the previous one has finished. Each result equals
 * that of the frame tracked alone (the batch changes only which CTA runs it). While a
 * server exists its context must not be used by other calls (nor references added). */
typedef struct ccst_server ccst_server;

typedef struct ccst_server_stats {
    uint64_t submitted, completed, rejected;   /* since the last reset                       */
    uint64_t batches;                          /* kernel launches                            */
    double   mean_batch;                       /* frames per launch                          */
    double   p50_us, p99_us, max_us;           /* submit -> result available (host clock)   */
    int64_t  in_flight;                        /* admitted, not yet completed               */
    int64_t  bytes_in_flight;                  /* arena bytes held by admitted frames now    */
    int64_t  max_bytes_in_flight;              /* most held since the last reset             */
    int64_t  budget_bytes;                     /* the arena's size                           */
} ccst_server_stats;

typedef struct ccst_server_config {
    int32_t max_batch;       /* frames per launch, >= 1                                       */
    int32_t max_in_flight;   /* batches in flight at once, 1 .. 4                            */
    int64_t budget_bytes;    /* admission arena, >= 256 (rounded up to a multiple of 256)    */
    uint32_t flags;          /* 0                                                             */
    int32_t reserved;
} ccst_server_config;

/* Start a server over ctx (ctx keeps ownership of its references and must outlive it).
 * A camera whose frame is larger than the budget is refused at submit (CCST_E_INVALID).
 * Errors: CCST_E_INVALID (bad configuration, no reference usable by ROI batches),
 * CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_server_create_ex(ccst_ctx* ctx, const ccst_server_config* cfg, ccst_server** out);

/* The same with a budget of `slots` frames of the largest reference present now, at most
 * min(max_batch, slots) frames per launch, and 4 batches in flight.
 * Errors: CCST_E_INVALID (slots or max_batch < 1, no reference usable by ROI batches),
 * CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_server_create(ccst_ctx* ctx, int slots, int max_batch, ccst_server** out);

/* Submit one frame of camera ref_id from host memory (rows pitch_elems apart, 0 = W; copied
 * before the call returns). With ticket non-NULL the result is kept for ccst_server_poll;
 * with NULL it is only counted in the statistics. Thread-safe.
 * Errors: CCST_E_INVALID, CCST_E_BUSY (the budget is full: retry later), CCST_E_CUDA. */
int ccst_server_submit(ccst_server* srv, int ref_id, const void* frame_host, int64_t pitch_elems,
                       uint64_t* ticket);

/* Wait up to timeout_us for a ticket's result. CCST_OK: *done = 1, *out holds the record
 * and the ticket is released. CCST_E_TIMEOUT: *done = 0. CCST_E_INVALID: unknown ticket.
 * Thread-safe. */
int ccst_server_poll(ccst_server* srv, uint64_t ticket, int timeout_us, ccst_result* out, int* done);

/* Statistics since the last reset (reset != 0 clears them after reading). Returns the
 * server's sticky error, if any. */
int ccst_server_read_stats(ccst_server* srv, int reset, ccst_server_stats* out);

/* Measurement helper: offered load from ncams host threads. Camera k submits frames of
 * its pool (pool_len[k] frames of its size, contiguous, host memory), cycled, at
 * exponential inter-arrival times of mean 1/rates_hz[k] for `seconds`, seeded by seed;
 * refused frames are dropped and counted. Returns after all admitted frames completed,
 * with the statistics of the run in *out. */
int ccst_server_loadgen(ccst_server* srv, int ncams, const int* ref_ids, const double* rates_hz,
                        const void* const* pools, const int* pool_len, double seconds, uint64_t seed,
                        ccst_server_stats* out);

/* Stop the worker after the admitted frames complete, and free the server. NULL is a no-op. */
void ccst_server_destroy(ccst_server* srv);

/* Real-time reference (Sec. III B, Eq. (9)): start a filtered reference from frame 0.
 *   frame0_dev   device memory, one H x W frame of the context's in_dtype, rows
 *                pitch_elems apart (0 means W). Read during the call's stream work.
 *   a0, b1       the filter's coefficients, a0 = 1 - exp(-T/tau), b1 = exp(-T/tau)
 *                for frame period T and time constant tau. Any finite values.
 * Sets F[E_0] = F[I_0] (CC-SN: F[I_0 + eps]) and makes E_0 the context's reference,
 * replacing the one given to ccst_create. The first call allocates the filter
 * state (2 x H x (W/2+1) complex doubles), owned and freed by the context.
 * Each reference update is one cooperative launch of at most W/2+1 CTAs whose grid
 * barriers wait a bounded time (see CCST_R_RT_STALE). Stream-ordered and asynchronous.
 * Errors: CCST_E_INVALID (null frame, pitch < W, a0 or b1 not finite),
 * CCST_E_UNSUPPORTED (no cooperative launch on the device), CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_rt_begin(ccst_ctx* ctx, const void* frame0_dev, int64_t pitch_elems, double a0, double b1);

/* Real-time tracking (Sec. III B): for i = 0 .. n-1, track frame i against the
 * current reference E, then update it with the frame aligned by the displacement
 * d just found, Eq. (9):
 *   F[E] <- a0 F[I_i](k) e^{+2 pi i (ky' dy / H + kx' dx / W)} + b1 F[E],
 * with fftfreq-signed ky', kx'; an even axis's Nyquist bin takes cos(pi d). The
 * aligned frame I_i(r + d) is the frame moved back onto the reference. CC-SN
 * filters E' = E + eps on I_i + eps and tracks against the operand 1/E'.
 * d is the record's displacement taken exactly, (p u + t) / u in FP64; a record
 * flagged CCST_R_TIMEOUT leaves E unchanged. A record flagged CCST_R_RT_STALE was
 * tracked, but the update after it did not complete.
 *   frames_dev   device memory, n frames of H rows pitch_elems apart (0 means W).
 *   out_dev      device memory, n records, as for ccst_track.
 * Each call continues the filter where the previous one ended. The frames are
 * sequential by construction: one frame is tracked at a time (latency, not
 * throughput, is this mode's figure). Stream-ordered and asynchronous.
 * Errors: CCST_E_INVALID (no ccst_rt_begin yet, n < 0, null pointers, pitch < W),
 * CCST_E_CUDA. */
int ccst_rt_track(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
                  ccst_result* out_dev);

/* Make frame_dev the reference: F[E] = F[frame] (CC-SN: F[frame + eps]), the E_0 of
 * Eqs. (8) and (9). It replaces the reference given to ccst_create (or any later one).
 *   frame_dev    device memory, one H x W frame of the context's in_dtype, rows
 *                pitch_elems apart (0 means W).
 * The first call of this, ccst_rt_begin or ccst_offline_update allocates the FP64 filter
 * state (2 x H x (W/2+1) complex doubles), owned by the context. Clears a stale flag (see
 * ccst_reference_status). Stream-ordered and asynchronous.
 * Errors: CCST_E_INVALID (null frame, pitch < W), CCST_E_UNSUPPORTED (no cooperative
 * launch on the device), CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_set_reference_frame(ccst_ctx* ctx, const void* frame_dev, int64_t pitch_elems);

/* Offline reference update (Sec. III A, Eq. (8)): make the context's reference the mean, in
 * Fourier space, of the n frames each moved back by its displacement,
 *   F[E] = (1/N) sum_i F[I_i](k) e^{+2 pi i (ky' dy_i / H + kx' dx_i / W)},
 * with d_i the displacement of record i (from tracking frame i against the previous
 * reference), taken exactly as (p u + t) / u in FP64, and the signed frequencies and
 * Nyquist bins of ccst_rt_track. CC-SN takes the mean of I_i + eps and tracks against
 * the operand 1 / that. Records flagged CCST_R_TIMEOUT are left out of the sum and of N;
 * with none left the reference stays.
 *   frames_dev   device memory, n frames of H rows pitch_elems apart (0 means W).
 *   rec_dev      device memory, n records (ccst_track's output for these frames).
 * The sum runs in FP64 in one CTA per SM (per-CTA partial sums, added in a fixed order:
 * the result does not depend on timing). The first call allocates 2 x SMs x H x (W/2+1)
 * complex doubles of workspace, owned by the context. Stream-ordered and asynchronous.
 * Errors: CCST_E_INVALID (n < 0, null pointers, pitch < W), CCST_E_UNSUPPORTED,
 * CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_offline_update(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
                        const ccst_result* rec_dev);

/* The offline method of Sec. III A: E_0 = frame 0; for p = 0 .. passes, track all n frames
 * against E_p (in batches of max_batch) and, for p < passes, set E_{p+1} by
 * ccst_offline_update. out_dev receives the records of the last pass (against E_passes);
 * the reference stays E_passes. n may exceed max_batch.
 * Errors: CCST_E_INVALID (n < 1, passes < 0, null pointers, pitch < W), and those of
 * ccst_set_reference_frame and ccst_offline_update. */
int ccst_offline_track(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems, int passes,
                       ccst_result* out_dev);

/* Whether a reference update of ccst_rt_track or ccst_offline_update gave up at a bounded
 * wait since the last ccst_set_reference_frame / ccst_rt_begin (*stale = 1): the reference
 * is then out of date. Synchronises the context's stream.
 * Errors: CCST_E_INVALID (null stale), CCST_E_CUDA. */
int ccst_reference_status(ccst_ctx* ctx, int* stale);

/* Drift removal (Sec. III B) over n tracking records/* Drift removal (Sec. III B) over n tracking records, r_i = (dx_i, dy_i).
 *   alpha <= 0   Eq. (10): R_0 = a0 r_0, R_i = a0 r_i + b1 R_{i-1}.
 *   alpha > 0    Eqs. (11)-(12): the step a0 r_i + (b1 - 1) R_{i-1} of R is cut to
 *                length alpha / u when longer; R_0 = a0 r_0 as in Eq. (10).
 * Writes out_dev[2i] = dx_i - R_i.x, out_dev[2i+1] = dy_i - R_i.y (doubles).
 *   rec_dev, out_dev   device memory owned by the caller.
 *   stream             cudaStream_t to run on (NULL: the default stream).
 * The recurrence is sequential; one GPU thread runs it. Asynchronous.
 * Errors: CCST_E_INVALID (n < 0, null pointers, non-finite a0/b1, NaN alpha,
 * alpha > 0 with u < 1), CCST_E_CUDA. */
int ccst_drift_correct(const ccst_result* rec_dev, int64_t n, double a0, double b1, double alpha, int u,
                       double* out_dev, void* stream);

/* Continuous peak: the stationary point s* of the band-limited interpolant of the
 * correlation surface (Sec. III; Eqs. (4), (7)),
 *   f(s) = (1/HW) Re sum_k X(k) e^{2 pi i (ky' sy / H + kx' sx / W)},
 * over all H x W frequencies (fftfreq-signed), X the product spectrum of the method,
 * found by Newton's method from the grid peak of each record (row sums in double-float,
 * about 2^-46 a term; steps until one is below 1e-11 px): the u -> infinity
 * limit of the tracker's estimate, and the quantity ccst_backward differentiates. The
 * paper's estimate itself is the grid point; this is an addition to it.
 *   frames_dev   device memory, n frames of H rows pitch_elems apart (0 means W).
 *   rec_dev      device memory, the n records ccst_track gave for these frames against
 *                the context's current reference.
 *   peak_dev     device memory, n x 2 doubles (dx, dy) of s*, or NULL.
 *   status_dev   device memory, n words, or NULL: 0, or a sum of 1 (Newton did not
 *                settle in 50 steps), 2 (s* is not a maximum for CC-U / minimum for
 *                CC-SN), 4 (s* is more than 1 px from the grid peak).
 * One CTA per frame (up to one per SM, frames strided), FP64 throughout. The first call
 * allocates the workspace of ccst_offline_update plus H x (W/2+1) complex doubles.
 * Stream-ordered and asynchronous.
 * Errors: CCST_E_INVALID (n < 0, null pointers, no output, pitch < W), CCST_E_NOMEM,
 * CCST_E_CUDA. */
int ccst_peak_continuous(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
                         const ccst_result* rec_dev, double* peak_dev, int32_t* status_dev);

/* Vector-Jacobian product of the continuous peak (ccst_peak_continuous) with respect to
 * the frame pixels and the reference. From grad f(s*) = 0: with the Hessian Hf of f at
 * s* and the upstream gradient g = dL/ds*, w = -Hf^{-1} g and
 *   dL/da(r) = (1/HW) Re sum_k (2 pi i w.k'/N) conj F[b](k) e^{2 pi i k.(s* - r)/N},
 *   dL/db(r) = (1/HW) Re sum_k (2 pi i w.k'/N) F[a](k) e^{2 pi i k.(s* + r)/N},
 * for the surface operands (a, b) = (I, E) (CC-U) or ((I + eps)^2, 1/(E + eps)) (CC-SN),
 * then the chain rule to I and E.
 *   frames_dev, rec_dev   as for ccst_peak_continuous.
 *   g_dxdy_dev    device memory, n x 2 floats (dL/ddx, dL/ddy).
 *   g_frames_dev  device memory, n x H x W floats dL/dI (row-major, pitch W), or NULL.
 *   g_ref_dev     device memory, H x W floats dL/dE summed over the n frames, or NULL.
 * A frame whose status would be non-zero contributes zero gradient. The sum over frames
 * runs in per-CTA partials added in a fixed order: the result does not depend on timing.
 * Stream-ordered and asynchronous.
 * Errors: CCST_E_INVALID (n < 0, null pointers, pitch < W), CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_backward(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
                  const ccst_result* rec_dev, const float* g_dxdy_dev, float* g_frames_dev, float* g_ref_dev);

/* Set the context's reference from an FP64 image: image_dev is device memory, H x W
 * doubles, row-major with pitch W, holding E (the template itself, not the CC-SN offset
 * E + eps: the context adds eps for CC-SN). All resident copies of the reference spectrum
 * and operand are recomputed from it in the FP64 pipeline of the reference updates
 * (Sec. III; the same pipeline as ccst_set_reference_frame, with FP64 input). This is
 * how a caller moves the reference after a gradient step of its own (for example a
 * torch optimiser on dL/dE from ccst_backward). Power-of-two contexts only.
 * Stream-ordered. Errors: CCST_E_INVALID (null image), CCST_E_UNSUPPORTED (general
 * shape, no cooperative launch), CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_set_reference_image(ccst_ctx* ctx, const double* image_dev);

/* Refinement of the reference template by the adjoint of the displacement. It is not in
 * the paper, whose own reference refinements are the offline mean of Eq. (8) and the
 * real-time filter of Eq. (9). Here the template E is fitted to calibration frames whose
 * displacements d_i are known, by gradient descent on
 *   L(E) = (1/n) sum_i |s*_i(E) - d_i|^2
 * over the frames whose continuous peak s* (ccst_peak_continuous) has status 0.
 * dL/dE comes from ccst_backward with dL/ds*_i = 2 (s*_i - d_i) / n.
 * Starting from the context's current reference, each evaluation k = 0 .. steps does this:
 *   1. tracks every frame (ccst_track), then finds s* and L(E_k), then dL/dE;
 *   2. if L(E_k) exceeds the loss of the last accepted template, rejects E_k: it goes
 *      back to that template and its gradient, and halves the step h;
 *      otherwise it accepts E_k;
 *   3. unless k = steps, takes the step E <- E - h |E|_2 / |dL/dE|_2 dL/dE from the
 *      accepted template and sets the reference from it (ccst_set_reference_image).
 * At the end the context's reference is the last accepted template. Arguments:
 *   frames_dev    device memory, n frames (in_dtype) of H rows pitch_elems apart (0 = W).
 *   target_dev    device memory, n x 2 doubles, the known (dx, dy) of each frame.
 *   steps         gradient steps (>= 0); steps + 1 evaluations.
 *   step_rel      the first step h, relative to |E| (> 0); 0.01 suits 64 x 64 spots.
 *   hist_dev      device memory, 2 (steps + 1) doubles: for evaluation k, L(E_k) and the
 *                 step h that produced E_k.
 *   ref_out_dev   device memory for the final template, H x W doubles, or NULL.
 * The first call allocates a workspace for n frames (records, peaks, gradients and four
 * H x W images); a larger n later reallocates it after a stream synchronisation.
 * Everything runs on the context's stream, with no host synchronisation.
 * Power-of-two contexts only.
 * Errors: CCST_E_INVALID (n < 1, steps < 0, step_rel not finite and positive, null
 * pointers, pitch < W), CCST_E_UNSUPPORTED (general shape), CCST_E_NOMEM, CCST_E_CUDA. */
int ccst_refine_reference(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
                          const double* target_dev, int steps, double step_rel, double* hist_dev,
                          double* ref_out_dev);

/* Free everything the context owns. NULL is a no-op. Synchronises its stream first. */
void ccst_destroy(ccst_ctx* ctx);

/* Last error message of this context (or of the last failed create when ctx is NULL).
 * Valid until the next call on the same context. Never NULL. */
const char* ccst_last_error(ccst_ctx* ctx);

/* Profiling (CCST_FLAG_PROFILE): total device time of the FP32 tracking kernel
 * and the number of launches it covers. Each captured graph owns one event pair
 * and contributes its latest replay. Direct launches use a ring of 1024 pairs
 * and contribute every launch since the last reset. Synchronises the stream.
 * Errors: CCST_E_INVALID (profiling off, NULL pointers), CCST_E_CUDA. */
int ccst_profile_kernel_ms(ccst_ctx* ctx, double* sum_ms, int64_t* launches);
int ccst_profile_reset(ccst_ctx* ctx);

/* Number of grid points per axis of the refinement square, M = ceil(1.5 u)
 * (Sec. III); CCST_E_INVALID for a NULL context. */
int ccst_grid_size(ccst_ctx* ctx);

/* Diagnostic form of ccst_track, for tests.
 * It runs without graphs and, when the pointers are non-NULL, also writes:
 *   int_surf_dev  n x H x W floats: the FP32 integer surface H*W*c(s)
 *                 (unnormalised), s in 0..H-1 x 0..W-1 (Eq. (4)/(7));
 *   sub_surf_dev  n x M x M floats: the FP32 upsampled surface relative to the
 *                 integer peak, H*W*(cu(j) - cu(centre)), row = y offset (Sec. III).
 * Both buffers are caller-owned device memory. On a general-shape context with the FP32
 * general-size kernel (see ccst_create) the surfaces are that kernel's; a frame it sends
 * to the double-float kernel may leave them unwritten, and still gets its record.
 * Errors: as ccst_track; CCST_E_UNSUPPORTED on other general-shape contexts. */
int ccst_debug_surfaces(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
                        ccst_result* out_dev, float* int_surf_dev, float* sub_surf_dev);

/* Allocation-free tracking, for callers that must not allocate device memory
 * while they run.
 *
 * No counterpart in the paper: this is a deployment form of ccst_create +
 * ccst_track. Typical callers are a real-time camera or feedback loop that
 * reserves all GPU memory when it starts and cannot afford a cudaMalloc later
 * (it may synchronise the device and has no time bound), or a plug-in inside a
 * host program that owns the device's memory pool.
 *
 * It computes the same results as ccst_create(ref, H, W, p) followed by
 * ccst_track(frames, n, pitch, out). Everything the context would own
 * (reference spectra, upsampling tables, twiddles, the FP64 FFT workspace) is
 * rebuilt on each call inside one file-scope device array of 2 MiB per device.
 *
 * Arguments:
 *   ref_dev     H*W float32 reference, device memory.
 *   p           parameters; p->max_batch and CCST_FLAG_GRAPHS / CCST_FLAG_PROFILE
 *               are ignored. NULL means the defaults.
 *   frames_dev  device memory, laid out as for ccst_track.
 *   out_dev     n ccst_result records, device memory.
 *   n           any count >= 0.
 * The work is enqueued on p->stream and the call returns without waiting.
 *
 * Limits: H, W powers of two in [8, 128]. The scratch of the requested H, W and
 * upsample must fit in the 2 MiB array (128 x 128 fits up to upsample ~1000);
 * larger requests return CCST_E_SHAPE.
 *
 * Rules:
 *   - The first call on each device resolves the array's device address and sets
 *     the kernel's shared-memory limit. Make that first call before any stream
 *     capture.
 *   - Every call on a device shares the one array, which keeps the last call's
 *     contents; each call rewrites all of it before use. Calls whose GPU work
 *     overlaps (different streams, or different host threads) race on it and
 *     must be serialised by the caller.
 *   - No cudaMalloc, cudaFree or other allocating call is made, on the device or
 *     the host.
 * Errors: CCST_E_INVALID, CCST_E_SHAPE, CCST_E_UNSUPPORTED, CCST_E_CUDA; the message
 * is in ccst_static_last_error(). */
int ccst_track_static(const float* ref_dev, int H, int W, const ccst_params* p,
                      const void* frames_dev, int64_t n, int64_t pitch_elems,
                      ccst_result* out_dev);

/* FP32 FMA throughput of the current device, for the roofline of the tracking kernel.
 * Not in the paper: the paper's dense work (the FFTs of Eq. (4) and the upsampled DFT of
 * Sec. III) needs FP32 accuracy, so its bound is the rate of the FP32 FMA pipes.
 *   stream          cudaStream_t to run on (NULL = default stream); the call blocks until done.
 *   iters           loop trips of the timing kernel (each thread does iters x 128 FMAs;
 *                   about 20000 gives a 20 ms launch on a 148-SM B300).
 *   tflops          out: measured rate, the best of three timed launches after one warm-up
 *                   (every SM full, independent FMA chains), in TFLOP/s (1 FMA = 2 flop).
 *   nominal_tflops  out: SMs x 128 FP32 lanes x 2 x the device's reported peak clock.
 * Allocates nothing. Errors: CCST_E_INVALID (null outputs, iters < 1), CCST_E_CUDA. */
int ccst_fp32_fma_peak(void* stream, int iters, double* tflops, double* nominal_tflops);

/* Message of the last failed ccst_track_static call in this process. Never NULL. */
const char* ccst_static_last_error(void);

/* Diagnostic entry, for tests that calibrate the tie guard.
 * For frame f it computes v(jb) - v(ja) of the upsampled surface (Sec. III),
 * unnormalised and relative to the frame's integer peak, for the flat grid
 * indices ja = pairs_dev[2f] and jb = pairs_dev[2f+1], two ways:
 *   d32_dev[f]  by the FP32 pair-difference guard;
 *   d64_dev[f]  accumulated in FP64 from the same FP32 product spectrum (NaN on a
 *               general-shape context, whose FP32 general-size kernel has no such sum).
 * No tracking results are written. All buffers are caller-owned device memory.
 * Errors: as ccst_track, plus CCST_E_INVALID for NULL buffers; CCST_E_UNSUPPORTED on
 * general-shape contexts without the FP32 general-size kernel. */
int ccst_debug_pairs(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
                     const int32_t* pairs_dev, float* d32_dev, double* d64_dev);

/* Diagnostic copy of the context's FP64 reference operand, H x W doubles into ref_dev
 * (device memory): E for CC-U, 1 / (E + eps) for CC-SN. Stream-ordered.
 * Errors: CCST_E_INVALID (null buffer), CCST_E_CUDA. */
int ccst_debug_reference(ccst_ctx* ctx, double* ref_dev);

/* Diagnostic entry, for tests of the real-time update's bounded waits. It runs one
 * reference update for the frame frame_dev (record rec_dev) with grid barriers that wait
 * for one more CTA than the launch has, so every wait must run out (after 2^12 polls here;
 * 2^22 in normal runs).
 *   The record gains CCST_R_RT_STALE; so does every later ccst_rt_track record, and the
 *   reference is left as it was or partly updated, until ccst_rt_begin starts it again.
 * No fault is raised; the context stays usable.
 * Errors: CCST_E_INVALID (no ccst_rt_begin yet, null pointers, pitch < W), CCST_E_CUDA. */
int ccst_debug_rt_timeout(ccst_ctx* ctx, const void* frame_dev, int64_t pitch_elems, ccst_result* rec_dev);

/* Diagnostic entry, for tests of the kernel's bounded waits. It runs ccst_track's
 * kernel with the bulk copies of the stage tables withheld, so the wait for them must run
 * out (after 2^10 polls here; 2^22 in normal runs).
 *   Each frame a CTA reached gets CCST_R_TIMEOUT, and that CTA stops.
 *   Frames no CTA reached keep their previous out_dev contents.
 *   With n <= the number of SMs, every frame is reached.
 * No fault is raised; the context stays usable.
 * Errors: as ccst_track. */
int ccst_debug_timeout(ccst_ctx* ctx, const void* frames_dev, int64_t n, int64_t pitch_elems,
                       ccst_result* out_dev);

#ifdef __cplusplus
}
#endif

#endif /* CCST_H */
