/*
 * bf_gp.h -- C ABI of the GB300 (sm_103a) Gauss-polynomial bilateral filter.
 *
 * Method: K. N. Chaudhury, "Fast and Accurate Bilateral Filtering using
 * Gauss-Polynomial Decomposition".  The Gaussian bilateral filter of Eq. (1)
 * (kernels of Eq. (2)) is approximated by replacing the translated range
 * kernel with its Gauss-polynomial of degree N (Eqs. (3)-(5)).  The filter
 * then becomes K = N + 2 spatial Gaussian filterings of the auxiliary images
 * of Eq. (7) (Eq. (8)), a per-pixel combine (Eqs. (9)-(10)) and a division
 * (Eq. (11)), after centring the intensities at t_c (Sec. 2, Eq. (6)).
 * Algorithm 1 lists the steps.
 *
 * Implementation form (mathematically identical to Eqs. (7)-(11)): with
 * h = f - t_c, R = max |h|, u = h / R in [-1, 1], s^2 = (R / sigma_r)^2,
 * E = exp(-s^2 u^2 / 2) and channels Phi_k = E u^k (k = 0..N+1),
 *     Q = sum_{n=0..N} (s^2 u)^n / n! * S Phi_n,
 *     P = sum_{n=0..N} (s^2 u)^n / n! * S Phi_{n+1},
 *     y = t_c + R * P / Q,
 * where S is the separable spatial Gaussian (truncated FIR on the window
 * [-w, w], w = ceil(3 sigma_s) by default (Sec. 1), or Deriche's recursive
 * Gaussian named in Sec. 3), each applied with zero extension at the image
 * border.  Everything on the device runs in FP32; FP64 is used only for the
 * expansion coefficients, the centre/scale and the filter coefficients.
 *
 * Conventions for every entry point below:
 *  - Pointers marked "device" must point to device memory of the current
 *    CUDA device; "host" pointers to host memory.  The caller owns every
 *    buffer; the library never allocates device memory.
 *  - Images are FP32, `planes` planes of H rows x W columns, row-major.
 *    Row r of plane c starts at  base + (c * H + r) * pitch  (elements), so
 *    planes are stacked with stride H * pitch; pitch >= W.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *    device work is enqueued asynchronously on it; the call returns after
 *    enqueueing.  Argument errors are detected on the host before anything
 *    is enqueued and returned synchronously.
 *  - The workspace `ws` (device, 256-byte aligned, size from
 *    bf_gp_workspace_size) is scratch owned by the caller.  It must not be
 *    used by two calls that run concurrently.  It also carries the device
 *    status word of the last call (bf_gp_get_device_status).
 *  - No entry point synchronises the device unless it says so.
 */
#ifndef BF_GP_H
#define BF_GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BF_OK = 0,
    BF_ERR_INVALID_ARG = 1,  /* null or misaligned (not 4-byte) pointer, bad size, sigma or order */
    BF_ERR_WORKSPACE = 2,    /* workspace too small or misaligned */
    BF_ERR_CUDA = 3,         /* a CUDA runtime call failed (see bf_gp_last_cuda_error) */
    BF_ERR_UNSUPPORTED = 4,  /* valid request outside what the kernels cover (e.g. a line too long) */
    BF_ERR_TIMEOUT = 5       /* a bounded device wait gave up (see the device status bits) */
} bf_status;

/* Bits of the device status word, set by the kernels of the last call. */
#define BF_DEV_NONPOS_Q 0x1u      /* some pixel had Q <= 0, where Eq. (11) is undefined (odd N; with the recursive filter, whose kernel has a slightly negative tail, also large (R/sigma_r)^2): it kept its own value */
#define BF_DEV_NONFINITE_IN 0x2u  /* the input held NaN/Inf; the plane was passed through unchanged */
#define BF_DEV_RANGE 0x4u         /* (R/sigma_r)^2 / 2 > 80: exp(-s^2 u^2 / 2) underflows FP32 */
#define BF_DEV_TIMEOUT 0x8u       /* a bounded inter-block wait gave up */

typedef enum {
    BF_SPATIAL_AUTO = 0, /* FIR for w <= 12, recursive otherwise */
    BF_SPATIAL_FIR = 1,  /* window sum of Eq. (8), taps exp(-d^2 / 2 sigma_s^2), |d| <= w */
    BF_SPATIAL_IIR = 2,  /* Deriche's 4th-order recursive Gaussian, causal + anticausal */
    BF_SPATIAL_BOX = 3   /* the paper's constant-time alternative (Sec. 3: any constant-time filter,
                            e.g. a box): box_passes passes of a flat kernel of half-width r
                            (fir_halfwidth, or chosen so that box_passes ((2r + 1)^2 - 1) / 12 is
                            closest to sigma_s^2), zero extension; box_passes * r <= 12; forward
                            (bf_gp_forward, fused kernel) only */
} bf_spatial;

typedef enum {
    BF_CENTRE_MEAN = 0,  /* t_c = mean of the plane (Algorithm 1, first step) */
    BF_CENTRE_GIVEN = 1  /* t_c = opts.t_c for every plane */
} bf_centre;

typedef struct {
    int order;          /* N >= 0, N <= 62 (K = N + 2 channels).  The paper uses N = 20 (Sec. 4). */
    int spatial;        /* bf_spatial */
    int centre;         /* bf_centre */
    int fir_halfwidth;  /* w for FIR; 0 selects ceil(3 sigma_s) (Sec. 1) */
    double t_c;         /* centre when centre == BF_CENTRE_GIVEN */
    int engine;         /* recursive filter only: how the chunk-local products run.
                           0 = auto (row pass on mma.sync tensor cores, column pass on CUDA cores: the
                               fastest pair measured on GB300; the backward's row pass on CUDA cores,
                               faster for it), 1 = FP32 CUDA cores for both passes,
                           2 = mma.sync tensor cores (TF32 x 3 products) for both passes,
                           3 = column pass on tcgen05 (TF32 x 3, accumulators in tensor memory),
                               row pass on CUDA cores */
    int fir_two_pass;   /* FIR forward only: 0 = one fused kernel per output tile (channels, row and
                           column filters and combine in shared memory, no row-filtered planes in
                           HBM), 1 = the separate row and column passes (what bf_gp_phase_rows /
                           bf_gp_phase_cols always run) */
    int box_passes;     /* BF_SPATIAL_BOX: passes of the flat kernel, 1..3 (0 selects 3) */
    int tc5_wait_test;  /* engine 3 only, to test its bounded wait: 0 = normal; n > 0 = the column pass
                           issues no tensor-core product and gives up each wait for one after n polls:
                           the call reports BF_DEV_TIMEOUT and writes every plane as copied */
    int row_threads;    /* threads per CTA of the row pass (recursive filter, two-pass FIR): 0 = the
                           default (256, or one row when a row needs more); 256 or 512.  A CTA holds
                           row_threads / (threads per row) rows.  The autotuner chooses it */
    int fir_tile;       /* fused FIR forward: output tile height, 0 (= 32), 16, 32 or 64 rows, tile
                           width 32; a taller tile shares its halo among more outputs, a shorter one
                           gives small images more CTAs.  The autotuner chooses it */
    int reserved[2];    /* must be zero */
} bf_gp_opts;

/* Fill *opts with the defaults: N = 20, AUTO spatial operator, mean centre. */
void bf_gp_default_opts(bf_gp_opts *opts);

/* Human-readable name of a status code (static string). */
const char *bf_status_string(bf_status s);

/* Text of the last CUDA error seen by this thread's calls (static buffer). */
const char *bf_gp_last_cuda_error(void);

/* Library version, e.g. 100 for 0.1.0. */
int bf_gp_version(void);

/*
 * Workspace bytes a forward call on `planes` planes of H x W needs with these
 * options (sigma_s matters only for the spatial-operator choice; pass the
 * value you will use).  Returns BF_ERR_INVALID_ARG for bad sizes and
 * BF_ERR_UNSUPPORTED outside the sizes the kernels cover: W <= 8192 (a row is
 * at most 512 threads of 16 samples); with the recursive filter a column is
 * one thread-block cluster of 512-row CTAs, so H <= 8192 with engines 0 and 1
 * (clusters of more than 8 CTAs use the non-portable cluster size; a device
 * that cannot hold such a cluster makes the call return BF_ERR_UNSUPPORTED)
 * and H <= 4096 with engines 2 and 3; FIR half-width <= 12; box passes x
 * half-width <= 12.
 */
bf_status bf_gp_workspace_size(int planes, int H, int W, float sigma_s, const bf_gp_opts *opts,
                               size_t *bytes);

/*
 * Forward filter (Algorithm 1 / Eqs. (7)-(11)).
 *   f     device, input,  planes x H x W at `pitch` (elements)
 *   y     device, output, same layout and pitch; may not alias f
 *   sigma_s > 0 (finite), sigma_r > 0 (+inf allowed: plain normalised Gaussian)
 *   opts  may be NULL (defaults)
 * Each plane is filtered independently with its own centre t_c and scale R.
 * A constant plane (R = 0) is copied.  A plane holding NaN/Inf is copied and
 * BF_DEV_NONFINITE_IN is raised.
 */
bf_status bf_gp_forward(const float *f, float *y, int planes, int H, int W, int pitch,
                        float sigma_s, float sigma_r, const bf_gp_opts *opts,
                        void *ws, size_t ws_bytes, void *stream);

/*
 * The three phases of bf_gp_forward as separate calls, for per-kernel timing
 * and for testing each half of the separable filter.  Same arguments as
 * bf_gp_forward; calling stats, rows and cols in this order on one stream
 * with one workspace is exactly bf_gp_forward.
 *   stats: Algorithm 1 step 1 (centre t_c = mean) plus min/max -> R, s^2 and
 *          the per-channel scale factors, written into ws.
 *   rows:  steps 2-4, 7, 12 (channels Phi_k = E u^k generated on the fly) and
 *          the row half of steps 8 and 13 (Eq. (8)); K row-filtered planes
 *          are written into ws.
 *   cols:  the column half of Eq. (8) fused with the sums of Eqs. (9)-(10)
 *          and the division of Eq. (11) (steps 11, 14-16, 18); writes y.
 */
bf_status bf_gp_phase_stats(const float *f, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                            const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream);
bf_status bf_gp_phase_rows(const float *f, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                           const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream);
bf_status bf_gp_phase_cols(const float *f, float *y, int planes, int H, int W, int pitch, float sigma_s,
                           float sigma_r, const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream);

/*
 * Joint (cross) bilateral filter: Eq. (1) with the range kernel evaluated on a
 * guide image g and the weights applied to the data image f (the extension
 * the paper's conclusion names).  By the same decomposition (Eqs. (3)-(5)) on
 * the centred guide, with u = (g - t_c) / R, E = exp(-s^2 u^2 / 2) and
 * d = (f - t_c) / R:
 *   y = t_c + R (sum_n a_n S(E u^n d)) / (sum_n a_n S(E u^n)),  a_n = (s^2 u)^n / n!,
 * i.e. K = 2 (N + 1) filterings (so N <= 31).  t_c and R are the guide's
 * (mean or the given centre; R = max |g - t_c|); a constant guide gives the
 * normalised Gaussian filter of f; a guide with NaN/Inf passes f through and
 * raises BF_DEV_NONFINITE_IN.  f, g, y: device, layout and pitch of
 * bf_gp_forward, y may alias neither input.  Recursive filter or FIR (two
 * passes) with the CUDA-core kernels (opts.engine and opts.fir_two_pass are
 * not used).  ws: bf_gp_joint_workspace_size bytes.  Async on `stream`.
 */
bf_status bf_gp_joint_workspace_size(int planes, int H, int W, float sigma_s, const bf_gp_opts *opts,
                                     size_t *bytes);
bf_status bf_gp_forward_joint(const float *f, const float *g, float *y, int planes, int H, int W, int pitch,
                              float sigma_s, float sigma_r, const bf_gp_opts *opts, void *ws, size_t ws_bytes,
                              void *stream);

/*
 * Training support (no counterpart in the paper, which has no derivative):
 * reverse-mode derivative of bf_gp_forward with respect to the image and
 * sigma_r.
 *
 * bf_gp_forward_train: bf_gp_forward that also writes, per pixel, the four
 *   sums the backward pass needs into `saved` (device, 4 * planes * H * W
 *   floats, layout [planes][4][H][W], dense).  A constant plane is filtered
 *   (result equal to its value) instead of copied, so its derivative exists.
 *
 * bf_gp_backward: given grad_y = dL/dy (device, layout and pitch of f),
 *   writes grad_f = dL/df (device, same layout; may not alias f) and, if
 *   grad_sigma_r is not NULL, dL/dsigma_r per plane (device, planes floats).
 *   f, saved, sigma_s, sigma_r and opts must be those of the matching
 *   bf_gp_forward_train call; ws needs bf_gp_workspace_size bytes (it may be
 *   the forward's workspace; its contents are not needed).  The derivative of
 *   the centre t_c (the plane mean, Algorithm 1 step 1) is included; a given
 *   centre is held fixed.  R gets no derivative (the result does not depend
 *   on it).  A pixel whose forward kept its own value (Q <= 0) passes dL/dy
 *   to its own input (dy/df = 1 there) and nothing else.
 *   Enqueues four kernels: stats, adjoint row pass, adjoint column pass
 *   (the same spatial operator, which is symmetric), finish.
 */
bf_status bf_gp_forward_train(const float *f, float *y, float *saved, int planes, int H, int W, int pitch,
                              float sigma_s, float sigma_r, const bf_gp_opts *opts, void *ws, size_t ws_bytes,
                              void *stream);
bf_status bf_gp_backward(const float *f, const float *grad_y, const float *saved, float *grad_f,
                         float *grad_sigma_r, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                         const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream);

/*
 * Forward filter on HOST buffers: brings f (host) into the device workspace
 * and runs bf_gp_forward there, all on `stream`; returns once the result is
 * in y (host) (it synchronises `stream`).  A buffer "mapped" here is 4-byte
 * aligned and lies wholly in pinned host memory mapped into the device's
 * address space (cudaHostAlloc, or cudaHostRegister with
 * cudaHostRegisterMapped).  A mapped f is read by the statistics pass itself,
 * which stores the device copy; any other f is copied first.  A mapped y
 * receives the result straight from the last pass, overlapping the transfer
 * with the pass; any other y gets it from a copy of a staged result.  Either
 * way y gets the same bytes as bf_gp_forward's device output, and nothing
 * outside y's planes * H * W floats is written.
 * ws must hold bf_gp_workspace_size(...) + 2 * planes * H * W * 4 bytes
 * (bf_gp_host_workspace_size).  pitch of the host buffers is W.
 */
bf_status bf_gp_host_workspace_size(int planes, int H, int W, float sigma_s, const bf_gp_opts *opts,
                                    size_t *bytes);
bf_status bf_gp_forward_host(const float *f_host, float *y_host, int planes, int H, int W,
                             float sigma_s, float sigma_r, const bf_gp_opts *opts,
                             void *ws, size_t ws_bytes, void *stream);

/*
 * Forward filter for callers that cannot allocate device memory.  The paper
 * has no counterpart; this is a calling convenience.
 *
 * Some callers can't call cudaMalloc and can't be handed a workspace: plug-in
 * hosts that give a filter only its input and output buffers, code running
 * while a stream is being captured (where allocation is not allowed), and
 * latency-bound loops where cudaMalloc/cudaFree would synchronise the device.
 * This entry point takes the same arguments as bf_gp_forward minus the
 * workspace and uses instead one scratch array of BF_GP_NOALLOC_SCRATCH_BYTES
 * that lives in the library itself (a static device array: every GPU that
 * loads the library holds it until the process exits).  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 *  - Limit: the request needs bf_gp_workspace_size(planes, H, W, sigma_s,
 *    opts) bytes of scratch; anything above BF_GP_NOALLOC_SCRATCH_BYTES is
 *    rejected with BF_ERR_WORKSPACE before anything is enqueued (the reason is
 *    also in bf_gp_last_cuda_error()).  With N = 20 that is about 380 000
 *    pixels per call (e.g. one 512 x 512 plane, or three 256 x 256 planes).
 *  - Set-up: the first call on a device looks up the array's device address
 *    (with that device current) and caches it; make that first call before
 *    any stream capture.  Later calls check the cached address against the
 *    current context and look it up again after a cudaDeviceReset.
 *  - Sharing: every call on a device uses the same array, which keeps the
 *    previous call's contents; the filter writes every scratch byte it reads
 *    before reading it, so nothing needs clearing.  Calls that overlap on the
 *    GPU (different streams, threads or processes sharing the context) race
 *    on the array: serialise them.  bf_gp_get_device_status and
 *    bf_gp_get_plane_stats cannot reach this scratch.
 */
#define BF_GP_NOALLOC_SCRATCH_BYTES (32u << 20)
bf_status bf_gp_forward_noalloc(const float *f, float *y, int planes, int H, int W, int pitch,
                                float sigma_s, float sigma_r, const bf_gp_opts *opts, void *stream);

/*
 * Batched filtering: many planes of different sizes, each with its own
 * sigma_s, sigma_r and order, filtered with the recursive Gaussian: every
 * plane's forward (the launches of bf_gp_forward) on a few streams, one
 * graph-capturable call.  Same method and per-plane result as bf_gp_forward
 * with BF_SPATIAL_IIR (the paper filters one image at a time; batching is an
 * implementation choice).
 *
 *   bf_gp_batched_plan_create: validates the planes (the limits of
 *     bf_gp_forward with BF_SPATIAL_IIR; pitch >= W; f, y device pointers
 *     that stay valid while the plan is used) and builds the per-plane tables
 *     on the host (filter coefficients in FP64 rounded to FP32).  opts.spatial
 *     must be AUTO or IIR; opts.order is ignored (each plane's own order is
 *     used); the centre and engine options apply to every plane (until
 *     bf_gp_batched_plan_tune picks an engine per plane).  The plan
 *     owns host memory and BF_GP_BATCH_STREAMS CUDA streams and events of the
 *     current device (released by bf_gp_batched_plan_destroy).
 *   bf_gp_batched_plan_workspace: device bytes the plan needs (tables and
 *     every plane's bf_gp_workspace_size).
 *   bf_gp_batched_plan_upload: copies the tables into ws (synchronises
 *     `stream`); must be called once per workspace before bf_gp_batched.
 *   bf_gp_batched: enqueues every plane's forward (statistics, row pass,
 *     column pass: the launches of bf_gp_forward, in its own part of ws) on the
 *     plan's streams, which fork from `stream` and join back into it, then
 *     one launch on `stream` that ORs the planes' status words into ws's.  No
 *     copies and no host synchronisation, so the call can be captured into a
 *     CUDA graph (the fork and join become graph dependencies) and replayed.
 *     ws must be the uploaded workspace; calls on one plan must not overlap.
 *   bf_gp_batched_plan_destroy: frees the plan.
 *
 * Per-plane centre and scale, for choosing each plane's order before the
 * plan that filters (the error of Eq. (5) on [-R, R] depends on R / sigma_r,
 * and R is known only from the data):
 *   bf_gp_batched_plan_stats_workspace: device bytes bf_gp_batched_plane_stats
 *     needs (tables and statistics only, no channel planes).
 *   bf_gp_batched_plane_stats: runs the plan's statistics pass (Algorithm 1
 *     step 1 and the scale R = max |f - t_c|) in ws, waits for it and writes
 *     t_c[i] and R[i] for each of the plan's n planes (host arrays, n
 *     entries, either may be NULL).  It uploads its own copy of the tables
 *     into ws; ws needs no other preparation and is not usable by
 *     bf_gp_batched afterwards unless uploaded again.  Pair it with
 *     bf_gp_order_for_tol(sigma_r, R[i], eps) and a second plan created with
 *     those orders.
 */
typedef struct {
    const float *f;  /* device input plane */
    float *y;        /* device output plane (may not alias f) */
    int H, W, pitch;
    float sigma_s, sigma_r;
    int order;
} bf_gp_plane;

typedef struct bf_gp_plan bf_gp_plan;
#define BF_GP_BATCH_STREAMS 8

bf_status bf_gp_batched_plan_create(const bf_gp_plane *planes, int n, const bf_gp_opts *opts, bf_gp_plan **out);
bf_status bf_gp_batched_plan_workspace(const bf_gp_plan *plan, size_t *bytes);
bf_status bf_gp_batched_plan_upload(bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream);
bf_status bf_gp_batched(const bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream);
void bf_gp_batched_plan_destroy(bf_gp_plan *plan);
bf_status bf_gp_batched_plan_stats_workspace(const bf_gp_plan *plan, size_t *bytes);
bf_status bf_gp_batched_plane_stats(const bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream, double *t_c,
                                    double *R);

/*
 * Autotuner.  The engines of the recursive filter (opts.engine 0..3) and the
 * fused or two-pass form of the FIR filter (opts.fir_two_pass) compute the
 * same filter with different kernels; which is fastest depends on the shape.
 *
 *   bf_gp_autotune: for the shape class of the call (device, planes, H, W,
 *     pitch, the spatial operator opts resolves to, K and the FIR half-width)
 *     returns the fastest candidate in opts->engine / opts->fir_two_pass (the
 *     other fields are left as given).  On the first call for a class it
 *     times every candidate the workspace can hold: one untimed forward, then
 *     `reps` forwards (<= 0 selects 5) between two CUDA events on `stream`,
 *     on the caller's f, y and ws (y is overwritten), and waits for them;
 *     later calls return the stored choice without launching anything.  ms
 *     (NULL, or BF_GP_TUNE_CANDIDATES floats) gets each candidate's mean time
 *     in milliseconds in candidate order (recursive: engine e with row_threads
 *     256 at 2 e and 512 at 2 e + 1; FIR: fused with 32-row tiles, two-pass
 *     with 256 and with 512 row threads, fused with 16- and with 64-row
 *     tiles), -1 where nothing was timed.  The choice (engine or FIR form,
 *     row_threads and fir_tile) is written into opts.  Not capturable into a graph.
 *     BF_ERR_UNSUPPORTED if no candidate runs.
 *   bf_gp_autotune_clear: forgets every stored choice.
 *   bf_gp_batched_plan_tune: runs bf_gp_autotune for every plane of an
 *     uploaded plan (on the plane's own buffers and part of ws, so the planes'
 *     outputs are overwritten) and makes bf_gp_batched use each plane's choice.
 *   bf_gp_batched_plan_engines: the engine each plane runs with (n entries).
 */
#define BF_GP_TUNE_CANDIDATES 8
bf_status bf_gp_autotune(const float *f, float *y, int planes, int H, int W, int pitch, float sigma_s,
                         float sigma_r, bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream, int reps,
                         float *ms);
void bf_gp_autotune_clear(void);
bf_status bf_gp_batched_plan_tune(bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream, int reps);
bf_status bf_gp_batched_plan_engines(const bf_gp_plan *plan, int *engines);

/*
 * Batched filtering in one persistent launch.  The same per-plane forward as
 * bf_gp_batched with engine 0 (tensor-core row pass, CUDA-core column pass,
 * the recursive Gaussian of Sec. 3 applied along rows then columns, Algorithm
 * 1), run by one launch of resident thread-block clusters that take work
 * items from a counter in ws: every plane's statistics partials, then its
 * centre and scale, its row groups, its column strips, in that order.  An
 * item that needs an earlier one (the row pass needs the plane's centre, the
 * column pass all of its rows) waits on that plane's readiness counter in ws
 * for at most a bounded number of clock cycles; a wait that gives up sets
 * BF_DEV_TIMEOUT in the plane's status word, counts one in its counter 3 and
 * skips the item (its output is then not written), so the launch always
 * ends.  Each plane's status word and counters are then gathered into ws's,
 * as bf_gp_batched does.
 *
 *   bf_gp_batched_persistent: enqueues a zeroing of the counters, the
 *     persistent launch and the gather on `stream`; no host synchronisation,
 *     graph-capturable.  ws must be the workspace the plan was uploaded to
 *     (bf_gp_batched_plan_upload), at least bf_gp_batched_plan_workspace
 *     bytes (BF_ERR_WORKSPACE otherwise).  BF_ERR_UNSUPPORTED when a plane
 *     has rows of more than 4096 samples or more than 4096 rows (the one
 *     launch's CTA and cluster shapes), or when no cluster fits on the device.
 *     The per-plane results equal bf_gp_batched's with engine 0 bit for bit
 *     (same kernels' arithmetic in the same order).  Calls on one plan must
 *     not overlap, nor overlap bf_gp_batched on the same workspace.
 *   bf_gp_batched_plan_set_wait: the wait budget of one readiness wait in SM
 *     clock cycles (>= 1; the plan starts with 2^32, about two seconds), and,
 *     for testing the timeout, a plane (0..n-1; -1 for none) whose column
 *     items wait for one row group more than the plane has, so that they give
 *     up.  BF_ERR_INVALID_ARG for a budget < 1 or a plane out of range.
 */
bf_status bf_gp_batched_persistent(const bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream);
bf_status bf_gp_batched_plan_set_wait(bf_gp_plan *plan, long long wait_cycles, int starve_plane);

/*
 * Read the device status word written by the last call that used `ws`
 * (BF_DEV_* bits).  Synchronises `stream` first.
 */
bf_status bf_gp_get_device_status(const void *ws, void *stream, uint32_t *bits);

/*
 * Counts behind the status bits of the last call that used `ws` (for a batch:
 * summed over its planes), into counters[BF_GP_NCOUNTERS]:
 *   [0] pixels whose Q <= 0 (they kept their own value; BF_DEV_NONPOS_Q)
 *   [1] non-finite input values (BF_DEV_NONFINITE_IN)
 *   [2] planes whose exponentials leave the FP32 range (BF_DEV_RANGE)
 *   [3] bounded waits that gave up (BF_DEV_TIMEOUT)
 * Synchronises `stream` first.
 */
#define BF_GP_NCOUNTERS 4
bf_status bf_gp_get_device_counters(const void *ws, void *stream, unsigned long long *counters);

/*
 * Read back, for plane `plane` of the last forward call that used `ws`, the
 * centre t_c and the scale R the device computed (FP64).  Synchronises
 * `stream`.
 */
bf_status bf_gp_get_plane_stats(const void *ws, int plane, void *stream, double *t_c, double *R);

/*
 * The order rule offered when the caller wants a kernel accuracy rather than
 * a fixed N (the paper fixes N = 20 and leaves the choice open, Sec. 4):
 * the smallest even N such that for all t, tau in [-R, R]
 *     | g_{sigma_r}(t - tau) - GP_N(t, tau) | <= eps,
 * with GP_N the Gauss-polynomial of Eq. (5), evaluated in FP64 on a grid of
 * the interval.  Returns -1 if no N <= 62 reaches eps.  Host only.
 */
int bf_gp_order_for_tol(double sigma_r, double R, double eps);

/* Largest even order N <= 62 for which a plane with scale R = max |f - t_c|
 * keeps every term beta_k Phi_k of the scaled channels inside FP32 (the
 * statistics pass raises BF_DEV_RANGE beyond it; this host copy of that test
 * keeps one bit of margin), or -1 if none does.  The Taylor terms of Eq. (4)
 * grow like (s^2)^n / n! with s^2 = (R / sigma_r)^2, so large R / sigma_r
 * bounds the order FP32 can carry. */
int bf_gp_order_fp32_limit(double sigma_s, double sigma_r, double R);

#ifdef __cplusplus
}
#endif

#endif /* BF_GP_H */
