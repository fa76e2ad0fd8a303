/*
 * ppf.h -- C ABI of the GB300 SIR particle filter for single-spot tracking
 * ("PPF - A Parallel Particle Filtering Library", Demirel et al.).
 *
 * One context = one particle filter of N particles on the current CUDA
 * device.  The library owns every particle buffer (allocated in ppf_create);
 * frames are caller-owned.  Every call returns a ppf_status; nothing throws
 * across the ABI.  Unless stated otherwise a call only enqueues work on the
 * context's stream and returns at once; device-side failures found by the
 * kernels are reported by the next synchronising call (ppf_estimate).
 *
 * Layouts:
 *   frame      row-major H x W (pixel (i, j) = column i <-> x, row j <-> y,
 *              centres at integer coordinates), element type model.frame_dtype.
 *   state      structure of arrays, 6 x N float32: x, y, vx, vy, I0, lw
 *              (lw = unnormalised log-weight).
 *   ancestors  N int32: slot i of the next propagation takes particle anc[i].
 */
#ifndef PPF_H
#define PPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PPF_OK = 0,
    PPF_EINVAL = 1,      /* bad argument (size, radius, pointer, scheme)        */
    PPF_ENOMEM = 2,      /* device or host allocation failed                    */
    PPF_ECUDA = 3,       /* a CUDA runtime call failed (see ppf_last_error)      */
    PPF_ETIMEOUT = 4,    /* a bounded device-side wait gave up: the binned
                            likelihood waits (about a second at most) for the
                            tensor copies of its tile windows; no kernel waits
                            on another.  The host fault injection
                            PPF_FAULT=timeout makes ppf_estimate report it   */
    PPF_EDEGENERATE = 5, /* every weight was zero or NaN: nothing was resampled */
    PPF_ESTATE = 6       /* call out of order (e.g. resample before a step)     */
} ppf_status;

/* Resampling schemes (Alg. 1 resampling step; Sec. 3; Sec. 4). */
typedef enum {
    PPF_SYSTEMATIC = 0, /* global systematic resampling                        */
    PPF_RPA_GS = 1,     /* proportional allocation + Greedy Scheduler (Alg. 2)  */
    PPF_RPA_SGS = 2,    /* proportional allocation + Sorted Greedy (Alg. 3)     */
    PPF_RPA_LGS = 3,    /* proportional allocation + Largest Gradient (Alg. 4)  */
    PPF_RNA = 4,        /* non-proportional allocation + ring migration (Sec. 3)*/
    /* Two-stage proportional allocation (Sec. 3 RPA, in the stratified form
     * of Bolic et al.): group g receives the same number N_g of offspring as
     * with one global draw (so the same schedules and routing), but draws
     * them inside the group with its own systematic offset. */
    PPF_RPA2_GS = 5,
    PPF_RPA2_SGS = 6,
    PPF_RPA2_LGS = 7,
    /* Adaptive RNA (Sec. 7, described there in words only; the reading
     * taken): RNA whose exchange ratio is exchange_ratio * (1 - |I| / G),
     * I the groups that proportional allocation (the global systematic
     * tickets of RPA) would give at least their own size, and whose ring is
     * a permutation of the groups kept between calls.  When the step's
     * log-evidence is negative (the object counts as lost) the ring is first
     * redrawn: the groups in increasing order of the first Philox word of
     * (seed; g, frame, filter, 4), ties by group index.  At most 16384
     * groups. */
    PPF_ARNA = 8
} ppf_scheme;

typedef enum { PPF_F32 = 0, PPF_BF16 = 1, PPF_F16 = 2 } ppf_dtype;

/* Model of Sec. 7: NCV dynamics (7.1), Gaussian-PSF appearance eq. 3 and
 * patch likelihood eq. 4 (7.2).  All lengths in pixels, per frame. */
typedef struct {
    int32_t width, height;    /* frame size W, H                                 */
    int32_t patch_radius;     /* r: S_x is the (2r+1)^2 box around the particle, 0..8 */
    int32_t frame_dtype;      /* ppf_dtype of the frames given to ppf_step       */
    float psf_sigma;          /* sigma_PSF of eq. 3                              */
    float amplitude;          /* prior scale of I0: I0 ~ U[A/2, 3A/2]            */
    float background;         /* I_bg of eq. 3                                   */
    float sigma_xi;           /* sigma_xi of eq. 4                               */
    float sigma_m;            /* position noise std                              */
    float sigma_v;            /* velocity noise std                              */
    float sigma_I;            /* intensity noise std                             */
    float v0_max;             /* prior velocity range: v ~ U[-v0, v0]            */
    uint64_t seed;            /* Philox key                                      */
    uint32_t filter_id;       /* Philox counter word 2 (independent filters)     */
    uint32_t likelihood;      /* 0: eq. 4 at the particle's position;
                                 1: pcSIR (Sec. 6), the likelihood held constant
                                    on every pixel cell at its value for the
                                    cell centre c = floor((x, y) + 1/2): one
                                    lookup per particle in a per-frame map of
                                    the patch sums of every anchor.  Not for
                                    ppf_loglik_grad or batches.                 */
} ppf_model;

/* Per-frame results (Alg. 1 normalisation / N_eff; MMSE estimate of Sec. 2). */
typedef struct {
    double mean[5];           /* posterior mean of x, y, vx, vy, I0 (before resampling) */
    double log_evidence;      /* log sum e^lw - log sum e^lw_prev (eq. 4 scale)  */
    double ess;               /* 1 / sum w_i^2                                   */
    double max_log_weight;    /* max_i lw_i                                      */
    int32_t frame;            /* frame index of the last ppf_step                */
    int32_t status_flags;     /* bit 0 degenerate weights, 1 wait timeout,
                                 2 inconsistent routing (copy skipped),
                                 3 caller ancestor out of range (identity used),
                                 4 resampling skipped by the N_eff test
                                   (ppf_resample_if),
                                 5 ARNA redrew its ring (object lost)           */
    int64_t links;            /* routing links of the last resample (Sec. 4-5)   */
    int64_t moved;            /* particles moved between groups by that resample */
    int64_t max_group;        /* largest / smallest group after it               */
    int64_t min_group;
} ppf_estimate_t;

typedef struct ppf_ctx ppf_ctx;

/* Alg. 1 initialisation (k = 0): allocates the context and draws N particles
 * uniformly (Sec. 7.3): x, y ~ U[-1/2, W-1/2) x U[-1/2, H-1/2),
 * v ~ U[-v0, v0]^2, I0 ~ U[A/2, 3A/2], equal weights.
 *   model       host pointer, copied.
 *   n           1 <= n <= 2^31 - 1 particles.
 *   group_size  particles per group (the paper's process, Sec. 3); the groups
 *               are a balanced partition of the N slots, ceil(N/group_size)
 *               of them; 1 <= group_size <= n.
 *   cuda_stream cudaStream_t to enqueue on (NULL = legacy default stream).
 *   out         receives the context; untouched on error.
 * Errors: PPF_EINVAL (sizes, radius > 8, non-positive sigma_PSF / sigma_xi,
 * unknown dtype), PPF_ENOMEM, PPF_ECUDA.  No context exists after an error,
 * so there is no ppf_last_error text; with the environment variable
 * PPF_VERBOSE set, the failing step is printed to stderr. */
ppf_status ppf_create(const ppf_model *model, int64_t n, int32_t group_size,
                      void *cuda_stream, ppf_ctx **out);

/* Frees every buffer of the context (synchronises its stream).  NULL is a no-op. */
void ppf_destroy(ppf_ctx *ctx);

/* One SIS step of Alg. 1 for frame k: every slot draws its particle from the
 * dynamics applied to its ancestor (bootstrap proposal), is weighted by the
 * patch likelihood eq. 4, and the weights are normalised (log-sum-exp with an
 * FP64 cross-group total), giving the estimate, N_eff and log-evidence.
 *   frame_dev   device pointer, H x W of model.frame_dtype; must stay valid
 *               until the stream has run the step.
 *   k           frame index (counter word of the random stream), k >= 1.
 * A step that follows another step without ppf_resample keeps the weights
 * (pure SIS).  Errors: PPF_EINVAL (NULL frame, k < 1), PPF_ECUDA. */
ppf_status ppf_step(ppf_ctx *ctx, const void *frame_dev, int32_t k);

/* ppf_step for a frame in host memory (H x W of model.frame_dtype).  The
 * frame is copied into one of two library-owned device buffers on a second,
 * library-owned stream, so that the copy of one frame overlaps the kernels of
 * the previous one; the step waits for its copy.  With page-locked memory the
 * call returns before the copy has run and frame_host must stay valid until
 * the context's stream has run the step; with pageable memory the copy is
 * synchronous.  Not for stream capture (the copy stream is not captured). */
ppf_status ppf_step_host(ppf_ctx *ctx, const void *frame_host, int32_t k);

/* The resampling step of Alg. 1 on the weights of the last step, using the
 * scheme's allocation (Sec. 3) and, for RPA, the scheme's routing schedule
 * (Sec. 4).  exchange_ratio: RNA, the fraction alpha of the smallest group
 * that migrates to the next group of the ring; ARNA, the largest such
 * fraction (0 <= alpha <= 1; ignored by the other schemes).
 * Systematic and RPA reset the weights to equal; RNA gives every offspring
 * its group's weight / group size.  LGS may leave the groups unequal.
 * Errors: PPF_ESTATE (no step since the last resample), PPF_EINVAL, PPF_ECUDA.
 * All-zero or NaN weights are reported as PPF_EDEGENERATE by the next
 * ppf_estimate; the particles are then kept as they are. */
ppf_status ppf_resample(ppf_ctx *ctx, ppf_scheme scheme, float exchange_ratio);

/* The resampling step of Alg. 1 under its effective-sample-size test: the
 * particles are resampled (as by ppf_resample) only when the N_eff of the
 * last step is below ess_threshold.  Otherwise they are kept -- identity
 * ancestry, group layout unchanged -- and the next step carries their
 * weights, as in sequential importance sampling.  The test runs on the
 * device (no host round trip); ppf_estimate reports a kept step in bit 4 of
 * status_flags and with links = moved = 0.  ess_threshold = +inf resamples
 * every time (ppf_resample), 0 never.
 * Errors: as ppf_resample; PPF_EINVAL for a NaN threshold. */
ppf_status ppf_resample_if(ppf_ctx *ctx, ppf_scheme scheme, float exchange_ratio, double ess_threshold);

/* Copies the results of the last step and of the last resample to the host
 * (synchronises the stream).  Returns PPF_EDEGENERATE / PPF_ETIMEOUT when the
 * device flagged such a condition since the previous call, PPF_EINVAL when it
 * found a caller-supplied ancestor out of range or an inconsistent routing
 * schedule (the values are still filled in; the flags are then cleared), and
 * PPF_ESTATE before the first step. */
ppf_status ppf_estimate(ppf_ctx *ctx, ppf_estimate_t *out);

/* ppf_estimate without waiting: enqueues, on the context's stream, a copy of
 * the same fields into out_host and returns.  out_host must be host memory
 * the device can write (page-locked or registered) and must stay valid until
 * the stream has run the copy; read it after synchronising the stream.  The
 * device flags are reported in status_flags but not cleared (ppf_estimate
 * clears them).  This lets a caller read every frame's result while the
 * next frames are already queued.
 * Errors: PPF_EINVAL (NULL), PPF_ESTATE before the first step, PPF_ECUDA. */
ppf_status ppf_estimate_async(ppf_ctx *ctx, ppf_estimate_t *out_host);

/* Copies the current particles (those of the last step, or the initial ones)
 * into caller-owned device buffers, each optional (NULL = skip):
 *   state_dev   6 x N float32 SoA (x, y, vx, vy, I0, lw),
 *   anc_dev     N int32 ancestors the next step will use (identity if none),
 *   lw_prev_dev N float32 log-weights the next step starts from.
 * Enqueued on the context's stream. */
ppf_status ppf_get_particles(ppf_ctx *ctx, float *state_dev, int32_t *anc_dev, float *lw_prev_dev);

/* Replaces the current particles (test and restart hook), enqueued on the
 * context's stream; the buffers are copied:
 *   state_dev   6 x N float32 SoA, required,
 *   anc_dev     ancestors for the next step, NULL = identity,
 *   lw_prev_dev N float32 starting log-weights for the next step; NULL means
 *               "carry lw" when anc_dev is NULL (pure SIS) and "equal
 *               weights" (as after systematic resampling) when it is not.
 * The next call must be ppf_step.  Errors: PPF_EINVAL, PPF_ECUDA. */
ppf_status ppf_set_particles(ppf_ctx *ctx, const float *state_dev, const int32_t *anc_dev,
                             const float *lw_prev_dev);

/* Number of groups G and their current slot offsets (G + 1 int64 values to a
 * host buffer; synchronises).  offsets may be NULL to query G only. */
ppf_status ppf_get_groups(ppf_ctx *ctx, int32_t *n_groups, int64_t *offsets_host);

/* Replaces the group layout (restart hook, with ppf_set_particles): G + 1
 * host int64 offsets, offsets[0] = 0, offsets[G] = N, non-decreasing (LGS
 * leaves groups unequal).  Synchronises.  Errors: PPF_EINVAL, PPF_ECUDA. */
ppf_status ppf_set_groups(ppf_ctx *ctx, const int64_t *offsets_host);

/* The ARNA ring order: G int32 group indices, ring[p] sending its migrants
 * to ring[(p + 1) mod G] (identity when the context is created and after
 * ppf_set_groups).  ppf_get_ring copies it to a host buffer (synchronises);
 * ppf_set_ring replaces it (restart hook) and returns PPF_EINVAL unless the
 * values are a permutation of 0..G-1.  Errors: PPF_EINVAL, PPF_ECUDA. */
ppf_status ppf_get_ring(ppf_ctx *ctx, int32_t *ring_host);
ppf_status ppf_set_ring(ppf_ctx *ctx, const int32_t *ring_host);

/* Gradient of the log marginal likelihood estimate (the sum over frames of
 * the per-frame log-evidence of Alg. 1) with respect to
 * theta = (sigma_PSF, A, I_bg, sigma_m).  It runs K frames from a fresh prior
 * draw: propagation, likelihood (intensity fixed at I0 = A, so A is a
 * parameter), normalisation, and systematic resampling after every frame but
 * the last.  Resampling is a stop-gradient: ancestors and patch anchors are
 * held fixed.  The sigma_m derivative follows each particle's ancestry
 * forward (a per-particle tangent), the others come from the frame
 * likelihoods; all cross-block sums are FP64.
 *   frames_dev  K x H x W of model.frame_dtype (device), frames 1..K.
 *   theta       host float[4] overriding the model's (psf_sigma, amplitude,
 *               background, sigma_m) for this call; NULL = the model's.
 *   loglik      receives L = sum_k [log sum_i w_i e^{l_k^i} ... ] (eq. 4 scale).
 *   grad        receives dL/dtheta (host double[4]).
 *   anc_dev     optional K x N int32 (device): row k holds the ancestors that
 *               frame k+1 used (row 0 is the identity) -- the checkpoint of
 *               the stop-gradient path.
 *   anchors_dev optional K x 2 x N int32 (device): the patch anchors
 *               (cx row, cy row) of every frame.
 * Synchronous.  It re-draws and overwrites the context's particles; afterwards
 * they are frame K's weighted particles (ppf_resample may follow).
 * Errors: PPF_EINVAL, PPF_ENOMEM, PPF_ECUDA; PPF_EDEGENERATE if some frame had
 * no usable weight (the values are still written). */
ppf_status ppf_loglik_grad(ppf_ctx *ctx, const void *frames_dev, int32_t K, const float *theta, double *loglik,
                           double *grad, int32_t *anc_dev, int32_t *anchors_dev);

/* ------------------------------------------------------------------------
 * Batched filters: F independent SIR filters (the bank of independent
 * filters of Sec. 3, MPF) with uneven particle counts, stepped together.
 * All filters share the frame size, patch radius and frame dtype; every other
 * model field is per filter.  Filter f draws its random numbers with its
 * model's seed and filter_id, so its results equal those of a single-filter
 * context created with the same model and n_f (systematic resampling).  A
 * filter whose resample keeps its particles (no usable weight, or the N_eff
 * test of ppf_batch_set_ess_threshold) continues them with their weights.
 * ------------------------------------------------------------------------ */
typedef struct ppf_batch ppf_batch;

/* Per-filter results of a step (same meaning as ppf_estimate_t's fields). */
typedef struct {
    double mean[5];
    double log_evidence;
    double ess;
    float max_log_weight;
    int32_t degenerate;      /* 1: no usable weight in this filter */
} ppf_filter_estimate_t;

/* models: host array of F models; n: host array of F particle counts (>= 1,
 * sum <= 2^31 - 1).  Draws every filter's prior (synchronises).
 * Errors: PPF_EINVAL (geometry differs between filters, bad values), PPF_ENOMEM,
 * PPF_ECUDA. */
ppf_status ppf_batch_create(const ppf_model *models, const int64_t *n, int32_t F, void *cuda_stream,
                            ppf_batch **out);
void ppf_batch_destroy(ppf_batch *b);

/* One SIS step of every filter (frames_dev: F x H x W, filter-major), then
 * ppf_batch_resample for frame k (systematic, per filter).  A step must follow
 * the prior draw or a resample (PPF_ESTATE otherwise). */
ppf_status ppf_batch_step(ppf_batch *b, const void *frames_dev, int32_t k);
ppf_status ppf_batch_resample(ppf_batch *b, int32_t k);

/* K frames (frames_dev: K x F x H x W) of step + resample, frame indices
 * k0 .. k0+K-1.  Every kernel of a frame iteration reads its frame, frame
 * index and estimate slot from a device-side cursor, so with use_graph != 0
 * one iteration is captured as a CUDA graph once (on the first such call, or
 * after the launch shape changed) and replayed K times; use_graph == 0
 * launches the kernels directly.  Both give identical results.  est_host
 * (optional, K x F, host) receives every filter's estimate of every frame.
 * Synchronous. */
ppf_status ppf_batch_run(ppf_batch *b, const void *frames_dev, int32_t k0, int32_t K, int32_t use_graph,
                         ppf_filter_estimate_t *est_host);

/* Estimates of the last step (F entries, host; synchronises).  Returns
 * PPF_EDEGENERATE when some filter had no usable weight since the last call. */
ppf_status ppf_batch_estimates(ppf_batch *b, ppf_filter_estimate_t *out_host);

/* Copies the concatenated state (6 x Ntot float32, filter-major slots) and
 * the pending ancestors (Ntot int32, global slot indices); each optional. */
ppf_status ppf_batch_get_particles(ppf_batch *b, float *state_dev, int32_t *anc_dev);

/* Times launch shapes of the batched step on frame k (frames_dev F x H x W)
 * -- work-unit size {512, 1024, 2048, 4096} particles, block {128, 256, 512}
 * threads, {2, 4, 8} blocks per SM -- and keeps the fastest.  The filters'
 * state is not advanced.  config_out (optional, 3 ints) receives the choice. */
ppf_status ppf_batch_autotune(ppf_batch *b, const void *frames_dev, int32_t k, int32_t *config_out);

/* Alg. 1's effective-sample-size test for every filter of the batch: from
 * the next resample on, filter f is resampled only while its N_eff is below
 * fraction x n_f; otherwise it keeps its particles and its next step carries
 * their weights (as ppf_resample_if does for one filter).  fraction = +inf
 * (the default) resamples every frame, 0 never.  Synchronises the batch's
 * stream; a cached graph of ppf_batch_run stays valid.
 * Errors: PPF_EINVAL (NaN or negative fraction), PPF_ECUDA. */
ppf_status ppf_batch_set_ess_threshold(ppf_batch *b, double fraction);

const char *ppf_batch_last_error(const ppf_batch *b);

/* Phase timing and launch counting (measurement hook; no effect on results).
 * When enabled, a pair of CUDA events is recorded on the context's stream
 * around each phase of every step / resample (up to `capacity` calls per
 * phase; later calls are counted but not timed). */
typedef struct {
    int64_t launches;        /* kernels launched by the library since enabling     */
    int64_t steps;           /* ppf_step calls                                      */
    int64_t resamples;       /* ppf_resample calls                                  */
    int64_t timed_steps;     /* steps whose events were recorded                    */
    double prepare_ms;       /* frame preparation kernels, summed device time       */
    double step_ms;          /* fused propagate + likelihood + partials kernels     */
    double finalize_ms;      /* FP64 normalisation kernels                          */
    double resample_ms;      /* all kernels of the resampling calls                 */
    int64_t h2d_bytes;       /* host-to-device bytes copied by ppf_step_host        */
    int64_t d2h_bytes;       /* device-to-host bytes copied by ppf_estimate         */
} ppf_profile_t;

/* enable != 0: reset the counters and start recording (capacity >= 1);
 * enable == 0: stop recording.  Errors: PPF_EINVAL, PPF_ENOMEM, PPF_ECUDA. */
ppf_status ppf_profile_enable(ppf_ctx *ctx, int enable, int32_t capacity);

/* Synchronises the stream and sums the recorded event pairs. */
ppf_status ppf_profile_read(ppf_ctx *ctx, ppf_profile_t *out);

/* The likelihood path of the steps (Sec. 6.3, input-space decomposition).
 * Both paths compute the same step and give the same results bit for bit;
 * they differ in how the patch of eq. 4 is read:
 *   PPF_PATH_DIRECT  one fused kernel; each particle reads its patch from the
 *                    prepared frame through the L1 cache.  Fastest when the
 *                    particles of neighbouring slots lie close together (after
 *                    resampling from a concentrated posterior).
 *   PPF_PATH_BINNED  the particles are binned by image tile (T x T patch
 *                    anchors, T = 32 up to 512 x 512 frames), each tile's
 *                    window (tile plus patch halo) is copied once into shared
 *                    memory by the tensor-memory accelerator, and every patch
 *                    is read from there.  Fastest when the particles are
 *                    spread over the frame (the prior draw, a lost object).
 *   PPF_PATH_AUTO    (the default) each step's path is chosen on the device
 *                    from the previous step: binned when more than a quarter
 *                    of its warps held particles whose patch anchors spanned
 *                    more than 64 pixels, unless a systematic or RPA
 *                    resampling after it had N_eff below N / 64 (its
 *                    offspring then fill every warp with the children of a
 *                    few parents: direct).  The first step after ppf_create
 *                    or ppf_set_particles is binned.
 * Errors: PPF_EINVAL (path out of range; PPF_PATH_BINNED for a pcSIR context
 * or a frame whose tiles would exceed 3072). */
enum { PPF_PATH_AUTO = 0, PPF_PATH_DIRECT = 1, PPF_PATH_BINNED = 2 };
ppf_status ppf_set_likelihood_path(ppf_ctx *ctx, int32_t path);

/* Whether the last step took the binned path (1) or the direct one (0).
 * Synchronises the context's stream. */
ppf_status ppf_get_likelihood_path(ppf_ctx *ctx, int32_t *last_step_binned);

/* Measurement hook, not part of the method: the FP32 fused multiply-add
 * throughput of the current device, the peak the likelihood's ALU roofline
 * is taken against.  Every thread runs eight independent FMA chains
 * (packed != 0: four chains of packed two-lane FMAs) over a grid of eight
 * 256-thread blocks per SM; an FMA counts two flops.  One warm-up launch,
 * then `repeats` timed launches (CUDA events on the legacy default stream);
 * the fastest is reported.  Synchronous; allocates and frees a small output
 * buffer.
 *   tflops_out  host: the best rate in TFLOP/s.
 *   ms_out      host, optional: that launch's duration.
 * Errors: PPF_EINVAL (NULL tflops_out, repeats outside 1..100), PPF_ENOMEM,
 * PPF_ECUDA. */
ppf_status ppf_fp32_peak(int32_t packed, int32_t repeats, double *tflops_out, double *ms_out);

/* Systematic resampling of n device log-weights with no device allocation.
 * (A library addition for callers that cannot allocate; the paper has no
 * counterpart.)  Some callers cannot call cudaMalloc: serving or real-time
 * loops that pre-plan all device memory (cudaMalloc may block and
 * synchronise the device), or hosts whose device memory belongs to another
 * runtime's allocator.  This call computes exactly what ppf_resample
 * (PPF_SYSTEMATIC) computes for the same log-weights, seed, filter id and
 * frame, using a fixed scratch array inside the library instead of
 * allocated buffers.
 *   lw_dev     n float32 log-weights (device), read only.
 *   n          1 <= n <= 16,777,216 (2^24, the scratch array's capacity);
 *              larger n returns PPF_EINVAL and enqueues nothing.
 *   anc_dev    n int32 (device, caller-owned): ancestor of every slot; the
 *              identity when every weight is zero or NaN.
 *   cuda_stream stream to enqueue on (NULL = legacy default stream).
 * The scratch array (about 113 KB) lives on every device that loads the
 * library until the process exits.  The first call on a device looks up its
 * address (with that device current), and so does the first call after the
 * device's context changed (a cudaDeviceReset); make those calls before any
 * stream capture.  Every call shares the array and it keeps the
 * last call's contents (each call clears what must start at zero): calls
 * whose work overlaps on the GPU race and must be serialised by the caller.
 * Errors: PPF_EINVAL (NULL pointers, n out of range, frame < 0), PPF_ECUDA. */
ppf_status ppf_systematic_resample_noalloc(const float *lw_dev, int64_t n, uint64_t seed, uint32_t filter_id,
                                           int32_t frame, int32_t *anc_dev, void *cuda_stream);

/* Human-readable name of a status code (static string). */
const char *ppf_status_string(ppf_status s);

/* Text of the last error recorded on this context ("" if none).  Valid until
 * the next call on the context. */
const char *ppf_last_error(const ppf_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PPF_H */
