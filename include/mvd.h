/*
 * mvd.h - C ABI of the GB300 (sm_103a) efficient Bayesian multi-view
 * deconvolution library (Preibisch et al., "Efficient Bayesian-based
 * multi-view deconvolution", arXiv:1308.0730).
 *
 * The library runs, on one GPU, the sequential (OSEM-order) efficient
 * Bayesian update of the paper (Suppl. Note "Alternative iteration for faster
 * convergence", applied to Eq. 220):
 *
 *   for each iteration, for each view v of the schedule:
 *     b   = psi * P_v                     forward blur        (Eq. 51)
 *     r   = phi_v / max(b, eps)           ratio               (Eq. 15)
 *     c   = r * P_v^comp                  back-projection     (Eq. 220)
 *     psi = max(psi . c, eps)             multiplicative step (Eq. 15)
 *
 * with P_v^comp the compound kernel of Eq. 222 (or of Eq. 230, Eq. 240, or
 * the plain mirrored PSF of Eq. 51). "*" is periodic (circular) convolution
 * on the volume grid, (f * k)(x) = sum_d k(d) f((x - d) mod dims), unless the
 * context has a zero or mirror boundary (mvd_boundary).
 *
 * Conventions shared by every entry point
 *   Layout   FP32 volumes, x fastest: voxel (x,y,z) at index x + X*(y + Y*z).
 *            dims = {X, Y, Z}. PSFs are FP32 boxes {Kx, Ky, Kz}, each size
 *            odd, centre at ((Kx-1)/2, (Ky-1)/2, (Kz-1)/2), same layout.
 *   Memory   Caller buffers are read during the call only and never
 *            retained. The context owns all device memory it allocates and
 *            mvd_destroy frees it.
 *   Order    create -> precompute_kernels -> (set_estimate) -> iterate* ->
 *            result. A call out of order returns MVD_ERR_STATE.
 *   Streams  All device work is ordered on the stream given at create
 *            (NULL = the legacy default stream). Entry points that return
 *            data to the host synchronise that stream; the others only
 *            enqueue work (errors of enqueued kernels surface at the next
 *            synchronising call).
 *   Errors   Every call returns an mvd_status; nothing aborts, exits or
 *            throws across the ABI. mvd_last_error() gives a message for the
 *            last failing call on the calling thread.
 *   Threads  A context may be used from one thread at a time.
 */
#ifndef MVD_H
#define MVD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mvd_ctx mvd_ctx; /* opaque; owns all device memory of one problem */

typedef enum {
    MVD_OK = 0,
    MVD_ERR_ARG = 1,         /* invalid argument value (NULL, negative/NaN view, PSF sum <= 0, ...) */
    MVD_ERR_SHAPE = 2,       /* inconsistent sizes (even PSF size, PSF larger than the volume, ...) */
    MVD_ERR_STATE = 3,       /* call out of order */
    MVD_ERR_OOM = 4,         /* a device allocation failed */
    MVD_ERR_CUDA = 5,        /* a CUDA runtime call or kernel failed */
    MVD_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    MVD_ERR_UNSUPPORTED = 7  /* valid request this build does not handle */
} mvd_status;

/* Back-projection kernel variant (what mvd_precompute_kernels builds). */
typedef enum {
    MVD_PLAIN = 0,     /* P_v^*  (Eq. 51; with one view, classic Richardson-Lucy, Eq. 15) */
    MVD_EFFICIENT = 1, /* P_v^* . prod_{w!=v} (P_v^* * P_w * P_w^*)   (Eq. 222) */
    MVD_OPT1 = 2,      /* P_v^* . prod_{w!=v} (P_v^* * P_w)           (Eq. 230) */
    MVD_OPT2 = 3       /* (P_v^*)^N                                    (Eq. 240) */
} mvd_variant;

/* Convolution engine. AUTO lets the autotuner pick per (dims, PSF boxes). */
typedef enum { MVD_PATH_AUTO = 0, MVD_PATH_DIRECT = 1, MVD_PATH_FFT = 2 } mvd_path;

/* Arithmetic of the FFT engine.
 *   MVD_PRECISE: double-float (pairs of FP32; inside the FFT lines every
 *     high part sits on one power-of-two grid per line, which keeps the error
 *     near 2^-43 of the line's largest value) for the whole forward blur
 *     b = psi * P_v and for the back-projection's y, z and inverse x passes; the back-projection's forward x pass transforms
 *     r - 1 in FP32 (c = (r - 1) * K + 1 holds because K sums to 1, and r - 1
 *     is small where the estimate fits). FP32 FFT rounding is absolute (it
 *     scales with the whole volume's norm), so in FP32 the dim voxels of b
 *     carry large relative errors that the ratio phi / b and the iteration
 *     amplify; double-float removes them.
 *   MVD_MIXED: the forward blur as in MVD_PRECISE, the back-projection in FP32
 *     (1.3x faster). Its rounding is absolute against r - 1: within 1e-4 of
 *     an exact computation where r - 1 stays moderate, but a count where b is
 *     near eps (low-count data, no background) makes |r - 1| large and its
 *     rounding spreads over the volume (4e-4 seen after 15 iterations).
 *   MVD_FAST: everything in FP32 (faster; after tens of iterations dim voxels
 *     differ from an exact computation by about 1e-3 relative). */
typedef enum { MVD_PRECISE = 0, MVD_FAST = 1, MVD_MIXED = 2 } mvd_precision;

/* How the image convolutions continue the volume past its faces.
 *   MVD_BOUNDARY_PERIODIC: periodic (circular) convolution on the X*Y*Z grid.
 *   MVD_BOUNDARY_ZERO: the volume is continued by zeros (the camera sees
 *     nothing of the object outside the grid). The context pads every axis
 *     internally by the largest PSF half-width h (to a {2,3,5}-smooth
 *     length), and the update divides the back-projected ratio by the view's
 *     sensitivity 1 * P_v^comp, which falls below 1 within h of a face: the
 *     ML-EM step of Shepp and Vardi (1982) for this forward model.
 *   MVD_BOUNDARY_MIRROR: the volume is continued by its half-sample
 *     symmetric reflection (... x1 x0 | x0 x1 ... ). Padding 2h; the forward
 *     blur sees the reflected estimate, the back-projection folds what lands
 *     past a face back onto the reflected voxel, and the update divides by
 *     the folded sensitivity (1 wherever P_v^comp is symmetric under the
 *     face's reflection).
 *   Far from the faces both updates are the periodic one. Estimates,
 *   results and view weights keep the X*Y*Z layout. View weights and
 *   regularisation compose with the sensitivity-normalised factor as in the
 *   periodic update (factor (c_v / s_v) / (1 + lambda psi), fraction w_v of
 *   the change), and mvd_iterate_combined multiplies the factors c_v / s_v.
 *   The unrolled (differentiable) form and the persistent batch kernel
 *   return MVD_ERR_UNSUPPORTED on a context with a zero or mirror boundary. */
typedef enum { MVD_BOUNDARY_PERIODIC = 0, MVD_BOUNDARY_ZERO = 1, MVD_BOUNDARY_MIRROR = 2 } mvd_boundary;

typedef struct {
    float eps;           /* floor of b and psi; <= 0 selects 1e-4 * psi0 */
    int path;            /* mvd_path */
    void* stream;        /* cudaStream_t to order all work on; NULL = default stream */
    int views_on_device; /* 1: `views` are device pointers (copied device-to-device) */
    int device;          /* CUDA device ordinal; -1 = the calling thread's current device */
    int precision;       /* mvd_precision (FFT engine) */
    int boundary;        /* mvd_boundary */
} mvd_options;

/* Fills *opt with eps = 0 (auto), path = AUTO, stream = NULL, host views,
 * device -1, precision = MVD_PRECISE, boundary = MVD_BOUNDARY_PERIODIC. */
void mvd_default_options(mvd_options* opt);

/*
 * Creates a context for one deconvolution problem.
 *   views     n_views pointers to X*Y*Z floats (observed views phi_v on the
 *             common registered grid, Eq. 51's identity-transform assumption);
 *             host pointers, or device pointers if opt->views_on_device.
 *             Values must be finite and >= 0 (Eq. 3), else MVD_ERR_ARG.
 *   psfs      n_views host pointers to Kx*Ky*Kz floats (P_v); values >= 0 and
 *             sum > 0, else MVD_ERR_ARG. Each PSF is normalised to sum 1
 *             (Eq. 3) when copied.
 *   psf_dims  3*n_views ints {Kx,Ky,Kz} per view; odd and <= dims, else
 *             MVD_ERR_SHAPE.
 *   dims      {X, Y, Z}, each >= 1.
 *   opt       may be NULL (defaults).
 *   out       receives the context; *out is NULL on failure.
 * Copies the views to the device (the context owns the copies), computes
 * psi0 = mean over all voxels of all views (the flat estimate, Eq. 15 text)
 * and eps, and sets psi = psi0.
 */
mvd_status mvd_create(const float* const* views, int n_views, const float* const* psfs,
                      const int* psf_dims, const int dims[3], const mvd_options* opt,
                      mvd_ctx** out);

/*
 * Builds P_v^comp for every view on the device (FP32) for the given
 * mvd_variant (Eq. 222 / Eq. 230 / Eq. 240 / Eq. 51), normalised to sum 1,
 * on P_v's own box; chooses the convolution engine (with MVD_PATH_AUTO: the
 * autotuner's cached choice for this shape if MVD_TUNE_CACHE holds one, else
 * a cost model of both engines; see mvd_autotune) and, for the FFT engine,
 * builds the two kernel spectra per view.
 * May be called again to switch variant.
 */
mvd_status mvd_precompute_kernels(mvd_ctx* ctx, int variant);

/* Sets the estimate: psi = psi0 (flat) if psi == NULL, else copies X*Y*Z
 * floats (> 0) from psi (a device pointer if on_device, else host). */
mvd_status mvd_set_estimate(mvd_ctx* ctx, const float* psi, int on_device);

/*
 * Loads new observed views into the context: the next time point of a series
 * recorded with the same PSFs (the paper's time-lapse recordings of hundreds
 * of time points, processed in parallel per time point; main text and the
 * table of experiments). Keeps the compound kernels, the spectra, the
 * engine choice, view weights and regularisation; recomputes psi0 (the mean
 * of the new views) and, unless eps was given at create, eps = 1e-4 psi0
 * (then the captured iteration graphs are rebuilt on the next iterate); resets
 * psi to the flat psi0 (mvd_set_estimate afterwards warm-starts instead).
 *   views     n_views pointers to X*Y*Z floats, host or (on_device) device
 *             pointers; finite and >= 0, not all zero, else MVD_ERR_ARG.
 * Synchronises the context's stream (it reads the views' sum back). After a
 * rejected load the context holds invalid views: iterate, autotune, the
 * unrolled form and batch creation return MVD_ERR_STATE until a load
 * succeeds. A batch already built from the context keeps the eps it was
 * built with.
 */
mvd_status mvd_set_views(mvd_ctx* ctx, const float* const* views, int on_device);

/*
 * Runs n_iter iterations of the sequential update. One iteration applies the
 * update of every view in `schedule` once, in order (schedule_len entries in
 * [0, n_views)); schedule == NULL or schedule_len == 0 means 0..n_views-1.
 * Enqueues work only. On a non-NULL stream, one iteration of a given
 * schedule is captured once as a CUDA graph (kept by the context until the
 * next mvd_precompute_kernels or mvd_destroy) and replayed per iteration;
 * while per-kernel timing is enabled, or with MVD_NO_GRAPH=1 in the
 * environment, kernels are launched one by one instead.
 */
mvd_status mvd_iterate(mvd_ctx* ctx, int n_iter, const int* schedule, int schedule_len);

/*
 * Partially overlapping views (Suppl. Note "Partially overlapping datasets").
 * weights: n_views pointers to X*Y*Z floats in [0, 1] (host, or device if
 * on_device), each view's blending image (1 where the view has data, falling
 * to 0 towards its boundary; else MVD_ERR_ARG). They are copied and, per
 * voxel, scaled by min(1, T / sum_v w_v), so the sum over views is at most T
 * and no weight ever grows; T (written to *target when non-NULL) is
 *   MVD_WEIGHTS_SUM_ONE     1 (the most uniform update),
 *   MVD_WEIGHTS_MIN_OVERLAP the minimal number of views overlapping at a voxel,
 *   MVD_WEIGHTS_AVG_OVERLAP the average number,
 *   MVD_WEIGHTS_USER        value (> 0),
 * counting at each voxel covered by some view the views with w_v > 0.
 * From then on every view update of mvd_iterate applies the fraction w_v of
 * the change of the Richardson-Lucy step: psi = max(psi (1 + w_v (c_v - 1)), eps).
 * weights == NULL removes them. With a zero or mirror boundary the images
 * are in the user's X*Y*Z layout and weigh the sensitivity-normalised
 * factor (mvd_boundary). The combined update, the unrolled differentiation
 * and the persistent batch kernel return MVD_ERR_UNSUPPORTED for a context
 * with weights. Synchronises the stream.
 * mvd_get_weights copies view v's normalised weights (X*Y*Z floats) to host.
 */
/*
 * Tikhonov regularisation of the sequential update (the paper's lambda,
 * 0.0006 to 0.06 in its experiments; it prints no update rule). This library
 * uses the one-step-late MAP-EM of P. J. Green (IEEE Trans. Med. Imaging 9,
 * 1990) with the quadratic prior lambda/2 |psi|^2: each view update's factor
 * becomes c_v / (1 + lambda psi), i.e.
 *   psi = max(psi (1 + w_v (c_v / (1 + lambda psi) - 1)), eps)
 * with the view weight w_v (1 without weights). lambda must be finite and
 * >= 0 (0 = none, the default). The combined update, the unrolled
 * differentiation and the persistent batch kernel return MVD_ERR_UNSUPPORTED
 * for lambda > 0.
 */
mvd_status mvd_set_regularization(mvd_ctx* ctx, float lambda);

typedef enum {
    MVD_WEIGHTS_SUM_ONE = 0,
    MVD_WEIGHTS_MIN_OVERLAP = 1,
    MVD_WEIGHTS_AVG_OVERLAP = 2,
    MVD_WEIGHTS_USER = 3
} mvd_weight_norm;
mvd_status mvd_set_weights(mvd_ctx* ctx, const float* const* weights, int on_device, int norm, float value,
                           float* target);
mvd_status mvd_get_weights(mvd_ctx* ctx, int v, float* out, size_t n_elems);

/*
 * Runs n_iter iterations of the combined (simultaneous) update of Eq. 50 /
 * Eq. 220: every view's factor c_v = (phi_v / max(psi * P_v, eps)) * P_v^comp
 * is computed from the same psi, then
 *   psi = max(psi . prod_v c_v, eps)               (root == 0, Eq. 50 as printed)
 *   psi = max(psi . (prod_v c_v)^(1/N), eps)       (root != 0, the geometric
 *        mean of the factors, as in the paper's convergence proof).
 * With a zero or mirror boundary each factor is c_v / s_v (s_v the view's
 * sensitivity, see mvd_boundary). View weights or lambda > 0 return
 * MVD_ERR_UNSUPPORTED (they belong to the sequential update).
 * Needs one more volume on the device (the product, allocated on first use;
 * with the mirror boundary a second one for the back-projection).
 * Enqueues work only; graph capture as in mvd_iterate.
 */
mvd_status mvd_iterate_combined(mvd_ctx* ctx, int n_iter, int root);

/* Copies psi (X*Y*Z floats) to host memory `out`; n_elems must be >= X*Y*Z.
 * Synchronises the context's stream. With a zero or mirror boundary the
 * estimate is first cropped out of the padded grid on the device. */
mvd_status mvd_result(mvd_ctx* ctx, float* out, size_t n_elems);

/* Hands out the device pointer of psi (X*Y*Z floats, borrowed; valid until
 * the next call that mutates or destroys the context). Does not synchronise;
 * with a zero or mirror boundary it enqueues the crop into a staging volume
 * (whose pointer it returns) on the context's stream. */
mvd_status mvd_result_device(mvd_ctx* ctx, const float** dptr);

/* Waits for all work enqueued on the context's stream. */
mvd_status mvd_synchronize(mvd_ctx* ctx);

/* Frees everything the context owns. NULL is ignored. */
void mvd_destroy(mvd_ctx* ctx);

/* Message for the last failing call on this thread ("" if none). */
const char* mvd_last_error(void);

/* Introspection. */
float mvd_get_eps(const mvd_ctx* ctx);  /* floor in use */
float mvd_get_psi0(const mvd_ctx* ctx); /* flat estimate value */
int mvd_get_path(const mvd_ctx* ctx);   /* MVD_PATH_DIRECT or MVD_PATH_FFT once precomputed */

/* Copies the compound kernel of view v (Kx*Ky*Kz floats, PSF layout) to host
 * memory `out` (n_elems >= that size). Synchronises the stream. */
mvd_status mvd_get_compound_kernel(mvd_ctx* ctx, int v, float* out, size_t n_elems);

/* Number of kernels this library has launched in the process so far. */
unsigned long long mvd_launch_count(void);

/*
 * The radix plan the FFT engine's shared-memory (Stockham) passes use for an
 * axis of length L under `precision` (mvd_precision): the stage radices, in
 * order, into radices[0..n-1]. Host only; needs no GPU.
 * Returns n >= 1, 0 if L is not {2,3,5}-smooth (or L < 2), or -1 if
 * max_stages < n or radices is NULL or precision is unknown. Powers of two
 * take radix 8 stages with one 4 or 2 (4 4 when that avoids a 2); other
 * lengths the cheapest product of radices 2, 3, 4, 5, 6, 8, 9 and 10 (no 10
 * for MVD_PRECISE and MVD_MIXED, whose double-float passes would spill with
 * it), largest radix first.
 */
int mvd_fft_plan(int L, int precision, int* radices, int max_stages);

/*
 * Per-kernel timing for measurement. While enabled, every launch of the
 * update's kernels is bracketed by two CUDA events recorded on the launching
 * stream. mvd_profile_read synchronises on the recorded events and returns,
 * per kernel class, the class name (static string), the number of timed
 * launches and their summed duration in milliseconds; it returns the number
 * of classes written (<= max). Enabling again discards earlier records.
 * Classes: x_forward, y, z_mul, x_ratio, x_update, direct_ratio,
 * direct_update, setup.
 */
void mvd_profile_enable(int on);
int mvd_profile_read(const char** names, unsigned long long* launches, double* ms, int max);

/*
 * Batched form: many independent problems of uneven size and view count
 * (time points, tiles of a large specimen; the paper processes such units
 * independently, Suppl. Table 1 and main text) advanced together by one
 * launch of a CUDA graph. Two executions (mvd_batch_mode):
 *   MVD_BATCH_BRANCHES    one graph in which each volume's whole run (the
 *                         single-volume engine's kernels) is an independent
 *                         branch; kernels of different volumes run side by
 *                         side. Needs a non-NULL stream and per-kernel timing
 *                         off. Any engine.
 *   MVD_BATCH_PERSISTENT  one persistent kernel over a global work queue of
 *                         FFT-pass tiles of all volumes, with bounded
 *                         per-volume dependency waits. FFT engine only.
 *   MVD_BATCH_AUTO        BRANCHES where it is allowed, else PERSISTENT.
 *   ctxs    n distinct contexts, each precomputed, all on one device and one
 *           stream (else MVD_ERR_ARG / MVD_ERR_STATE / MVD_ERR_UNSUPPORTED).
 *           The batch keeps pointers into them: destroy the batch before any
 *           of its contexts, and do not re-precompute or autotune a context
 *           while a batch uses it.
 *   n_iter  iterations of each context's default schedule (views 0..N-1)
 *           per mvd_batch_run.
 * mvd_batch_run enqueues the job on the shared stream (each context's psi
 * advances by n_iter iterations from its current value); mvd_batch_wait
 * synchronises and returns MVD_ERR_TIMEOUT if a persistent block gave up
 * waiting for a dependency (a bounded wait; MVD_BATCH_POLL_LIMIT sets the
 * poll count). mvd_batch_tasks gives the work items of one run (tiles of the
 * persistent queue, or kernels of the branch graph); mvd_batch_mode the
 * execution chosen. mvd_batch_create = mvd_batch_create_mode(..., AUTO, ...).
 */
typedef enum { MVD_BATCH_AUTO = 0, MVD_BATCH_PERSISTENT = 1, MVD_BATCH_BRANCHES = 2 } mvd_batch_mode_t;
typedef struct mvd_batch mvd_batch;
mvd_status mvd_batch_create(mvd_ctx* const* ctxs, int n, int n_iter, mvd_batch** out);
mvd_status mvd_batch_create_mode(mvd_ctx* const* ctxs, int n, int n_iter, int mode, mvd_batch** out);
int mvd_batch_mode(const mvd_batch* batch);
mvd_status mvd_batch_run(mvd_batch* batch);
mvd_status mvd_batch_wait(mvd_batch* batch);
long long mvd_batch_tasks(const mvd_batch* batch);
void mvd_batch_destroy(mvd_batch* batch);

/*
 * Autotuner: picks the engine (direct tiled convolution or FFT) and its tile
 * shape for this problem by timing one pass of view updates per candidate on
 * the context's own data (the estimate is restored afterwards), then sets the
 * fastest on the context. Candidates: the FFT engine with register-resident
 * power-of-two passes and with mixed-radix Stockham passes (where the dims
 * are {2,3,5}-smooth), and the direct engine with output tiles of 32 x ty x 4
 * for every ty in {8,4,2,1} whose staging fits in shared memory.
 * The choice is persisted per (dims, precision, PSF boxes, GPU model) as one
 * text line appended to cache_path (NULL = the MVD_TUNE_CACHE environment
 * variable; neither = not persisted). An existing entry is applied without
 * timing (from_cache = 1), and mvd_precompute_kernels with MVD_PATH_AUTO
 * applies a cached entry for its shape when MVD_TUNE_CACHE names a file.
 * Needs a precomputed context (MVD_ERR_STATE); synchronises the stream; out
 * may be NULL. Drops the context's captured graphs.
 */
typedef struct {
    int path;             /* MVD_PATH_DIRECT or MVD_PATH_FFT */
    int direct_tile_y;    /* direct engine: output tile height ty; 0 for FFT */
    int fft_engine;       /* FFT: 1 register-resident passes, 0 Stockham passes; -1 for direct */
    int from_cache;       /* 1 when read from the cache without timing */
    double ms_per_update; /* measured time of one view update (ms) */
} mvd_tune_result;
mvd_status mvd_autotune(mvd_ctx* ctx, const char* cache_path, mvd_tune_result* out);

/*
 * Differentiation of the unrolled iteration, for calibrating PSF parameters
 * or views against a target (the paper's update, Eq. 15 with the kernels of
 * Eq. 222 / 230 / 240 / 51, read as a differentiable function of the views
 * and PSFs; the paper itself does not differentiate it).
 *   mvd_unrolled_forward   n_iter >= 0 iterations of the default schedule
 *            (views 0..N-1) from the flat start psi0 = mean of the views,
 *            keeping the estimate before every view update on the device
 *            (n_iter * N volumes, freed by the next call or mvd_destroy).
 *            Afterwards the context's estimate is psi_K (mvd_result*).
 *            Needs a precomputed context (else MVD_ERR_STATE).
 *   mvd_unrolled_backward  reverse pass for the last forward run.
 *            grad_psi    device, X*Y*Z floats: dL/dpsi_K.
 *            grad_views  N device pointers, X*Y*Z floats each, written with
 *                        dL/dphi_v (including the flat start's share).
 *            grad_psfs   N HOST pointers, Kx*Ky*Kz floats each (the PSF
 *                        box), written with dL/dp_v for the RAW PSF as
 *                        passed to mvd_create (through the normalisation of
 *                        Eq. 3 and the compound kernel).
 *            The floors max(., eps) pass gradient only where inactive; eps
 *            is held fixed. Volume work runs on the direct engine in FP32
 *            (MVD_ERR_UNSUPPORTED for PSF boxes it cannot stage, or more than
 *            32 views). Synchronises the stream. MVD_ERR_STATE without a
 *            forward run.
 */
mvd_status mvd_unrolled_forward(mvd_ctx* ctx, int n_iter);
mvd_status mvd_unrolled_backward(mvd_ctx* ctx, const float* grad_psi, float* const* grad_views,
                                 float* const* grad_psfs);

/*
 * Gaussian PSF model (host, FP64 arithmetic, FP32 output) for calibration:
 * p(d) = exp(-0.5 * u^T diag(1/v) u) / sum, u = R^T d, R the rotation about
 * y by angle_deg (x towards z), v = sigma_xy^2 on the two lateral axes and
 * sigma_ax^2 on axis (0 = x, 1 = y, 2 = z), on a centred box (odd sizes;
 * MVD_ERR_SHAPE otherwise). mvd_gaussian_psf_vjp returns
 * grad_sigma = {dL/dsigma_xy, dL/dsigma_ax} for grad_psf = dL/dp (host,
 * box layout). Sigmas must be > 0 (MVD_ERR_ARG).
 */
mvd_status mvd_gaussian_psf(double sigma_xy, double sigma_ax, double angle_deg, int axis, const int box[3],
                            float* out);
mvd_status mvd_gaussian_psf_vjp(double sigma_xy, double sigma_ax, double angle_deg, int axis, const int box[3],
                                const float* grad_psf, double grad_sigma[2]);

/*
 * Allocation-free view update. The paper has no counterpart: this entry point
 * serves callers that cannot call cudaMalloc, such as applications whose
 * device memory belongs to a caching allocator that must see every
 * allocation (a raw cudaMalloc or cudaFree also synchronises the device), or
 * acquisition loops that allocate at start-up only. It runs one view update
 * with the direct engine and allocates nothing:
 *   psi = max(psi . ((phi / max(psi * psf, eps)) * comp), eps)
 * All pointers are device pointers the caller owns, on the current device
 * (host, pinned or another device's memory returns MVD_ERR_ARG, checked with
 * cudaPointerGetAttributes): psi (X*Y*Z floats,
 * updated in place), phi (X*Y*Z floats), psf and comp (Kx*Ky*Kz floats each,
 * PSF layout; used as given, so pass a normalised PSF and its compound
 * kernel, e.g. from mvd_get_compound_kernel). dims = {X,Y,Z}, kdims =
 * {Kx,Ky,Kz} (odd, <= dims), eps > 0, stream = cudaStream_t or NULL.
 * Limit: X*Y*Z <= 2^21 voxels (8 MiB of ratio scratch); larger volumes
 * return MVD_ERR_SHAPE, PSF boxes the direct engine cannot stage return
 * MVD_ERR_UNSUPPORTED.
 * The ratio scratch is one file-scope device array per GPU, held until the
 * process exits and shared by every call: calls whose work overlaps on the
 * GPU (other streams, other host threads) race on it. Order them on one
 * stream. The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. Enqueues work only.
 */
mvd_status mvd_update_direct_noalloc(float* psi, const float* phi, const float* psf, const float* comp,
                                     const int dims[3], const int kdims[3], float eps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MVD_H */
