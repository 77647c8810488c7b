/*
 * pnp_ms2g.h — C ABI of the GB300 (sm_103a) implementation of the hot path of
 * "Accelerating Plug-and-Play Image Reconstruction via Multi-Stage Sketched
 * Gradients" (Tang, arXiv 2203.07308): the data-fidelity gradient A^T(Ax - b)
 * for 2-D fan-beam X-ray CT, used full-grid, image-sketched and angle-subset,
 * inside the multi-stage PnP loop of Algorithm 1.
 *
 * Conventions shared by every entry point
 *   Units      lengths in fine pixels (pixel side 1); the image is centred at the
 *              origin.  Level s (sketch factor s in {1,2,4,8}, Eq. 4's S_k) has
 *              n/s pixels per side of size s.
 *   Images     float32, row-major [batch][n_s][n_s], x (column) index fastest;
 *              pixel (ix,iy) of level s is centred at
 *              ((ix - (n_s-1)/2) s, (iy - (n_s-1)/2) s).
 *   Sinograms  float32 [batch][views][n_det], detector index fastest.  A
 *              sinogram "of subset p of P" holds the views v = p, p+P, p+2P, ...
 *              in increasing order (Alg. 1 Option 2 with angle subsets); P = 1
 *              means all views.  The data b is always the full [batch][n_views][n_det].
 *   Operator   A_s (Eq. 1 / Eq. 4): ray (v, j) from the source at
 *              dso (cos b_v, sin b_v), b_v = angle0 + angle_span v / n_views,
 *              to the flat-detector bin centre -ddo (cos b_v, sin b_v)
 *              + u_j (-sin b_v, cos b_v), u_j = (j - (n_det-1)/2) det_pitch;
 *              samples q_k = F + (k + 1/2) (step s) d for every integer k, F the
 *              point of the ray nearest the origin, d its unit direction; each
 *              sample adds (step s) times the bilinear interpolant of the level-s
 *              image (zero outside it).  A_s^T is the exact transpose.
 *   Pointers   d_* are device pointers, h_* host pointers.  The caller owns every
 *              buffer and the stream; the library allocates no device memory.
 *              Buffers passed to one call must not overlap unless stated.
 *   Streams    `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *              are asynchronous on it unless they return host results (stated).
 *   Workspace  d_ws of at least pnp_workspace_size() bytes, 256-byte aligned,
 *              prepared once per geometry by pnp_setup().  Calls that take it
 *              use it as scratch: calls sharing one workspace must be ordered
 *              on one stream.
 *   Errors     every int-returning call returns PNP_OK or a PNP_E* code and
 *              leaves a message for pnp_last_error() (thread-local).  Invalid
 *              arguments are rejected before anything is launched.
 */
#ifndef PNP_MS2G_H
#define PNP_MS2G_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PNP_OK = 0,
    PNP_EINVAL = 1,        /* bad argument (size, pointer, factor, subset, geometry) */
    PNP_ECUDA = 2,         /* a CUDA runtime call or launch failed */
    PNP_ETIMEOUT = 3,      /* a bounded device-side wait gave up */
    PNP_EUNSUPPORTED = 4,  /* valid request the library does not handle */
    PNP_ESTATE = 5         /* workspace not prepared by pnp_setup for this geometry */
};

/* Fan-beam geometry (Sec. 3: fan-beam X-ray CT, views equally spaced over
 * angle_span).  All lengths in fine pixels, angles in radians. */
typedef struct {
    int32_t n;          /* fine image side; divisible by every sketch factor used */
    int32_t n_views;    /* projection angles */
    int32_t n_det;      /* detector bins */
    int32_t batch;      /* independent images sharing this geometry */
    double dso;         /* source to rotation centre */
    double ddo;         /* rotation centre to detector */
    double det_pitch;   /* bin spacing on the detector */
    double angle0;      /* angle of view 0 */
    double angle_span;  /* views cover [angle0, angle0 + angle_span) */
    double step;        /* ray-march step in level pixels (0.5 = half a pixel) */
} pnp_geom;

/* Sketch operators S_k (and U_k = S_k^T).  POOL: s x s average pooling.
 * BICUBIC: the paper's bicubic resize (Sec. 3), read as the separable Keys
 * cubic convolution kernel (a = -1/2) widened by s, normalised to sum to one
 * over the fine pixels inside the image. */
#define PNP_SKETCH_POOL 0
#define PNP_SKETCH_BICUBIC 1

/* Subset gradient estimates for Option 2 (P_k > 1).  Sec. 2 uses the vanilla
 * minibatch estimate and names variance-reduced ones as alternatives:
 *   SVRG (Johnson & Zhang 2013): snapshot yt and its full sketched gradient mu at
 *     the start of every epoch of P_k iterations; v = G_p(y) - G_p(yt) + mu.
 *   SAGA (Defazio, Bach & Lacoste-Julien 2014): the last gradient of every subset
 *     is kept (filled at the stage's first iterate); v = G_p(y) - T_p + mean_j T_j,
 *     then T_p = G_p(y).
 * Both need a buffer registered with pnp_set_vr_buffer. */
#define PNP_EST_MINIBATCH 0
#define PNP_EST_SVRG 1
#define PNP_EST_SAGA 2

/* One stage of Algorithm 1: sketch factor s_k (m_k = d / s_k^2), N_k inner
 * iterations, P_k interleaved angle subsets (1 = Option 1, >1 = Option 2), the
 * sketch kind and the subset estimate. */
typedef struct {
    int32_t factor;
    int32_t iters;
    int32_t n_subsets;
    int32_t kind;       /* PNP_SKETCH_POOL or PNP_SKETCH_BICUBIC (ignored for factor 1) */
    int32_t estimator;  /* PNP_EST_* (ignored when n_subsets == 1) */
} pnp_stage;

/* Loop parameters of Algorithm 1. */
typedef struct {
    float alpha;        /* RED-PRO relaxation x = (1-alpha) z + alpha D(z), alpha in (0,1] */
    float lambda;       /* TV weight of the denoiser D = TV-prox (Sec. 2, after Eq. 5) */
    int32_t tv_iters;   /* FGP iterations of D (Beck & Teboulle 2009); 0 = identity */
    int32_t momentum;   /* 0: a_i = 0 (Eq. 5); 1: a_i = (i-1)/(i+3) (Sec. 3) */
    int32_t flags;      /* PNP_RUN_* bits */
    uint64_t subset_seed; /* seed of the subset order of problems given without a
                             subset sequence (pnp_subset_sequence) */
} pnp_run_params;

/* pnp_run / pnp_run_many: capture the whole launch sequence as a CUDA graph the
 * first time a call with identical arguments (pointers, geometry, schedule,
 * step sizes, subset sequence, parameters, stream) is made, and replay it on
 * later identical calls.  Ignored on the legacy default stream (NULL).  The
 * library keeps up to 16 instantiated graphs. */
#define PNP_RUN_GRAPH 1

/* pnp_run / pnp_run_many: bracket every phase launch of every iteration with a
 * pair of CUDA events on the run's stream, so that pnp_kernel_times can report
 * the device time of each phase.  Not combinable with PNP_RUN_GRAPH. */
#define PNP_RUN_KERNEL_TIMES 2
/* Flag for pnp_run_params.flags: every phase kernel of the run (coefficient
 * image, forward projector, gather backprojector, FGP denoiser) launches in its
 * persistent form: only as many CTAs as the GPU holds at once, each walking
 * the phase's work table of (geometry class, instance, tile / ray block) items
 * with a stride of the grid (no waits between CTAs).  Every item computes what
 * it computes in the direct form, so the results are the same bits; what
 * changes is who schedules the items (the kernel instead of the hardware's CTA
 * dispatcher).  Combines with PNP_RUN_GRAPH. */
#define PNP_RUN_PERSISTENT 4

/* Phases of one iteration of Algorithm 1, as timed by PNP_RUN_KERNEL_TIMES. */
#define PNP_PHASE_PREP 0      /* sketch S and the bilinear coefficient image */
#define PNP_PHASE_FORWARD 1   /* A_s^{(p)} (S y) - b^{(p)} */
#define PNP_PHASE_BACKWARD 2  /* A_s^{(p)T}, U and the gradient step z = y - eta g */
#define PNP_PHASE_DENOISE 3   /* TV prox by FGP, relaxation and momentum */
#define PNP_N_PHASES 4

/* One geometry class of a batched run: a uniform batch of images sharing one
 * geometry, with its own schedule, data, iterate and prepared workspace. */
typedef struct {
    pnp_geom geom;
    const pnp_stage* stages;
    int32_t n_stages;
    const double* h_eta;          /* [n_stages], or NULL: eta_k = 1/L_k as pnp_step_sizes computes it */
    const int32_t* h_subset_seq;  /* [sum iters], or NULL: pnp_subset_sequence(params.subset_seed) */
    const float* d_b;             /* [batch][n_views][n_det] */
    float* d_x;                   /* in: x_0, out: x */
    const float* d_xtrue;         /* optional, with h_psnr_log */
    double* h_psnr_log;           /* optional, [sum iters][batch] (entries before start_iter untouched) */
    void* d_ws;                   /* pnp_setup-prepared workspace of this geometry */
    int32_t start_iter;           /* checkpoint/resume: iterations already done (0 = fresh run) */
    float* d_y;                   /* optional: in, y_{start_iter} (default: x); out, y after the run */
} pnp_problem;

/* Maximum total iterations of one pnp_run call when a PSNR log is requested. */
#define PNP_MAX_LOG_ITERS 65536

/* Bytes of device workspace for geometry g (all sketch levels in {1,2,4,8}
 * that divide n with n/s >= 4).  Returns PNP_EINVAL for an invalid geometry. */
int pnp_workspace_size(const pnp_geom* g, size_t* bytes);

/* Prepares d_ws for geometry g: computes the FP64 per-ray tables of every
 * level on the device (foot point, direction, sample range) and registers the
 * (workspace, geometry) pair.  Must precede every call that takes d_ws with
 * this geometry; redo it after reusing the memory for another geometry.
 * Asynchronous on `stream`. */
int pnp_setup(const pnp_geom* g, void* d_ws, size_t ws_bytes, void* stream);

/* Weighted least squares.  Sec. 3 simulates transmission data b ~ Poisson(I0
 * exp(-A x)) and takes the logarithm; the matching data fidelity is
 * f = 1/2 sum_j w_j ((A x)_j - b_j)^2 with w_j the inverse variance of b_j
 * (proportional to the measured counts for log transmission data).  After this
 * call every gradient, step size (power iteration; instance 0's weights) and
 * objective computed with d_ws uses the weights d_w [batch][n_views][n_det]
 * (the caller keeps them alive); pnp_project stays unweighted.  NULL returns to
 * plain least squares.  pnp_setup clears it. */
int pnp_set_weights(const pnp_geom* g, const float* d_w, void* d_ws);

/* Forward projection (Eq. 1, Eq. 4): d_sino = A_s^{(p)} d_img, or the residual
 * A_s^{(p)} d_img - b^{(p)} when d_b is not NULL.
 *   factor   sketch level s; d_img is the level-s image [batch][n/s][n/s]
 *   d_b      NULL or the full data [batch][n_views][n_det]
 *   d_sino   out, [batch][views of subset][n_det]
 *   subset, n_subsets   0 <= subset < n_subsets <= n_views (1 = all views) */
int pnp_project(const pnp_geom* g, int factor, const float* d_img, const float* d_b,
                float* d_sino, int subset, int n_subsets, void* d_ws, void* stream);

/* Backprojection, the exact transpose of pnp_project (the A^T of Eq. 5):
 * d_img = A_s^{(p)T} d_sino, computed as a deterministic pixel-driven gather
 * (no atomics; bitwise repeatable).
 *   d_sino   [batch][views of subset][n_det];  d_img out, [batch][n/s][n/s] */
int pnp_backproject(const pnp_geom* g, int factor, const float* d_sino, float* d_img,
                    int subset, int n_subsets, void* d_ws, void* stream);

/* Sketch S (Eq. 4, Alg. 1 "v = S_k(y)"): s x s average pooling,
 * d_fine [batch][n][n] -> d_coarse [batch][n/s][n/s]. */
int pnp_sketch(const pnp_geom* g, int factor, const float* d_fine, float* d_coarse, void* stream);

/* Upsampler U = S^T (Alg. 1 "U_k"): each coarse value replicated over its
 * s x s block and divided by s^2, d_coarse -> d_fine. */
int pnp_upsample(const pnp_geom* g, int factor, const float* d_coarse, float* d_fine, void* stream);

/* pnp_sketch / pnp_upsample with the sketch kind. */
int pnp_sketch_kind(const pnp_geom* g, int factor, int kind, const float* d_fine, float* d_coarse, void* stream);
int pnp_upsample_kind(const pnp_geom* g, int factor, int kind, const float* d_coarse, float* d_fine,
                      void* stream);

/* Full data-fidelity gradient (Eq. 5): d_g = A^T (A d_x - d_b), all views,
 * fine grid.  d_x, d_g [batch][n][n]; d_b [batch][n_views][n_det]. */
int pnp_full_grad(const pnp_geom* g, const float* d_x, const float* d_b, float* d_g,
                  void* d_ws, void* stream);

/* Sketched (minibatch) gradient estimate of Alg. 1 on the fine grid:
 *   d_g = c S^T A_s^{(p)T} (A_s^{(p)} S d_y - b^{(p)}),   c = n_subsets,
 * i.e. U G with U = S^T, G = Option 1 (n_subsets = 1) or Option 2 (angle
 * subset p scaled by P so that its mean over p is the Option 1 gradient).
 * For factor 1 and n_subsets 1 it equals pnp_full_grad. */
int pnp_sketch_grad(const pnp_geom* g, int factor, const float* d_y, const float* d_b, float* d_g,
                    int subset, int n_subsets, void* d_ws, void* stream);

/* pnp_sketch_grad with the sketch kind (S and U = S^T of that kind). */
int pnp_sketch_grad_kind(const pnp_geom* g, int factor, int kind, const float* d_y, const float* d_b,
                         float* d_g, int subset, int n_subsets, void* d_ws, void* stream);

/* Bytes of workspace for pnp_tv_denoise on [batch][n][n]. */
int pnp_tv_workspace_size(int n, int batch, size_t* bytes);

/* TV-prox denoiser D (Sec. 2, after Eq. 5: "TV-prox"): iters iterations of FGP
 * (Beck & Teboulle 2009, isotropic TV, forward differences, zero past the last
 * row/column, dual step 1/(8 lambda), no box constraint) applied to each image:
 *   d_x ~= argmin_x 1/2 ||x - d_z||^2 + lambda TV(x).
 * d_z, d_x [batch][n][n] (may not alias).  d_ws (pnp_tv_workspace_size bytes)
 * carries the dual state between launches when iters > 8; it may be NULL
 * otherwise. */
int pnp_tv_denoise(const float* d_z, float* d_x, int n, int batch, float lambda, int iters,
                   void* d_ws, size_t ws_bytes, void* stream);

/* Step-size constant L = ||A_s S||^2 (Sec. 3: eta = O(1/L)) by power iteration
 * on S^T A_s^T A_s S from the normalised all-ones image, FP32 operators and FP64
 * inner products; stops when the Rayleigh quotient changes by less than tol
 * (relative) or after max_iters.  Uses batch instance 0's buffers only (L does
 * not depend on the data).  Synchronous: writes *h_L and *h_iters. */
int pnp_power_iter(const pnp_geom* g, int factor, int max_iters, double tol, double* h_L,
                   int* h_iters, void* d_ws, void* stream);

/* pnp_power_iter for L = ||A_s S||^2 with S of the given kind. */
int pnp_power_iter_kind(const pnp_geom* g, int factor, int kind, int max_iters, double tol, double* h_L,
                        int* h_iters, void* d_ws, void* stream);

/* Bytes of the estimator-state buffer that pnp_run needs for this schedule
 * (0 when no stage uses SVRG or SAGA): snapshot, difference image, the running
 * sums and, for SAGA, P_k level-grid images per image of the batch. */
int pnp_vr_buffer_size(const pnp_geom* g, const pnp_stage* stages, int n_stages, size_t* bytes);

/* Registers (d_buf != NULL) or clears the estimator-state buffer of a prepared
 * workspace; caller-owned device memory of `bytes` bytes (256-byte aligned).
 * The buffer carries the SVRG snapshot and the SAGA table between calls, so a run
 * resumed with start_iter continues bit for bit when the buffer is the one the
 * interrupted run left.  PNP_ESTATE from pnp_run when a stage needs a larger one. */
int pnp_set_vr_buffer(const pnp_geom* g, void* d_buf, size_t bytes, void* d_ws);

/* Step sizes of Algorithm 1 for a schedule (Sec. 3: eta = O(1/L)):
 * h_eta[k] = 1 / L_k, L_k = ||W^{1/2} A_{s_k} S_k||^2 for stage k's level and
 * sketch kind (W the weights of pnp_set_weights, else I), by the power iteration
 * of pnp_power_iter_kind with at most 100 iterations and relative tolerance 1e-6.
 * Each L is cached in the workspace's registry entry (per level and sketch kind)
 * until pnp_setup or pnp_set_weights; computing one is synchronous on `stream`
 * and uses the workspace's scratch buffers, so call it outside stream capture.
 * pnp_run and pnp_run_many use it for problems given without step sizes. */
int pnp_step_sizes(const pnp_geom* g, const pnp_stage* stages, int n_stages, double* h_eta, void* d_ws,
                   void* stream);

/* The iteration schedule of Algorithm 1 as a caller that unrolls it walks it
 * (the differentiable form): for iteration i = 1..T, T = the sum of the stages'
 * iters (written to *h_total),
 *   h_stage[i-1]   index k of its stage (factor s_k, subsets P_k, eta_k)
 *   h_subset[i-1]  its angle subset: h_subset_seq[i-1] when P_k > 1, else 0
 *   h_amom[i-1]    its momentum coefficient a_i = (i-1)/(i+3) (Sec. 3) when
 *                  momentum != 0, else 0 (Eq. 5) -- the a_i that pnp_run uses.
 * The arrays hold `capacity` entries; PNP_EINVAL (with *h_total set) when T
 * exceeds it, or when a subset id lies outside its stage's [0, P_k).
 * Host only; launches nothing. */
int pnp_schedule(const pnp_stage* stages, int n_stages, const int32_t* h_subset_seq, int momentum,
                 int32_t* h_stage, int32_t* h_subset, float* h_amom, int64_t capacity, int64_t* h_total);

/* The subset order of Algorithm 1's minibatches (Sec. 2: each iteration's
 * minibatch is drawn at random, Eq. 6-7), read as sampling the P angle subsets
 * without replacement per epoch.  Writes the subset id of every iteration
 * i = 1..T (T = sum of the stages' iters, written to *h_total) to h_seq[i-1]:
 * stage by stage, a stage with P = n_subsets > 1 runs in epochs of P
 * iterations, each a uniform permutation of 0..P-1 (a shorter last epoch takes
 * the first entries of its permutation); a stage with P = 1 gives zeros.
 * Permutation: Durstenfeld's Fisher-Yates shuffle of the identity, for
 * j = P-1 down to 1 swapping entries j and r, r uniform in [0, j].  Uniform
 * integers in [0, m): the next number u of a SplitMix64 stream (Steele, Lea &
 * Flood 2014: the t-th number, t = 1, 2, ..., is SplitMix64's finaliser of
 * seed + t * 0x9e3779b97f4a7c15), redrawn while u < 2^64 mod m, taken mod m.
 * One stream serves the whole schedule.  h_seq holds `capacity` entries (it
 * may be NULL with capacity 0 to ask for T); PNP_EINVAL (with *h_total set)
 * when T exceeds it or a stage has iters < 0 or n_subsets < 1.
 * Host only; launches nothing. */
int pnp_subset_sequence(const pnp_stage* stages, int n_stages, uint64_t seed, int32_t* h_seq, int64_t capacity,
                        int64_t* h_total);

/* Algorithm 1 (PnP-MS2G) on every image of the batch.
 *   stages[n_stages]   the schedule; h_eta[n_stages] step sizes eta_k, or NULL
 *                      for eta_k = 1/L_k from pnp_step_sizes (the first run
 *                      that needs a level's L then synchronises `stream`)
 *   h_subset_seq       subset id of every iteration (length sum iters), or
 *                      NULL for the order pnp_subset_sequence draws from
 *                      params->subset_seed
 *   params             alpha, lambda, tv_iters, momentum
 *   d_b                data [batch][n_views][n_det]
 *   d_x                in: x_0 (= y_0), out: x after the last iteration
 *   d_xtrue, h_psnr_log  optional (both or neither): per-iteration PSNR
 *                      (peak 1) of every instance, [total_iters][batch];
 *                      the call then synchronises `stream` before returning
 * Iteration i: v = S_k y_{i-1}; r = A_s^{(p_i)} v - b^{(p_i)};
 *   z = y_{i-1} - eta_k c S_k^T A_s^{(p_i)T} r;  x_i = (1-alpha) z + alpha D(z);
 *   y_i = x_i + a_i (x_i - x_{i-1}).
 * S_k and U_k = S_k^T follow the stage's sketch kind; with an SVRG or SAGA
 * stage the gradient term is that estimator's (see PNP_EST_*), which needs an
 * estimator buffer (pnp_set_vr_buffer; PNP_ESTATE without one). */
int pnp_run(const pnp_geom* g, const pnp_stage* stages, int n_stages, const double* h_eta,
            const int32_t* h_subset_seq, const pnp_run_params* params, const float* d_b,
            float* d_x, const float* d_xtrue, double* h_psnr_log, void* d_ws, void* stream);

/* Algorithm 1 on several geometry classes at once (images of uneven size,
 * views and bins): every iteration runs each projector and denoiser phase as
 * ONE launch covering up to 4 classes that are still iterating (more classes:
 * one launch per phase for each group of 4, in class order); classes may have
 * schedules of different lengths; iteration i of every class uses the same
 * momentum a_i and params.  One denoiser launch serves every class, so the
 * classes share its variant (the register-resident ones only when every class
 * was tuned to one); a class whose own tuned variant differs can then differ
 * from its single-class pnp_run in the last bits (both within the reconstruction
 * tolerance).  A class given without a subset sequence takes the order
 * pnp_subset_sequence draws for its stages from params->subset_seed.
 * Workspaces and outputs must be distinct per class.  Synchronous only when some class logs PSNR.  PNP_EUNSUPPORTED for
 * more than 1024 classes.
 * Checkpoint/resume: a class with start_iter = k continues Algorithm 1 from
 * iteration k + 1 with d_x = x_k and d_y = y_k (both returned by an earlier run
 * that stopped after k iterations, e.g. a schedule cut at k); the result is
 * bitwise identical to an uninterrupted run. */
int pnp_run_many(const pnp_problem* problems, int n_problems, const pnp_run_params* params, void* stream);

/* Launch shapes of a prepared workspace, per sketch level (index 0..3 for the
 * factors 1, 2, 4, 8), 0 meaning the built-in heuristic:
 *   lanes   forward projector lanes per ray: 4, 8 or 16
 *   back    backprojector CTA: G view groups (1..32) of 8 x 4 pixel blocks, or
 *           PNP_BACK_TILE4 | G: G view groups (1..64) of 4 x 4 pixel blocks
 *           (the pixel-driven gather), or PNP_BACK_SCATTER | TS: the
 *           sample-driven scatter on TS x TS tiles, TS in {12, 16, 22, 32};
 *           a gather shape | PNP_BACK_BATCH(BC), BC in {4, 8, 16}, selects the
 *           batched gather: each thread applies every hat product it computes to
 *           the residuals of BC images of the batch (the images of one geometry
 *           share all rays and samples), with at most 512 threads per CTA
 *           (G x 32 or G x 16 for 8 x 4 or 4 x 4 blocks); its results are bitwise
 *           those of the same gather shape without PNP_BACK_BATCH
 *   tile    FGP denoiser: side of the shared-memory tile (8..40), 1 for the
 *           register-resident warp tiles (five iterations per launch), or 2 / 3 / 4
 *           for the register-resident strips (64 columns x 64 / 96 / 128 rows per
 *           CTA, two columns per lane, ten iterations per launch)
 * The gather's view groups fix its summation order: results are bitwise
 * reproducible for fixed shapes.  The scatter adds each sample's four bilinear
 * terms as 32-bit fixed-point integers (scale: the tile's largest |residual|
 * maps to at most 2^21, lower where the geometry lets more terms reach one
 * pixel within a chunk of views), so its sums do not depend on the order of
 * the adds and are bitwise reproducible too; they differ from the gather's by
 * that quantisation: about 2^-21 of the tile's largest |residual| per term, so
 * the error grows with the residual's dynamic range within a tile (measured
 * 2-3e-6 relative for residuals spread over three decades, 8e-7 for the FP32
 * gather, which has no such dependence and is the shape to pin where that
 * matters); a non-finite residual turns the outputs of every scatter tile its
 * ray can reach into NaN.  pnp_autotune sets the
 * shapes, choosing among the gather's shapes only (the scatter's error depends
 * on the data, so it runs only where pnp_set_launch_shapes pins it);
 * pnp_set_launch_shapes pins them (PNP_EINVAL for a shape outside these sets).
 * PNP_BACK_TABLE | PNP_BACK_BATCH(BC) | G (G 1..16, BC in {2, 4, 8, 16}; 0 counts
 * as 2) reads the stored gather table of pnp_set_gather_table instead of
 * evaluating the hats: CTAs of 32 blocks x G view groups, bitwise the sums of
 * the gather with the same G; without a registered table it runs as that
 * gather (batched for BC >= 4). */
#define PNP_BACK_TILE4 (1 << 8)
#define PNP_BACK_SCATTER (1 << 9)
#define PNP_BACK_BATCH(bc) ((bc) << 16)
#define PNP_BACK_TABLE (1 << 10)
typedef struct {
    int32_t lanes[4];
    int32_t back[4];
    int32_t tile;
} pnp_launch_shapes;
int pnp_get_launch_shapes(const pnp_geom* g, pnp_launch_shapes* out, void* d_ws);
int pnp_set_launch_shapes(const pnp_geom* g, const pnp_launch_shapes* in, void* d_ws);

/* Stored gather table of A_s^T (Eq. 5's transpose, with the weights of the
 * pixel-driven gather): the gather's weights depend on the geometry alone, so
 * they can be computed once per geometry and read back from HBM instead of
 * being re-evaluated in every backprojection.  For every sketch level present
 * in the workspace, every view and 2x2 pixel block: the bins of the rays that
 * meet the block's support (in increasing order) and the four summed hat
 * products of each, in groups of 32 blocks stored slot by slot (a group takes
 * as many slots as its block with the most rays).  About 2.3 entries of 20 B
 * per block and view: 2.6 GB for the full grid of 512^2 / 720 x 768, 3.4 GB for
 * all its levels.
 * pnp_gather_table_size: bytes the table of d_ws's geometry needs (runs the
 *   counting kernel on the workspace's ray tables; overwrites the workspace's
 *   denoiser state buffers; synchronous).
 * pnp_set_gather_table: builds the table into d_table (caller-owned, at least
 *   that many bytes, 256-byte aligned; PNP_EINVAL otherwise) and registers it
 *   with d_ws, so that launch shapes with PNP_BACK_TABLE (and pnp_autotune,
 *   which then times them) use it; d_table == NULL unregisters.  The caller
 *   keeps the buffer alive while the workspace uses it; pnp_setup on the
 *   workspace drops the registration.  Synchronous.  Library instrumentation
 *   of the path, no counterpart in the paper (which evaluates A^T matrix-free). */
int pnp_gather_table_size(const pnp_geom* g, void* d_ws, size_t* bytes, void* stream);
int pnp_set_gather_table(const pnp_geom* g, void* d_table, size_t bytes, void* d_ws, void* stream);

/* Times the launch shapes of this geometry's kernels on d_ws's own buffers
 * (forward lanes per ray 4/8/16 and the gather backprojector's view groups for each
 * sketch level of the schedule, using its first angle subset; the FGP tile side
 * around the cost-model choice) and records the fastest for later calls that
 * use d_ws.  Shapes change only the order of floating-point sums (results stay
 * within rounding of each other and deterministic for fixed shapes).
 * Synchronous; overwrites the workspace's scratch buffers. */
int pnp_autotune(const pnp_geom* g, const pnp_stage* stages, int n_stages, const pnp_run_params* params,
                 void* d_ws, void* stream);

/* Final FP64 reductions for every instance: h_out[3*i + 0] = 1/2 ||A x - b||^2,
 * h_out[3*i + 1] = TV(x) (isotropic, as in the denoiser), h_out[3*i + 2] =
 * PSNR(x, xtrue) (peak 1; NaN when d_xtrue is NULL).  Synchronous. */
int pnp_objective(const pnp_geom* g, const float* d_x, const float* d_b, const float* d_xtrue,
                  double* h_out, void* d_ws, void* stream);

/* Exact number of in-image samples (inside |x|,|y| < (n_s/2 + 1/2) s) over the
 * rays of the subset, one instance: the work unit of GRay-samples/s.
 * Synchronous. */
int pnp_sample_count(const pnp_geom* g, int factor, int subset, int n_subsets, double* h_count,
                     void* d_ws, void* stream);

/* ---------------------------------------------------------------------------
 * Differentiable form.  Sec. 2 of the paper remarks that the sketched
 * iterations (and their denoiser and sampling operators) can be unrolled and
 * trained end to end.  These calls give one iteration of Algorithm 1 as a
 * differentiable function of (y_{i-1}, x_{i-1}, lambda) and its exact
 * vector-Jacobian product; the VJP recomputes the iteration's forward pass, so
 * a caller that unrolls T iterations keeps only each iteration's inputs
 * (per-iteration checkpointing).  The FGP reverse sweep follows the FGP
 * recurrence of pnp_tv_denoise backwards (projection Jacobian
 * (I - a a^T/|a|^2)/|a| where |a| > 1, identity elsewhere).
 * --------------------------------------------------------------------------- */

/* Bytes of VJP workspace for pnp_tv_vjp on [batch][n][n] with `iters` FGP
 * iterations (all pre-projection points of the forward pass are stored). */
int pnp_tv_vjp_workspace_size(int n, int batch, int iters, size_t* bytes);

/* Reverse mode of pnp_tv_denoise: d_zbar = (dx/dz)^T d_xbar and, if h_lambar is
 * not NULL, h_lambar[b] = <d_xbar[b], dx[b]/dlambda> for each instance
 * (synchronous then).  lambda > 0 when iters > 0.  d_ws of
 * pnp_tv_vjp_workspace_size bytes. */
int pnp_tv_vjp(const float* d_z, const float* d_xbar, float* d_zbar, double* h_lambar, int n, int batch,
               float lambda, int iters, void* d_ws, size_t ws_bytes, void* stream);

/* Bytes of the second (VJP) workspace of pnp_unrolled_step_vjp. */
int pnp_vjp_workspace_size(const pnp_geom* g, int tv_iters, size_t* bytes);

/* One iteration of Algorithm 1 with sketch factor `factor`, angle subset
 * (subset, n_subsets), step eta, momentum coefficient amom (the a_i of that
 * iteration) and params alpha, lambda, tv_iters (momentum field unused):
 *   z = y - eta c S^T A_s^{(p)T}(A_s^{(p)} S y - b^{(p)});
 *   x_out = (1 - alpha) z + alpha D(z);  y_out = x_out + amom (x_out - x_prev).
 * Inputs are not modified; outputs must not alias inputs. */
int pnp_unrolled_step(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                      const pnp_run_params* params, float amom, const float* d_y, const float* d_xprev,
                      const float* d_b, float* d_xout, float* d_yout, void* d_ws, void* stream);

/* VJP of pnp_unrolled_step: given d_xbar, d_ybar (gradients of a loss with
 * respect to x_out and y_out) returns d_ybar_in = dJ/dy, d_xpbar = dJ/dx_prev
 * and, if h_lambar is not NULL, h_lambar[b] = dJ/dlambda for each instance
 * (synchronous then).  d_vjp_ws of pnp_vjp_workspace_size bytes.  The data b
 * is treated as a constant. */
int pnp_unrolled_step_vjp(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                          const pnp_run_params* params, float amom, const float* d_y, const float* d_b,
                          const float* d_xbar, const float* d_ybar, float* d_ybar_in, float* d_xpbar,
                          double* h_lambar, void* d_ws, void* d_vjp_ws, size_t vjp_ws_bytes, void* stream);

/* pnp_unrolled_step that also stores z = y - eta c S^T A_s^{(p)T}(...) into
 * d_zout [batch][n][n] (may not alias the other arguments), so that the VJP can
 * start from it instead of recomputing the gradient step. */
int pnp_unrolled_step_save(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                           const pnp_run_params* params, float amom, const float* d_y, const float* d_xprev,
                           const float* d_b, float* d_xout, float* d_yout, float* d_zout, void* d_ws,
                           void* stream);

/* pnp_unrolled_step_vjp from the z that pnp_unrolled_step_save stored (d_z)
 * instead of recomputing it from y: one projector pair fewer per iteration. */
int pnp_unrolled_step_vjp_saved(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                                const pnp_run_params* params, float amom, const float* d_z,
                                const float* d_xbar, const float* d_ybar, float* d_ybar_in, float* d_xpbar,
                                double* h_lambar, void* d_ws, void* d_vjp_ws, size_t vjp_ws_bytes,
                                void* stream);

/* Bytes of scratch inside the library for pnp_full_grad_noalloc (per GPU that
 * loads the library, held until the process exits). */
#define PNP_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The full gradient of pnp_full_grad, d_g = A^T (A d_x - d_b), for callers that
 * cannot allocate device memory: a real-time scanner service that fixes its
 * memory at start-up so no request can fail or stall on allocation, or a
 * plug-in inside an application whose allocator owns all of the GPU's memory.
 * The paper has no counterpart; it is an interface for such callers.
 *   It allocates nothing and takes no workspace: its scratch lives in a fixed
 *   PNP_NOALLOC_SCRATCH_BYTES array compiled into the library.  A geometry needs
 *   32 B per ray (rayf 16, rayi 8, rayk 8) and 16 B per view (ray tables), plus
 *   per batch image 16 (n+3)^2 B (coefficient image) and 4 B per ray (residual),
 *   each part rounded up to 256 B; e.g. 256x256 with 360 views x 512 bins needs
 *   about 7.7 MB.  Geometries that need more are rejected with PNP_EINVAL and a
 *   message.
 *   It is always the unweighted gradient: weights registered with
 *   pnp_set_weights belong to a workspace and do not apply here, so it equals
 *   pnp_full_grad only for a workspace without weights.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current) and keeps it for the life of the process;
 *   make that first call before any stream capture.  The address is not valid
 *   across cudaDeviceReset: a process that resets a device must not call this
 *   entry point on it afterwards.
 *   All calls share the array: calls that overlap on the GPU (other streams or
 *   host threads) race and give wrong results; order them on one stream.
 *   Every call rewrites all the scratch it reads, so nothing needs clearing.
 *   d_x, d_g [batch][n][n], d_b [batch][n_views][n_det]; asynchronous on `stream`. */
int pnp_full_grad_noalloc(const pnp_geom* g, const float* d_x, const float* d_b, float* d_g, void* stream);

/* Read bandwidth (GB/s) of the on-chip memory levels of the current GPU,
 * measured with this library's probe kernels and CUDA events (best of three
 * timed launches each, after a warm-up): h_gbs[0] L2 (a 24 MiB buffer streamed
 * by every SM with L1-bypassing 16-byte loads), h_gbs[1] L1 (each block
 * re-reading a private 16 KB window), h_gbs[2] shared memory (each block
 * re-reading 32 KB, conflict-free 16-byte words).  These are the denominators of
 * the projector kernels' on-chip rooflines.  d_buf: caller-owned scratch of at
 * least 32 MiB (PNP_EINVAL names the size needed when it is short), 256-byte
 * aligned, overwritten.  Synchronous.  Library instrumentation; the paper has no
 * counterpart. */
int pnp_onchip_bandwidth(void* d_buf, size_t bytes, double* h_gbs, void* stream);

/* Device time (ms, summed) and number of timed launches of each phase over all
 * runs with PNP_RUN_KERNEL_TIMES since the last reset, indexed by PNP_PHASE_*.
 * h_ms and h_launches hold PNP_N_PHASES entries each (either may be NULL).
 * Waits for the recorded events to complete.  reset != 0 clears the totals
 * afterwards.  Library instrumentation; the paper has no counterpart. */
int pnp_kernel_times(double* h_ms, int64_t* h_launches, int reset);

/* Number of kernels this library has launched in this process. */
uint64_t pnp_launch_count(void);

/* Message of the last failed call on this thread ("" if none). */
const char* pnp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PNP_MS2G_H */
