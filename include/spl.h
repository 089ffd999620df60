/*
 * libspl — GB300 (sm_103a) engine for the stationary timestamp pmf of an
 * asynchronous single-photon LiDAR pixel under SPAD dead time
 * (Zhang, Weerasooriya, Chennuri, Chan, "Real-Time Markov Modeling for
 * Single-Photon LiDAR", arXiv 2509.20500).
 *
 * Problem (Sec. 2.2): given theta = (t_r, t_d, sigma, tau, S, B, n_b), return
 * the registration pmf f_r over the n_b TCSPC bins, computed as the stationary
 * distribution pi of the timestamp Markov chain, pi P~ = pi (Sec. 2.3).
 *
 * Conventions shared by every call:
 *  - Times (t_r, t_d, tau, sigma) are in one unit of the caller's choice.
 *  - Bins are 0-based, bin j covers ((j) Delta, (j+1) Delta] with centre
 *    s_j = (j + 1/2) Delta, Delta = t_r / n_bins (state set, Sec. 2.3; the
 *    discretiser D of Sec. 3.1).  The bin width is never passed: the dead-time
 *    shift is computed from n_bins and t_r as
 *        q = fmod(t_d, t_r) * n_bins / t_r   (IEEE FP64, in that order)
 *        l = ceil(q)                         (Theorem 2)
 *    so dead times on the bin grid give exact integer shifts.
 *  - Lambda is the flux of one laser period of the Eq. 1 flux, F(t_r): the
 *    Gaussian pulse is truncated to [0, t_r) and not renormalised.
 *  - Device pointers are CUDA device addresses owned by the caller (PyTorch
 *    allocates them); host pointers are ordinary host memory.  "stream" is a
 *    cudaStream_t passed as void*; NULL means the legacy default stream.
 *  - Every call returns an spl_status_t and never aborts the process.  On
 *    SPL_ECUDA the CUDA error is kept for spl_last_cuda_error().
 *  - Results are FP32 pmfs (sum 1).  Matrix entries and power iterations run
 *    in FP32; the cumulative flux F, Lambda and the exponentials that turn them
 *    into per-bin factors run in FP64 on the GPU.
 *  - Threads: the batch calls of one device share the library's workspace for
 *    that device and take its lock, so they may come from several host
 *    threads (they run one at a time; spl_batch_stationary_noalloc shares one
 *    static scratch area instead, see there).  A chain (spl_chain_t) or a
 *    network (spl_mlp_t) is used by one thread at a time; distinct objects are
 *    independent.  The per-pixel host work of a large batch call runs on a
 *    small pool of library threads (up to 7, started on the first such call,
 *    idle between calls, never joined); in a process forked after they
 *    started, that work runs on the calling thread.
 */
#ifndef SPL_H
#define SPL_H

#include <stdint.h>

#if defined(__GNUC__)
#define SPL_API __attribute__((visibility("default")))
#else
#define SPL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* One pixel.  n_bins >= 2.  shift_override = -1 uses the paper's row shift
 * l = ceil(q) (Theorem 2); a value >= 0 forces that shift (for example
 * ceil(q + 1/2) - 1, which reproduces the sequential shift-then-quantise
 * construction of Eq. 4 exactly).  Valid input: t_r > 0, sigma > 0, t_d >= 0,
 * S >= 0, B >= 0, S + B > 0, 0 <= tau < t_r, all finite, Lambda <= 120. */
typedef struct {
    double t_r, t_d, tau, sigma, S, B;
    int32_t n_bins;
    int32_t shift_override;
} spl_pixel_t;

typedef enum {
    SPL_OK = 0,
    SPL_EINVAL = 1,    /* invalid argument: bad theta, NULL pointer, n < 0, size limit */
    SPL_ENOMEM = 2,    /* device or host allocation failed */
    SPL_ECUDA = 3,     /* a CUDA runtime/driver call failed */
    SPL_ENOCONV = 4,   /* max_iter steps did not meet the stop rule, or the iterate settled on an FP32
                          rounding floor above the tolerance; result is the last iterate */
    SPL_ETIMEOUT = 5,  /* a bounded device-side wait gave up; result undefined */
} spl_status_t;

typedef enum {
    SPL_MATERIALIZED = 0,  /* P stored in HBM (FP32, 4 N^2 bytes); power step is a TMA-staged GEMV */
    SPL_FUSED = 1,         /* P never stored; power step regenerates each tile of P~ in registers */
} spl_mode_t;

/* Per-pixel outcome of an iteration. */
typedef struct {
    int32_t iters;          /* power steps taken */
    int32_t status;         /* spl_status_t of this pixel */
    float last_step_l1;     /* ||pi_k - pi_{k-1}||_1 of the last step */
    float err_bound;        /* estimated L1 distance of the result to the exact pi */
    float lambda2_abs;      /* estimate of |lambda_2| of P~ (Sec. 4.1); -1 if none */
    float lambda2_phase;    /* estimate of arg(lambda_2) in radians, [0, pi] (Sec. 4.2) */
} spl_report_t;

typedef struct spl_chain spl_chain_t;   /* opaque; owned by the library */

/*
 * Build the chain of one pixel (Sec. 3.2-3.4).
 *   Computes, on `stream`, the per-bin flux lambda(s_j) (Eq. 1), the
 *   cumulative flux F(s_j) and Lambda = F(t_r) (Theorem 1) in FP64, and from
 *   them the factors of Eq. 6.  mode SPL_MATERIALIZED additionally writes the
 *   N x N matrix P_ij = lambda(s_j) exp(F(s_p) - F(s_j) - Lambda 1{p > j}),
 *   p = (i + l) mod N (Eq. 6 after the row roll E = J_l E_base, Sec. 3.4),
 *   with the roll folded into the row address, plus its row sums.
 *   *out receives a chain that owns all device scratch it needs; release it
 *   with spl_free.  The call is asynchronous on `stream` except for its
 *   device allocations.
 * Errors: SPL_EINVAL (theta, p == NULL, out == NULL), SPL_ENOMEM, SPL_ECUDA.
 */
SPL_API spl_status_t spl_build(const spl_pixel_t *p, spl_mode_t mode, void *stream, spl_chain_t **out);

/*
 * Stationary pmf of a built chain by power iteration, pi <- pi P~ with
 * renormalisation (Sec. 2.3, Sec. 3.4).
 *   tol      : target L1 error of the result (for example 1e-6).  The stop
 *              rule bounds the remaining error with the last steps and the
 *              estimate of lambda_2 (modulus and phase, Sec. 4).
 *   max_iter : step limit (> 0).
 *   d_warm   : NULL for the uniform start, else a device vector of n_bins
 *              nonnegative weights with positive sum (normalised here).
 *   d_pi     : device output, n_bins floats.
 *   rep      : host pointer (may be NULL) for the report.
 * Synchronises the chain's stream (it reads convergence flags back).
 * Errors: SPL_EINVAL, SPL_ECUDA, SPL_ENOCONV (d_pi holds the last iterate).
 */
SPL_API spl_status_t spl_stationary(spl_chain_t *c, double tol, int32_t max_iter, const float *d_warm,
                            float *d_pi, spl_report_t *rep);

/*
 * Stationary pmfs of many independent pixels with uneven n_bins in one
 * persistent launch (matrix-free; one thread block per pixel at a time,
 * largest pixels first).
 *   h_pixels  : host array of n pixels.
 *   tol, max_iter : as in spl_stationary, per pixel.
 *   d_warm    : NULL or a device array packed like d_out (nonnegative weights).
 *   d_out     : device output, packed: pixel k occupies
 *               d_out[d_offsets[k] .. d_offsets[k] + n_bins_k).
 *   d_offsets : device int64 array [n + 1] of those offsets (caller-owned).
 *   h_reports : host array [n] or NULL.  When non-NULL the call synchronises
 *               `stream` to fill it; when NULL the call is asynchronous.
 * Returns the worst per-pixel status (SPL_ENOCONV < SPL_ETIMEOUT), or
 * SPL_EINVAL for any invalid pixel (nothing is launched then).
 */
SPL_API spl_status_t spl_batch_stationary(const spl_pixel_t *h_pixels, int32_t n, double tol, int32_t max_iter,
                                  const float *d_warm, float *d_out, const int64_t *d_offsets,
                                  spl_report_t *h_reports, void *stream);

/* Kinds of warm start for spl_batch_stationary_ex (d_warm). */
typedef enum {
    SPL_WARM_WEIGHTS = 0,   /* nonnegative weights packed like d_out; start = weights / sum */
    SPL_WARM_LOGITS = 1,    /* logits packed like d_out; start = softmax */
    SPL_WARM_LEARNED = 2,   /* rows of warm_ld floats per pixel (caller order) in the learned frame:
                               start_j ~ exp(z[(j - c) mod N] + log lambda(s_j)), c = floor(tau / Delta) */
} spl_warm_kind_t;

/* Form of the power step of the batch kernel. */
typedef enum {
    SPL_PASS_DENSE = 0,       /* every entry of P~ regenerated and used (N^2 FFMA per step) */
    SPL_PASS_STRUCTURED = 1,  /* the same step through the triangular structure of Eq. 6:
                                 y_j = w_j (P_j + e^-Lambda (T - P_j)) with P a prefix sum
                                 (O(N) per step; row sums by prefix and suffix scans) */
    SPL_PASS_DENSE_ROWSCAN = 2, /* dense power steps as SPL_PASS_DENSE (N^2 FFMA per step), with the
                                 row sums of P~'s normalisation taken from the same triangular
                                 structure: r'_k = u_k (sum_{j>=k} w_j + e^-Lambda sum_{j<k} w_j), a
                                 suffix and a prefix scan (O(N) once per pixel, instead of one more
                                 dense pass) */
} spl_pass_kind_t;

/* Column weights of P~ (how the detection density enters bin j). */
typedef enum {
    SPL_FLUX_POINT = 0,       /* the paper's form (Sec. 3.4): lambda(s_j) exp(-F(s_j)) at the bin centre */
    SPL_FLUX_BININT = 1,      /* an ablation beyond the paper: the exact integral of the detection density
                                 over the bin, exp(-F(j Delta)) - exp(-F((j+1) Delta)) (the point form is its
                                 midpoint rule; the two agree to O(Delta^2)) */
} spl_flux_kind_t;

/* Options for spl_batch_stationary_ex. */
typedef struct {
    int32_t warm_kind;        /* spl_warm_kind_t, used when d_warm != NULL */
    int32_t warm_ld;          /* row stride of SPL_WARM_LEARNED logits (>= n_bins) */
    int32_t min_iter;         /* steps always taken before the stop rule may fire (>= 1) */
    int32_t threads;          /* threads per block, 0 = library default */
    int32_t time_kernel;      /* 1: record CUDA events around the batch kernel (see spl_batch_kernel_ms) */
    int32_t pass_kind;        /* spl_pass_kind_t */
    int32_t flux_kind;        /* spl_flux_kind_t */
    int32_t tune;             /* launch configuration: 0 (default) measured on the first batch of at least
                                 1024 pixels of a kind (padded n_bins, pass kind, SM count) and cached, also in
                                 the file SPL_TUNE_CACHE names if set: block size (256 or 512 threads) and
                                 columns per thread (8 or 4; dense passes only), state level, blocks per SM.
                                 1 fixed heuristic (256 threads, 8 columns); 2 explicit threads, state_level and
                                 cols.  State level and blocks per SM leave the pmfs unchanged bit for bit; the
                                 block size (order of the block reductions) and the columns per thread (where
                                 the diagonal span splits each column's sum) change them within rounding. */
    int32_t state_level;      /* tune == 2: per-pixel vectors in shared memory (2 all, 1 three, 0 one) */
    int32_t cols;             /* tune == 2, dense passes: columns per thread, 8 or 4 (0 = 8) */
} spl_batch_opts_t;

/* spl_batch_stationary with options (opts may be NULL for the defaults). */
SPL_API spl_status_t spl_batch_stationary_ex(const spl_pixel_t *h_pixels, int32_t n, double tol, int32_t max_iter,
                                     const float *d_warm, float *d_out, const int64_t *d_offsets,
                                     spl_report_t *h_reports, void *stream, const spl_batch_opts_t *opts);

/*
 * Spectral analysis of many pixels (Sec. 4, Fig. 4 columns 1-2): the modulus
 * and phase of lambda_2, the subdominant eigenvalue of P~ that sets the
 * spectral gap 1 - |lambda_2| and the oscillation of the convergence.
 * Per pixel: pi by power iteration, then `subspace_iters` steps of
 * orthogonal iteration on two vectors deflated against pi with a 2 x 2
 * Rayleigh-Ritz projection (complex pairs resolved); every product with P~
 * uses the O(N) structured form of Eq. 6.  FP32; accuracy about 1e-4 when
 * |lambda_3| / |lambda_2| is well below 1.
 *   d_out : device [n][2] floats: |lambda_2|, |arg lambda_2| in [0, pi].
 * n_bins <= 4096.  Synchronises `stream`.
 */
SPL_API spl_status_t spl_batch_spectral(const spl_pixel_t *h_pixels, int32_t n, int32_t subspace_iters,
                                        float *d_out, void *stream);

/*
 * Event Monte Carlo reference histograms (Sec. 5, Fig. 3b/3c; the detector
 * model of Sec. 2.2): for each pixel, `runs` independent runs of `cycles`
 * laser cycles each.  Per cycle, Poisson(S) Gaussian signal photons (kept
 * inside [0, t_r)) and Poisson(B) uniform background photons, in time order,
 * pass a non-paralysable dead time t_d that carries across cycles; each
 * registration counts in bin floor(t N / t_r).  Random numbers: Philox4x64-10
 * with key (seed, k 2^32 + r) for run r of pixel k and counter
 * (cycle, block, 0, 0); the experiment is exactly specified (FP64, no
 * contraction), so the same seed gives the same histograms on any
 * implementation of it.  shift_override is ignored.
 *   d_hist : device uint32, run r of pixel k at runs * off_k + r * N_k,
 *            off_k = sum of n_bins of pixels 0..k-1 (caller-owned, fully
 *            written).
 * Limits: n_bins <= 16384, S <= 16, B <= 16 (at most 64 photons per source
 * and cycle; more has probability < 1e-18), n * runs < 2^31.
 * Errors: SPL_EINVAL for invalid pixels or limits, SPL_ENOMEM, SPL_ECUDA.
 * Allocates a small parameter buffer; synchronises `stream`.
 */
SPL_API spl_status_t spl_mc_histograms(const spl_pixel_t *h_pixels, int32_t n, int32_t runs, int64_t cycles,
                                       uint64_t seed, uint32_t *d_hist, void *stream);

/* The measured launch configuration cached for batches whose largest pixel
 * has n_bins_max bins and pass kind pass_kind on the current device:
 * SPL_OK with *threads, *state_level, *blocks_per_sm and *cols (columns per
 * thread; cols may be NULL), or SPL_ENOCONV if none is cached yet. */
SPL_API spl_status_t spl_batch_tune_lookup(int32_t n_bins_max, int32_t pass_kind, int32_t *threads,
                                           int32_t *state_level, int32_t *blocks_per_sm, int32_t *cols);

/* Device time in ms of the batch kernel of the last spl_batch_stationary_ex
 * call on the current device that set time_kernel (events recorded on that
 * call's stream just before and after the kernel launch).  Waits for the end
 * event.  SPL_EINVAL if no timed call was made. */
SPL_API spl_status_t spl_batch_kernel_ms(float *ms);

/*
 * Same computation as spl_batch_stationary with HOST buffers: h_warm (NULL or
 * packed host floats), h_out (packed host floats, offsets from the n_bins of
 * h_pixels in order) and h_reports (may be NULL).  Copies inputs to the device
 * and results back inside the call; synchronises `stream`.  One launch; in
 * a batch of one size the kernel counts the finished pixels of each of eight
 * caller ranges, the calling thread polls the counts and copies a range back
 * on a library-owned stream as soon as it is complete, while the kernel runs
 * on (same pmfs bit for bit as the device-buffer call).
 */
SPL_API spl_status_t spl_batch_stationary_host(const spl_pixel_t *h_pixels, int32_t n, double tol, int32_t max_iter,
                                       const float *h_warm, float *h_out, spl_report_t *h_reports,
                                       void *stream);

/*
 * spl_batch_stationary without any allocation.  The paper has no counterpart;
 * this entry point exists for callers that may not allocate device memory:
 * real-time pipelines that ban allocation once running (cudaMalloc can
 * synchronise the device and its latency is unbounded) and plug-ins inside
 * an application whose own allocator owns the GPU memory budget.
 *   Arguments are those of spl_batch_stationary (d_warm: NULL or packed
 *   nonnegative weights; d_out and d_offsets caller-owned device arrays;
 *   h_reports NULL or host [n]).
 *   The kernel's device scratch (queue counter, work list, reports and the
 *   per-pixel flux constants) is a fixed file-scope device array of
 *   15,204,608 bytes (about 15.2 MB) that every GPU loading the library holds
 *   until the process exits; host staging is static too.  No cudaMalloc,
 *   cudaFree or other allocating routine is called.
 *   Limits: n <= 65536 pixels and 2 <= n_bins <= 3072 per pixel; larger
 *   requests return SPL_EINVAL before any device work.
 *   The first call on a device looks up the array's device address for that
 *   device (cudaGetSymbolAddress).  With lazy module loading (the CUDA
 *   default) that lookup loads the library's module on the device, which is
 *   when the array is reserved: the first call per device may allocate and
 *   synchronise the device.  Make it during start-up, before any stream
 *   capture; later calls allocate nothing.  All calls share the array and it keeps the previous call's
 *   contents (the queue counter is cleared by each call); calls whose work
 *   overlaps on the GPU race on it, so issue them one after the other.
 *   With h_reports the call synchronises `stream`; without, it is
 *   asynchronous.  Returns the worst per-pixel status, as the batch call.
 */
SPL_API spl_status_t spl_batch_stationary_noalloc(const spl_pixel_t *h_pixels, int32_t n, double tol,
                                                  int32_t max_iter, const float *d_warm, float *d_out,
                                                  const int64_t *d_offsets, spl_report_t *h_reports,
                                                  void *stream);

/*
 * Learned warm start (the paper has no network; this follows its batched use
 * case).  A 5 -> 4 x 512 (GELU, tanh form) -> 2000 MLP, BF16 weights with FP32
 * accumulation on the tensor cores, maps (sub-bin pulse position, sigma,
 * log S, log B, x_d / t_r) of an n_bins = 2000 pixel to a log-correction of
 * the flux prior lambda(s_j) in a frame rolled to the pulse bin; its softmax
 * starts the power iteration, which always runs to the stop rule (so the
 * network changes how many steps are needed, never the accuracy of the
 * result).
 *   spl_mlp_create   : device network for batches of up to max_batch pixels,
 *                      seeded uniform fan-in initialisation; owns its scratch
 *                      (device memory, and a pinned host buffer of max_batch
 *                      pixels through which the pixels are uploaded).
 *   spl_mlp_param_count / set_params / get_params : packed FP32 parameters,
 *                      per layer W (rows x cols, row-major) then b.
 *   spl_mlp_forward  : logits [n][2048] of pixels with n_bins == 2000 (B > 0);
 *                      d_logits may be NULL (kept inside the network).
 *   spl_mlp_loss_grad: mean cross-entropy of the start vector against d_target
 *                      ([n][2000] pmfs on the device) and, into h_grads
 *                      (packed like the parameters, may be NULL), its gradient.
 *   spl_mlp_train_step: one AdamW step on that loss (lr, weight_decay).
 *   spl_batch_stationary_learned: forward pass, then spl_batch_stationary
 *                      started from the network's warm start; stream must be
 *                      the network's stream.
 * All run on the network's stream; errors as the other calls.
 */
typedef struct spl_mlp spl_mlp_t;
SPL_API spl_status_t spl_mlp_create(int32_t max_batch, uint64_t seed, void *stream, spl_mlp_t **out);
SPL_API int64_t spl_mlp_param_count(void);
SPL_API spl_status_t spl_mlp_set_params(spl_mlp_t *m, const float *h_params, int64_t count);
SPL_API spl_status_t spl_mlp_get_params(spl_mlp_t *m, float *h_params, int64_t count);
/* AdamW state for checkpoints: h_state holds 2 x spl_mlp_param_count()
 * floats, the first moments then the second moments, each packed like the
 * parameters; *step / step is the optimiser step count (bias correction).
 * With the parameters it resumes training exactly. */
SPL_API spl_status_t spl_mlp_get_state(spl_mlp_t *m, float *h_state, int64_t count, int32_t *step);
SPL_API spl_status_t spl_mlp_set_state(spl_mlp_t *m, const float *h_state, int64_t count, int32_t step);
SPL_API spl_status_t spl_mlp_forward(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n, float *d_logits);
/* Device time of the forward pass alone: uploads the pixels once, then times
 * `reps` forward passes (features and the five GEMMs, logits kept inside the
 * network) with CUDA events on the network's stream; *ms_per_forward gets the
 * mean.  Synchronises the stream. */
SPL_API spl_status_t spl_mlp_time_forward(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n, int32_t reps,
                                          float *ms_per_forward);
SPL_API spl_status_t spl_mlp_loss_grad(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n, const float *d_target,
                                       float *h_loss, float *h_grads);
SPL_API spl_status_t spl_mlp_train_step(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n, const float *d_target,
                                        float lr, float weight_decay, float *h_loss);
SPL_API const float *spl_mlp_logits(spl_mlp_t *m);
SPL_API void spl_mlp_free(spl_mlp_t *m);
SPL_API spl_status_t spl_batch_stationary_learned(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n, double tol,
                                                  int32_t max_iter, float *d_out, const int64_t *d_offsets,
                                                  spl_report_t *h_reports, void *stream,
                                                  const spl_batch_opts_t *opts /* nullable; warm fields ignored */);
/* The same from and to host memory: pmfs into h_out (packed in caller order,
 * sum of n_bins floats; pinned memory copies fastest).  As
 * spl_batch_stationary_host, each of eight caller ranges of a batch of one
 * size is copied back as soon as the kernel has finished it (same pmfs bit
 * for bit). */
SPL_API spl_status_t spl_batch_stationary_learned_host(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n,
                                                       double tol, int32_t max_iter, float *h_out,
                                                       spl_report_t *h_reports, void *stream,
                                                       const spl_batch_opts_t *opts /* nullable */);

/*
 * Stationary pmfs of several fused chains in one launch (Sec. 3.4, the
 * matrix-free power iteration of Eq. 6, as spl_stationary with a uniform
 * start, for many pixels at once).
 *   chains: n distinct chains built with SPL_FUSED on one and the same stream
 *   (the call runs on that stream).  One cooperative launch (at most 32
 *   chains per launch; more run as consecutive launches) runs the chains in
 *   lockstep: at every power step the work of the chains still iterating
 *   (256-column tile x 32-row units, chain after chain) is split evenly over
 *   all resident CTAs, then their bins likewise for the normalisation, with
 *   one grid barrier per step.  Each chain has its own stop rule; a chain that
 *   stops leaves the step's work to the others, so no CTA idles while any
 *   chain iterates.
 *   d_out: device [sum of n_bins] FP32, the pmfs packed in chain order.
 *   h_reports: NULL or host [n]; with it the call synchronises the stream and
 *   returns the worst per-chain status, without it the call is asynchronous.
 *   Each chain's pmf is the one spl_stationary gives (same steps, same stop
 *   rule; its column pass is split over other CTAs, so sums are added in
 *   another order).  A chain may need more partial and statistics slots than
 *   its own single-chain plan: the first such call grows them (a device
 *   allocation, after a stream synchronisation).
 * Errors: SPL_EINVAL (NULL chain, a materialised chain, a chain given twice,
 * chains on different streams, n < 0, tol <= 0, max_iter < 1), SPL_ENOMEM,
 * SPL_ECUDA; per chain SPL_ENOCONV, SPL_ETIMEOUT as spl_stationary.
 */
SPL_API spl_status_t spl_chains_stationary(spl_chain_t *const *chains, int32_t n, double tol, int32_t max_iter,
                                           float *d_out, spl_report_t *h_reports);

/* Partial slots per column tile of each chain of a lockstep multi-chain
 * launch (host arithmetic only, no GPU needed): on a GPU with `sms` SMs
 * keeping `blocks_per_sm` CTAs resident (grid G = sms x blocks_per_sm), a
 * step's units are split as [b U / G', (b+1) U / G') over G' = min(G, U) CTAs
 * with U >= the chain's own units T x RB, so one tile of RB units meets at
 * most ceil(RB / max(1, floor(T RB / G))) + 1 CTAs (at most RB, at most G);
 * slots[g] is that bound for chain g (n_bins[g] bins).  1 <= n <= 32, else
 * SPL_EINVAL. */
SPL_API spl_status_t spl_chains_plan(const int32_t *n_bins, int32_t n, int32_t sms, int32_t blocks_per_sm,
                                     int32_t *slots);

/* Plan of a fused chain's persistent iteration (host arithmetic only, no GPU
 * needed): on a GPU with `sms` SMs keeping `blocks_per_sm` CTAs resident, a
 * chain of n_bins bins runs on `grid` CTAs; its column pass is cut into
 * tiles x row_blocks equal units (256 columns x 32 rows, vlen = rows padded),
 * CTA b taking units [b U / grid, (b+1) U / grid) with U = tiles x
 * row_blocks; `segs` partial slots per CTA; at most `chunk` rows staged in
 * shared memory at once.  SPL_EINVAL on bad arguments. */
typedef struct {
    int32_t grid, tiles, row_blocks, segs, chunk, vlen;
} spl_run_plan_t;
SPL_API spl_status_t spl_chain_run_plan(int32_t n_bins, int32_t sms, int32_t blocks_per_sm, spl_run_plan_t *out);

/* Self-test of the device-side bounded waits, for tests: an mbarrier phase
 * that nothing completes (the wait gives up after a short limit), and a grid
 * barrier of a three-CTA cooperative launch that one CTA never reaches (the
 * two waiting CTAs give up after the limit, set the error flag and poison the
 * arrival count, which would release any other waiter).  No fault, trap or hang is
 * involved.  SPL_OK if every wait gave up as designed, SPL_EINVAL if one did
 * not, SPL_ECUDA on a CUDA error.
 *
 * Fault injection for tests (host side, nothing reaches the GPU): with the
 * environment variable SPL_FAULT=alloc every batch call fails as if its first
 * device allocation had failed (SPL_ENOMEM); with SPL_FAULT=launch as if its
 * kernel launch had failed (SPL_ECUDA). */
SPL_API spl_status_t spl_selftest_bounded_waits(void *stream);

/* Measurement: the FP32 FMA throughput of the current device, the
 * denominator of the FP32 rooflines of the matrix-free passes.  A kernel of
 * 4 blocks x 256 threads per SM runs 16 independent FMA chains per thread for
 * `iters` rounds (2 x 16 x iters FLOP per thread); one untimed launch, then
 * `reps` launches timed one by one with CUDA events on `stream`.
 * *tflops_median / *tflops_best (may be NULL) get the median and fastest
 * launch in TFLOP/s, *sms_out (may be NULL) the SM count used.  The paper has
 * no counterpart: it is the roofline denominator, not part of the method.
 * SPL_EINVAL for iters < 1, reps < 1 or tflops_median == NULL; SPL_ENOMEM,
 * SPL_ECUDA. */
SPL_API spl_status_t spl_fp32_fma_peak(int32_t iters, int32_t reps, void *stream, double *tflops_median,
                                       double *tflops_best, int32_t *sms_out);

/* The MLP's tensor-core GEMM on its own, for tests: D[M][N] = A[M][K] B[N][K]^T
 * with row-major BF16 device matrices A, B and an FP32 device output D.
 * M % 128 == 0, K % 64 == 0, N % 32 == 0. */
SPL_API spl_status_t spl_gemm_bf16(const void *d_A, const void *d_B, int32_t M, int32_t N, int32_t K, float *d_D,
                                   void *stream);

/* Materialised chains only: copy P (the paper's unnormalised P of Eq. 4/6,
 * lambda_j E_ij without the constant 1/(1 - e^-Lambda)) to d_P, row-major
 * [n_bins][n_bins].  SPL_EINVAL for fused chains. */
SPL_API spl_status_t spl_matrix(spl_chain_t *c, float *d_P);

/* Measurement: device time of one dense power-step pass of a chain (the
 * TMA GEMV over the stored P, or the split regenerating column pass),
 * averaged over `reps` passes captured in one CUDA graph (so no host launch
 * overhead) and replayed after one untimed replay; CUDA events on the
 * chain's stream.  Leaves the chain's iterate reset. */
SPL_API spl_status_t spl_chain_time_pass(spl_chain_t *c, int32_t reps, float *ms_per_pass);

/* Measurement: device time of one whole power step of a chain (the dense
 * pass, the reduction of its partials, normalisation, step statistics, stop
 * rule and next broadcast vector) with the stop rule held open: materialised
 * chains as reps steps replayed from a captured graph, fused chains as one
 * persistent launch of reps steps (which makes one more pass for its lagged
 * stop decision), each after an untimed run.  Leaves the chain's iterate
 * reset. */
SPL_API spl_status_t spl_chain_time_step(spl_chain_t *c, int32_t reps, float *ms_per_step);

/* Measurement: device time of the materialised build (the write of P and its
 * row sums, Eq. 6 with the roll in the row address), averaged over `reps`
 * rebuilds after one warm-up; the stored P is rewritten with the same
 * values.  SPL_EINVAL for fused chains. */
SPL_API spl_status_t spl_chain_time_build(spl_chain_t *c, int32_t reps, float *ms_per_build);

/* Per-bin vectors of a built chain, for inspection: d_lambda (FP32 lambda(s_j)),
 * d_F (FP64 F(s_j)); either may be NULL.  h_Lambda (host, may be NULL) gets
 * Lambda; h_shift (may be NULL) the row shift in use. */
SPL_API spl_status_t spl_chain_flux(spl_chain_t *c, float *d_lambda, double *d_F, double *h_Lambda,
                            int32_t *h_shift);

/* Release a chain (NULL is ignored). */
SPL_API void spl_free(spl_chain_t *c);

/* Static text for a status. */
SPL_API const char *spl_strerror(spl_status_t s);

/* Text of the last CUDA error seen by this thread's calls ("" if none). */
SPL_API const char *spl_last_cuda_error(void);

/* Library version string. */
SPL_API const char *spl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPL_H */
