/*
 * saa.h -- C ABI of libsaa: GPU Monte Carlo sample-average (SAA) estimation
 * of the mean-variance objective, its gradient, and the Frank-Wolfe loop of
 * arXiv 2404.11631 ("A Preliminary Study on Accelerating Simulation
 * Optimization with GPU Implementation"), Sec. 3.1.
 *
 * Problem (Sec. 3.1, Eq. 3): minimise f(w) = (1/2) Var[w'R] - E[w'R] over
 * W = {w >= 0, 1'w <= 1}, R ~ D(mu, Sigma).  The SAA estimate (Eq. 4, with
 * the sample mean R_bar of Eq. 5) over N samples R_i is
 *
 *     f_hat(w) = lambda * (1/(N-1)) sum_i (w'(R_i - R_bar))^2 - w'R_bar,
 *
 * lambda = 1/2 reproducing Eq. 3 (Eq. 4 as printed has lambda = 1).  The
 * library evaluates f_hat and grad_w f_hat for K candidate decisions at once
 * and runs Algorithm 1 (Frank-Wolfe with resampling every M iterations).
 *
 * Samples.  R_i = mu + s_i C zhat_i, C the lower Cholesky factor of Sigma,
 * zhat_i innovations drawn in-kernel from a counter-based Philox4x32-10
 * stream (Salmon et al., SC'11) keyed by `seed`, with counter
 * (dimension block, i, epoch, (tag << 24) | instance).  Nothing of size N
 * is ever stored: every kernel regenerates the samples it needs.
 *   law GAUSS        zhat ~ N(0, I), s = 1             (R ~ N(mu, Sigma), Sec. 3.1)
 *   law LOGN_STD     zhat = standardised lognormal(sigma=1) innovations, s = 1
 *                    (mean mu, covariance Sigma, heavy right tail)
 *   law STUDENT_T    zhat ~ N(0, I), s = sqrt(nu / chi2_nu)  (multivariate t)
 *   law MIX          i < N/2 GAUSS, i >= N/2 LOGN_STD
 * Precision FP64 draws FP64 normals; every other precision draws FP32
 * normals.  Both are bit-exact with the project's CPU oracle.
 *
 * Conventions.
 *   - Array arguments are caller-owned DEVICE memory unless stated.  Dense
 *     matrices are row-major.  The library allocates only inside saa_ctx.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  The returned status covers argument validation and
 *     launch; device-side flags (bounds, timeouts) surface at the next call on
 *     the same context or at saa_ctx_sync().
 *   - Calls on one context must not run concurrently from several host
 *     threads.  Results are deterministic: the same inputs and device give
 *     bitwise-identical outputs.
 *   - The workspace `ws` (device memory, 256-byte aligned, at least
 *     saa_workspace_size() bytes) is scratch owned by the caller; it may be
 *     reused after the call's work on `stream` has completed.
 *   - On error the call returns a non-zero saa_status and saa_last_error()
 *     gives a thread-local message.
 */
#ifndef SAA_H
#define SAA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SAA_OK = 0,
    SAA_EINVAL = 1,       /* invalid argument (message in saa_last_error) */
    SAA_ENOMEM = 2,       /* workspace too small or host allocation failed */
    SAA_ECUDA = 3,        /* CUDA runtime error */
    SAA_ETIMEOUT = 4,     /* a bounded device wait gave up */
    SAA_EDEVICE = 5,      /* a device-side check flagged an error */
    SAA_EUNSUPPORTED = 6  /* size or precision outside what the library supports */
} saa_status;

typedef enum {
    SAA_LAW_GAUSS = 0,
    SAA_LAW_LOGN_STD = 1,
    SAA_LAW_STUDENT_T = 2,
    SAA_LAW_MIX = 3
} saa_law;

typedef enum {
    SAA_FP64 = 0,   /* FP64 normals, FP64 contraction (DFMA): the plain FP64 GPU path */
    SAA_FP32 = 1,   /* FP32 normals, FP32 contraction (FFMA), FP64 cross-block reduction */
    SAA_BF16X3 = 2, /* FP32 normals, BF16 hi/lo split contraction on tcgen05 tensor cores
                       (hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM), FP64 reduction;
                       relative error of the estimates within 5e-5 */
    SAA_FP8X = 3,   /* streamed mode only (saa_eval_samples): E4M3 contraction, samples split
                       hi + lo, decisions in three terms, four products (A1 B1 + A1 B2 +
                       A2 B1 + A1 B3) on kind::f8f6f4, power-of-two column and decision
                       scales, FP32 accumulation in TMEM; centred and scaled samples
                       required.  The sample-side rounding (2^-8 per element) averages over
                       the scenarios: relative error of the estimates within 1e-4 from
                       N of a few thousand; every other entry point returns
                       SAA_EUNSUPPORTED for it */
    SAA_F16X3 = 4   /* as SAA_BF16X3 with FP16 hi/lo operands and a power-of-two scale per
                       decision: relative error of the estimates within 1e-6 */
} saa_prec;

typedef struct saa_ctx saa_ctx;

/* One SAA problem (Sec. 3.1).  A host struct holding device pointers. */
typedef struct {
    int32_t d;          /* dimension of w and R (number of assets), 1 <= d */
    int32_t law;        /* saa_law */
    int64_t N;          /* number of samples per resample, 2 <= N < 2^32 */
    int32_t nu;         /* degrees of freedom of the t law: even, >= 2 (else ignored) */
    int32_t reserved;   /* must be 0 */
    double lambda;      /* variance weight; 0.5 gives Eq. 3 */
    uint64_t seed;      /* Philox key */
    uint32_t instance;  /* stream id, low 24 bits used (counter word 3) */
    uint32_t epoch;     /* resample index (counter word 2) */
    const double* mu;   /* device [d]: mean of R */
    const double* chol; /* device [d*d] row-major lower-triangular C, C C' = Sigma;
                           entries above the diagonal are ignored.  A diagonal
                           entry that is not positive and finite is flagged on
                           the device (SAA_EDEVICE at the next saa_ctx_sync).
                           NULL selects the diagonal form below. */
    const double* sd;   /* device [d] or NULL: with chol NULL, Sigma = diag(sd^2)
                           (C = diag(sd)), the independent assets of Sec. 4.1.
                           This form has no dimension limit (Sec. 4.1 runs up
                           to 10^5 assets): saa_eval, saa_grad and saa_solve
                           take it at SAA_FP32 with K <= 4; the other entry
                           points need chol.  A spread that is not positive
                           and finite is flagged like a bad chol diagonal. */
} saa_problem;

/* Context: device properties, tuned launch shapes, a device error word and
 * cached CUDA graphs.  `device` is a CUDA ordinal; the call makes it current. */
saa_status saa_ctx_create(saa_ctx** out, int device);
void saa_ctx_destroy(saa_ctx* ctx);

/* Waits for `stream`, then reads and clears the device error word:
 * SAA_OK, SAA_EDEVICE or SAA_ETIMEOUT. */
saa_status saa_ctx_sync(saa_ctx* ctx, void* stream);

/* Workspace bytes needed by saa_eval (want_grad = 0), saa_grad (1) or
 * saa_solve (2) for this problem, K decisions and precision; 0 if the
 * arguments are invalid. */
size_t saa_workspace_size(const saa_ctx* ctx, const saa_problem* prob, int32_t K, saa_prec prec, int want_grad);

/* Eq. 4 for K decisions at once.
 *   X     device [K*d]: row k is the decision w_k (need not lie in W)
 *   f     device [K]: f_hat(w_k)
 *   pbar  device [K] or NULL: w_k'R_bar (Eq. 5)
 *   var   device [K] or NULL: (1/(N-1)) sum_i (w_k'(R_i - R_bar))^2
 * At SAA_F16X3 / SAA_BF16X3 a K larger than one tensor-core launch takes
 * (256 up to d = 128, 128 up to d = 256, 64 above it and for gradients)
 * runs as consecutive chunks of that size in the same workspace (which
 * saa_workspace_size sizes for one chunk); every chunk draws the same
 * scenarios, so the time grows with the number of chunks, and a decision's
 * result does not depend on the other decisions up to FP32 summation order.
 * Errors: SAA_EINVAL for d < 1, N < 2, N >= 2^32, K outside [1, 65535], a bad law/nu, NULL
 * required pointers; SAA_ENOMEM if ws_bytes is too small; SAA_EUNSUPPORTED
 * for d beyond the precision's limit (saa_max_dim). */
saa_status saa_eval(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X, saa_prec prec,
                    double* f, double* pbar, double* var, void* ws, size_t ws_bytes, void* stream);

/* saa_eval for a caller whose data live in HOST memory (the end-to-end
 * call of a program that keeps mu, C and the decisions on the host).
 *   prob->mu, prob->chol (or prob->sd), X   HOST arrays, laid out as for
 *                                          saa_eval
 *   f, pbar, var                           HOST [K] (pbar, var optional)
 *   ws   DEVICE scratch of saa_eval_host_workspace_size() bytes, 256-byte
 *        aligned: saa_eval's workspace followed by room for the copies
 * The call copies the inputs into `ws` on `stream`, runs saa_eval there,
 * copies the outputs back, then waits for `stream` and reads the device
 * error word as saa_ctx_sync does: when it returns, the outputs are on the
 * host and device-side flags (SAA_EDEVICE, SAA_ETIMEOUT) are reported.
 * Page-locked host arrays (cudaHostAlloc) are copied by DMA directly;
 * pageable ones go through the driver's staging.  Errors as saa_eval; the
 * size query returns 0 for invalid arguments. */
size_t saa_eval_host_workspace_size(const saa_ctx* ctx, const saa_problem* prob, int32_t K, saa_prec prec);
saa_status saa_eval_host(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X, saa_prec prec,
                         double* f, double* pbar, double* var, void* ws, size_t ws_bytes, void* stream);

/* Eq. 4 and its gradient in w (the paper uses it in Algorithm 1 without
 * writing it out; differentiating Eq. 4 gives
 *   grad f_hat(w) = lambda (2/(N-1)) sum_i (R_i - R_bar)(R_i - R_bar)'w - R_bar).
 *   f     device [K] or NULL
 *   grad  device [K*d]: row k is grad f_hat(w_k)
 * K beyond 64 runs in chunks at the tensor-core precisions, as saa_eval.
 * Errors as saa_eval. */
saa_status saa_grad(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X, saa_prec prec,
                    double* f, double* grad, void* ws, size_t ws_bytes, void* stream);

/* Algorithm 1 (Frank-Wolfe for mean-variance optimisation) from global
 * iteration t0 for T iterations.  Iteration t uses the samples of resample
 * index prob->epoch + t / M (a fresh draw every M iterations), evaluates
 * g = grad f_hat(w_t), takes the LMO vertex s_t over W (e_j for the first
 * j minimising g_j if g_j < 0, else 0), gamma_t = 2/(t+2) and
 * w_{t+1} = w_t + gamma_t (s_t - w_t).  Resuming with (t0, w_t0) continues
 * a run bit for bit.
 *   w0        device [d], in W
 *   w_out     device [d]: w_{t0+T}
 *   f_trace   device [T] or NULL: f_hat(w_t) on iteration t's samples
 *   gap_trace device [T] or NULL: Frank-Wolfe gap g'(w_t - s_t) >= 0
 * The T iterations run as replays of one captured CUDA graph. */
saa_status saa_solve(saa_ctx* ctx, const saa_problem* prob, const double* w0, int32_t T, int32_t M, int64_t t0,
                     saa_prec prec, double* w_out, double* f_trace, double* gap_trace, void* ws, size_t ws_bytes,
                     void* stream);

/* Algorithm 1 with a sample size per epoch (the resampling step allows the
 * sample size N_k to depend on the epoch k).  Epoch k0 + k, for k = 0 ..
 * n_epochs-1, draws N_sched[k] samples of resample index prob->epoch + k0 + k
 * and runs M iterations at the global iteration t = (k0 + k) M + m, so
 * gamma_t = 2/(t+2) and the resampling follow the global count; prob->N is
 * ignored.  Each run of epochs with equal N_k is one captured graph
 * replayed over those epochs.  Resuming with (k0, w) continues a run bit
 * for bit; a constant schedule gives saa_solve's iterates.
 *   N_sched    HOST [n_epochs]: 2 <= N_k < 2^32
 *   w0, w_out  device [d] (w0 in W)
 *   f_trace, gap_trace  device [n_epochs*M] or NULL, as saa_solve's
 *   ws         device scratch of saa_solve_adaptive_workspace_size() bytes
 *              (the largest epoch's saa_solve workspace), 256-byte aligned
 * Errors as saa_solve; the workspace query returns 0 for invalid arguments. */
size_t saa_solve_adaptive_workspace_size(const saa_ctx* ctx, const saa_problem* prob, const int64_t* N_sched,
                                         int32_t n_epochs, saa_prec prec);
saa_status saa_solve_adaptive(saa_ctx* ctx, const saa_problem* prob, const double* w0, const int64_t* N_sched,
                              int32_t n_epochs, int32_t M, int32_t k0, saa_prec prec, double* w_out,
                              double* f_trace, double* gap_trace, void* ws, size_t ws_bytes, void* stream);

/* A ragged batch of B independent problems (Eq. 4 for each), in one
 * persistent launch: problem b has its own d, N, law, stream, K[b]
 * decisions X[b] and outputs f[b] (pbar[b], var[b] optional; pass NULL for
 * the whole array or per entry).  SAA_FP32 or SAA_FP64, d <= 1024.
 *   probs, K, X, f, pbar, var   HOST arrays of length B; X[b], f[b], ...
 *                               are device pointers
 * Each problem's scenarios are cut into chunks that a persistent grid takes
 * from a queue; every chunk has its own partial slot, merged per problem in
 * chunk order, so results are deterministic for a given tile shape.  On the
 * first call for a batch shape the context's autotuner (on by default, see
 * saa_ctx_set_autotune) times the candidate tile shapes on the batch itself
 * and caches the fastest for the process; that first call must not be
 * inside a stream capture (it synchronises).  The descriptor tables go
 * through a pinned staging buffer owned by the context. */
size_t saa_workspace_size_batched(const saa_ctx* ctx, int32_t B, const saa_problem* probs, const int32_t* K,
                                  saa_prec prec);
saa_status saa_eval_batched(saa_ctx* ctx, int32_t B, const saa_problem* probs, const int32_t* K,
                            const double* const* X, saa_prec prec, double* const* f, double* const* pbar,
                            double* const* var, void* ws, size_t ws_bytes, void* stream);
saa_status saa_ctx_set_autotune(saa_ctx* ctx, int enable);

/* Sample store of the diagonal-covariance gradient (saa_problem.chol NULL):
 * when its FP32 samples, N * round_up(d, 4) * 4 bytes, take at most
 * max_bytes, the forward pass writes them to the workspace and the adjoint
 * pass reads them back instead of drawing them again (the results are
 * bitwise the same either way).  The default is 2^35 bytes (32 GiB), which
 * holds Sec. 4.1's 10^5 assets at N = 2^16; 0 always draws twice.  The
 * workspace size follows the setting, so query it after changing it. */
saa_status saa_ctx_set_sample_store(saa_ctx* ctx, size_t max_bytes);

/* A ragged batch planned once and replayed as a CUDA graph.  Same problems,
 * decisions and value outputs as saa_eval_batched; with `grad` non-NULL
 * (host [B] array of device [K_b*d_b] outputs) it also writes each problem's
 * gradient of Eq. 4 in w, as saa_grad does.  SAA_FP32 or SAA_FP64.
 *   saa_batch_workspace_size  bytes of `ws` (0 for invalid arguments)
 *   saa_batch_create  validates, picks the tile shape (the context's
 *       autotuner, on the first batch of this shape), uploads the
 *       descriptor tables into `ws`, waits for `stream`, and captures the
 *       launch sequence (prologue, persistent main kernel, finalize, and the
 *       gradient kernels) into a CUDA graph.  X, outputs and ws are bound
 *       by address: later launches read the current contents of X, mu and
 *       chol and overwrite the outputs.  ws must outlive the batch.
 *   saa_batch_launch  replays the graph on `stream` (asynchronous).
 *   saa_batch_destroy  waits for the device and frees the graph.
 * Per-problem limits as saa_eval_batched.  Results are deterministic. */
typedef struct saa_batch saa_batch;
size_t saa_batch_workspace_size(const saa_ctx* ctx, int32_t B, const saa_problem* probs, const int32_t* K,
                                saa_prec prec, int want_grad);
saa_status saa_batch_create(saa_ctx* ctx, int32_t B, const saa_problem* probs, const int32_t* K,
                            const double* const* X, saa_prec prec, double* const* f, double* const* pbar,
                            double* const* var, double* const* grad, void* ws, size_t ws_bytes, void* stream,
                            saa_batch** out);
saa_status saa_batch_launch(saa_batch* batch, void* stream);
void saa_batch_destroy(saa_batch* batch);

/* Scenario-range partial sums: the sums over i in Eq. 4 and Eq. 5
 * (Sec. 3.1) split by scenario, so that one problem's N samples can be
 * shared across devices or calls.  Ranges that cover [0, N) without overlap
 * add up, element by element, to the whole sample's sums, from which
 * saa_finalize_partials gives what saa_eval / saa_grad give (up to the
 * rounding of a different summation order).  With D_i = R_i - mu (the
 * samples centred at the law's mean) and p_ik = w_k'D_i:
 *   part  device [2K + d + (want_grad ? K*d : 0)] FP64, written in order
 *         P1 [K]    sum_i p_ik
 *         P2 [K]    sum_i p_ik^2
 *         P3 [d]    sum_i D_i
 *         P4 [K*d]  sum_i D_i p_ik (row k), with want_grad
 * over i = i0 .. i0+n-1 of resample index prob->epoch (prob->N is the whole
 * sample's size: the mixed law's split at N/2 does not move).  prec as
 * saa_eval / saa_grad (F16X3 / BF16X3 gradients need d <= 1024, K <= 64);
 * chol must be given (the diagonal form returns SAA_EUNSUPPORTED).
 *   ws   device scratch of saa_partials_workspace_size() bytes (0 for
 *        invalid arguments), 256-byte aligned
 * Errors as saa_eval, and SAA_EINVAL for a range outside [0, N).
 * Deterministic for a given range, device and precision. */
size_t saa_partials_workspace_size(const saa_ctx* ctx, const saa_problem* prob, int64_t n, int32_t K, saa_prec prec,
                                   int want_grad);
saa_status saa_partials(saa_ctx* ctx, const saa_problem* prob, int64_t i0, int64_t n, int32_t K, const double* X,
                        saa_prec prec, int want_grad, double* part, void* ws, size_t ws_bytes, void* stream);

/* Totals of R partial vectors of length len (device [R*len], row r = the
 * partials of one range; total device [len]): element e is the
 * Neumaier-compensated sum over r = 0 .. R-1 in that order, so the totals
 * are the same bit for bit whichever device or collective produced the
 * rows.  The merge step when the ranges' partials have been gathered. */
saa_status saa_partials_merge(saa_ctx* ctx, int32_t R, int64_t len, const double* parts, double* total,
                              void* stream);

/* Eq. 4, Eq. 5 and the gradient of Eq. 4 from the totals of saa_partials
 * over the whole sample (FP64, no workspace):
 *   pbar_k = w_k'mu + P1_k/N,  V_k = (P2_k - P1_k^2/N) / (N-1),
 *   f_k = lambda V_k - pbar_k,
 *   grad_k = lambda (2/(N-1)) (P4_k - P1_k P3/N) - (mu + P3/N)
 * (R_bar = mu + P3/N, and sum_i (R_i - R_bar)(R_i - R_bar)'w_k =
 * P4_k - P3 P1_k/N).  X device [K*d]; part device, laid out as above (P4
 * needed only for grad); f, pbar, var device [K], grad device [K*d], each
 * optional (at least one).  prob->chol is not read. */
saa_status saa_finalize_partials(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X,
                                 const double* part, double* f, double* pbar, double* var, double* grad,
                                 void* stream);

/* The scenario generator on its own (debugging, streamed mode, parity):
 * scenarios i0 .. i0+n-1 of resample index prob->epoch.
 *   prec     SAA_FP64 (double outputs) or SAA_FP32 (float outputs)
 *   z_out    device [n*d]: innovations zhat_i after the law transform
 *   s_out    device [n] or NULL: scales s_i
 *   xi_out   device [n*d] or NULL: samples R_i = mu + s_i C zhat_i at the
 *            same precision, xi_ij = fma(s_i, acc_j, mu_j) with acc_j the fma
 *            chain over l = 0..j of C_jl zhat_il (C, mu rounded first). */
saa_status saa_generate(saa_ctx* ctx, const saa_problem* prob, int64_t i0, int64_t n, saa_prec prec, void* z_out,
                        void* s_out, void* xi_out, void* stream);

/* Streamed mode: Eq. 4 / Eq. 5 on samples held in device memory instead of
 * regenerated (the sample set {R_i} of Sec. 3.1 materialised, e.g. by
 * saa_generate's xi_out or supplied by the caller), for d <= 256 and
 * K <= 256 on the tensor cores, the sample tiles brought in by TMA.
 *   R        device [N*d] FP32, row-major (scenario i = row i); 16-byte
 *            aligned, d a multiple of 4 (rows of 16-byte multiples)
 *   center   device [d] FP64 or NULL (0): subtracted from every row before
 *            the split-precision contraction, in FP32; p_ik = c'x_k +
 *            (R_i - c)'x_k with c = center rounded to FP32, so the result
 *            does not depend on it beyond rounding; pass the samples' mean
 *            (or mu): without it the FP32 accumulation error of the
 *            contraction, relative to |R_i'x_k|, reaches V multiplied by
 *            (pbar^2 + V) / V
 *   sigma    device [d] FP64 or NULL (1): per-column spreads; column j is
 *            multiplied by 2^-a_j and x_kj by 2^a_j, 2^(a_j-1) < sigma_j <=
 *            2^a_j (exact), so the split products stay in range.  At
 *            SAA_F16X3 every |R_ij - c_j| 2^-a_j must be below 2^15, at
 *            SAA_FP8X at most 448 (E4M3's largest finite value); violations
 *            and sigma_j outside [2^-100, 2^100] or not finite are reported
 *            by the next saa_ctx_sync as SAA_EDEVICE
 *   X        device [K*d] FP64 decisions w_k (the scenario vector already
 *            holds the returns: no mu or C is applied)
 *   lambda   risk weight of Eq. 2
 *   prec     SAA_F16X3, SAA_BF16X3 (operand type of the hi/lo products) or
 *            SAA_FP8X (E4M3 products; center and sigma must then both be
 *            given, else SAA_EINVAL)
 *   f, pbar, var  device [K] FP64, each optional: lambda V - pbar, the
 *            sample mean of R_i'x_k, and its unbiased sample variance
 *   ws       device scratch of saa_eval_samples_workspace_size() bytes,
 *            256-byte aligned
 * 2 <= N < 2^31.  The workspace query returns 0 for invalid or unsupported
 * arguments; the call returns SAA_EINVAL / SAA_EUNSUPPORTED for them.
 * Deterministic for a given device and N. */
size_t saa_eval_samples_workspace_size(const saa_ctx* ctx, int64_t N, int32_t d, int32_t K, saa_prec prec);
saa_status saa_eval_samples(saa_ctx* ctx, int64_t N, int32_t d, const float* R, const double* center,
                            const double* sigma, int32_t K, const double* X, double lambda, saa_prec prec,
                            double* f, double* pbar, double* var, void* ws, size_t ws_bytes, void* stream);

/* The binary-classification task of Sec. 3.3 (logistic model):
 *   t = x_i'omega_k, c = 1 / (1 + e^-t)
 *   F_k    = -(1/b) sum_S [ z log c + (1 - z) log(1 - c) ]
 *   grad_k = (1/b) sum_S (c - z) x_i            (the mini-batch gradient)
 *   hvp_k  = (1/b) sum_S c (1 - c) (x_i'v_k) x_i (sub-sampled Hessian times v_k)
 * over a sample S of a binary data set, for K parameter vectors at once.
 *
 * Data layout: row i of X holds saa_logistic_pitch(n) 32-bit words; feature
 * j of point i is bit j % 32 of word j / 32 (bits past n are 0); z [N]
 * holds the labels (0 or 1).
 *
 * saa_logistic_generate writes rows i0 .. i0+rows-1 of the synthetic data
 * set of Sec. 4.1's setup (X starts at row i0; z optional): feature j =
 * 128 b + 32 q + t of point i is bit t of word q of Philox4x32-10(counter
 * (b, i, 0, (4 << 24) | instance), key seed), and the label is [2 x_i'w* >
 * 1'w*] (integer arithmetic) flipped when word 0 of Philox(counter (0, i,
 * 0, (5 << 24) | instance)) is below `flip` (429496730 for the paper's 10 %
 * label noise).  X must be 16-byte aligned.
 *
 * saa_logistic_eval: idx device [b] int64 row indices of S (repeats
 * allowed), or NULL for every row (b = N); W device [K*n] FP64; V device
 * [K*n] FP64 (needed for hvp); F [K], grad [K*n], hvp [K*n] device FP64,
 * each optional.  Scratch: saa_logistic_workspace_size(n, b, K, has_v)
 * bytes, 256-byte aligned (has_v = V and hvp both given).  EUNSUPPORTED for
 * n > 43648.  Deterministic for a given device. */
typedef struct {
    int32_t n;            /* features */
    int32_t reserved;     /* must be 0 */
    int64_t N;            /* data points, 1 <= N < 2^32 */
    uint64_t seed;        /* Philox key */
    uint32_t instance;    /* low 24 bits used (counter word 3) */
    uint32_t flip;        /* label-noise threshold on a 32-bit word */
    const int32_t* wstar; /* device [n]: integer weights of the labelling rule */
} saa_logistic;
int32_t saa_logistic_pitch(int32_t n);
saa_status saa_logistic_generate(saa_ctx* ctx, const saa_logistic* prob, int64_t i0, int64_t rows, uint32_t* X,
                                 uint8_t* z, void* stream);
size_t saa_logistic_workspace_size(const saa_ctx* ctx, int32_t n, int64_t b, int32_t K, int has_v);
saa_status saa_logistic_eval(saa_ctx* ctx, int32_t n, int64_t N, const uint32_t* X, const uint8_t* z,
                             const int64_t* idx, int64_t b, int32_t K, const double* W, const double* V, double* F,
                             double* grad, double* hvp, void* ws, size_t ws_bytes, void* stream);

/* Moments of the generator: per-dimension sums of the innovations zhat_ij
 * (after the law transform, before the t law's scale s_i) and of their
 * squares over scenarios i0 .. i0+n-1 of resample index prob->epoch, drawn
 * by the estimator kernels' own in-kernel generator (the samples of
 * Sec. 3.1).  The standardised laws give mean 0 and variance 1 per
 * coordinate, so this checks the law on the device at any scale; it is also
 * the generator-only kernel that the roofline's per-normal figure is
 * measured on.
 *   prec     SAA_FP32 or SAA_FP64 (which generator mode draws)
 *   sum      device [d] FP64: sum_i zhat_ij
 *   sumsq    device [d] FP64 or NULL: sum_i zhat_ij^2
 *   ws       device scratch of saa_generate_moments_workspace_size() bytes,
 *            8-byte aligned
 * 1 <= d <= 2048, 1 <= n, i0 + n <= N.  Deterministic for a given device.
 * The workspace-size query returns 0 for invalid arguments. */
size_t saa_generate_moments_workspace_size(const saa_ctx* ctx, const saa_problem* prob, int64_t i0, int64_t n,
                                           saa_prec prec);
saa_status saa_generate_moments(saa_ctx* ctx, const saa_problem* prob, int64_t i0, int64_t n, saa_prec prec,
                                double* sum, double* sumsq, void* ws, size_t ws_bytes, void* stream);

/* Covariance-first form (Sec. 3.1: the sample mean and covariance formed
 * once per resample), for d <= 1024 on the tensor cores.  With the whitened
 * samples a_i = s_i zhat_i of resample prob->epoch:
 *   saa_moments       M = sum_i a_i a_i' (device [d*d] FP64, row-major) and
 *                     mt = sum_i a_i (device [d] FP64); prec SAA_F16X3 or
 *                     SAA_BF16X3 (the hi/lo operand type of A'A).  Scratch:
 *                     saa_moments_workspace_size() bytes, 256-byte aligned.
 *   saa_eval_moments  for K decisions X [K*d]: y_k = C'w_k, S1 = mt'y_k,
 *                     S2 = y_k'M y_k, and f, pbar, var (each optional) as
 *                     saa_eval computes them, plus grad [K*d] (optional) =
 *                     C[lambda 2/(N-1) (M y_k - S1 m) - m] - mu, m = mt/N,
 *                     all in FP64.  Scratch: saa_eval_moments_workspace_size().
 * The moments' work does not depend on K: evaluating many decisions, or
 * many iterations of Algorithm 1 on one resample, costs K d^2 FP64
 * multiply-adds each after one saa_moments.  Above d = 128, M is formed in
 * 128 x 128 blocks, each block's CTAs drawing the two dimension slices it
 * needs (every normal drawn up to ceil(d/128) times at d = 1024); SAA_EINVAL
 * for d > 1024. */
size_t saa_moments_workspace_size(const saa_ctx* ctx, const saa_problem* prob, saa_prec prec);
saa_status saa_moments(saa_ctx* ctx, const saa_problem* prob, saa_prec prec, double* M, double* mt, void* ws,
                       size_t ws_bytes, void* stream);
size_t saa_eval_moments_workspace_size(const saa_problem* prob, int32_t K);
saa_status saa_eval_moments(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X, const double* M,
                            const double* mt, double* f, double* pbar, double* var, double* grad, void* ws,
                            size_t ws_bytes, void* stream);

/* The newsvendor's Monte Carlo gradient (Sec. 3.2, the approximated
 * gradient), for n products with normal demands:
 *   grad_kj = (k_j - v_j) + (h_j + v_j) * (count_kj / S),
 *   count_kj = #{s < S : z_js <= tau_kj},  tau_kj = RN_f32((x_kj - mu_j) / sigma_j)
 * (subtraction and division in FP64), z_js the generator's FP32 normals on
 * counter (s / 4, j, epoch, (3 << 24) | instance), element s mod 4 -- the
 * comparison d_js = mu_j + sigma_j z_js <= x_kj taken on the standardised
 * demand in one fixed precision, so the counts are exact integers.
 *   X     device [K*n] FP64, K decision vectors (1 <= K <= 8), row-major
 *   grad  device [K*n] FP64 output
 *   ws    device scratch of saa_newsvendor_workspace_size() bytes (the
 *         counts, uint32 [K][n]), 4-byte aligned
 * Deterministic.  A sigma_j that is not positive is flagged on the device
 * (SAA_EDEVICE at the next saa_ctx_sync). */
typedef struct {
    int64_t n;            /* products, 1 <= n < 2^32 */
    int64_t S;            /* demand samples per product, 1 <= S < 2^30 */
    uint64_t seed;        /* Philox key */
    uint32_t instance;    /* stream id (counter word 3, low 24 bits) */
    uint32_t epoch;       /* resample index (counter word 2) */
    const double* mu;     /* device [n] demand means */
    const double* sigma;  /* device [n] demand standard deviations, > 0 */
    const double* k;      /* device [n] unit ordering costs */
    const double* h;      /* device [n] unit holding costs */
    const double* v;      /* device [n] unit shortage costs */
} saa_newsvendor;
size_t saa_newsvendor_workspace_size(const saa_newsvendor* prob, int32_t K);
saa_status saa_newsvendor_grad(saa_ctx* ctx, const saa_newsvendor* prob, int32_t K, const double* X, double* grad,
                               void* ws, size_t ws_bytes, void* stream);

/* Lower Cholesky factor C of Sigma (C C' = Sigma), the map from standard
 * normals to the samples of the normal law of Sec. 3.1 (R = mu + C z): the
 * `chol` input of saa_problem.  FP64, blocked right-looking factorization
 * with a fixed summation order (deterministic), on `stream`.
 *   d       1 <= d <= 46340
 *   Sigma   device [d*d] row-major symmetric positive definite; only the
 *           lower triangle (j <= i) is read
 *   chol    device [d*d] row-major: receives C, zeros above the diagonal.
 *           May equal Sigma (in place); must not partially overlap it.
 * Returns SAA_EINVAL for bad arguments, SAA_ECUDA on a launch failure.  A
 * pivot that is not positive (Sigma not positive definite, NaN) is found on
 * the device: the next saa_ctx_sync reports SAA_EDEVICE and `chol` is
 * undefined. */
saa_status saa_cholesky(saa_ctx* ctx, int32_t d, const double* Sigma, double* chol, void* stream);

/* saa_eval without a context or a workspace, for callers that cannot
 * allocate device memory: a real-time loop that cannot afford cudaMalloc's
 * implicit device synchronisation, a plug-in inside a host framework that
 * owns all device memory through its own allocator, or code held to a
 * device-memory budget by another component.  The paper has no
 * counterpart: this is a deployment convenience, not part of the method.
 *
 * Same arguments and results as saa_eval, on the CURRENT device, for
 * SAA_FP32 and SAA_FP64 with a dense chol; the diagonal form (chol NULL)
 * returns SAA_EUNSUPPORTED.  Scratch comes from one array of
 * SAA_STATIC_SCRATCH_BYTES in device memory defined by the library, which
 * every GPU that loads libsaa holds until the process exits; problems whose
 * scratch would not fit (large K times d, or very many CTAs) return
 * SAA_ENOMEM with the needed size in saa_last_error().  The call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).  Its
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the process, so do not use this
 * entry point across a cudaDeviceReset.  A diagonal entry of chol that is not positive and
 * finite cannot be reported through a context here: the call writes NaN to
 * f (and to pbar, var when given) instead.  All calls share the array:
 * calls whose GPU work overlaps (other streams, other host threads) race on
 * it.  The call clears the part that must start at zero (its error word);
 * every other value is written before it is read. */
#define SAA_STATIC_SCRATCH_BYTES (16u << 20)
saa_status saa_eval_static(const saa_problem* prob, int32_t K, const double* X, saa_prec prec, double* f,
                           double* pbar, double* var, void* stream);

/* Failure-path self-test: launches one warp that waits, with the same
 * bounded mbarrier wait the tensor-core kernel uses and a budget of
 * `budget_us` microseconds (1 .. 100000), on a barrier that nothing
 * completes.  The wait gives up, sets the timeout bit of the context's
 * error word and returns: the next saa_ctx_sync reports SAA_ETIMEOUT and
 * clears it, and the context stays usable.  No fault, trap or hang. */
saa_status saa_selftest_timeout(saa_ctx* ctx, uint32_t budget_us, void* stream);

/* Index-checked build.  Compiled with SAA_BOUNDS_CHECK defined (the package
 * builds it as libsaa_bounds.so), the tensor-core value, gradient and
 * streamed kernels check the indices of their partial-sum writes against
 * the workspace regions the host carved, and of their shared-memory stage
 * stores against the stage; an index at or past its bound raises the bounds
 * bit of the context's error word (the next saa_ctx_sync returns
 * SAA_EDEVICE) and the access is skipped, instead of faulting.  The results
 * of every call are otherwise the same, bit for bit, as the normal build's.
 * saa_bounds_check_enabled returns 1 in that build, 0 in the normal one.
 * saa_selftest_bounds launches one warp that stores, through the same
 * check, past the declared capacity of a device array twice that size (so
 * no build writes outside it): the checked build flags every store and
 * skips it, and the next saa_ctx_sync returns SAA_EDEVICE; the normal build
 * returns SAA_EUNSUPPORTED without launching.  Not in the paper: a tool for
 * this library's own checking. */
int32_t saa_bounds_check_enabled(void);
saa_status saa_selftest_bounds(saa_ctx* ctx, void* stream);

/* Arithmetic self-test of the FP32 generator: for every one of its 2^23
 * uniforms u = (2k + 1) 2^-24 it compares the LOG's quotient (m - 1)/(m + 1)
 * and the Box-Muller root sqrt(-2 LOG(u)), which the generator forms by
 * Markstein's correction of the hardware approximations, with the IEEE
 * round-to-nearest division and square root.  mismatches: device [2]
 * (quotient, root), zeroed and then filled asynchronously on `stream`; both
 * are 0 when the generator's results are the IEEE ones bit for bit. */
saa_status saa_selftest_arith(saa_ctx* ctx, unsigned long long* mismatches, void* stream);

/* Kernel timing (tracing).  While enabled, every saa_eval / saa_grad call
 * records a CUDA event pair on its stream around its main sample kernel (the
 * generation + contraction + epilogue kernel) and counts the kernels it
 * launches.  saa_profile_read waits for the recorded events, returns the
 * summed main-kernel time in milliseconds, the number of main-kernel
 * launches timed and the total kernels launched since the last read, then
 * resets the counters.  Not recorded inside saa_solve's captured graph. */
saa_status saa_profile_enable(saa_ctx* ctx, int enable);
saa_status saa_profile_read(saa_ctx* ctx, double* main_ms, int64_t* main_launches, int64_t* kernels_launched);

/* Launch shape that saa_eval (want_grad = 0) or saa_grad (1) would use for
 * this problem: CTAs of the main kernel (grid), CTAs per thread-block
 * cluster (1 unless the path splits the dimensions across a cluster) and
 * scenario tiles.  Any output may be NULL.  For tracing and tuning. */
saa_status saa_plan_info(const saa_ctx* ctx, const saa_problem* prob, int32_t K, saa_prec prec, int want_grad,
                         int32_t* grid, int32_t* cluster, int64_t* tiles);

/* Largest d that `prec` supports.  For SAA_F16X3 and SAA_BF16X3 that is
 * 1024: up to d = 256 one launch takes K <= 256 (k_tc_value, K <= 128 above
 * d = 128), above it K <= 64 (the cluster kernel that splits the dimensions,
 * without its adjoint for values); saa_eval and saa_grad run larger K in
 * chunks of that size, saa_partials does not. */
int32_t saa_max_dim(saa_prec prec);

const char* saa_status_string(saa_status s);
/* Message of the last failed call on this host thread ("" if none). */
const char* saa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SAA_H */
