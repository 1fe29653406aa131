/*
 * tdo.h — C ABI of the GB300 (sm_103a) transformer density-operator library (libtdo.so).
 *
 * The method (arxiv 2502.20723): the density operator of an open spin chain is vectorised as a state
 * in the doubled Hilbert space, |rho>> = sum rho(s, s') |s>|s'> (vectorisation appendix), and its
 * matrix elements are given by a transformer: log rho(s, s') = log(exp z(s,s') + conj exp z(s',s))
 * (Eq. log_sum_exp_conjugate).  The steady state minimises Cost = ||Lhat rho||^2 / ||rho||^2
 * (Eq. lossnetk) where Lhat is the vectorised Lindbladian (Eq. VecLin), estimated by Metropolis
 * sampling of |rho|^2 and the local estimator L_loc, and optimised by stochastic reconfiguration.
 *
 * Conventions for every entry point
 *  - Configurations: a doubled configuration (s, s') is two uint32 words; bit i is site i; bit value 0
 *    is |0> (sigma^z = +1), 1 is |1> (sigma^z = -1); sigma^- = |1><0|.  N <= 32.
 *  - Buffers are owned by the caller.  Every data pointer may be a device pointer or a host pointer
 *    (pageable or pinned); the library detects host memory and stages it through its own device
 *    workspace.  Calls are ordered on the context's stream; a call with a host output (or a host
 *    pointer in any argument) synchronises that stream before returning, a call with only device
 *    pointers is asynchronous.
 *  - log rho values are float pairs (re, im), the imaginary part in (-pi, pi] (principal branch).
 *  - Parameters theta: a flat FP64 vector in this order (rows = input features, row-major):
 *      token embedding E[4][d] (token = 2*bit(first channel) + bit(second channel)), or
 *        conv embedding Wc1[2][2][C1], bc1[C1], Wc2[2][C1][d], bc2[d];
 *      per layer: Wq, Wk, Wv, Wo [d][d] (no bias); if mlp_ratio r > 0: W1[d][r d], b1[r d], W2[r d][d], b2[d];
 *      head Wh[d][2], bh[2].
 *  - Every call returns a tdo_status; tdo_last_error() gives a message.  No exception crosses the ABI.
 *    A context is used by one host thread at a time.
 */
#ifndef TDO_H
#define TDO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdo_ctx tdo_ctx;

typedef enum {
  TDO_OK = 0,
  TDO_EINVAL = -1,        /* bad argument (null pointer, size out of range, inconsistent spec) */
  TDO_ENOMEM = -2,        /* device allocation failed */
  TDO_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed */
  TDO_ENUMERIC = -4,      /* a non-finite value was produced (e.g. rho = 0 exactly, NaN parameters) */
  TDO_ETIMEOUT = -5,      /* a bounded device-side wait gave up */
  TDO_EUNSUPPORTED = -6   /* valid request outside what the kernels implement (e.g. N > 32) */
} tdo_status;

enum { TDO_EMBED_TOKEN = 0, TDO_EMBED_CONV = 1 };
/* Precision of a context: TDO_FP32 = FP32 CUDA-core path; TDO_BF16 and TDO_FP16 = tensor-core path
 * (tcgen05 GEMMs with FP32 accumulation) whose GEMM operands are BF16 or FP16 respectively.  TDO_FP8 =
 * the tensor-core path whose evaluations of log rho (tdo_log_rho, tdo_log_rho_ragged, the local
 * estimator's connected rows, tdo_sample and the observables) run on E4M3 operands (kind::f8f6f4, FP32
 * accumulation; one power-of-two scale per weight matrix, one per tile for each activation image, set
 * from the largest magnitude so that scaled values stay below 256); its gradient, log-derivatives and SR
 * step use the FP16 kernels.  E4M3 keeps 4 significant bits: its log rho error is stated beside its
 * throughput, not bounded like the 16-bit paths'. */
enum { TDO_FP32 = 0, TDO_BF16 = 1, TDO_FP16 = 2, TDO_FP8 = 3 };

/* Problem statement: a chain of N spins, a Hamiltonian given as a sum of real multiples of Pauli strings
 * on at most two sites, and single-site jump operators with rates (Eq. Lindblad / Eq. VecLin). */
typedef struct {
  int n_sites;                /* N, 1..32 */
  int n_terms;                /* Hamiltonian terms */
  const int *term_sites;      /* [n_terms][2] site indices; second entry -1 for a single-site term */
  const char *term_paulis;    /* [n_terms][2] in {'I','X','Y','Z'} (second ignored when its site is -1) */
  const double *term_coef;    /* [n_terms] real coefficients */
  int n_jumps;                /* jump operators */
  const int *jump_site;       /* [n_jumps] */
  const double *jump_op;      /* [n_jumps][2][2][2]: L[row][col] as (re, im), basis (|0>, |1>) */
  const double *jump_rate;    /* [n_jumps] gamma_i >= 0 */
} tdo_problem;

/* Transformer hyper-parameters (architecture appendix). */
typedef struct {
  int embed;                  /* TDO_EMBED_TOKEN or TDO_EMBED_CONV */
  int conv_channels;          /* C1 for the conv embedding */
  int d_model;                /* 16, 32 or 64 */
  int n_heads;                /* divides d_model; head dim <= 16 */
  int n_layers;               /* 1..8 */
  int mlp_ratio;              /* 0 (the paper's block: no MLP) or 1..4 */
  int precision;              /* TDO_FP32, TDO_BF16, TDO_FP16 or TDO_FP8 (tensor-core GEMM operand type) */
} tdo_model;

/* Number of real parameters of a model (the length of theta). 0 for an invalid model. */
size_t tdo_model_num_params(const tdo_model *model);

/* Create a context on the current CUDA device: copies the problem and theta (host FP64, n_theta values),
 * builds the Lindbladian connection rules, uploads parameters.  stream: a cudaStream_t (NULL = legacy
 * default stream).  The context owns its device workspace; tdo_destroy frees it. */
tdo_status tdo_create(const tdo_problem *problem, const tdo_model *model, const double *theta,
                      size_t n_theta, void *stream, tdo_ctx **out);
tdo_status tdo_destroy(tdo_ctx *ctx);
size_t tdo_num_params(const tdo_ctx *ctx);
/* Largest number of connected configurations (diagonal included) of any row of Lhat. */
int tdo_max_connections(const tdo_ctx *ctx);

/* Replace / read theta (FP64, n = tdo_num_params values, host or device pointer). */
tdo_status tdo_set_params(tdo_ctx *ctx, const double *theta);
tdo_status tdo_get_params(tdo_ctx *ctx, double *theta);

/* Batched ansatz evaluation (architecture appendix; Eq. log_sum_exp_conjugate):
 * logrho[b] = log rho(sig[b], sigp[b]) as (re, im) floats, b < B.  B may be 0. */
tdo_status tdo_log_rho(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t B, float *logrho);

/* The ansatz over chains of different lengths in one batch (architecture appendix: the token embedding,
 * the attention and the mean pooling take a sequence of any length with the same theta, the
 * translation-invariant form of the appendix's global mean pooling): logrho[b] = log rho(sig[b], sigp[b])
 * for a chain of n_sites[b] sites, 1 <= n_sites[b] <= 32 (TDO_EUNSUPPORTED otherwise; the context's own
 * n_sites plays no part).  The batch is sorted into buckets of equal N on the device; tensor-core contexts
 * then run every bucket's tiles in one persistent launch whose shape (CTAs per SM, bucket order, static
 * or dynamic tile schedule) is chosen by timing four candidates on the first call with a new mix of
 * chain lengths and cached in the context (tdo_ragged_tuning reads it); FP32 contexts launch once per
 * bucket.  Synchronises the stream.  B < 2^32. */
tdo_status tdo_log_rho_ragged(tdo_ctx *ctx, const int32_t *n_sites, const uint32_t *sig, const uint32_t *sigp,
                              size_t B, float *logrho);
/* The launch shape the autotuner kept for a mix of chain lengths (bit N-1 of mix set for each N present):
 * CTAs per SM (1 or 2), descending-N tile order (0/1), dynamic tile schedule (0/1).  TDO_EINVAL if that
 * mix has not been seen. */
tdo_status tdo_ragged_tuning(const tdo_ctx *ctx, uint32_t mix, int *ctas_per_sm, int *descending,
                             int *dynamic_schedule);

/* Vector-Jacobian product of tdo_log_rho: grad[k] += sum_b Re(c_b * d log rho_b / d theta_k) with the
 * complex cotangents c_b = (cot[2b], cot[2b+1]); grad is FP64 [P], accumulated into (not zeroed). */
tdo_status tdo_log_rho_vjp(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t B,
                           const float *cot, double *grad);

/* Log-derivatives O[b][k] = d log rho(sig[b], sigp[b]) / d theta_k as (re, im) floats, layout
 * [B][P][2] (metric-tensor section: the Delta O_i of S). */
tdo_status tdo_jacobian(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t B, float *O);

/* Rows of Lhat (Eq. VecLin with A rho B -> (A (x) B^T)|rho>>): for sample s, count[s] entries
 * conn_sig/conn_sigp/conn_coef [s*M + j], j < count[s], M = tdo_max_connections(); entry 0 is always
 * the diagonal (s itself, coefficient possibly 0); the others have nonzero coefficients, in a fixed
 * order.  coef is (re, im) float. */
tdo_status tdo_connections(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t Ns,
                           int32_t *count, uint32_t *conn_sig, uint32_t *conn_sigp, float *conn_coef);

/* Local estimator L_loc(x) = sum_y Lhat_xy rho(y)/rho(x) (optimisation-procedure section) for Ns
 * samples: lloc [Ns][2] doubles (may be NULL); cost = mean |L_loc|^2 and its standard error
 * (Eq. lossnetk estimated on the samples; either output pointer may be NULL). */
tdo_status tdo_local_estimator(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t Ns,
                               double *lloc, double *cost, double *stderr_);

/* The local estimator above, for callers that must not allocate device memory while they run: a host
 * application whose device memory belongs to another allocator (a framework's caching pool holding the
 * free memory), or a latency-critical loop that cannot afford the device-wide synchronisation that
 * cudaMalloc / cudaFree may imply.  The paper has no counterpart; this is an interface convenience.
 * Same outputs as tdo_local_estimator, but sig, sigp and lloc must be device pointers (lloc 16-byte
 * aligned), and the call
 * allocates nothing: its scratch is one fixed device array (10,813,952 bytes, about 10.8 MB) that every GPU which loads
 * the library holds until the process exits.  Limits: Ns <= 16384 and Ns * tdo_max_connections()
 * <= 262144, else TDO_EINVAL.  The first call on a device looks up the array's device address (once
 * per device, with that device current); make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (other threads or streams) race and must not be
 * made; the array keeps the last call's contents. */
tdo_status tdo_local_estimator_noalloc(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t Ns,
                                       double *lloc, double *cost, double *stderr_);

/* Metropolis-Hastings on |rho|^2 with single-bit proposals (sampling section).  Chains are in/out in
 * sig/sigp [n_chains].  Proposal t of chain c draws Philox4x32-10(key = (seed lo, seed hi),
 * counter = (c, t lo, t hi, 0)) -> (x0, x1, ...): bit k = ((x0 >> 8) * 2N) >> 24 (k < N flips s_k,
 * else s'_{k-N}), u = (x1 >> 8) 2^-24, accept iff u < exp(min(0, 2 Re(log rho' - log rho))).
 * Proposals t = counter .. counter + n_sweeps*2N - 1 (a sweep is 2N proposals).  After each sweep the
 * chain states are stored to samples_sig/samples_sigp [sweep][n_chains] when those are not NULL.
 * accepted (may be NULL) receives the number of accepted moves. */
tdo_status tdo_sample(tdo_ctx *ctx, size_t n_chains, size_t n_sweeps, uint64_t seed, uint64_t counter,
                      uint32_t *sig, uint32_t *sigp, uint32_t *samples_sig, uint32_t *samples_sigp,
                      uint64_t *accepted);

/* Metropolis-Hastings on the diagonal of rho, P(alpha) proportional to |rho(alpha, alpha)| (supplement,
 * "Mixed-State Observables"; the sampler of the local estimator below).  Chains alpha [n_chains] in/out
 * (bit i = site i).  Same random stream as tdo_sample with N choices per draw: proposal t of chain c
 * takes Philox4x32-10(key = (seed lo, seed hi), counter = (c, t lo, t hi, 0)) -> (x0, x1, ...), flips
 * site k = ((x0 >> 8) * N) >> 24 of alpha (in both entries of the pair (alpha, alpha)), u = (x1 >> 8) 2^-24,
 * and accepts iff u < exp(min(0, Re(log rho(alpha', alpha') - log rho(alpha, alpha)))).  A sweep is N
 * proposals: t = counter .. counter + n_sweeps*N - 1.  samples [sweep][n_chains] (may be NULL) get the
 * states after each sweep; accepted (may be NULL) the number of accepted moves. */
tdo_status tdo_sample_diag(tdo_ctx *ctx, size_t n_chains, size_t n_sweeps, uint64_t seed, uint64_t counter,
                           uint32_t *alpha, uint32_t *samples, uint64_t *accepted);

/* Site-averaged magnetisations <sigma^a> = Tr(rho A) / Tr(rho), A = (1/N) sum_i sigma^a_i (supplement,
 * "Mixed-State Observables") from Ns samples alpha of |rho(alpha, alpha)| (tdo_sample_diag):
 * local estimator A~(alpha) = sum_beta rho(alpha, beta) / rho(alpha, alpha) <beta|A|alpha> over beta =
 * alpha and its N single flips (<alpha ^ e_i|sigma^x_i|alpha> = 1, <alpha ^ e_i|sigma^y_i|alpha> =
 * i (1 - 2 alpha_i), <alpha|sigma^z_i|alpha> = 1 - 2 alpha_i; bit 0 = |0>), reweighted by the sign s of
 * rho(alpha, alpha) (the ansatz does not force it positive): <A> = sum s A~ / sum s.
 * mag[3] = (<sigma^x>, <sigma^y>, <sigma^z>) (real parts); sign_mean (may be NULL) = mean of s;
 * local (may be NULL) = [Ns][4] complex doubles (s, A~x, A~y, A~z), each as (re, im).
 * TDO_EINVAL when the signs sum to zero. */
tdo_status tdo_magnetisation(tdo_ctx *ctx, const uint32_t *alpha, size_t Ns, double *mag, double *sign_mean,
                             double *local);

/* Purity Tr(rho^2) / Tr(rho)^2 from Ns samples (sigma, sigma') of |rho|^2 (tdo_sample):
 * Tr(rho)^2 / Tr(rho^2) = E[rho(sigma, sigma) rho(sigma', sigma') / |rho(sigma, sigma')|^2], estimated by
 * the sample mean m; purity = 1 / m, stderr_ (may be NULL) its standard error by the delta method.
 * TDO_EINVAL when m <= 0. */
tdo_status tdo_purity(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t Ns, double *purity,
                      double *stderr_);

/* Cost gradient for real parameters from Ns samples (derivative of Eq. lossnetk):
 * grad_k = 2 Re (1/Ns) sum_x [ conj(L_loc(x)) sum_y Lhat_xy (rho_y/rho_x) O_k(y) - Cost O_k(x) ],
 * grad FP64 [P] (overwritten); cost (may be NULL) = mean |L_loc|^2; O (may be NULL) receives the
 * samples' log-derivatives as in tdo_jacobian. */
tdo_status tdo_grad(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t Ns, double *grad,
                    double *cost, float *O);

/* Stochastic-reconfiguration solve (metric-tensor and regularisation sections):
 * (Re S + diag_shift I) x = rhs with S_ij = <O_i^* O_j> - <O_i^*><O_j> over the Ns rows of O
 * ([Ns][P][2] floats), by Jacobi-preconditioned conjugate gradients in FP64 until
 * ||r|| <= tol ||rhs|| or max_iter iterations.  iters / resid (may be NULL) report the iterations
 * and the final relative residual. */
tdo_status tdo_sr_solve(tdo_ctx *ctx, const float *O, size_t Ns, const double *rhs, double diag_shift,
                        double tol, int max_iter, double *x, int *iters, double *resid);

/* Optimiser applied to the SR direction delta = (Re S + diag_shift I)^-1 grad by tdo_sr_step and tdo_vmc_step
 * (optimisation-procedure section: "Stochastic Gradient Descent or Adam" combined with stochastic
 * reconfiguration as the gradient preconditioner).  TDO_OPT_SGD (default): theta <- theta - lr delta.
 * TDO_OPT_ADAM (Kingma and Ba, Algorithm 1, delta in the role of the gradient): with t the steps taken
 * since this call, m <- beta1 m + (1 - beta1) delta, v <- beta2 v + (1 - beta2) delta^2,
 * theta <- theta - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps); the moments are FP64 [P]
 * in the context.  Every call resets the moments and t (TDO_EINVAL on an unknown kind or beta outside
 * [0, 1), eps <= 0).  The paper uses Adam for its Heisenberg example with no values printed; the
 * usual 0.9, 0.999, 1e-8 are suggested. */
enum { TDO_OPT_SGD = 0, TDO_OPT_ADAM = 1 };
tdo_status tdo_set_optimizer(tdo_ctx *ctx, int kind, double beta1, double beta2, double eps);

/* Stopping rule of the CG solve inside tdo_sr_step: ||r|| <= tol ||rhs|| or max_iter iterations (defaults:
 * tol 1e-5, max_iter 100).  The solve
 * starts from the previous step's solution when there is one (reset by tdo_set_params). */
tdo_status tdo_set_sr_options(tdo_ctx *ctx, double tol, int max_iter);

/* One optimisation-workflow step on a given sample set: cost and gradient, log-derivatives,
 * SR solve with diag_shift, then the optimiser's update with the direction delta (tdo_set_optimizer;
 * default theta <- theta - lr * delta).  cost (may be NULL) gets the cost before the update. */
tdo_status tdo_sr_step(tdo_ctx *ctx, const uint32_t *sig, const uint32_t *sigp, size_t Ns, double lr,
                       double diag_shift, double *cost);

/* Learning-rate and SR-shift schedules (supplement, "Learning Rate Scheduling"): value(step) = v0 for
 * step < i_switch, else v0 (1 + cos(pi (step - i_switch) / i_decay)) / 2 + alpha v0.  Host arithmetic. */
double tdo_schedule_value(long long step, double v0, long long i_switch, long long i_decay, double alpha);

/* The two schedules of one optimisation run.  The paper's values: eta0 0.0061, i_switch 30000,
 * i_decay 40000, alpha 0.001; lambda0 0.004, i_switch_sr 30000, i_decay_sr 40000, alpha_sr 0.01. */
typedef struct {
  double eta0;
  long long i_switch, i_decay;
  double alpha;
  double lambda0;
  long long i_switch_sr, i_decay_sr;
  double alpha_sr;
} tdo_schedule;

/* One step of the optimisation workflow (supplement, optimisation procedure) with the schedules:
 * n_sweeps Metropolis sweeps of the chains (sig, sigp) [n_chains] (tdo_sample with *counter, which
 * advances by n_sweeps * 2N), then tdo_sr_step on the chain states with lr = eta(step) and diag_shift =
 * lambda(step) of sched (NULL: the paper's values).  cost (may be NULL) as in tdo_sr_step. */
tdo_status tdo_vmc_step(tdo_ctx *ctx, uint32_t *sig, uint32_t *sigp, size_t n_chains, size_t n_sweeps,
                        uint64_t seed, uint64_t *counter, long long step, const tdo_schedule *sched, double *cost);

/* Whole-step CUDA graph for tdo_vmc_step (the optimisation workflow's step: sweeps, connections, L_loc
 * and cost, gradient, log-derivatives, SR solve, update).  With enable != 0, tdo_vmc_step records its
 * step into a CUDA graph on first use and then launches that graph, with one host synchronisation per
 * step (to return the cost and the outcome) instead of one per host decision.  Results are those of the
 * call-by-call step, up to the order of floating-point atomics:
 *   - the connected-row count stays on the device: buffers and grids are sized for n_chains x
 *     tdo_max_connections rows, and the kernels read the count the connection scan left on the device;
 *   - the CG's iterations are a conditional while node; a failed warm-started solve is rerun from x = 0
 *     inside the same launch, and the update is skipped on the device when the solve fails, L_loc is not
 *     finite or a bounded wait gave up; the status is then reported as tdo_sr_step reports it;
 *   - the sampler's counter and Adam's bias corrections are read from device memory, written before each
 *     launch, so advancing *counter and Adam's step count needs no new recording.
 * The step is recorded again when anything it depends on changes: n_chains, n_sweeps, seed, lr and
 * diag_shift (the schedules' values), the SR options and product mode, the optimiser, the chain
 * buffers' addresses, or a reallocation of the context's device workspace.  Host chain buffers are
 * staged (copied in before and out after each launch).  Graph mode records no per-group timing
 * (tdo_timing).  Needs a tensor-core context whose gradient runs on the tensor cores (token embedding,
 * d = 64, N <= 32): TDO_EUNSUPPORTED otherwise.  enable = 0 frees the recorded graph. */
tdo_status tdo_set_step_graph(tdo_ctx *ctx, int enable);
/* How many times the step graph has been recorded and launched (each pointer may be NULL). */
tdo_status tdo_step_graph_stats(const tdo_ctx *ctx, long long *recordings, long long *launches);

/* Device timing of this context's kernels: with enable != 0, every kernel launch of the calls above is
 * bracketed by CUDA events on the context's stream (records from before are dropped).  Used by the
 * benchmark to time kernels inside a real step. */
tdo_status tdo_timing(tdo_ctx *ctx, int enable);
/* Total recorded device time (ms) and launches of a kernel group since tdo_timing(ctx, 1):
 * "fwd" (transformer forward), "sample" (Metropolis), "bwd_vjp" (gradient backward), "bwd_jac"
 * (log-derivatives), "conn" (connections, scan, compaction), "lloc" (L_loc, cost, cotangents),
 * "sr" (CG solve), "sr_mv" (the S' v products inside "sr", each launch bracketed on its own), "update"
 * (parameter update and refresh), or "all" (every group but "sr_mv").  Synchronises the stream. */
tdo_status tdo_timing_read(tdo_ctx *ctx, const char *group, double *ms, long long *launches);

/* Iterations and final relative residual of the last tdo_sr_step's CG solve. */
tdo_status tdo_sr_info(const tdo_ctx *ctx, int *iters, double *resid);

/* How the last tdo_sr_step's CG solve ended (each pointer may be NULL): outcome 0 = stopped at the
 * iteration limit, 1 = converged, 2 = breakdown (p . (S + shift I) p not positive), 3 = a non-finite
 * value (the step then returned TDO_ENUMERIC); last_pap = the last p . (S + shift I) p, formed as
 * (1/Ns) sum_s |t_s - tbar|^2 + shift |p|^2 with t = O p (never negative); restarts = 1 when the
 * warm-started solve failed and was solved again from x = 0. */
tdo_status tdo_sr_report(const tdo_ctx *ctx, int *outcome, double *last_pap, int *restarts);

/* How the CG solve forms each product (Re S + shift I) v (metric-tensor section; the S matrix is never
 * formed).  TDO_SR_PRODUCT_TWO_PASS (default): two streaming passes over the log-derivatives, t = O v
 * per sample, then w = Re(O^H t) per parameter (HBM-bound; on GB300 at about 0.94 of the measured copy
 * bandwidth).  TDO_SR_PRODUCT_ONE_PASS: where the log-derivatives are stored as BF16 pairs (tensor-core
 * contexts) with rows on 16-byte boundaries, one pass: thread-block clusters of up to 16 CTAs each own a
 * range of samples and every CTA of a cluster one parameter slice; t_s is exchanged inside the cluster
 * through distributed shared memory, and w is accumulated from the same copy of the row in shared
 * memory.  It reads O once, but each row costs two block barriers and one cluster exchange, and on a
 * GB300 it measured 1.3 times slower than two passes at the headline shape (198,274 parameters, 16,384
 * samples); it is kept as an option.  All give the same products up to the order of FP32 partial sums
 * (each within 3e-7 of an FP64 evaluation of the definition).
 * TDO_SR_PRODUCT_GRID: also one pass where the log-derivatives are BF16 pairs on 16-byte rows, without
 * clusters: one CTA per SM owns a parameter slab of every row; rows go in blocks of 8, bulk-copied into a
 * ring of shared-memory stages; every CTA publishes its partials of t_s for a block to global memory as
 * tagged 64-bit words, dedicated exchange warps sum the partials of all CTAs (the same bits in every CTA)
 * while the compute warps work eight blocks ahead; w is accumulated from a second copy of each block,
 * served from L2, so DRAM reads O once.  On a GB300 at the headline shape it measured 4.50 ms per product
 * against 4.08 ms for two passes: one CTA unpacks and multiplies every element twice within one read's
 * time, so the SM side, not DRAM, bounds it; it is kept as an option.  Its bounded waits
 * watch the context's error flag (TDO_ETIMEOUT), so a launch whose CTAs cannot all run at once ends with
 * that error instead of waiting. */
enum { TDO_SR_PRODUCT_TWO_PASS = 0, TDO_SR_PRODUCT_ONE_PASS = 1, TDO_SR_PRODUCT_GRID = 2 };
tdo_status tdo_set_sr_product(tdo_ctx *ctx, int mode);

/* One product of the CG solve outside it: Ap = (Re S + shift I) v, S_ij = <O_i^* O_j> - <O_i^*><O_j> over
 * the Ns rows of O (metric-tensor and regularisation sections), S never formed.  O: log-derivatives as
 * BF16 pairs, one uint32 per element (Re in the low 16 bits, Im in the high 16 bits), [Ns][ldo] with
 * ldo >= the parameter count P, device memory owned by the caller; v, Ap: FP64 [P], device memory.  The
 * product runs in the mode of tdo_set_sr_product for tensor-core contexts, and in two passes in FP32
 * contexts; tdo_sr_product_shape reports it.  v is rounded to FP32 for the products with O, as in the
 * solve.  TDO_EINVAL for NULL or host pointers, Ns = 0 or ldo < P; TDO_ETIMEOUT when a bounded wait of the
 * one-pass product gave up.  Synchronises the context's stream. */
tdo_status tdo_sr_apply(tdo_ctx *ctx, const uint32_t *O, size_t Ns, size_t ldo, const double *v, double shift,
                        double *Ap);

/* The last tdo_sr_step's (or tdo_sr_apply's) product shape (each pointer may be NULL): one_pass = 1 when
 * the cluster product ran, 2 for the grid product, 0 for two passes; cluster = CTAs per cluster (1 for
 * the grid product); clusters = clusters (or CTAs of the grid product) launched (0, 0 for two
 * passes).  A bounded wait of
 * the one-pass product that gives up makes tdo_sr_step return TDO_ETIMEOUT. */
tdo_status tdo_sr_product_shape(const tdo_ctx *ctx, int *one_pass, int *cluster, int *clusters);

/* Arithmetic peak of the current device measured by the library (no counterpart in the paper):
 * kind 0 = FP32 fused multiply-add on the CUDA cores, 1 = FP64 FMA; *tflops = the best of three timed
 * launches (CUDA events on `stream`, a cudaStream_t or NULL) of a kernel of independent FMA chains,
 * 2 FLOP per FMA.  Allocates and frees a few bytes of device memory; synchronises the stream.  Used as
 * the denominator of the FP32 path's roofline fraction. */
tdo_status tdo_measure_peak(int kind, void *stream, double *tflops);

/* Self-test of the bounded device waits (no counterpart in the paper): launches one CTA that sets up the
 * tensor-core control block of the forward (two mbarriers, a TMEM allocation) and waits, at most
 * spin_limit polls (1 .. 2^20), for an MMA completion that nothing signals; no copy and no MMA is in
 * flight.  The wait gives up, the kernel raises the context's error flag, frees its TMEM and returns, and
 * the call reports TDO_ETIMEOUT exactly as a timed-out production kernel does.  The context stays
 * usable.  BF16 contexts only (TDO_EUNSUPPORTED otherwise). */
tdo_status tdo_wait_selftest(tdo_ctx *ctx, long long spin_limit);

/* Message of the last failing call on this context (or of the last failed tdo_create when ctx is NULL). */
const char *tdo_last_error(const tdo_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* TDO_H */
