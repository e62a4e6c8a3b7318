/*
 * fram.h -- C ABI of the GB300 (sm_103a) FRAM solver.
 *
 * FRAM (Frobenius-Regularized Assignment Matching, arXiv 2508.00887) matches
 * two undirected graphs with nonnegative symmetric adjacency matrices A and
 * A~ (written B here) by the projected fixed-point iteration of eq. 3:
 *
 *     X     = A N B + lambda K                     (Alg. 1 step 5, eq. 3)
 *     D     = SDSN(X, theta)                       (Alg. 1 step 6, Alg. 2)
 *     N     = (1 - alpha) N + alpha D              (Alg. 1 step 7)
 *     delta = ||N_t - N_{t-1}||_F / ||N_t||_F      (Alg. 1 step 8)
 *
 * until delta <= delta_tol, then rounds N to a permutation (eq. 2, Alg. 1
 * step 10).  Every step runs in this library's own CUDA kernels.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 *  - Matrices are dense, row-major, contiguous n x n arrays of IEEE double.
 *  - perm[i] (int32) is the node of the second graph matched to node i of
 *    the first graph: the matching matrix has M[i][perm[i]] = 1.
 *  - The caller owns every buffer it passes.  The library never frees or
 *    keeps a caller pointer after the call returns (fram_submit copies its
 *    inputs before returning).
 *  - Pointer kinds: fram_solve and fram_solve_batched accept host or device
 *    pointers for each matrix/vector argument (the kind is detected per
 *    pointer); host buffers are staged through the context's device
 *    workspace.  The step-level entry points (fram_gradient, fram_sdsn,
 *    fram_assign) take device pointers only.
 *  - All work is ordered on the context's stream.  Calls return after their
 *    results are written (they synchronise that stream).
 *  - Errors are reported by status code only; no exception or abort crosses
 *    the ABI.  fram_last_error() gives a one-line description of the most
 *    recent failure on a context.  Outputs are unspecified when a call fails.
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef FRAM_H
#define FRAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fram_ctx fram_ctx;

typedef enum {
  FRAM_OK = 0,
  FRAM_NOT_READY = 1,       /* fram_poll: request still in flight            */
  FRAM_ERR_INVALID = -1,    /* bad argument or input outside the graph model */
  FRAM_ERR_OOM = -2,        /* workspace would exceed the HBM budget         */
  FRAM_ERR_CUDA = -3,       /* a CUDA runtime call failed                    */
  FRAM_ERR_DEGENERATE = -4, /* max(X) <= 0 in SDSN step 1 (e.g. no edges)    */
  FRAM_ERR_TIMEOUT = -5,    /* a device-side wait exceeded its time limit    */
  FRAM_ERR_BUSY = -6        /* fram_submit: admission queue is full          */
} fram_status;

typedef enum {
  FRAM_PREC_FP64 = 0,       /* every step in FP64 (the parity path)                 */
  FRAM_PREC_MIXED_TF32 = 1, /* TF32 tensor-core gradient, FP32 SDSN, FP64 update    */
  FRAM_PREC_MIXED_BF16 = 2  /* BF16 tensor-core gradient, FP32 SDSN, FP64 update    */
} fram_precision;

/* Step 6 projection.  FRAM_PROJ_SDSN is Alg. 2 as printed (alternating
 * projections, stopped by gamma or the sweep cap).  FRAM_PROJ_EXACT computes
 * the FRA solution of eq. 4 / Thm. 1 exactly (not in the paper: multipliers
 * a, b with D = max(0, Y0 - a 1^T - 1 b^T) by dual block coordinate ascent,
 * see fram_fra_exact); FP64 path only. */
typedef enum {
  FRAM_PROJ_SDSN = 0,
  FRAM_PROJ_EXACT = 1
} fram_projection;

/* Solver parameters.  fram_default_params() fills the paper's settings
 * (Sec. 7 "Setting": lambda = 1, alpha = 0.95, theta = 10 for sparse graphs;
 * use theta = 2 for dense ones) and the tolerances and caps that the paper
 * leaves open. */
typedef struct {
  double lambda;      /* weight of the node term K (eq. 1); unused when K is NULL   */
  double alpha;       /* damping step of eq. 3, in (0, 1]                           */
  double theta;       /* FRA scale (Thm. 1); > 0                                    */
  double delta_tol;   /* outer stop: delta <= delta_tol (default 1e-6)              */
  double gamma_tol;   /* SDSN stop: gamma <= gamma_tol (default 1e-14)              */
  double polish_tol;  /* mixed paths: FP64 polish runs while gamma > polish_tol     */
  double mixed_delta_tol; /* mixed paths stop at delta <= max(delta_tol, this)       */
                          /* (default 5e-4): BF16/TF32 rounding of N and T puts a    */
                          /* floor under delta (~1e-4 BF16, ~1e-5 TF32 at n = 1000)   */
  double stall_ratio; /* mixed paths, safeguard: also stop once delta <= stall_below */
  double stall_below; /* and delta > stall_ratio * previous delta (defaults 0.9 and  */
                      /* 1e-3, near the BF16 floor; stall_ratio = 0 disables).  The  */
                      /* FP64 path ignores all three.  A slowly contracting delta    */
                      /* far above the floor is progress, not a stall.               */
  int max_outer;      /* outer-iteration cap (default 100)                          */
  int max_sweeps;     /* SDSN sweep cap per call (default 200)                      */
  int max_polish;     /* mixed paths: FP64 polish sweep cap per call (default 0)    */
  int precision;      /* fram_precision                                             */
  int init;           /* 0 = auto (N0 = 0 with K, 11^T/n without), 1 = zero, 2 = uniform */
  int projection;     /* fram_projection (default FRAM_PROJ_SDSN).  EXACT stops at a */
                      /* row residual <= max(gamma_tol, 8 n eps), at most max_sweeps */
                      /* sweeps; its residual is reported as gamma                   */
} fram_params;

/* Per-solve diagnostics (all optional to read). */
typedef struct {
  int outer_iters;          /* outer iterations run                             */
  int total_sweeps;         /* SDSN sweeps summed over the outer iterations     */
  int polish_sweeps;        /* FP64 polish sweeps (mixed paths)                 */
  int sdsn_converged_last;  /* 1 if the last SDSN call reached gamma_tol        */
  int lap_augmentations;    /* rows placed by augmenting paths (0: argmax path) */
  int lap_auction_phases;   /* epsilon-scaling auction phases run before them,
                               -1 if the auction was not needed              */
  double delta;             /* last delta                                       */
  double gamma;             /* gamma of the last SDSN output                    */
  double objective;         /* Phi at the permutation, unscaled inputs (eq. 1)  */
  double match_error;       /* 1/2 ||A - M B M^T||_F, unscaled (Sec. 7)         */
  double assignment_value;  /* sum_i N[i][perm[i]] at the final N               */
  double ms_total;          /* device time of the solve, milliseconds           */
  double ms_gemm;           /* device time in the gradient GEMMs (step 5)       */
  double ms_sdsn;           /* device time in SDSN (step 6; FP32 phase if mixed)*/
  double ms_polish;         /* device time in the FP64 polish (mixed paths)     */
  double ms_update;         /* device time in the update + delta (steps 7-8)    */
  double ms_rounding;       /* device time of the discretisation (eq. 2)        */
} fram_info;

/* ---------------------------------------------------------------- lifetime */

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the
 * device workspace the context may hold (0 = no cap).  `cuda_stream` is a
 * cudaStream_t to order all work on, or NULL for a stream owned by the
 * context.  Returns FRAM_ERR_INVALID for a bad device or NULL ctx pointer,
 * FRAM_ERR_CUDA if the device cannot be used. */
fram_status fram_create(fram_ctx **ctx, int device, size_t hbm_budget_bytes, void *cuda_stream);

/* Release the context and all device memory it holds.  NULL is a no-op. */
fram_status fram_destroy(fram_ctx *ctx);

/* Fill `p` with the defaults described at fram_params. */
void fram_default_params(fram_params *p);

/* Text of the last error on `ctx` ("" if none); valid until the next call. */
const char *fram_last_error(const fram_ctx *ctx);

/* Number of this library's kernels launched on `ctx` since creation. */
uint64_t fram_kernel_launches(const fram_ctx *ctx);

/* Time limit of every device-side wait on `ctx` (grid barriers, mbarrier
 * waits), in milliseconds (default 4000).  On expiry the waiting kernel
 * records the failure, stops, and the call returns FRAM_ERR_TIMEOUT; the
 * context stays usable.  FRAM_ERR_INVALID for limit_ms < 1. */
fram_status fram_set_wait_limit(fram_ctx *ctx, int limit_ms);

/* Failure-path self-test: launches `blocks` CTAs that wait at the library's
 * grid barrier for one more CTA than exists, so the wait can only end by its
 * time limit.  Returns FRAM_ERR_TIMEOUT (the expected outcome) after about
 * the context's wait limit; FRAM_ERR_INVALID for blocks < 1 or > 64. */
fram_status fram_selftest_wait_timeout(fram_ctx *ctx, int blocks);

/* ------------------------------------------------------------ full solve */

/* Solve one matching problem with FRAM (Alg. 1 + Alg. 2 + eq. 2).
 *   n        number of nodes of each graph, n >= 1 (the paper's n = n~, Sec. 3)
 *   A, B     n x n adjacency matrices: symmetric, nonnegative, finite
 *            (Sec. 3 "Graph").  Host or device memory.
 *   K        optional n x n node-similarity matrix K = F F~^T (eq. 1), or NULL.
 *   params   solver parameters, or NULL for fram_default_params().
 *   X_out    optional n x n output: the final soft assignment N.
 *   perm_out n int32 outputs: the discretised matching (eq. 2).
 *   info     optional diagnostics.
 * Errors: FRAM_ERR_INVALID (n < 1, NULL A/B/perm_out, non-square shapes,
 * asymmetric |A - A^T| > 1e-12 max(A, 1), negative or non-finite entries,
 * bad params), FRAM_ERR_DEGENERATE (max(X) <= 0, e.g. edgeless graphs),
 * FRAM_ERR_OOM, FRAM_ERR_TIMEOUT, FRAM_ERR_CUDA. */
fram_status fram_solve(fram_ctx *ctx, int n, const double *A, const double *B, const double *K,
                       const fram_params *params, double *X_out, int32_t *perm_out,
                       fram_info *info);

/* Solve `count` independent problems of (possibly different) sizes n[i] in
 * one call.  Each problem follows fram_solve exactly (same parameters, no K).
 * Problems with n[i] <= 64 run inside one persistent kernel, several per SM;
 * larger ones run one after another through the single-problem path.
 * Arrays of pointers are host arrays; the pointed-to matrices may be host or
 * device memory.  X_out and infos may be NULL. */
fram_status fram_solve_batched(fram_ctx *ctx, int count, const int *n, const double *const *A,
                               const double *const *B, const fram_params *params,
                               double *const *X_out, int32_t *const *perm_out, fram_info *infos);

/* Kernel form of fram_solve_batched's persistent launch (an autotuning and
 * testing hook).  0 (default): on the first call per precision, time every
 * form on a sample of the batch (every k-th pair, up to 32 per SM) and keep
 * the fastest.  1, 2, 3: one pair per
 * CTA of 128, 256 or 512 threads (FP64 and mixed).  4: teams of two warps,
 * a pair with n <= 32 on one warp (tile edge 32), a larger one on both
 * (tile edge 64); 5: every pair on two warps (mixed precision only; an FP64
 * batch with 4 or 5 returns FRAM_ERR_INVALID).  FRAM_ERR_INVALID outside 0..5. */
fram_status fram_set_batched_kernel(fram_ctx *ctx, int variant);

/* The form the batched path uses for `precision` (0 before its first call). */
int fram_batched_kernel(const fram_ctx *ctx, int precision);

/* ------------------------------------------------------------- serving */

/* Enqueue one problem for the context's continuous-batching scheduler (a
 * thread the context starts on first use).  A and B (host or device) are
 * copied into library-owned memory before the call returns, so the caller
 * may free them.  The scheduler admits waiting requests into device slots
 * while the HBM budget (hbm_budget_bytes of fram_create; 0 = 60% of the
 * memory free at first use) has room, keeps A, B, N and X resident until the
 * request retires, and advances all admitted requests together, one outer
 * iteration per tick, with their SDSN sweeps in one grouped launch.  Each
 * request computes exactly what fram_solve computes with the same params (no
 * K).  Returns FRAM_ERR_BUSY when the waiting queue is full. */
fram_status fram_submit(fram_ctx *ctx, int n, const double *A, const double *B,
                        const fram_params *params, uint64_t *ticket);

/* Collect a submitted problem.  Waits up to wait_ms milliseconds (0 = do not
 * wait, < 0 = wait until done).  Returns FRAM_NOT_READY while in flight.  On
 * completion the ticket retires: FRAM_OK copies N (if X_out != NULL), perm
 * and info out (host or device buffers; info.ms_total is the request's
 * latency from submit to completion); a failed request returns its error.
 * Unknown or retired tickets give FRAM_ERR_INVALID. */
fram_status fram_poll(fram_ctx *ctx, uint64_t ticket, double *X_out, int32_t *perm_out,
                      fram_info *info, int wait_ms);

/* Number of scheduler ticks the context's serving loop has run (one tick =
 * one outer iteration of every admitted request); 0 before the first
 * fram_submit.  With fram_kernel_launches it gives the launches per tick. */
uint64_t fram_serve_ticks(const fram_ctx *ctx);

/* ---------------------------------------------------- step-level entry points
 * Single steps of the path on DEVICE buffers, for testing and composition. */

/* Gradient of eq. 3 in FP64: X = A N B + lambda K (K may be NULL). */
fram_status fram_gradient(fram_ctx *ctx, int n, const double *A, const double *N, const double *B,
                          const double *K, double lambda, double *X);

/* FP64 path (fram_solve, fram_gradient): the gradient of eq. 3 uses CSR
 * products for A_s and for B_s when their fraction of nonzero entries is at
 * most max_density (default 0.2; 0 always uses the dense GEMM).  The CSR
 * products add the same terms in the same order as the dense GEMM, so the
 * result does not change, only the time: 2 nnz n instead of 2 n^3 flops.
 * FRAM_ERR_INVALID outside [0, 1]. */
fram_status fram_set_sparse_density(fram_ctx *ctx, double max_density);

/* Node-attribute affinity K = F Ft^T: the node term <N, F F~^T> of eq. 1,
 * whose gradient lambda F F~^T enters eq. 3.  K[i][j] is the inner product
 * of node i's attribute vector in G with node j's in G~.
 *   F, Ft : n x d row-major FP64 device arrays (caller-owned, read only).
 *   K     : n x n row-major FP64 device array (caller-owned), written.
 * Pass K to fram_solve; nonnegative attributes (descriptor histograms, for
 * instance) give the nonnegative K it requires.  Each entry is summed in
 * FP64 over k = 0..d-1 in order.  Errors: FRAM_ERR_INVALID for n < 1, d < 1
 * or null/host pointers. */
fram_status fram_node_affinity(fram_ctx *ctx, int n, int d, const double *F, const double *Ft,
                               double *K);

/* Gradient of eq. 3 as the mixed paths form it: A, N, B (FP64, device) are
 * rounded to BF16 (precision = FRAM_PREC_MIXED_BF16) or TF32
 * (FRAM_PREC_MIXED_TF32); T = A N is accumulated in FP32 on the tensor cores
 * and rounded to the same input format; X = T B (+ lambda K) is accumulated
 * in FP32 and written as an n x n FP32 device array. */
fram_status fram_gradient_lowp(fram_ctx *ctx, int n, const double *A, const double *N,
                               const double *B, const double *K, double lambda, int precision,
                               float *X);

/* SDSN (Alg. 2) in FP64 on X, written to D (D may equal X):
 * D0 = (theta/2) X / max(X); repeat D <- max(0, P1(D)) (eq. 7); stop when
 * gamma = sum(D)/n - 1 <= gamma_tol or after max_sweeps sweeps.
 * sweeps_out / gamma_out (host pointers) may be NULL.
 * FRAM_ERR_DEGENERATE if max(X) <= 0. */
fram_status fram_sdsn(fram_ctx *ctx, int n, const double *X, double *D, double theta,
                      double gamma_tol, int max_sweeps, int *sweeps_out, double *gamma_out);

/* SDSN (Alg. 2) as the mixed paths run it (Alg. 1 step 6 in FP32, Sec. 6
 * "Mixed-precision architecture"): the same kernel and launch configuration
 * as the FP32 phase inside fram_solve, on FP32 data.
 *   X  n x n FP32 device array, row stride ldx >= n elements (read only
 *      unless D == X)
 *   D  n x n FP32 device array, row stride ldd >= n (D == X allowed, then
 *      ldd == ldx); the padding columns of either are not touched
 * D0 = (theta/2) X / max(X) (max taken over the n x n block); every sweep
 * D <- max(0, P1(D)) (eq. 7) in FP32 arithmetic with FP32 row and column
 * sums; the total S (from FP32 partial totals) and gamma = S/n - 1 carry
 * about twice FP32's precision: FP64 in the streamed form (n > 1024), a
 * double-float sum in the on-chip forms; stop when gamma <= gamma_tol
 * (after at least one sweep) or after max_sweeps sweeps.  sweeps_out / gamma_out (host) may be NULL.
 * Errors: FRAM_ERR_INVALID (bad sizes, strides or pointers),
 * FRAM_ERR_DEGENERATE (max(X) <= 0), FRAM_ERR_TIMEOUT, FRAM_ERR_CUDA. */
fram_status fram_sdsn_f32(fram_ctx *ctx, int n, const float *X, int ldx, float *D, int ldd,
                          double theta, double gamma_tol, int max_sweeps, int *sweeps_out,
                          double *gamma_out);

/* Exact FRA projection (eq. 4 / Thm. 1; a variant of Alg. 1 step 6, not in
 * the paper): D = argmin over doubly stochastic D of ||D - (theta/2) X/max X||_F,
 * computed as D = max(0, Y0 - a 1^T - 1 b^T) by block coordinate ascent on
 * the dual (each multiplier the exact root of its piecewise-linear equation,
 * over-relaxed while the residual falls), in FP64.  X, D: n x n device
 * arrays (D may equal X), n <= 12800.  Stops at the first point whose row
 * residual max_i |sum_j D_ij - 1| is <= tol and whose column multipliers
 * came from a plain step (column sums exact up to rounding), or after
 * max_sweeps sweeps.  sweeps_out and res_out (host) may be NULL.
 * FRAM_ERR_DEGENERATE if max(X) <= 0. */
fram_status fram_fra_exact(fram_ctx *ctx, int n, const double *X, double *D, double theta,
                           double tol, int max_sweeps, int *sweeps_out, double *res_out);

/* SDSN (as fram_sdsn) of `count` independent problems in ONE grouped,
 * cooperative launch: problem i (size n[i], device X[i] -> D[i]) runs on the
 * same sub-grid fram_sdsn would give it, with its own barrier and stop test.
 * This is the serving path's grouped SDSN.  Problems whose sub-grids do not
 * all fit one co-resident wave return FRAM_ERR_INVALID.  sweeps_out and
 * gamma_out (host arrays of count) may be NULL. */
fram_status fram_sdsn_grouped(fram_ctx *ctx, int count, const int *n, const double *const *X,
                              double *const *D, double theta, double gamma_tol, int max_sweeps,
                              int *sweeps_out, double *gamma_out);

/* Linear assignment of eq. 2 on W (n x n, device, finite): perm maximises
 * sum_i W[i][perm[i]] (device int32 output; among optimal permutations the
 * one returned is unspecified).  value_out (host) receives that sum and
 * auction_phases_out (host) the number of epsilon-scaling auction phases
 * run before the final augmenting paths (-1: none were needed); either may
 * be NULL.  FRAM_ERR_TIMEOUT if the search did not terminate (non-finite
 * W). */
fram_status fram_assign(fram_ctx *ctx, int n, const double *W, int32_t *perm, double *value_out,
                        int *auction_phases_out);

/* Concurrent searches of the assignment's exact completion (eq. 2) for
 * n >= 1024, on `ctx` (fram_assign, the rounding of fram_solve and of served
 * requests).  0 (default): 8.  1: one shortest-augmenting-path search at a
 * time.  2..16: that many clusters of 8 CTAs, capped by how many can be
 * resident; each searches from its own free row on a snapshot of the duals
 * and commits its path under a lock, unless a commit since its start
 * changed a column it popped, in which case it searches again.  Every
 * setting returns an optimal permutation; only the choice among tied optima
 * can differ from run to run.  FRAM_ERR_INVALID outside 0..16. */
fram_status fram_set_lap_searches(fram_ctx *ctx, int searches);

/* Statistics of the last assignment run by fram_assign or fram_solve on
 * `ctx`: augmenting paths applied, searches repeated after a conflicting
 * commit (always 0 for one search at a time) and Dijkstra steps of the last
 * completion pass, repeated searches included.  Any pointer may be NULL.
 * FRAM_ERR_INVALID if no assignment has run on ctx. */
fram_status fram_lap_last_stats(const fram_ctx *ctx, int *augmented, int *repeats,
                                long long *steps);

/* Largest n that fram_sdsn_static accepts. */
#define FRAM_SDSN_STATIC_MAX_N 4096

/* fram_sdsn without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory -- applications whose device memory belongs to another
 * allocator (a framework's caching allocator or a pool reserved up front,
 * which a foreign cudaMalloc would bypass or find empty) and loops that cannot
 * afford the device-wide synchronisation of cudaFree.
 *
 * Same computation, kernel and launch configuration as fram_sdsn, on DEVICE
 * buffers X and D (n x n row-major doubles, D may equal X), ordered on
 * `cuda_stream` (NULL = legacy default stream); returns after the result is
 * written.  No context is needed and nothing is allocated: the scratch (SDSN
 * partials, grid barrier, max(X), status; about 2 MiB) is a static device
 * array that every GPU loading this library holds until the process exits.
 *  - n > FRAM_SDSN_STATIC_MAX_N returns FRAM_ERR_INVALID with a message.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents (each call clears what must start at zero).  Calls that overlap
 *    on the GPU race on it: serialise them on one stream.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture begins.
 * sweeps_out / gamma_out (host) may be NULL; `err` (host, err_len bytes, may
 * be NULL) receives a one-line message on failure.  Other errors as fram_sdsn. */
fram_status fram_sdsn_static(int n, const double *X, double *D, double theta, double gamma_tol,
                             int max_sweeps, void *cuda_stream, int *sweeps_out, double *gamma_out,
                             char *err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* FRAM_H */
