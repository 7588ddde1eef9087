/*
 * lslu.h - C ABI of the GB300 (sm_103a) LSLU / Hybrid LSLU library.
 *
 * The library solves b = A x + e for a sparse rectangular A (m x n, CSR) with
 * the inner-product-free LSLU and Hybrid LSLU methods of Brown, Chung, Nagy
 * and Sabate Landman, "Inner Product Free Krylov Methods for Large-Scale
 * Inverse Problems" (arXiv 2409.05239):
 *   - the basis L_k (n-space) and D_{k+1} (m-space) come from the Hessenberg
 *     process with pivoting for rectangular systems (Algorithm 4), with
 *     A L_k = D_{k+1} H_{k+1,k} and A^T D_{k+1} = L_{k+1} W_{k+1}
 *     (Eqs. nhr, nhr2);
 *   - x_k = x_0 + L_k y_k with y_k = argmin ||beta e1 - H_{k+1,k} y||^2 +
 *     lambda_k^2 ||y||^2 (Eq. TSP, Algorithm 5); lambda_k = 0 is LSLU
 *     (Section 2.2), otherwise lambda_k is fixed or chosen by GCV (Eq. gcv2)
 *     or weighted GCV with omega = (k+1)/m (Eq. wgcv).
 *
 * Conventions shared by every entry point:
 *   - indices are 0-based; dense matrices are column-major;
 *   - every call returns an lslu_status; the library never aborts or traps;
 *     lslu_error_string() gives a one-line description of the last failure;
 *   - pointers marked "host or device" are read or written on the host when
 *     ptr_location is LSLU_HOST and on the current CUDA device when it is
 *     LSLU_DEVICE; the caller owns every buffer it passes, the library owns
 *     the memory behind a handle until lslu_destroy();
 *   - calls on one handle are not thread-safe; all device work of a handle is
 *     ordered on the stream given at creation (NULL = the legacy default
 *     stream); calls that return host data synchronise that stream.
 */
#ifndef LSLU_H
#define LSLU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lslu_ctx* lslu_handle;

typedef enum {
  LSLU_OK = 0,
  LSLU_ERR_INVALID_ARG = 1,  /* a size, pointer, CSR structure or option is invalid */
  LSLU_ERR_CUDA = 2,         /* a CUDA runtime call failed                         */
  LSLU_ERR_OOM = 3,          /* device memory allocation failed                    */
  LSLU_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up                  */
  LSLU_BREAKDOWN_BETA = 5,   /* r0 = b - A x0 is zero (Algorithm 4, initialisation) */
  LSLU_BREAKDOWN_W = 6,      /* q has no non-zero unpivoted entry (Algorithm 4)     */
  LSLU_BREAKDOWN_H = 7,      /* u has no non-zero unpivoted entry (Algorithm 4)     */
  LSLU_ERR_NONFINITE = 8     /* a pivot or the data is NaN or infinite             */
} lslu_status;

/* Storage of A's values.  F64 keeps the basis and all accumulation in FP64.
 * F32 and BF16 keep the basis vectors in FP32 and accumulate in FP32; the
 * Hessenberg entries (H, W), the projected solve, lambda and x stay FP64. */
typedef enum { LSLU_F64 = 0, LSLU_F32 = 1, LSLU_BF16 = 2 } lslu_value_type;

/* Choice of lambda_k in Algorithm 5 (Section 3.2.1). */
typedef enum {
  LSLU_LAMBDA_NONE = 0,  /* LSLU: lambda = 0                                  */
  LSLU_LAMBDA_FIXED = 1, /* the lambda argument for every k                   */
  LSLU_LAMBDA_GCV = 2,   /* minimiser of the projected GCV function, Eq. gcv2 */
  LSLU_LAMBDA_WGCV = 3   /* weighted GCV, omega = (k+1)/m, Eq. wgcv           */
} lslu_lambda_rule;

enum { LSLU_HOST = 0, LSLU_DEVICE = 1 };

/* Create a solver for the m x n CSR matrix A (row_ptr: m+1 int64 offsets,
 * col_idx: nnz int32 column indices in [0, n), vals: nnz FP64 values), all
 * host or device per ptr_location.  The values are rounded to value_type
 * (FP64 -> FP32 round-to-nearest-even; BF16 rounds that FP32 value to
 * nearest-even).  The library keeps its own copy of A and of A^T (a
 * transposed CSR, so A^T u needs no atomics) and allocates the bases for up to
 * max_iter iterations: (n + m) * (max_iter + 1) basis entries.
 * Errors: LSLU_ERR_INVALID_ARG for m, n < 1, nnz < 0, nnz >= 2^31,
 * max_iter < 1 or > 2048, a non-monotone row_ptr, a column out of range or a
 * non-finite value; LSLU_ERR_OOM; LSLU_ERR_CUDA.  *out is NULL on failure. */
lslu_status lslu_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                        const int32_t* col_idx, const double* vals, int32_t value_type,
                        int32_t max_iter, int32_t ptr_location, void* cuda_stream,
                        lslu_handle* out);

/* lslu_create with a renumbering of the rows and columns of A, for memory
 * locality of the sparse products (Algorithm 4 gathers the basis vector
 * through the column indices of every row).  row_order (m int32) and
 * col_order (n int32) are permutations: caller row i becomes internal row
 * row_order[i], caller column j internal column col_order[j]; NULL is the
 * identity.  Host or device per ptr_location, like the CSR arrays; copied.
 * The handle stores A_hat = P_r A P_c^T (each row's entries sorted by the new
 * column) and runs every solve on A_hat and b_hat = P_r b.  Every entry point
 * takes and returns vectors, bases and pivot indices in the caller's
 * numbering: the renumbering is applied on entry and undone on exit.  Max-abs
 * pivots pick the same entries in any numbering, and every pivot search
 * breaks ties by the caller's index (Algorithm 4's lowest index), so the
 * pivots are lslu_create's and the results equal up to the rounding order of
 * the products.  lslu_spmv is refused on such a handle.
 * Errors: those of lslu_create, and LSLU_ERR_INVALID_ARG when an order is not
 * a permutation of [0, m) or [0, n). */
lslu_status lslu_create_ordered(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                const int32_t* col_idx, const double* vals, int32_t value_type,
                                int32_t max_iter, const int32_t* row_order,
                                const int32_t* col_order, int32_t ptr_location,
                                void* cuda_stream, lslu_handle* out);

/* Run K iterations of Hybrid LSLU (Algorithm 5) on data b (length m, FP64)
 * from x0 (length n, FP64; NULL means x0 = 0).  rule is an lslu_lambda_rule;
 * lambda is used by LSLU_LAMBDA_FIXED only.  Outputs (host or device per
 * ptr_location, any may be NULL except x_out):
 *   x_out       n      FP64  x_k of the last completed iteration k = *k_done
 *   col_pivots  K      int32 g: pivot row of l_1..l_k (entries past k_done = -1)
 *   row_pivots  K+1    int32 t: pivot row of d_1..d_{k+1}
 *   lambda_hist K      FP64  lambda_j for j = 1..k (needs per-iteration solves)
 *   resid_hist  K      FP64  ||beta e1 - H_{j+1,j} y_j|| for j = 1..k
 *   k_done      1      int32 completed iterations (== K unless a breakdown)
 * When lambda_hist or resid_hist is non-NULL the projected problem is solved
 * for every j (all at once after the basis loop, since the basis never
 * depends on lambda); otherwise only for j = k_done.  x_out is the same bit
 * for bit either way.  A breakdown is not a failure of the call: it returns
 * LSLU_BREAKDOWN_* with x of the last completed iteration (x0 if none).  K
 * must satisfy 1 <= K <= max_iter. */
lslu_status lslu_solve(lslu_handle h, const double* b, const double* x0, int32_t K,
                       int32_t rule, double lambda, int32_t ptr_location, double* x_out,
                       int32_t* col_pivots, int32_t* row_pivots, double* lambda_hist,
                       double* resid_hist, int32_t* k_done);

/* Batched Hybrid LSLU (Algorithm 5 run independently on nprob problems that
 * share one launch sequence).  Problem p owns rows row_off[p] .. row_off[p+1]-1
 * and columns col_off[p] .. col_off[p+1]-1 of one block-diagonal CSR matrix
 * (row_ptr: row_off[nprob]+1 int64 offsets; col_idx: int32; vals: FP64; every
 * entry of a row of problem p must lie in problem p's column range).  All
 * arrays are host memory; row_off and col_off have nprob+1 entries, start at
 * 0 and are strictly increasing.  Values are stored as value_type, which must
 * be LSLU_F32 or LSLU_BF16 (the basis is FP32).  Internally every problem
 * starts on a 128-row boundary of the concatenated row and column spaces, so
 * each tile of the elimination kernels belongs to one problem; the padding
 * rows are masked out of every pivot search.
 * Errors: LSLU_ERR_INVALID_ARG (nprob < 1, bad offsets, a problem with no row
 * or column, an entry outside its block, a non-finite value, FP64 values,
 * max_iter outside [1, 2048]); LSLU_ERR_OOM; LSLU_ERR_CUDA. */
lslu_status lslu_create_batched(int32_t nprob, const int64_t* row_off, const int64_t* col_off,
                                const int64_t* row_ptr, const int32_t* col_idx,
                                const double* vals, int32_t value_type, int32_t max_iter,
                                void* cuda_stream, lslu_handle* out);

/* lslu_create_batched with every problem renumbered for memory locality, as
 * lslu_create_ordered does for one problem.  row_order (row_off[nprob] int32)
 * and col_order (col_off[nprob] int32), host memory, are permutations of the
 * concatenated rows and columns that map each problem's range onto itself:
 * caller row i becomes internal row row_order[i]; NULL is the identity.
 * lslu_solve_batched takes b and returns x and the pivot indices in the
 * caller's numbering; pivot searches break ties by the caller's index, as
 * without a renumbering.  Errors: those of lslu_create_batched, and LSLU_ERR_INVALID_ARG when
 * an order is not a permutation or moves an index out of its problem. */
lslu_status lslu_create_batched_ordered(int32_t nprob, const int64_t* row_off,
                                        const int64_t* col_off, const int64_t* row_ptr,
                                        const int32_t* col_idx, const double* vals,
                                        int32_t value_type, int32_t max_iter,
                                        const int32_t* row_order, const int32_t* col_order,
                                        void* cuda_stream, lslu_handle* out);

/* A batched handle for nrhs right-hand sides that share one m x n CSR matrix
 * (row_ptr m+1 int64, col_idx int32 in [0, n), vals FP64; host memory).  The
 * matrix and its transpose are stored once, and every sparse product reads
 * them once for all right-hand sides: the nrhs input vectors are interleaved
 * so that each non-zero fetches its nrhs operands together.  Solved with
 * lslu_solve_batched (problem r = right-hand side r: b holds nrhs x m values,
 * x_out nrhs x n); each right-hand side gets the result of a single-problem
 * solve, bit for bit.  value_type LSLU_F32 or LSLU_BF16; 1 <= nrhs <= 16.
 * Errors: as lslu_create_batched. */
lslu_status lslu_create_shared(int64_t m, int64_t n, const int64_t* row_ptr,
                               const int32_t* col_idx, const double* vals, int32_t nrhs,
                               int32_t value_type, int32_t max_iter, void* cuda_stream,
                               lslu_handle* out);

/* lslu_create_shared with the matrix renumbered for memory locality, as
 * lslu_create_ordered does: row_order (m int32) and col_order (n int32), host
 * memory, are permutations (NULL: the identity) applied to the one stored
 * matrix and so to every right-hand side.  lslu_solve_batched takes b and
 * returns x and the pivot indices in the caller's numbering; pivot searches
 * break ties by the caller's index.  Errors: those of lslu_create_shared, and
 * LSLU_ERR_INVALID_ARG when an order is not a permutation. */
lslu_status lslu_create_shared_ordered(int64_t m, int64_t n, const int64_t* row_ptr,
                                       const int32_t* col_idx, const double* vals, int32_t nrhs,
                                       int32_t value_type, int32_t max_iter,
                                       const int32_t* row_order, const int32_t* col_order,
                                       void* cuda_stream, lslu_handle* out);

/* K iterations of Hybrid LSLU on every problem of a batched handle, from
 * x0 = 0.  b has row_off[nprob] FP64 entries (problem p's data at
 * row_off[p]); rule and lambda as in lslu_solve (the same rule for every
 * problem; lambda_k is chosen per problem, and LSLU_LAMBDA_WGCV uses each
 * problem's own row count).  Outputs (host or device per ptr_location; all
 * but x_out may be NULL):
 *   x_out       col_off[nprob]  FP64  x of every problem at its k_done
 *   col_pivots  nprob x K       int32 g of problem p at p*K, indices local to
 *                                     the problem, -1 past its k_done
 *   row_pivots  nprob x (K+1)   int32 t, same layout with stride K+1
 *   k_done      nprob           int32 completed iterations per problem
 *   status      nprob           int32 lslu_status of each problem (OK or a
 *                                     LSLU_BREAKDOWN_* code)
 * A breakdown stops only its own problem.  The call returns LSLU_OK unless an
 * argument is invalid or CUDA fails; 1 <= K <= max_iter. */
lslu_status lslu_solve_batched(lslu_handle h, const double* b, int32_t K, int32_t rule,
                               double lambda, int32_t ptr_location, double* x_out,
                               int32_t* col_pivots, int32_t* row_pivots, int32_t* k_done,
                               int32_t* status);

/* lslu_solve with the sampled pivoting of Section 2.2: every pivot is the
 * largest |entry| among the unpivoted rows of a small sample instead of the
 * whole vector (ties: lowest index); when no sampled unpivoted entry is
 * non-zero the full search is used.  samples holds 2K+1 rows of nsamp int32
 * indices (row-major; host or device per ptr_location): row 0 for r0 and
 * row 2k+2 for u at iteration k index [0, m), row 2k+1 for q indexes [0, n).
 * The caller draws the random indices (any generator), so results are
 * reproducible from the table.  Single-problem handles; 1 <= nsamp <= 65536.
 * Outputs as lslu_solve. */
lslu_status lslu_solve_sampled(lslu_handle h, const double* b, const double* x0, int32_t K,
                               int32_t rule, double lambda, const int32_t* samples,
                               int32_t nsamp, int32_t ptr_location, double* x_out,
                               int32_t* col_pivots, int32_t* row_pivots, int32_t* k_done);

/* lslu_solve with the pivot lists given instead of searched: iteration k
 * takes row col_pivots[k] of the L-side vector and row row_pivots[k+1] of the
 * D-side vector as its pivots (row_pivots[0] for r0), whatever their
 * magnitude.  With the pivots of an earlier solve this is the map whose
 * derivative lslu_adjoint computes (finite differences with the pivots held
 * fixed).  col_pivots: K distinct indices in [0, n); row_pivots: K+1 distinct
 * indices in [0, m) (host or device per ptr_location, validated on the host).
 * A zero entry at a given pivot is a breakdown.  Outputs x_out (n) and
 * k_done (may be NULL) as in lslu_solve; the call leaves the same state for
 * lslu_get_state and lslu_adjoint. */
lslu_status lslu_solve_fixed_pivots(lslu_handle h, const double* b, const double* x0, int32_t K,
                                    int32_t rule, double lambda, int32_t ptr_location,
                                    const int32_t* col_pivots, const int32_t* row_pivots,
                                    double* x_out, int32_t* k_done);

/* Reverse-mode derivative of the last lslu_solve with its pivot lists held
 * fixed (with g and t fixed, Algorithm 5 is a smooth map (b, lambda) -> x_K).
 * Given x_bar = dJ/dx_K for any scalar loss J (n, FP64), returns
 *   b_bar       m  FP64  dJ/db = (dx_K/db)^T x_bar
 *   lambda_bar  1  FP64  dJ/dlambda for the lambda_K the solve used, taken as
 *                        an independent parameter (may be NULL)
 *   x0_bar      n  FP64  dJ/dx0 (may be NULL)
 * all host or device per ptr_location.  The sweep runs the transposed steps
 * on the device: per iteration two sparse products and passes over the
 * stored bases (about twice the bytes of the forward solve); the projected
 * adjoint uses a Cholesky factorisation of H^T H + lambda^2 I.  The first
 * call allocates a work space of the size of the two bases.
 * Errors: LSLU_ERR_INVALID_ARG for a batched handle, when the last
 * lslu_solve did not complete all K iterations (or lslu_projected ran since),
 * or when H^T H + lambda^2 I is not positive definite (lambda = 0 with a rank
 * deficient H); LSLU_ERR_OOM; LSLU_ERR_CUDA. */
lslu_status lslu_adjoint(lslu_handle h, const double* x_bar, int32_t ptr_location,
                         double* b_bar, double* lambda_bar, double* x0_bar);

/* Hybrid LSLU with the stopping criterion of Section 3.2.2: runs up to K_max
 * iterations (2 <= K_max <= max_iter), solves the projected problem of every
 * k with the lambda rule, evaluates
 *   G^(k) = n ||beta e1 - H_{k+1,k} y_k||^2 / ((m - k) + sum_i lam_k^2/(sigma_i^2 + lam_k^2))^2
 * (Eq. stop2, read with the filter factor multiplying [U^T e1]_i as in its
 * derivation) and stops at the first k with |G^(k+1) - G^(k)| / G^(1) < tol
 * (Eq. tol), else at the last completed iteration.  Outputs (host or device per
 * ptr_location): x_out (n) = x_k at that iteration (equal to lslu_solve with
 * K = k), k_stop (1), g_hist (K_max, may be NULL).  The graph loop mode
 * (the default) stops online: it runs the basis in chunks of 8 iterations,
 * solves the projected problems of each chunk's sizes and evaluates the
 * criterion after each chunk, so it computes at most 8 iterations past
 * k_stop + 1 (the test needs G^(k+1)); g_hist then holds G^(k) for the
 * iterations evaluated (at least through k_stop + 1, whole chunks or K_max)
 * and zero past them.  With the persistent or cluster loop (lslu_set_loop) it
 * runs all K_max iterations, g_hist holds every G^(k) (zero past k_done), and
 * x0 must be NULL.  Either way the basis of the first k iterations does not
 * depend on the later ones, so x and each G^(k) are those of the full run.
 * A breakdown ends the sequence at k_done. */
lslu_status lslu_solve_stopping(lslu_handle h, const double* b, const double* x0, int32_t K_max,
                                int32_t rule, double lambda, double tol, int32_t ptr_location,
                                double* x_out, int32_t* k_stop, double* g_hist);

/* Copy the state of the last lslu_solve (host or device per ptr_location;
 * any pointer may be NULL).  k = *k_done of that solve.
 *   H  (k+1) x k FP64 column-major, W k x k FP64 column-major, beta 1 FP64,
 *   L  n x k basis (FP64 for LSLU_F64, FP32 otherwise), column-major,
 *   D  m x (k+1) basis, column-major.
 * Errors: LSLU_ERR_INVALID_ARG if no lslu_solve has run (batched solves keep
 * no exportable state). */
lslu_status lslu_get_state(lslu_handle h, int32_t ptr_location, double* H, double* W,
                           double* beta, void* L, void* D);

/* One sparse product on the device (the first step of each half of an
 * Algorithm 4 iteration): y = A x (transpose = 0; x length n, y length m) or
 * y = A^T x (transpose = 1; x length m, y length n).  x and y are device
 * pointers of the basis type (FP64 for LSLU_F64, FP32 otherwise).  Launched
 * on the handle's stream without synchronising.  Single-problem handles only. */
lslu_status lslu_spmv(lslu_handle h, int32_t transpose, const void* x, void* y);

/* Solve the projected problem of Eq. (TSP) for one upper Hessenberg
 * H ((k+1) x k, FP64, column-major with leading dimension ldh >= k+1) and
 * beta, on the device, with the lambda rule of lslu_solve (m is the row
 * count used by LSLU_LAMBDA_WGCV for omega = (k+1)/m).  Outputs (any may be
 * NULL): y (k), sigma (k, descending singular values of H), c (k+1,
 * beta U^T e1), lambda_out (1), resid_out (1, ||beta e1 - H y||).  Uses the
 * handle's workspace; 1 <= k <= max_iter of the handle. */
lslu_status lslu_projected(lslu_handle h, int32_t k, const double* H, int32_t ldh, double beta,
                           int32_t rule, double lambda, int64_t m, int32_t ptr_location,
                           double* y, double* sigma, double* c, double* lambda_out,
                           double* resid_out);

/* The projected problems of a whole history (Algorithm 5 solves Eq. TSP at
 * every iteration): for every leading block H_{k+1,k}, k = 1..K, of one
 * H ((K+1) x K, FP64, column-major, ldh >= K+1; H_{k+1,k} is rows 0..k and
 * columns 0..k-1) with the same beta, lambda_k by the rule of lslu_solve and
 * the residual ||beta e1 - H_{k+1,k} y_k||.  The same launches as the
 * histories of lslu_solve, so a history can be recomputed under another rule
 * from lslu_get_state's H without running the basis again; lambda_hist[K-1]
 * equals lslu_projected's lambda_out for k = K bit for bit.  H, lambda_hist
 * (K) and resid_hist (K; either may be NULL) are host or device per
 * ptr_location.  Uses the handle's workspace; 1 <= K <= max_iter of the
 * handle.  Errors: LSLU_ERR_INVALID_ARG (K, ldh, H, rule, m, a negative
 * fixed lambda, ptr_location), LSLU_ERR_OOM, LSLU_ERR_CUDA. */
lslu_status lslu_projected_history(lslu_handle h, int32_t K, const double* H, int32_t ldh,
                                   double beta, int32_t rule, double lambda, int64_t m,
                                   int32_t ptr_location, double* lambda_hist, double* resid_hist);

/* Allocation-free variant of lslu_projected, for callers that cannot call
 * cudaMalloc (for example code that runs under a framework whose memory pool
 * must own every device allocation, or a time-critical loop that cannot
 * afford an allocation's implicit synchronisation).  The paper has no
 * counterpart: this is a deployment interface.
 *   - Same problem and outputs as lslu_projected, but every pointer (H, y,
 *     sigma, c, lambda_out, resid_out) is a device pointer, no handle is
 *     needed, and the work runs asynchronously on cuda_stream (NULL = the
 *     legacy default stream): the outputs are ready once that stream reaches
 *     this point.  Any output pointer may be NULL.  c holds |beta U^T e1|.
 *   - Work space: a fixed array of 1.12 MB of device memory that the library
 *     reserves when it is loaded, on every GPU that loads it, until the
 *     process exits.  It serves 1 <= k <= 256; larger k is rejected with
 *     LSLU_ERR_INVALID_ARG and a message naming the limit.  Nothing else is
 *     allocated.
 *   - The first call on a device looks up the array's device address and
 *     sets kernel attributes for that device; make it before any stream
 *     capture.
 *   - Every call shares the one array: calls whose work may overlap on the
 *     GPU (other streams, other host threads) race and must be serialised by
 *     the caller.  No part of the array needs to start at zero.
 * Errors: LSLU_ERR_INVALID_ARG, LSLU_ERR_CUDA; lslu_error_string(NULL) has
 * the message. */
lslu_status lslu_projected_noalloc(int32_t k, const double* H, int32_t ldh, double beta,
                                   int32_t rule, double lambda, int64_t m, double* y,
                                   double* sigma, double* c, double* lambda_out,
                                   double* resid_out, void* cuda_stream);

/* Per-kernel CUDA-event timing of later solves: enable != 0 records an
 * event pair around every sparse product launched by lslu_solve.
 * lslu_timing returns the number of such launches since the last reset and
 * their summed duration in milliseconds, then resets the counters. */
lslu_status lslu_profile(lslu_handle h, int32_t enable);
lslu_status lslu_timing(lslu_handle h, int32_t* spmv_launches, double* spmv_ms);

/* Number of kernel launches made by the last lslu_solve. */
int64_t lslu_last_launch_count(lslu_handle h);

/* K iterations of Hybrid LSLU with the optimal Tikhonov parameter of the
 * final projected problem, the one that minimises ||L_K y_K(lambda) - x_true||
 * (Eq. lambda of Section 3.2.1, the reference curves of Section 4.1; needs the
 * true solution): the error is
 * evaluated on the 257-point grid sigma_1 10^[-14, 2] and refined between the
 * best point's neighbours by 5 rounds of 63-point multisection in log(lambda)
 * (each round keeps its best point and that point's neighbours).
 * Outputs x_out (n) = x_K for that lambda (equal to lslu_solve with
 * LSLU_LAMBDA_FIXED and that lambda) and lambda_out (1, may be NULL); host or
 * device per ptr_location (b: m, x_true: n, FP64).  A breakdown before
 * iteration K is returned as its status. */
lslu_status lslu_solve_optimal(lslu_handle h, const double* b, int32_t K, const double* x_true,
                               int32_t ptr_location, double* x_out, double* lambda_out);

/* Low-rank uncertainty quantification of Section 4.2 on the state of the last
 * lslu_solve (k = its k_done): with A^T A ~ L_k W_k (D_k^T D_k)^-1 W_k^T L_k^T
 * (Eq. nhr2) and lambda = sigma / alpha, the posterior covariance
 * sigma^2 (lambda^2 I + A^T A)^-1 is approximated by
 *   Gamma_k = sigma^2 lambda^-2 (I - L_k M L_k^T),
 *   M = (L_k^T L_k + lambda^2 (G^T G)^-1)^-1,  G^T G = W_k (D_k^T D_k)^-1 W_k^T
 * (the paper's Woodbury form, with lambda^2 for its lambda).  Outputs (host
 * or device per ptr_location, either may be NULL): var_diag (n, FP64) the
 * diagonal of Gamma_k (posterior variances), var_sum (1) = 1^T Gamma_k 1.
 * sigma2 (noise variance) and lambda must be > 0.  Single-problem handles.
 * The k x k Cholesky factor runs on one thread-block cluster that keeps its
 * columns in shared memory: k up to about 640 with 16 CTAs (beyond that W_k is
 * numerically singular in FP64 for this method).
 * Errors: LSLU_ERR_INVALID_ARG when no solve has completed an iteration, the
 * k x k system is not positive definite, or k is above that limit;
 * LSLU_ERR_OOM; LSLU_ERR_CUDA. */
lslu_status lslu_uq(lslu_handle h, double sigma2, double lambda, int32_t ptr_location,
                    double* var_diag, double* var_sum);

/* Row shape of the sparse products: lanes per CSR row x chunks in flight per
 * lane.  Shapes 0-5 read 32-bit column indices in chunks of 4 entries:
 * 0: 16x2 (default for FP32/BF16 values), 1: 32x1, 2: 16x1 (default for
 * FP64 values), 3: 8x1, 4: 8x2, 5: 4x1; shapes 6-11 are the same lane shapes
 * on 16-bit column offsets in chunks of 8 entries (2.5 instead of 4 bytes per
 * entry; available when every 8-entry unit of the matrix spans fewer than
 * 2^16 columns, see lslu_spmv_config).  Shapes 12 ("32x8e") and 14
 * ("32x4e") put the 32 lanes of a warp on consecutive entries of one row (8
 * or 4 entries in flight per lane), so neighbouring columns share the sectors
 * of their x gathers; 13 and 15 are the same on 16-bit offsets.  Every shape
 * computes the same products with a different summation order, so results
 * change in rounding only; each is bitwise reproducible.  The shared-matrix
 * product of lslu_create_shared follows the default 16-lane shapes.
 * Errors: LSLU_ERR_INVALID_ARG for a shape outside [0, 16) or one the matrix
 * does not support. */
lslu_status lslu_set_spmv_shape(lslu_handle h, int32_t shape_A, int32_t shape_AT);

/* The sparse products' configuration (host outputs, any may be NULL): the
 * row shape of A and A^T and whether each has 16-bit column offsets. */
lslu_status lslu_spmv_config(lslu_handle h, int32_t* shape_A, int32_t* shape_AT,
                             int32_t* compressed_A, int32_t* compressed_AT);

/* Autotuner: times every row shape on the handle's A and A^T (each rep
 * launches A then A^T, as a solve does, each after a read of twice the L2
 * size that stands in for the elimination before every product of a solve;
 * CUDA events on the handle's stream, after one warm-up pair) and keeps the
 * fastest shape for each, or the default shape unless the fastest beats it
 * by more than 3% (closer times swap places from run to run).  Allocates
 * and frees the flush buffer (LSLU_ERR_OOM if it cannot).  Outputs (host, any may
 * be NULL): the chosen shapes and the average time of every shape in
 * microseconds (us[0..15] for A, us[16..31] for A^T; -1 where unavailable).
 * Drops captured solves (they hold the old kernels). */
lslu_status lslu_tune_spmv(lslu_handle h, int32_t reps, int32_t* shape_A, int32_t* shape_AT,
                           double* us);

/* How later solves on the handle run the basis loop of Algorithm 4:
 *   LSLU_LOOP_GRAPH       each step is its own kernel (six per iteration),
 *                         replayed from a captured CUDA graph (default);
 *   LSLU_LOOP_PERSISTENT  one cooperative launch runs the pivot of r0 and all
 *                         K iterations, with grid-wide barriers between the
 *                         dependent steps (four per iteration).  For
 *                         workloads whose steps are too short to fill the
 *                         GPU (small problems, small batches);
 *   LSLU_LOOP_CLUSTER     one thread-block cluster (16 CTAs where the device
 *                         allows, else 8) runs the same steps for one small
 *                         problem, keeping the current basis vector, T^-1 and
 *                         its rows of every vector in shared memory and
 *                         synchronising with hardware cluster barriers; single
 *                         problems whose vectors and T^-1 fit a CTA's shared
 *                         memory: about max(m, n) + 2 (max_iter+1)^2 entries
 *                         of the compute type (8 bytes with FP64 values, 4
 *                         otherwise), at most 200 KB (refused otherwise).
 *                         blocks and stall_first_barrier must be 0.
 * The projected solve and x = L y follow as in the graph mode.  A persistent
 * handle serves lslu_solve, lslu_solve_batched, lslu_solve_stopping and
 * lslu_solve_optimal with x0 = NULL and searched pivots; x0, replayed or
 * sampled pivots return LSLU_ERR_INVALID_ARG (set the graph mode for them).
 * Results equal the graph mode's up to the rounding order of the products
 * (identical pivots wherever no near-tie separates them).
 *   blocks          blocks of the launch; 0 = one per SM, or fewer for small
 *                   problems; at most the co-resident count (lslu_loop_config).
 *   wait_limit_ns   every barrier wait gives up after this many nanoseconds
 *                   (0 = one second); the solve then returns LSLU_ERR_TIMEOUT
 *                   with no completed iteration and the handle stays usable.
 *   stall_first_barrier  testing only: != 0 makes the first barrier wait on
 *                   a word nothing writes, so it runs out after wait_limit_ns
 *                   (which must then be given); use 0 otherwise.
 * Errors: LSLU_ERR_INVALID_ARG (unknown mode, shared-matrix handles, more than
 * 1024 problems, blocks or wait_limit_ns out of range; for the cluster mode a
 * batch or a problem that does not fit), LSLU_ERR_CUDA (no cooperative or
 * cluster launch on the device), LSLU_ERR_OOM.  Drops captured solves. */
enum { LSLU_LOOP_GRAPH = 0, LSLU_LOOP_PERSISTENT = 1, LSLU_LOOP_CLUSTER = 2 };
lslu_status lslu_set_loop(lslu_handle h, int32_t mode, int32_t blocks, int64_t wait_limit_ns,
                          int32_t stall_first_barrier);

/* The loop configuration (host outputs, any may be NULL): mode, blocks of the
 * persistent launch or CTAs of the cluster (0 in graph mode) and the largest
 * co-resident block count of the persistent launch on the handle's device (0
 * where that mode is unavailable). */
lslu_status lslu_loop_config(lslu_handle h, int32_t* mode, int32_t* blocks, int32_t* max_blocks);

/* One-line description of the last failure on h (h may be NULL for a failed
 * lslu_create on this thread).  The string stays valid until the next call. */
const char* lslu_error_string(lslu_handle h);

/* Free everything the handle owns.  NULL is allowed. */
void lslu_destroy(lslu_handle h);

#ifdef __cplusplus
}
#endif

#endif /* LSLU_H */
