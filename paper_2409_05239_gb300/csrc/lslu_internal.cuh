// Internal types of the LSLU library: device CSR, solver state, launchers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lslu.h"

namespace lslu {

// Programmatic dependent launch.  A kernel started with launch_pdl may begin
// while the previous kernel of its stream is still draining (this hides the
// launch latency between the short kernels of the iteration).  Such a kernel
// calls pdl_wait() before it touches anything an earlier kernel wrote or
// reads, and pdl_trigger() only after that, so that its own successor cannot
// start before every kernel ahead of it has completed.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Rows of the internal CSR start on a multiple of kRowAlign entries and are
// padded to that length (pad entries repeat the row's last column with value
// 0), so every row can be read with 16-byte vector loads.
constexpr int kRowAlign = 8;
// Within every full kPermBlock-entry block of a row the entries are stored
// transposed (4 x 16: stored position 4 l + i holds entry 16 i + l), so that
// a 16-lane row group reading one 4-entry chunk per lane gathers 16
// consecutive entries of the row in each step (neighbouring columns share L1
// sectors); the last partial block of a row keeps its order.  A sum over a
// row does not depend on the order, only its rounding does.
constexpr int kPermBlock = 64;

// Upper bound on max_iter (bounds the projected-problem workspace).
constexpr int kMaxIter = 2048;
// Problems one persistent basis loop serves (per-problem tables in shared
// memory).
constexpr int kMaxPersistProblems = 1024;

// Rows of one elimination tile.  Problems solved together (a batch) start on
// multiples of kTile in the concatenated row and column spaces, so every tile
// belongs to exactly one problem.
constexpr int kTile = 128;

// Row shapes of the sparse products (lanes per CSR row x chunks in flight per
// lane); each matrix has one, set at create (the default of its value type)
// or by lslu_tune_spmv / lslu_set_spmv_shape.  Shapes 0-5 read 32-bit column
// indices (chunks of 4 entries), shapes 6-11 the same lane shapes on 16-bit
// offsets (chunks of 8 entries; only for matrices that have them).
// Shapes 12-15 put the 32 lanes of a warp on consecutive entries of one row
// (8 or 4 entries in flight per lane; 32-bit columns and 16-bit offsets).
enum {
  kShapeG16U2 = 0,
  kShapeG32U1 = 1,
  kShapeG16U1 = 2,
  kShapeG8U1 = 3,
  kShapeG8U2 = 4,
  kShapeG4U1 = 5,
  kShapesPerFormat = 6,
  kShapeE8 = 12,
  kShapeE8Cmp = 13,
  kShapeE4 = 14,
  kShapeE4Cmp = 15,
  kNumShapes = 16
};
int default_shape(int vt);
// the shape reads 16-bit column offsets
inline bool shape_cmp(int sh) {
  return (sh >= kShapesPerFormat && sh < kShapeE8) || (sh >= kShapeE8 && (sh & 1));
}

struct DevCsr {
  int shape = kShapeG16U2;
  int compressed = 0;          // 16-bit column offsets available (off, ubase)
  int use_cmp = 0;             // the shape reads them (shape >= kShapesPerFormat)
  uint16_t* off = nullptr;     // nnz_padded: column - first column of its 8-entry unit
  int32_t* ubase = nullptr;    // nnz_padded / 8: first column of every unit
  int64_t rows = 0, cols = 0;
  int64_t nnz = 0;         // true non-zeros
  int64_t nnz_padded = 0;  // entries stored, including padding
  int32_t* row_ptr = nullptr;  // rows + 1 (padded offsets, multiples of kRowAlign)
  int32_t* row_len = nullptr;  // rows (padded length, multiple of kRowAlign)
  int32_t* col = nullptr;      // nnz_padded
  void* val = nullptr;         // nnz_padded, type per value type
};

// Device-resident state of one problem of a solve (one per problem of a
// batch).  Written by the pivot kernels.
struct DevState {
  int32_t status;   // lslu_status of this problem
  int32_t k_done;   // completed iterations when status != OK
  int32_t ticket;   // block counter of the grid-wide argmax reduction (entry 0 only)
  int32_t ticket2;  // block counter of this problem's pivot-row products
  double beta;      // signed max-abs entry of r0
  double pivot;     // value of the last pivot (FP64 copy)
  float pivot_f;    // same, FP32 copy for the FP32 scale kernel
  int32_t amin;     // lowest index attaining the maximum (exact r0 pivot search)
  unsigned long long amax;  // running argmax key of the pivot search
};

// Work space of the projected-problem kernel (global memory): one slot per
// problem; slot of problem size kk at base + offsets[kk] when packed.
struct ProjWork {
  double* base = nullptr;
  const int64_t* offsets = nullptr;  // device table, kmax+2 entries (packed only)
  int packed = 0;
  int cluster = 1;       // CTAs per cluster
  int slab_in_smem = 0;  // set by the launcher
  // set by the launcher for each launch that serves part of the problems:
  int prob0 = 0;  // problem index (k - k_first) of the launch's first problem
  int kcap = 0;   // largest k of a bidiagonalisation launch (sizes its shared
                  // memory; 0: k_last)
  int desc = 0;   // 1: bidiagonalisation clusters take the problems largest k first
  int64_t slot_stride = 0;  // doubles per problem of a batch
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t m = 0, n = 0, nnz = 0;  // padded concatenated sizes (= the problem's for nprob == 1)
  // batch of problems solved together (nprob == 1 for lslu_create)
  int nprob = 1;
  std::vector<int64_t> prob_m, prob_n, row_base, col_base;  // per problem (host)
  int64_t m_user = 0, n_user = 0;      // unpadded totals (the caller's layout)
  int32_t* tile_prob_m = nullptr;      // problem of each kTile rows of the m-space
  int32_t* tile_prob_n = nullptr;      // ... of the n-space
  uint8_t* pad_m = nullptr;            // 1 on padding rows (never pivots)
  uint8_t* pad_n = nullptr;
  int32_t* map_m = nullptr;            // caller row -> padded row
  int32_t* map_n = nullptr;            // caller column -> padded column
  double* xin_pad = nullptr;           // padded staging of b (batch)
  double* xout_user = nullptr;         // x in the caller's layout (batch)
  int64_t* mvec = nullptr;             // rows of every problem (weighted GCV)
  int64_t res_off = 0;                 // offset of the residual outputs in proj_out
  // right-hand sides sharing one matrix (lslu_create_shared): A and A^T are
  // stored once (m1 x n1); problem r's rows start at r * m1_pad, its columns
  // at r * n1_pad
  int shared_rhs = 0;
  int64_t m1 = 0, n1 = 0, m1_pad = 0, n1_pad = 0;
  float* xi = nullptr;                 // interleaved right-hand sides, max(m1, n1) x RS
  int value_type = LSLU_F64;
  int kmax = 0;
  DevCsr A, AT;  // A (m rows) and A^T (n rows)

  // bases, column-major: L is n x kmax with leading dimension ldl; D is
  // m x (kmax+1) with leading dimension ldd; entries of the basis type.
  void* L = nullptr;
  void* D = nullptr;
  int64_t ldl = 0, ldd = 0;
  double* H = nullptr;   // (kmax+1) x kmax, ld = kmax+1
  double* W = nullptr;   // kmax x kmax, ld = kmax
  // inverses of the pivot-row matrices T_L(i,j) = l_j(g_i), T_D(i,j) = d_j(t_i),
  // column-major, basis type, leading dimension ldt = kmax+1
  void* TLi = nullptr;
  void* TDi = nullptr;
  int64_t ldt = 0;
  int32_t* gp = nullptr;  // kmax per problem (padded-space row indices)
  int32_t* tp = nullptr;  // kmax+1 per problem
  int32_t* fixed_gp = nullptr;  // pivots replayed by lslu_solve_fixed_pivots (kmax)
  int32_t* fixed_tp = nullptr;  // (kmax + 1)
  int32_t* samples = nullptr;   // sampled-pivot table, (2 kmax + 1) x samples_cap
  int samples_cap = 0;
  // per-problem strides of the arrays above and below
  int64_t h_stride = 0, w_stride = 0, t_stride = 0, c_stride = 0, xp_stride = 0;
  uint8_t* gused = nullptr;  // n
  uint8_t* tused = nullptr;  // m
  void* q = nullptr;      // n work vector (compute type)
  void* u = nullptr;      // m work vector (compute type)
  double* r0 = nullptr;   // m, FP64
  double* xin = nullptr;  // max(m, n) FP64 staging for host inputs
  double* coef = nullptr; // kmax+1 elimination coefficients (FP64)
  void* xp = nullptr;     // partial coefficient sums: ceil((kmax+1)/8) x ldt
  double* part_val = nullptr;  // argmax partials
  int32_t* part_idx = nullptr;
  double* gstop = nullptr;  // G^(k) of the online stopping rule (max_iter entries)
  int part_cap = 0;
  DevState* st = nullptr;       // nprob entries
  DevState* st_host = nullptr;  // pinned mirror (nprob entries)
  double* pw_single = nullptr;   // projected work space, one problem of size <= kmax
  double* pw_batched = nullptr;  // all problem sizes 1..kmax (histories), on first use
  int64_t* pw_offsets = nullptr; // device offset table of pw_batched
  int pw_cluster = 1;
  double* proj_out = nullptr;  // per problem: lambda, resid (2 doubles)
  double* y = nullptr;         // kmax
  double* sig = nullptr;       // kmax per problem (histories)
  double* cvec = nullptr;      // (kmax+1) per problem
  double* xout = nullptr;      // n, FP64

  // captured solves: one instantiated CUDA graph per (K, rule, lambda,
  // histories, x0, profiling, replayed pivots) and the stream they are launched on
  struct GraphEntry {
    int K, rule, hist, has_x0;
    double lam;
    cudaGraphExec_t exec;
    int64_t launches;
    int prof;      // 1: event-record nodes around every sparse product
    int ev_pairs;  // number of such event pairs
    int fixed;     // 1: pivots replayed from fixed_gp / fixed_tp
    const void* samples;  // sample table of sampled pivoting (null: full search)
    int nsamp;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool use_graphs = true;
  unsigned long long* proj_tstamp = nullptr;  // LSLU_PROJ_TIMING diagnostics

  // reverse-mode work space (lslu_adjoint), allocated on first use
  void* adj_Vb = nullptr;      // adjoints of the L-side eliminated vectors, ldl x kmax
  void* adj_Zb = nullptr;      // adjoints of the D-side eliminated vectors, ldd x kmax
  void* adj_vec = nullptr;     // compute-type vectors: 3 of length ldl, 3 of length ldd
  double* adj_small = nullptr; // FP64 projected adjoint, pivot-row adjoints, scalars
  double* adj_part = nullptr;  // per-block partial sums
  int adj_part_rows = 0;       // blocks of the partial-sum array
  bool adj_valid = false;      // the last lslu_solve completed K iterations and its
                               // state (bases, H, W, y, lambda) is intact

  // renumbered handle (lslu_create_ordered): caller row i is internal row
  // ord_m[i], caller column j internal column ord_n[j]; the matrix, the bases
  // and every pivot search live in the internal numbering, and vectors and
  // pivot indices are mapped at the entry points
  int32_t* ord_m = nullptr;
  int32_t* ord_n = nullptr;
  std::vector<int32_t> ord_m_h, ord_n_h;  // caller -> internal (host)
  std::vector<int32_t> inv_m_h, inv_n_h;  // internal -> caller (host)
  double* ord_stage = nullptr;            // max(m, n) FP64 staging
  // pivot tie-breaking by the caller's index: stored row -> caller index
  // (owned; padding rows of a batch get INT32_MAX) and caller index -> stored
  // row (ord_m / ord_n, or the composed batch maps map_m / map_n)
  int32_t* rank_m = nullptr;
  int32_t* rank_n = nullptr;
  const int32_t* unrank_m = nullptr;
  const int32_t* unrank_n = nullptr;

  // persistent basis loop (lslu_set_loop): one cooperative launch runs the
  // whole basis generation of a solve, with bounded grid barriers
  int loop_mode = 0;            // LSLU_LOOP_GRAPH, _PERSISTENT or _CLUSTER
  int loop_blocks = 0;          // blocks of the persistent launch, CTAs of the cluster
  unsigned long long loop_wait_ns = 1000000000ull;  // limit of one barrier wait
  int loop_stall = 0;           // test only: the first barrier waits on a word nothing writes
  void* pq_v = nullptr;         // n eliminated q (compute type)
  void* pq_w = nullptr;         // m eliminated u
  int64_t* pq_row0 = nullptr;   // first m-space row of every problem (batches)
  int64_t* pq_col0 = nullptr;   // first n-space row of every problem
  unsigned long long* pq_keys = nullptr;  // 2 nprob pivot keys
  double* pq_slot_val = nullptr;          // one partial per block (FP64)
  int32_t* pq_slot_idx = nullptr;
  unsigned* pq_bar = nullptr;   // barrier counter, generation, stall word
  bool pq_no_graph = false;     // the persistent launch could not be captured
  int* pq_err = nullptr;        // 0 or LSLU_ERR_TIMEOUT

  int last_k = -1;  // k_done of the last solve, -1 if none
  int last_K = 0;
  int64_t launches = 0;
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  int ev_used = 0;
  int prof_launches = 0;
  double prof_ms = 0.0;
  std::string err;
  int num_sms = 0;
};

// ---- launchers (defined in the kernel translation units) -------------------

// y = A x for a device CSR; XT input vector type, YT output type; the
// accumulation type is YT.  vt selects the stored value type of the CSR.
template <typename XT, typename YT>
void launch_spmv(const DevCsr& A, int vt, const XT* x, YT* y, cudaStream_t s, int num_sms);

// Elimination coefficients computed inside the sparse product (see
// k_spmv_pivots): cnt pivot rows piv per problem, pivot-row inverse Tinv.
// Problem p's arrays sit at base + p * stride.
struct PivotCoef {
  const int32_t* piv;
  int64_t piv_stride;
  int cnt;
  const void* B;     // the basis (basis type), leading dimension ldb: T(i,j) = B(piv_i, j)
  int64_t ldb;
  double* coef;      // cnt coefficients (FP64 copy)
  int64_t coef_stride;
  double* hess_col;  // cnt Hessenberg entries of this column (W(:,k) or H(:,k))
  int64_t hess_stride;
  void* xp;          // partial sums, npiv_blocks x ldi (accumulation type)
  int64_t xp_stride;
  void* Tinv;        // column-major inverse of T (basis type = accumulation type), ld ldi
  int64_t ldi;
  int64_t tinv_stride;
  DevState* st;
  int nprob;
  int npiv_blocks;   // per problem, set by the launcher
};
template <typename XT, typename YT>
void launch_spmv_pivots(const DevCsr& A, int vt, const XT* x, YT* y, PivotCoef pc,
                        cudaStream_t s);

// Several right-hand sides sharing one matrix (lslu_create_shared): the R
// vectors x[r * xstride + j] are interleaved into xi[j * RS + r] (RS = R rounded
// up to 4, 8 or 16), then one pass over the CSR writes y[r * ystride + row]
// and the elimination coefficients of every right-hand side (as
// launch_spmv_pivots, with problem p's output rows at p * ystride + row).
int rhs_stride(int R);
// Streams `bytes` of buf through L2 (reads only), so that a timed product
// starts with the matrix out of L2 and no dirty lines to write back.
void launch_l2_flush(const void* buf, size_t bytes, int* sink, cudaStream_t s, int num_sms);
void launch_interleave(const float* x, int64_t xstride, int64_t count, int R, float* xi,
                       cudaStream_t s, int num_sms);
void launch_spmm_pivots(const DevCsr& A, int vt, const float* xi, float* y, int64_t ystride,
                        int R, PivotCoef pc, cudaStream_t s);

// Products in a non-default row shape, native vector type only (FP64 for FP64
// values, FP32 otherwise): shapes 0-2 in lslu_spmv_shapes_a.cu, 3-5 in _b.cu.
void launch_spmv_shape_a(int shape, const DevCsr& A, int vt, const void* x, void* y,
                         cudaStream_t s);
void launch_spmv_pivots_shape_a(int shape, const DevCsr& A, int vt, const void* x, void* y,
                                const PivotCoef& pc, cudaStream_t s);
void launch_spmv_shape_b(int shape, const DevCsr& A, int vt, const void* x, void* y,
                         cudaStream_t s);
void launch_spmv_pivots_shape_b(int shape, const DevCsr& A, int vt, const void* x, void* y,
                                const PivotCoef& pc, cudaStream_t s);
void launch_spmv_shape_c(int shape, const DevCsr& A, int vt, const void* x, void* y,
                         cudaStream_t s);
void launch_spmv_pivots_shape_c(int shape, const DevCsr& A, int vt, const void* x, void* y,
                                const PivotCoef& pc, cudaStream_t s);
inline void launch_spmv_shape(int shape, const DevCsr& A, int vt, const void* x, void* y,
                              cudaStream_t s) {
  if (shape >= kShapeE8) {
    launch_spmv_shape_c(shape, A, vt, x, y, s);
    return;
  }
  const int g = shape % kShapesPerFormat;  // the format follows A.use_cmp
  if (g <= kShapeG16U1)
    launch_spmv_shape_a(g, A, vt, x, y, s);
  else
    launch_spmv_shape_b(g, A, vt, x, y, s);
}
inline void launch_spmv_pivots_shape(int shape, const DevCsr& A, int vt, const void* x,
                                     void* y, const PivotCoef& pc, cudaStream_t s) {
  if (shape >= kShapeE8) {
    launch_spmv_pivots_shape_c(shape, A, vt, x, y, pc, s);
    return;
  }
  const int g = shape % kShapesPerFormat;
  if (g <= kShapeG16U1)
    launch_spmv_pivots_shape_a(g, A, vt, x, y, pc, s);
  else
    launch_spmv_pivots_shape_b(g, A, vt, x, y, pc, s);
}

// Build the padded CSR of A and of A^T (host-side layout, then upload).
cudaError_t build_csr_pair(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                           const double* vv, int vt, DevCsr* A, DevCsr* AT, cudaStream_t s);
void free_csr(DevCsr* c);

// Basis-step kernels; see lslu_basis.cu.  Problem p's arrays sit at
// base + p * stride; tile_prob maps every kTile rows to their problem
// (nullptr when nprob == 1).
struct PivotArgs {
  int32_t* piv_list;     // pivot list (gp or tp)
  int64_t piv_stride;
  int piv_slot;          // index written in piv_list (== number of earlier vectors)
  uint8_t* used;         // pivoted-row mask
  double* hess_entry;    // where the pivot value goes (W(k,k) or H(k+1,k)); may be null
  int64_t hess_stride;
  int64_t ldt;           // leading dimension of Tinv
  int breakdown_code;    // status to set when no non-zero candidate is left
  int k_on_breakdown;    // k_done to record on breakdown
  int is_init;           // 1 for the r0 pivot (records beta)
  void* Tinv;            // inverse of T (basis type, column-major): its diagonal entry is set
  int64_t tinv_stride;
  const double* coef;    // elimination coefficients (cnt per problem)
  int64_t coef_stride;
  int nprob;
  const int32_t* tile_prob;
  const int32_t* fixed;  // replayed pivot list (same layout as piv_list), or null: argmax
  const int32_t* samples;  // sampled pivoting (single problem): nsamp candidate rows, or null
  int nsamp;
  // renumbered handles: rank[i] = the caller's index of row i, unrank its
  // inverse; a tie of a pivot search goes to the lowest caller index (both
  // null: the row index itself)
  const int32_t* rank;
  const int32_t* unrank;
};

template <typename XT, typename BT, typename CT>
void launch_eliminate_argmax(const XT* x, const BT* B, int64_t ld, int cnt, int64_t rows, CT* v,
                             const PivotArgs& pa, double* part_val, int32_t* part_idx,
                             int part_cap, DevState* st, cudaStream_t s, int num_sms);

// Exact pivot of r0 for every problem (largest |r0|, lowest index; FP64):
// sets beta, the first row pivot, its mask entry and T_D^-1(0,0).
template <typename BT>
void launch_init_pivot(const double* r0, int64_t rows, const PivotArgs& pa, DevState* st,
                       cudaStream_t s, int num_sms);

template <typename CT, typename BT>
void launch_scale(const CT* v, BT* out, int64_t rows, DevState* st, int nprob,
                  const int32_t* tile_prob, cudaStream_t s, int num_sms);

void launch_residual0(const double* b, const double* Ax0, double* r0, int64_t m, cudaStream_t s);
// G^(k) of Eq. (stop2) for k = 1..K from the projected residuals and traces
// (G may alias tr), and the stopping iteration of Eq. (tol) into *k_stop.
void launch_stop_select(const double* res, const double* tr, double* G, int K, double n,
                        double m, double tol, const DevState* st, int32_t* k_stop,
                        cudaStream_t s);
void launch_init_state(DevState* st, int nprob, int K, cudaStream_t s);
void launch_scatter(const double* src, const int32_t* map, int64_t count, double* dst,
                    cudaStream_t s);
void launch_gather(const double* src, const int32_t* map, int64_t count, double* dst,
                   cudaStream_t s);
// dst(i, j) = src(map[i], j) for i < rows, j < cols (column-major, leading
// dimensions lds and ldd, elements of elem_bytes = 4 or 8 bytes)
void launch_gather_rows(const void* src, int64_t lds, const int32_t* map, int64_t rows,
                        int64_t cols, void* dst, int64_t ldd, int elem_bytes, cudaStream_t s);
// Vectors across the entry points (lslu_api.cu): a caller vector (rows: m
// entries, else n; host or device) into a device vector of the internal
// numbering, and back.  Plain copies on a handle without a renumbering.
cudaError_t vec_in(Ctx* c, bool rows, const double* src, bool host, double* dst);
cudaError_t vec_out(Ctx* c, bool rows, const double* src, bool host, double* dst);

// Projected problem (lslu_projected.cu).
struct ProjArgs {
  const double* H;  // ld = ldh
  int64_t ldh;
  double beta_val;          // used when st is null (otherwise st[p].beta)
  const int64_t* mvec;      // rows of each batch entry (weighted GCV), or null: m
  int nbatch;               // > 1: one final problem per batch entry p (strides below)
  int64_t strideH;          // batch stride of H
  int64_t ldy;              // batch stride of y
  int rule;
  double lambda;
  int64_t m;
  int k_first;   // problems k_first..k_last (one CTA each)
  int k_last;
  int want_y;    // write y for k_last
  double* y;
  double* sig;   // per problem stride ldsig (may be null)
  int64_t ldsig;
  double* cvec;  // per problem stride ldc (may be null)
  int64_t ldc;
  double* lam_out;  // per problem (may be null), index k-1
  double* res_out;  // per problem (may be null), index k-1
  double* tr_out;   // sum_i lam^2/(sigma_i^2+lam^2) per problem (may be null), index k-1
  const DevState* st;  // if non-null (per batch entry), problems with k > k_done
                       // are skipped and the y problem uses k = k_done
  unsigned long long* tstamp;  // optional phase timestamps (ns) of the last problem
};
// nlaunch (may be null) receives the number of kernels launched.
cudaError_t launch_projected(const ProjArgs& a, ProjWork& w, cudaStream_t s,
                             int* nlaunch = nullptr);
int64_t projected_slot_doubles(int kk, int CL);
// Optimal lambda of the last projected problem of size K in slot w (needs
// G = L^T L and g = L^T x_true, k x k and k, FP64): E on the 257-point grid
// into Eg, then the refined minimiser into *lam_out (device).
int optimal_lambda_work_doubles();  // round values of the refinement (Er below)
cudaError_t launch_optimal_lambda(const ProjWork& w, int K, const DevState* st, const double* G,
                                  const double* g, double* Eg, double* Er, double* lam_out,
                                  cudaStream_t s);
// G = L_k^T L_k and g = L_k^T v (v: n FP64 on the device) for the bases of a
// handle (lslu_uq.cu); allocates and frees its own work space.
lslu_status basis_gram_products(struct Ctx* c, int k, const double* v, double* G, double* g);
int projected_cluster_size();

// Persistent basis loop (lslu_persistent.cu): the r0 pivot and K iterations
// of the basis steps of every problem of c in one cooperative launch of
// `blocks` blocks, from r0 (FP64, m; x0 = 0) into the handle's bases, H, W,
// pivot lists and state.  Barrier waits give up after wait_ns (stall != 0:
// the first barrier waits on a word nothing writes, for testing) and the
// problems then end with LSLU_ERR_TIMEOUT.  persistent_max_blocks sets the
// kernel up on the current device and returns its co-resident block count
// (0: the launch cannot be resident); call it before the first launch.
cudaError_t launch_persistent_basis(Ctx* c, const double* r0, int K, int blocks,
                                    unsigned long long wait_ns, int stall, cudaStream_t s);
int persistent_max_blocks(int vt, int K, int nprob, int num_sms);

// Basis loop of one small problem on one thread-block cluster
// (lslu_cluster.cu).  cluster_loop_setup sets the kernels up on the current
// device and returns the cluster size they run with (0: unavailable);
// cluster_loop_fits tells whether an m x n problem with K iterations fits the
// CTAs' shared memory; launch_cluster_basis runs the r0 pivot and K
// iterations (x0 = 0) into the handle's bases, H, W, pivot lists and state.
int cluster_loop_setup(int vt);
bool cluster_loop_fits(int vt, int64_t m, int64_t n, int K, int C);
cudaError_t launch_cluster_basis(Ctx* c, const double* r0, int K, int C, cudaStream_t s);

template <typename BT>
void launch_recombine(const BT* L, int64_t ldl, const double* y, int64_t ldy, const double* x0,
                      double* x, int64_t n, const DevState* st, int nprob,
                      const int32_t* tile_prob, int K, cudaStream_t s, int num_sms);

}  // namespace lslu

// The opaque handle type of the C ABI is the solver context.
struct lslu_ctx : public lslu::Ctx {};
