// Internal types of the LSLU library: device CSR, solver state, launchers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lslu.h"

namespace lslu {

// Rows of the internal CSR start on a multiple of kRowAlign entries and are
// padded to that length (pad entries repeat the row's last column with value
// 0), so every row can be read with 16-byte vector loads.
constexpr int kRowAlign = 8;

// Upper bound on max_iter (bounds the projected-problem workspace).
constexpr int kMaxIter = 2048;

struct DevCsr {
  int64_t rows = 0, cols = 0;
  int64_t nnz = 0;         // true non-zeros
  int64_t nnz_padded = 0;  // entries stored, including padding
  int32_t* row_ptr = nullptr;  // rows + 1 (padded offsets, multiples of kRowAlign)
  int32_t* row_len = nullptr;  // rows (padded length, multiple of kRowAlign)
  int32_t* col = nullptr;      // nnz_padded
  void* val = nullptr;         // nnz_padded, type per value type
};

// Device-resident state of one solve.  Written by the pivot kernels.
struct DevState {
  int32_t status;   // lslu_status of the running solve
  int32_t k_done;   // completed iterations when status != OK
  int32_t ticket;   // block counter of the grid-wide argmax reduction
  int32_t ticket2;  // block counter of the pivot-row products
  double beta;      // signed max-abs entry of r0
  double pivot;     // value of the last pivot (FP64 copy)
  float pivot_f;    // same, FP32 copy for the FP32 scale kernel
  float pad1;
  unsigned long long amax;  // running argmax key of the FP32 pivot search
};

// Work space of the projected-problem kernel (global memory): one slot per
// problem; slot of problem size kk at base + offsets[kk] when packed.
struct ProjWork {
  double* base = nullptr;
  const int64_t* offsets = nullptr;  // device table, kmax+2 entries (packed only)
  int packed = 0;
  int cluster = 1;       // CTAs per cluster
  int slab_in_smem = 0;  // set by the launcher
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t m = 0, n = 0, nnz = 0;
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
  int32_t* gp = nullptr;  // kmax
  int32_t* tp = nullptr;  // kmax+1
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
  int part_cap = 0;
  DevState* st = nullptr;
  DevState* st_host = nullptr;  // pinned mirror
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
  // histories, x0) and the stream they are launched on
  struct GraphEntry {
    int K, rule, hist, has_x0;
    double lam;
    cudaGraphExec_t exec;
    int64_t launches;
    int prof;      // 1: event-record nodes around every sparse product
    int ev_pairs;  // number of such event pairs
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool use_graphs = true;
  unsigned long long* proj_tstamp = nullptr;  // LSLU_PROJ_TIMING diagnostics

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
// k_spmv_pivots): cnt pivot rows piv, pivot-row matrix T.
struct PivotCoef {
  const int32_t* piv;
  int cnt;
  const void* B;     // the basis (basis type), leading dimension ldb: T(i,j) = B(piv_i, j)
  int64_t ldb;
  double* coef;      // cnt coefficients (FP64 copy)
  double* hess_col;  // cnt Hessenberg entries of this column (W(:,k) or H(:,k))
  void* xp;          // partial sums, npiv_blocks x ldi (accumulation type)
  void* Tinv;        // column-major inverse of T (basis type = accumulation type), ld ldi
  int64_t ldi;
  DevState* st;
  int npiv_blocks;   // set by the launcher
};
template <typename XT, typename YT>
void launch_spmv_pivots(const DevCsr& A, int vt, const XT* x, YT* y, PivotCoef pc,
                        cudaStream_t s);

// Build the padded CSR of A and of A^T (host-side layout, then upload).
cudaError_t build_csr_pair(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                           const double* vv, int vt, DevCsr* A, DevCsr* AT, cudaStream_t s);
void free_csr(DevCsr* c);

// Basis-step kernels; see lslu_basis.cu.
struct PivotArgs {
  int32_t* piv_list;     // pivot list (gp or tp)
  int piv_slot;          // index written in piv_list (== number of earlier vectors)
  uint8_t* used;         // pivoted-row mask
  double* hess_entry;    // where the pivot value goes (W(k,k) or H(k+1,k)); may be null
  int64_t ldt;           // leading dimension of Tinv
  int breakdown_code;    // status to set when no non-zero candidate is left
  int k_on_breakdown;    // k_done to record on breakdown
  int is_init;           // 1 for the r0 pivot (records beta)
  void* Tinv;            // inverse of T (basis type, row-major): its diagonal entry is set
};

template <typename XT, typename BT, typename CT>
void launch_eliminate_argmax(const XT* x, const BT* B, int64_t ld, int cnt, const double* coef,
                             int64_t rows, CT* v, const PivotArgs& pa, double* part_val,
                             int32_t* part_idx, int part_cap, DevState* st, cudaStream_t s,
                             int num_sms);

template <typename CT, typename BT>
void launch_scale(const CT* v, BT* out, int64_t rows, DevState* st, cudaStream_t s, int num_sms);

void launch_residual0(const double* b, const double* Ax0, double* r0, int64_t m, cudaStream_t s);
void launch_init_state(DevState* st, int K, cudaStream_t s);

// Projected problem (lslu_projected.cu).
struct ProjArgs {
  const double* H;  // ld = ldh
  int64_t ldh;
  double beta_val;          // used when beta_ptr is null
  const double* beta_ptr;   // device beta (from the solve) or null
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
  const DevState* st;  // if non-null, problems with k > k_done are skipped and
                       // the y problem uses k = k_done
  unsigned long long* tstamp;  // optional phase timestamps (ns) of the last problem
};
cudaError_t launch_projected(const ProjArgs& a, ProjWork& w, cudaStream_t s);
int64_t projected_slot_doubles(int kk, int CL);
int projected_cluster_size();

template <typename BT>
void launch_recombine(const BT* L, int64_t ldl, const double* y, const double* x0, double* x,
                      int64_t n, const DevState* st, int K, cudaStream_t s, int num_sms);

}  // namespace lslu

// The opaque handle type of the C ABI is the solver context.
struct lslu_ctx : public lslu::Ctx {};
