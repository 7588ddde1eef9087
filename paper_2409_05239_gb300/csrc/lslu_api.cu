// C ABI of the LSLU library (include/lslu.h): handle management and the
// iteration driver of Hybrid LSLU (Algorithm 5).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lslu_internal.cuh"

using namespace lslu;

namespace {
thread_local std::string g_create_err_store;
}

namespace lslu {
// Last failure of a call that has no handle (lslu_create, allocation-free
// entry points); read by lslu_error_string(NULL).
std::string& thread_error() { return g_create_err_store; }
}  // namespace lslu

namespace {


lslu_status set_err(Ctx* c, lslu_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    lslu::thread_error() = msg;
  return st;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return set_err(c, e_ == cudaErrorMemoryAllocation ? LSLU_ERR_OOM : LSLU_ERR_CUDA, \
                     std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

size_t basis_bytes(int vt) { return vt == LSLU_F64 ? 8 : 4; }

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count ? count * sizeof(T) : 16);
}

void destroy_ctx(lslu_ctx* c) {
  if (!c) return;
  free_csr(&c->A);
  free_csr(&c->AT);
  if (c->proj_tstamp) cudaFree(c->proj_tstamp);
  void* ptrs[] = {c->L, c->D, c->H, c->W, c->gp, c->tp, c->gused, c->tused,
                  c->q, c->u, c->r0, c->xin, c->coef, c->xp, c->part_val, c->part_idx, c->st,
                  c->TLi, c->TDi,
                  c->pw_single, c->pw_batched, c->pw_offsets, c->proj_out, c->y, c->sig,
                  c->cvec, c->xout};
  for (void* p : ptrs) cudaFree(p);
  if (c->st_host) cudaFreeHost(c->st_host);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}


}  // namespace

extern "C" lslu_status lslu_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                   const int32_t* col_idx, const double* vals,
                                   int32_t value_type, int32_t max_iter, int32_t ptr_location,
                                   void* cuda_stream, lslu_handle* out) {
  lslu_ctx* c = nullptr;
  if (!out) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (m < 1 || n < 1 || nnz < 0 || nnz >= (int64_t)INT32_MAX)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "invalid m, n or nnz");
  if (m >= (int64_t)INT32_MAX || n >= (int64_t)INT32_MAX)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "m and n must be below 2^31");
  if (max_iter < 1 || max_iter > kMaxIter)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "max_iter must be in [1, 2048]");
  if (value_type < LSLU_F64 || value_type > LSLU_BF16)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "unknown value_type");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  if (!row_ptr || (nnz > 0 && (!col_idx || !vals)))
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL CSR array");

  // bring the CSR to the host for validation and layout
  std::vector<int64_t> rp(m + 1);
  std::vector<int32_t> ci(nnz);
  std::vector<double> vv(nnz);
  if (ptr_location == LSLU_DEVICE) {
    cudaError_t e = cudaMemcpy(rp.data(), row_ptr, (m + 1) * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nnz)
      e = cudaMemcpy(ci.data(), col_idx, nnz * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nnz) e = cudaMemcpy(vv.data(), vals, nnz * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
      return set_err(nullptr, LSLU_ERR_CUDA, std::string("copying CSR: ") + cudaGetErrorString(e));
  } else {
    std::memcpy(rp.data(), row_ptr, (m + 1) * 8);
    if (nnz) {
      std::memcpy(ci.data(), col_idx, nnz * 4);
      std::memcpy(vv.data(), vals, nnz * 8);
    }
  }
  if (rp[0] != 0 || rp[m] != nnz)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[m] == nnz");
  for (int64_t r = 0; r < m; ++r)
    if (rp[r + 1] < rp[r])
      return set_err(nullptr, LSLU_ERR_INVALID_ARG, "row_ptr is not monotone");
  for (int64_t i = 0; i < nnz; ++i) {
    if (ci[i] < 0 || ci[i] >= n)
      return set_err(nullptr, LSLU_ERR_INVALID_ARG, "column index out of range");
    if (!std::isfinite(vv[i]))
      return set_err(nullptr, LSLU_ERR_INVALID_ARG, "non-finite matrix value");
  }

  c = new lslu_ctx();
  c->m = m;
  c->n = n;
  c->nnz = nnz;
  c->value_type = value_type;
  c->kmax = max_iter;
  c->stream = (cudaStream_t)cuda_stream;
  lslu_status st = LSLU_OK;
  auto fail = [&](lslu_status s2) {
    lslu::thread_error() = c->err;
    destroy_ctx(c);
    return s2;
  };
#define CKC(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      st = e_ == cudaErrorMemoryAllocation ? LSLU_ERR_OOM : LSLU_ERR_CUDA; \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return fail(st);                              \
    }                                               \
  } while (0)
  CKC(cudaGetDevice(&c->device));
  CKC(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  CKC(build_csr_pair(m, n, rp.data(), ci.data(), vv.data(), value_type, &c->A, &c->AT,
                     c->stream));
  const int K = max_iter;
  const size_t bb = basis_bytes(value_type);
  c->ldl = round_up(n, 128);  // whole 128-row tiles of the elimination kernel
  c->ldd = round_up(m, 128);
  c->ldt = K + 1;
  CKC(cudaMalloc(&c->L, (size_t)c->ldl * K * bb));
  CKC(cudaMalloc(&c->D, (size_t)c->ldd * (K + 1) * bb));
  CKC(cudaMemset(c->L, 0, (size_t)c->ldl * K * bb));
  CKC(cudaMemset(c->D, 0, (size_t)c->ldd * (K + 1) * bb));
  CKC(dmalloc(&c->H, (size_t)(K + 1) * K));
  CKC(dmalloc(&c->W, (size_t)K * K));
  CKC(cudaMalloc(&c->TLi, (size_t)(K + 1) * (K + 1) * bb));
  CKC(cudaMalloc(&c->TDi, (size_t)(K + 1) * (K + 1) * bb));
  CKC(dmalloc(&c->gp, K));
  CKC(dmalloc(&c->tp, K + 1));
  CKC(dmalloc(&c->gused, n));
  CKC(dmalloc(&c->tused, m));
  CKC(cudaMalloc(&c->q, n * bb));
  CKC(cudaMalloc(&c->u, m * bb));
  CKC(dmalloc(&c->r0, m));
  CKC(dmalloc(&c->xin, m + n));
  CKC(dmalloc(&c->coef, K + 1));
  CKC(cudaMalloc(&c->xp, (size_t)((K + 8) / 8 + 1) * (K + 1) * bb));
  c->part_cap = c->num_sms * 16;
  CKC(dmalloc(&c->part_val, c->part_cap));
  CKC(dmalloc(&c->part_idx, c->part_cap));
  CKC(dmalloc(&c->st, 1));
  CKC(cudaMallocHost((void**)&c->st_host, sizeof(DevState)));
  std::memset(c->st_host, 0, sizeof(DevState));
  CKC(cudaMemset(c->st, 0, sizeof(DevState)));
  // projected workspace for the single final problem (k <= K); the batched
  // workspace for histories is allocated on first use
  c->pw_cluster = projected_cluster_size();
  // LSLU_NO_GRAPHS=1: launch every kernel directly instead of replaying
  // captured graphs (for kernel-level profilers)
  if (const char* ng = std::getenv("LSLU_NO_GRAPHS")) c->use_graphs = ng[0] == '0';
  if (std::getenv("LSLU_PROJ_TIMING")) {
    CKC(cudaMallocManaged(&c->proj_tstamp, 16 * sizeof(unsigned long long)));
    std::memset(c->proj_tstamp, 0, 16 * sizeof(unsigned long long));
  }
  if (std::getenv("LSLU_VERBOSE"))
    std::fprintf(stderr, "lslu: %d SMs, projected-solve cluster of %d CTAs\n", c->num_sms,
                 c->pw_cluster);
  CKC(dmalloc(&c->pw_single, (size_t)projected_slot_doubles(K, c->pw_cluster)));
  CKC(dmalloc(&c->proj_out, 2 * (size_t)K));
  CKC(dmalloc(&c->y, K));
  CKC(dmalloc(&c->sig, K));
  CKC(dmalloc(&c->cvec, K + 1));
  CKC(dmalloc(&c->xout, n));
  CKC(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  CKC(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  CKC(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  CKC(cudaStreamSynchronize(c->stream));
#undef CKC
  *out = c;
  return LSLU_OK;
}

namespace {

// CUDA-event timing of the sparse products (lslu_profile).  Inside a stream
// capture the events become external event-record nodes of the graph, so a
// profiled solve replays the same graph of kernels.
void ensure_events(Ctx* c, int need) {
  while ((int)c->ev_pool.size() < need) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
}
void record_event(Ctx* c, cudaStream_t s, bool capturing, cudaEvent_t e) {
  if (capturing)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}
void record_spmv_start(Ctx* c, cudaStream_t s, bool capturing, cudaEvent_t* e0) {
  *e0 = nullptr;
  if (!c->profile) return;
  ensure_events(c, c->ev_used + 2);
  *e0 = c->ev_pool[c->ev_used];
  record_event(c, s, capturing, *e0);
}
void record_spmv_end(Ctx* c, cudaStream_t s, bool capturing, cudaEvent_t e0) {
  if (!e0) return;
  record_event(c, s, capturing, c->ev_pool[c->ev_used + 1]);
  c->ev_used += 2;
}
void collect_spmv_times(Ctx* c, int pairs) {
  for (int i = 0; i < pairs; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]) == cudaSuccess) {
      c->prof_ms += ms;
      c->prof_launches += 1;
    }
  }
  cudaGetLastError();
}

// Enqueues one whole solve on stream s (no host synchronisation, capturable):
// state reset, r0 and its pivot, K basis iterations, the projected problems
// and x = x0 + L y.  Inputs are read from the handle's staging buffers.
template <typename BT, typename CT>
int64_t enqueue_solve(Ctx* c, cudaStream_t s, const double* db, const double* dx0, int K,
                      int rule, double lam, bool hist, bool capturing) {
  c->ev_used = 0;
  const int64_t m = c->m, n = c->n;
  const int vt = c->value_type;
  BT* L = (BT*)c->L;
  BT* D = (BT*)c->D;
  CT* q = (CT*)c->q;
  CT* u = (CT*)c->u;
  const int64_t ldh = c->kmax + 1, ldw = c->kmax;
  int64_t launches = 0;

  launch_init_state(c->st, K, s);
  cudaMemsetAsync(c->gused, 0, n, s);
  cudaMemsetAsync(c->tused, 0, m, s);
  cudaMemsetAsync(c->gp, 0xff, sizeof(int32_t) * c->kmax, s);
  cudaMemsetAsync(c->tp, 0xff, sizeof(int32_t) * (c->kmax + 1), s);
  launches += 1;

  // r0 = b - A x0
  if (dx0) {
    launch_spmv<double, double>(c->A, vt, dx0, c->r0, s, c->num_sms);
    launch_residual0(db, c->r0, c->r0, m, s);
    launches += 2;
  } else {
    launch_residual0(db, nullptr, c->r0, m, s);
    launches += 1;
  }
  // beta = signed max-abs entry of r0, d_1 = r0 / beta, t(1)
  {
    PivotArgs pa{c->tp, 0, c->tused, nullptr, c->ldt, LSLU_BREAKDOWN_BETA, 0, 1, c->TDi};
    launch_eliminate_argmax<double, BT, double>(c->r0, D, c->ldd, 0, c->coef, m, c->r0, pa,
                                                c->part_val, c->part_idx, c->part_cap, c->st, s,
                                                c->num_sms);
    launch_scale<double, BT>(c->r0, D, m, c->st, s, c->num_sms);
    launches += 2;
  }
  for (int k = 0; k < K; ++k) {
    // q = A^T d_k (with the coefficients W(0:k, k) from its pivot rows);
    // eliminate l_0..l_{k-1}; pivot; l_k
    cudaEvent_t e0;
    PivotCoef pcw{c->gp, k, L, c->ldl, c->coef, c->W + k * ldw, c->xp, c->TLi, c->ldt, c->st, 0};
    record_spmv_start(c, s, capturing, &e0);
    launch_spmv_pivots<BT, CT>(c->AT, vt, D + (int64_t)k * c->ldd, q, pcw, s);
    record_spmv_end(c, s, capturing, e0);
    PivotArgs paw{c->gp, k, c->gused, c->W + k + k * ldw, c->ldt, LSLU_BREAKDOWN_W, k, 0, c->TLi};
    launch_eliminate_argmax<CT, BT, CT>(q, L, c->ldl, k, c->coef, n, q, paw, c->part_val,
                                        c->part_idx, c->part_cap, c->st, s, c->num_sms);
    launch_scale<CT, BT>(q, L + (int64_t)k * c->ldl, n, c->st, s, c->num_sms);
    // u = A l_k (with H(0:k+1, k)); eliminate d_0..d_k; pivot; d_{k+1}
    PivotCoef pch{c->tp, k + 1, D, c->ldd, c->coef, c->H + k * ldh, c->xp, c->TDi, c->ldt, c->st,
                  0};
    record_spmv_start(c, s, capturing, &e0);
    launch_spmv_pivots<BT, CT>(c->A, vt, L + (int64_t)k * c->ldl, u, pch, s);
    record_spmv_end(c, s, capturing, e0);
    PivotArgs pah{c->tp, k + 1, c->tused, c->H + (k + 1) + k * ldh, c->ldt, LSLU_BREAKDOWN_H, k,
                  0, c->TDi};
    launch_eliminate_argmax<CT, BT, CT>(u, D, c->ldd, k + 1, c->coef, m, u, pah, c->part_val,
                                        c->part_idx, c->part_cap, c->st, s, c->num_sms);
    launch_scale<CT, BT>(u, D + (int64_t)(k + 1) * c->ldd, m, c->st, s, c->num_sms);
    launches += 6;
  }
  // projected problems: every k (histories) or only k = k_done
  ProjArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.H = c->H;
  pa.ldh = ldh;
  pa.beta_ptr = &c->st->beta;
  pa.rule = rule;
  pa.lambda = lam;
  pa.m = m;
  pa.k_first = hist ? 1 : K;
  pa.k_last = K;
  pa.want_y = 1;
  pa.y = c->y;
  pa.lam_out = c->proj_out;
  pa.res_out = c->proj_out + c->kmax;
  pa.st = c->st;
  pa.tstamp = c->proj_tstamp;
  ProjWork w;
  w.cluster = c->pw_cluster;
  if (hist) {
    w.base = c->pw_batched;
    w.offsets = c->pw_offsets;
    w.packed = 1;
  } else {
    w.base = c->pw_single;
    w.packed = 0;
  }
  launch_projected(pa, w, s);
  launch_recombine<BT>(L, c->ldl, c->y, dx0, c->xout, n, c->st, K, s, c->num_sms);
  launches += 2;
  return launches;
}

lslu_status ensure_batched_workspace(Ctx* c) {
  if (c->pw_batched) return LSLU_OK;
  std::vector<int64_t> off(c->kmax + 2, 0);
  for (int kk = 1; kk <= c->kmax; ++kk)
    off[kk + 1] = off[kk] + projected_slot_doubles(kk, c->pw_cluster);
  CK(dmalloc(&c->pw_batched, (size_t)off[c->kmax + 1]));
  CK(dmalloc(&c->pw_offsets, off.size()));
  CK(cudaMemcpy(c->pw_offsets, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
  return LSLU_OK;
}

template <typename BT, typename CT>
lslu_status solve_impl(Ctx* c, const double* db, const double* dx0, int K, int rule, double lam,
                       bool hist) {
  if (hist) {
    lslu_status st = ensure_batched_workspace(c);
    if (st != LSLU_OK) return st;
  }
  cudaStream_t s = c->stream;
  int ev_pairs = 0;
  if (c->profile) ensure_events(c, 4 * K + 8);
  if (!c->use_graphs) {
    c->launches = enqueue_solve<BT, CT>(c, s, db, dx0, K, rule, lam, hist, false);
    ev_pairs = c->ev_used / 2;
    CK(cudaGetLastError());
  } else {
    const int has_x0 = dx0 != nullptr;
    const int prof = c->profile ? 1 : 0;
    Ctx::GraphEntry* ge = nullptr;
    for (auto& g : c->graphs)
      if (g.K == K && g.rule == rule && g.hist == (int)hist && g.has_x0 == has_x0 &&
          g.lam == lam && g.prof == prof)
        ge = &g;
    if (!ge) {
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int64_t nl =
          enqueue_solve<BT, CT>(c, c->cap_stream, db, dx0, K, rule, lam, hist, true);
      const int pairs = c->ev_used / 2;
      cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, LSLU_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      }
      cudaGraphExec_t exec;
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess)
        return set_err(c, LSLU_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      if (c->graphs.size() >= 8) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
      }
      c->graphs.push_back({K, rule, (int)hist, has_x0, lam, exec, nl, prof, pairs});
      ge = &c->graphs.back();
    }
    CK(cudaEventRecord(c->ev_in, s));
    CK(cudaStreamWaitEvent(c->cap_stream, c->ev_in, 0));
    CK(cudaGraphLaunch(ge->exec, c->cap_stream));
    CK(cudaEventRecord(c->ev_out, c->cap_stream));
    CK(cudaStreamWaitEvent(s, c->ev_out, 0));
    c->launches = ge->launches;
    ev_pairs = ge->ev_pairs;
  }
  CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (c->profile) collect_spmv_times(c, ev_pairs);
  if (c->proj_tstamp) {
    const unsigned long long* t = c->proj_tstamp;
    std::fprintf(stderr,
                 "lslu projected k=%d: bidiag %.1f us, sturm grid %.1f us, newton+weights %.1f us, "
                 "lambda %.1f us, lsqr %.1f us, Q %.1f us\n",
                 K, (t[1] - t[0]) * 1e-3, (t[2] - t[1]) * 1e-3, (t[3] - t[2]) * 1e-3,
                 (t[4] - t[3]) * 1e-3, (t[6] - t[5]) * 1e-3, (t[7] - t[6]) * 1e-3);
    std::fprintf(stderr,
                 "  bidiag sections: norms %.1f, cluster syncs %.1f, right house+partials %.1f, "
                 "right update + left house %.1f, left update %.1f us\n",
                 t[8] * 1e-3, t[9] * 1e-3, t[10] * 1e-3, t[11] * 1e-3, t[12] * 1e-3);
  }
  return LSLU_OK;
}

}  // namespace

extern "C" lslu_status lslu_solve(lslu_handle h, const double* b, const double* x0, int32_t K,
                                  int32_t rule, double lambda, int32_t ptr_location,
                                  double* x_out, int32_t* col_pivots, int32_t* row_pivots,
                                  double* lambda_hist, double* resid_hist, int32_t* k_done) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (K < 1 || K > c->kmax) return set_err(c, LSLU_ERR_INVALID_ARG, "K must be in [1, max_iter]");
  if (rule < LSLU_LAMBDA_NONE || rule > LSLU_LAMBDA_WGCV)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown lambda rule");
  if (rule == LSLU_LAMBDA_FIXED && !(lambda >= 0.0 && std::isfinite(lambda)))
    return set_err(c, LSLU_ERR_INVALID_ARG, "fixed lambda must be finite and >= 0");
  if (!b || !x_out) return set_err(c, LSLU_ERR_INVALID_ARG, "b and x_out are required");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  const bool host = ptr_location == LSLU_HOST;
  const int64_t m = c->m, n = c->n;
  cudaStream_t s = c->stream;
  // inputs are staged in the handle's buffers (captured solves read fixed
  // addresses)
  if (host)
    for (int64_t i = 0; i < m; ++i)
      if (!std::isfinite(b[i])) return set_err(c, LSLU_ERR_NONFINITE, "b has a non-finite entry");
  const cudaMemcpyKind h2d = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(c->xin, b, m * 8, h2d, s));
  const double* db = c->xin;
  const double* dx0 = nullptr;
  if (x0) {
    CK(cudaMemcpyAsync(c->xin + m, x0, n * 8, h2d, s));
    dx0 = c->xin + m;
  }
  const bool hist = lambda_hist || resid_hist;
  const double lam = rule == LSLU_LAMBDA_FIXED ? lambda : 0.0;
  lslu_status st = c->value_type == LSLU_F64
                       ? solve_impl<double, double>(c, db, dx0, K, rule, lam, hist)
                       : solve_impl<float, float>(c, db, dx0, K, rule, lam, hist);
  if (st != LSLU_OK) return st;
  const DevState ds = *c->st_host;
  const int kd = ds.k_done < 0 ? 0 : (ds.k_done > K ? K : ds.k_done);
  c->last_k = kd;
  c->last_K = K;
  const cudaMemcpyKind d2o = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(x_out, c->xout, n * 8, d2o, s));
  if (col_pivots) {
    CK(cudaMemcpyAsync(col_pivots, c->gp, (size_t)kd * 4, d2o, s));
    if (K > kd) {
      if (host)
        std::memset(col_pivots + kd, 0xff, (size_t)(K - kd) * 4);
      else
        CK(cudaMemsetAsync(col_pivots + kd, 0xff, (size_t)(K - kd) * 4, s));
    }
  }
  if (row_pivots) {
    const int nt = (ds.status == LSLU_BREAKDOWN_BETA) ? 0 : kd + 1;
    CK(cudaMemcpyAsync(row_pivots, c->tp, (size_t)nt * 4, d2o, s));
    if (K + 1 > nt) {
      if (host)
        std::memset(row_pivots + nt, 0xff, (size_t)(K + 1 - nt) * 4);
      else
        CK(cudaMemsetAsync(row_pivots + nt, 0xff, (size_t)(K + 1 - nt) * 4, s));
    }
  }
  for (int which = 0; which < 2; ++which) {
    double* dst = which == 0 ? lambda_hist : resid_hist;
    if (!dst) continue;
    const double* src = c->proj_out + (which == 0 ? 0 : c->kmax);
    CK(cudaMemcpyAsync(dst, src, (size_t)kd * 8, d2o, s));
    if (K > kd) {
      if (host)
        std::memset(dst + kd, 0, (size_t)(K - kd) * 8);
      else
        CK(cudaMemsetAsync(dst + kd, 0, (size_t)(K - kd) * 8, s));
    }
  }
  if (k_done) {
    if (host)
      *k_done = kd;
    else
      CK(cudaMemcpyAsync(k_done, &c->last_k, 4, cudaMemcpyHostToDevice, s));
  }
  CK(cudaStreamSynchronize(s));
  if (ds.status != LSLU_OK) {
    const char* what = ds.status == LSLU_BREAKDOWN_BETA ? "breakdown: r0 = 0"
                       : ds.status == LSLU_BREAKDOWN_W  ? "breakdown in the W step"
                       : ds.status == LSLU_BREAKDOWN_H  ? "breakdown in the H step"
                                                        : "non-finite pivot";
    return set_err(c, (lslu_status)ds.status, what);
  }
  return LSLU_OK;
}

extern "C" lslu_status lslu_get_state(lslu_handle h, int32_t ptr_location, double* H, double* W,
                                      double* beta, void* L, void* D) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (c->last_k < 0) return set_err(c, LSLU_ERR_INVALID_ARG, "no solve has run");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  const int k = c->last_k;
  const cudaMemcpyKind kind =
      ptr_location == LSLU_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  cudaStream_t s = c->stream;
  const size_t bb = basis_bytes(c->value_type);
  if (H && k > 0)
    CK(cudaMemcpy2DAsync(H, (k + 1) * 8, c->H, (c->kmax + 1) * 8, (k + 1) * 8, k, kind, s));
  if (W && k > 0) CK(cudaMemcpy2DAsync(W, k * 8, c->W, c->kmax * 8, k * 8, k, kind, s));
  if (beta) {
    DevState ds;
    CK(cudaMemcpyAsync(&ds, c->st, sizeof(ds), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ptr_location == LSLU_HOST)
      *beta = ds.beta;
    else
      CK(cudaMemcpyAsync(beta, &c->st->beta, 8, cudaMemcpyDeviceToDevice, s));
  }
  if (L && k > 0)
    CK(cudaMemcpy2DAsync(L, c->n * bb, c->L, c->ldl * bb, c->n * bb, k, kind, s));
  if (D)
    CK(cudaMemcpy2DAsync(D, c->m * bb, c->D, c->ldd * bb, c->m * bb, k + 1, kind, s));
  CK(cudaStreamSynchronize(s));
  return LSLU_OK;
}

extern "C" lslu_status lslu_spmv(lslu_handle h, int32_t transpose, const void* x, void* y) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (!x || !y) return set_err(c, LSLU_ERR_INVALID_ARG, "NULL vector");
  const DevCsr& A = transpose ? c->AT : c->A;
  if (c->value_type == LSLU_F64)
    launch_spmv<double, double>(A, c->value_type, (const double*)x, (double*)y, c->stream,
                                c->num_sms);
  else
    launch_spmv<float, float>(A, c->value_type, (const float*)x, (float*)y, c->stream,
                              c->num_sms);
  CK(cudaGetLastError());
  return LSLU_OK;
}

extern "C" lslu_status lslu_projected(lslu_handle h, int32_t k, const double* H, int32_t ldh,
                                      double beta, int32_t rule, double lambda, int64_t m,
                                      int32_t ptr_location, double* y, double* sigma, double* cv,
                                      double* lambda_out, double* resid_out) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (k < 1 || k > c->kmax || ldh < k + 1 || !H)
    return set_err(c, LSLU_ERR_INVALID_ARG, "invalid k, ldh or H");
  if (rule < LSLU_LAMBDA_NONE || rule > LSLU_LAMBDA_WGCV || m < 1)
    return set_err(c, LSLU_ERR_INVALID_ARG, "invalid rule or m");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  cudaStream_t s = c->stream;
  const double* dH = H;
  double* stage = nullptr;
  if (ptr_location == LSLU_HOST) {
    CK(dmalloc(&stage, (size_t)(k + 1) * k));
    CK(cudaMemcpy2DAsync(stage, (k + 1) * 8, H, (size_t)ldh * 8, (k + 1) * 8, k,
                         cudaMemcpyHostToDevice, s));
    dH = stage;
    ldh = k + 1;
  }
  ProjArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.H = dH;
  pa.ldh = ldh;
  pa.beta_val = beta;
  pa.rule = rule;
  pa.lambda = rule == LSLU_LAMBDA_FIXED ? lambda : 0.0;
  pa.m = m;
  pa.k_first = k;
  pa.k_last = k;
  pa.want_y = 1;
  pa.y = c->y;
  pa.sig = c->sig;
  pa.ldsig = c->kmax;
  pa.cvec = c->cvec;
  pa.ldc = c->kmax + 1;
  pa.lam_out = c->proj_out;
  pa.res_out = c->proj_out + c->kmax;
  ProjWork w;
  w.base = c->pw_single;
  w.cluster = c->pw_cluster;
  CK(launch_projected(pa, w, s));
  const cudaMemcpyKind kind =
      ptr_location == LSLU_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (y) CK(cudaMemcpyAsync(y, c->y, k * 8, kind, s));
  if (sigma) CK(cudaMemcpyAsync(sigma, c->sig, k * 8, kind, s));
  if (cv) CK(cudaMemcpyAsync(cv, c->cvec, (k + 1) * 8, kind, s));
  if (lambda_out) CK(cudaMemcpyAsync(lambda_out, c->proj_out + (k - 1), 8, kind, s));
  if (resid_out) CK(cudaMemcpyAsync(resid_out, c->proj_out + c->kmax + (k - 1), 8, kind, s));
  CK(cudaStreamSynchronize(s));
  if (stage) cudaFree(stage);
  return LSLU_OK;
}

extern "C" lslu_status lslu_profile(lslu_handle h, int32_t enable) {
  if (!h) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  h->profile = enable != 0;
  return LSLU_OK;
}

extern "C" lslu_status lslu_timing(lslu_handle h, int32_t* spmv_launches, double* spmv_ms) {
  if (!h) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (spmv_launches) *spmv_launches = h->prof_launches;
  if (spmv_ms) *spmv_ms = h->prof_ms;
  h->prof_launches = 0;
  h->prof_ms = 0.0;
  return LSLU_OK;
}

extern "C" int64_t lslu_last_launch_count(lslu_handle h) { return h ? h->launches : 0; }

extern "C" const char* lslu_error_string(lslu_handle h) {
  return h ? h->err.c_str() : lslu::thread_error().c_str();
}

extern "C" void lslu_destroy(lslu_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  destroy_ctx(h);
}
