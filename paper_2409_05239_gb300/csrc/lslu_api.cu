// C ABI of the LSLU library (include/lslu.h): handle management and the
// iteration driver of Hybrid LSLU (Algorithm 5).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <algorithm>
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

cudaError_t vec_in(Ctx* c, bool rows, const double* src, bool host, double* dst) {
  const int64_t len = rows ? c->m : c->n;
  const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (!c->ord_m) return cudaMemcpyAsync(dst, src, len * 8, kind, c->stream);
  cudaError_t e = cudaMemcpyAsync(c->ord_stage, src, len * 8, kind, c->stream);
  if (e != cudaSuccess) return e;
  launch_scatter(c->ord_stage, rows ? c->ord_m : c->ord_n, len, dst, c->stream);
  return cudaGetLastError();
}

cudaError_t vec_out(Ctx* c, bool rows, const double* src, bool host, double* dst) {
  const int64_t len = rows ? c->m : c->n;
  const cudaMemcpyKind kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (!c->ord_m) return cudaMemcpyAsync(dst, src, len * 8, kind, c->stream);
  launch_gather(src, rows ? c->ord_m : c->ord_n, len, c->ord_stage, c->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(dst, c->ord_stage, len * 8, kind, c->stream);
}
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
                  c->q, c->u, c->r0, c->xin, c->coef, c->xp, c->part_val, c->part_idx, c->gstop, c->st,
                  c->TLi, c->TDi,
                  c->pw_single, c->pw_batched, c->pw_offsets, c->proj_out, c->y, c->sig,
                  c->cvec, c->xout, c->tile_prob_m, c->tile_prob_n, c->pad_m, c->pad_n,
                  c->map_m, c->map_n, c->xin_pad, c->xout_user, c->mvec,
                  c->adj_Vb, c->adj_Zb, c->adj_vec, c->adj_small, c->adj_part,
                  c->fixed_gp, c->fixed_tp, c->xi, c->samples, c->ord_m, c->ord_n,
                  c->ord_stage, c->rank_m, c->rank_n, c->pq_v, c->pq_w, c->pq_row0,
                  c->pq_col0, c->pq_keys, c->pq_slot_val, c->pq_slot_idx, c->pq_bar,
                  c->pq_err};
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

namespace {

// Device state of a handle whose padded concatenated CSR (c->m x c->n rows,
// c->nprob problems) is rp/ci/vv; every per-problem array is strided.
lslu_status create_common(lslu_ctx* c, const int64_t* rp, const int32_t* ci, const double* vv,
                          int64_t csr_m = -1, int64_t csr_n = -1) {
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
  const int64_t m = c->m, n = c->n;
  const int P = c->nprob;
  CKC(cudaGetDevice(&c->device));
  CKC(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  CKC(build_csr_pair(csr_m < 0 ? m : csr_m, csr_n < 0 ? n : csr_n, rp, ci, vv, c->value_type,
                     &c->A, &c->AT, c->stream));
  if (c->shared_rhs)
    CKC(dmalloc(&c->xi, (size_t)std::max(c->m1, c->n1) * rhs_stride(c->shared_rhs)));
  const int K = c->kmax;
  const size_t bb = basis_bytes(c->value_type);
  c->ldl = round_up(n, 128);  // whole 128-row tiles of the elimination kernel
  c->ldd = round_up(m, 128);
  c->ldt = K + 1;
  c->h_stride = (int64_t)(K + 1) * K;
  c->w_stride = (int64_t)K * K;
  c->t_stride = (int64_t)(K + 1) * (K + 1);
  c->c_stride = K + 2;
  c->xp_stride = (int64_t)((K + 8) / 8 + 1) * (K + 1);
  CKC(cudaMalloc(&c->L, (size_t)c->ldl * K * bb));
  CKC(cudaMalloc(&c->D, (size_t)c->ldd * (K + 1) * bb));
  CKC(cudaMemset(c->L, 0, (size_t)c->ldl * K * bb));
  CKC(cudaMemset(c->D, 0, (size_t)c->ldd * (K + 1) * bb));
  CKC(dmalloc(&c->H, (size_t)P * c->h_stride));
  CKC(dmalloc(&c->W, (size_t)P * c->w_stride));
  CKC(cudaMalloc(&c->TLi, (size_t)P * c->t_stride * bb));
  CKC(cudaMalloc(&c->TDi, (size_t)P * c->t_stride * bb));
  CKC(dmalloc(&c->gp, (size_t)P * K));
  CKC(dmalloc(&c->tp, (size_t)P * (K + 1)));
  CKC(dmalloc(&c->fixed_gp, (size_t)K));
  CKC(dmalloc(&c->fixed_tp, (size_t)K + 1));
  CKC(dmalloc(&c->gused, n));
  CKC(dmalloc(&c->tused, m));
  CKC(cudaMalloc(&c->q, n * bb));
  CKC(cudaMalloc(&c->u, m * bb));
  CKC(dmalloc(&c->r0, m));
  CKC(dmalloc(&c->xin, m + n));
  CKC(dmalloc(&c->coef, (size_t)P * c->c_stride));
  CKC(cudaMalloc(&c->xp, (size_t)P * c->xp_stride * bb));
  // one FP64 pivot partial per elimination block (one block per 64-row tile)
  c->part_cap = (int)std::max<int64_t>((int64_t)c->num_sms * 16, (std::max(m, n) + 63) / 64 + 1);
  CKC(dmalloc(&c->part_val, c->part_cap));
  CKC(dmalloc(&c->part_idx, c->part_cap));
  CKC(dmalloc(&c->st, P));
  CKC(cudaMallocHost((void**)&c->st_host, sizeof(DevState) * P));
  std::memset(c->st_host, 0, sizeof(DevState) * P);
  CKC(cudaMemset(c->st, 0, sizeof(DevState) * P));
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
  // projected work space: one slot of size K per problem (the histories work
  // space is allocated on first use)
  CKC(dmalloc(&c->pw_single, (size_t)P * projected_slot_doubles(K, c->pw_cluster)));
  c->res_off = K > P ? K : P;
  CKC(dmalloc(&c->proj_out, 3 * (size_t)c->res_off));  // lambda, residual, trace
  CKC(dmalloc(&c->y, (size_t)P * K));
  CKC(dmalloc(&c->sig, K));
  CKC(dmalloc(&c->cvec, K + 1));
  CKC(dmalloc(&c->xout, n));
  CKC(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  CKC(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  CKC(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  CKC(cudaStreamSynchronize(c->stream));
#undef CKC
  return LSLU_OK;
}

}  // namespace

namespace {

// Caller -> internal renumbering of one index space (row or column orders of
// lslu_create_ordered): copied to the host, checked to be a permutation of
// [0, len); inv receives its inverse.  NULL means the identity.
lslu_status read_order(const int32_t* order, int64_t len, bool device, std::vector<int32_t>& fwd,
                       std::vector<int32_t>& inv, const char* what) {
  fwd.resize(len);
  inv.assign(len, -1);
  if (!order) {
    for (int64_t i = 0; i < len; ++i) fwd[i] = inv[i] = (int32_t)i;
    return LSLU_OK;
  }
  if (device) {
    cudaError_t e = cudaMemcpy(fwd.data(), order, len * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
      return set_err(nullptr, LSLU_ERR_CUDA, std::string("copying ") + what + ": " +
                                                 cudaGetErrorString(e));
  } else {
    std::memcpy(fwd.data(), order, len * 4);
  }
  for (int64_t i = 0; i < len; ++i) {
    const int32_t v = fwd[i];
    if (v < 0 || v >= len || inv[v] >= 0)
      return set_err(nullptr, LSLU_ERR_INVALID_ARG, std::string(what) + " is not a permutation");
    inv[v] = (int32_t)i;
  }
  return LSLU_OK;
}

// A host CSR renumbered: stored row r holds caller row inv_row[r], with its
// columns mapped through col_new and sorted ascending (stable for repeats).
void renumber_csr(int64_t rows, const int64_t* rp, const int32_t* ci, const double* vv,
                  const std::vector<int32_t>& inv_row, const std::vector<int32_t>& col_new,
                  std::vector<int64_t>& rp_o, std::vector<int32_t>& ci_o,
                  std::vector<double>& vv_o) {
  rp_o.assign(rows + 1, 0);
  for (int64_t r = 0; r < rows; ++r)
    rp_o[r + 1] = rp_o[r] + (rp[inv_row[r] + 1] - rp[inv_row[r]]);
  ci_o.resize(rp_o[rows]);
  vv_o.resize(rp_o[rows]);
  std::vector<uint64_t> key;
  for (int64_t r = 0; r < rows; ++r) {
    const int64_t a = rp[inv_row[r]], len = rp[inv_row[r] + 1] - a, o = rp_o[r];
    key.resize(len);
    for (int64_t i = 0; i < len; ++i)
      key[i] = ((uint64_t)(uint32_t)col_new[ci[a + i]] << 32) | (uint64_t)i;
    std::sort(key.begin(), key.end());
    for (int64_t i = 0; i < len; ++i) {
      ci_o[o + i] = (int32_t)(key[i] >> 32);
      vv_o[o + i] = vv[a + (int64_t)(key[i] & 0xffffffffull)];
    }
  }
}

lslu_status create_single(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                          const int32_t* col_idx, const double* vals, int32_t value_type,
                          int32_t max_iter, const int32_t* row_order, const int32_t* col_order,
                          int32_t ptr_location, void* cuda_stream, lslu_handle* out) {
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
  const bool ordered = row_order || col_order;
  std::vector<int32_t> om, on, im, in;
  if (ordered) {
    lslu_status st = read_order(row_order, m, ptr_location == LSLU_DEVICE, om, im, "row_order");
    if (st == LSLU_OK)
      st = read_order(col_order, n, ptr_location == LSLU_DEVICE, on, in, "col_order");
    if (st != LSLU_OK) return st;
    std::vector<int64_t> rp2;
    std::vector<int32_t> ci2;
    std::vector<double> vv2;
    renumber_csr(m, rp.data(), ci.data(), vv.data(), im, on, rp2, ci2, vv2);
    rp.swap(rp2);
    ci.swap(ci2);
    vv.swap(vv2);
  }

  c = new lslu_ctx();
  c->nprob = 1;
  c->m = m;
  c->n = n;
  c->m_user = m;
  c->n_user = n;
  c->prob_m = {m};
  c->prob_n = {n};
  c->row_base = {0};
  c->col_base = {0};
  c->nnz = nnz;
  c->value_type = value_type;
  c->kmax = max_iter;
  c->stream = (cudaStream_t)cuda_stream;
  lslu_status st = create_common(c, rp.data(), ci.data(), vv.data());
  if (st != LSLU_OK) return st;
  if (ordered) {
    cudaError_t e = dmalloc(&c->ord_m, m);
    if (e == cudaSuccess) e = dmalloc(&c->ord_n, n);
    if (e == cudaSuccess) e = dmalloc(&c->rank_m, m);
    if (e == cudaSuccess) e = dmalloc(&c->rank_n, n);
    if (e == cudaSuccess) e = dmalloc(&c->ord_stage, std::max(m, n));
    if (e == cudaSuccess) e = cudaMemcpy(c->ord_m, om.data(), m * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->ord_n, on.data(), n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->rank_m, im.data(), m * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->rank_n, in.data(), n * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      destroy_ctx(c);
      return set_err(nullptr, e == cudaErrorMemoryAllocation ? LSLU_ERR_OOM : LSLU_ERR_CUDA,
                     std::string("renumbering maps: ") + cudaGetErrorString(e));
    }
    c->unrank_m = c->ord_m;
    c->unrank_n = c->ord_n;
    c->ord_m_h.swap(om);
    c->ord_n_h.swap(on);
    c->inv_m_h.swap(im);
    c->inv_n_h.swap(in);
  }
  *out = c;
  return LSLU_OK;
}

}  // namespace

extern "C" lslu_status lslu_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                   const int32_t* col_idx, const double* vals,
                                   int32_t value_type, int32_t max_iter, int32_t ptr_location,
                                   void* cuda_stream, lslu_handle* out) {
  return create_single(m, n, nnz, row_ptr, col_idx, vals, value_type, max_iter, nullptr, nullptr,
                       ptr_location, cuda_stream, out);
}

extern "C" lslu_status lslu_create_ordered(int64_t m, int64_t n, int64_t nnz,
                                           const int64_t* row_ptr, const int32_t* col_idx,
                                           const double* vals, int32_t value_type,
                                           int32_t max_iter, const int32_t* row_order,
                                           const int32_t* col_order, int32_t ptr_location,
                                           void* cuda_stream, lslu_handle* out) {
  return create_single(m, n, nnz, row_ptr, col_idx, vals, value_type, max_iter, row_order,
                       col_order, ptr_location, cuda_stream, out);
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
// A part of it (graph loop mode only): iterations k_begin .. k_end-1, with the
// reset and r0 when k_begin == 0 and the projected problems and x when finish.
template <typename BT, typename CT>
int64_t enqueue_solve(Ctx* c, cudaStream_t s, const double* db, const double* dx0, int K,
                      int rule, double lam, bool hist, bool capturing, bool fixed, int nsamp,
                      int k_begin = 0, int k_end = -1, bool finish = true) {
  if (k_end < 0) k_end = K;
  // sampled pivoting: pick t uses row t of the sample table (t = 0 for r0,
  // 2k+1 for q and 2k+2 for u at iteration k)
  auto samp = [&](int t) -> const int32_t* {
    return nsamp > 0 ? c->samples + (int64_t)t * nsamp : nullptr;
  };
  c->ev_used = 0;
  const int64_t m = c->m, n = c->n;
  const int vt = c->value_type;
  const int P = c->nprob;
  const int32_t* tpm = c->tile_prob_m;  // nullptr for a single problem
  const int32_t* tpn = c->tile_prob_n;
  BT* L = (BT*)c->L;
  BT* D = (BT*)c->D;
  CT* q = (CT*)c->q;
  CT* u = (CT*)c->u;
  const int64_t ldh = c->kmax + 1, ldw = c->kmax;
  int64_t launches = 0;

  if (k_begin == 0) {
  launch_init_state(c->st, P, K, s);
  if (P == 1) {
    cudaMemsetAsync(c->gused, 0, n, s);
    cudaMemsetAsync(c->tused, 0, m, s);
  } else {  // padding rows and columns are never pivots
    cudaMemcpyAsync(c->gused, c->pad_n, n, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->tused, c->pad_m, m, cudaMemcpyDeviceToDevice, s);
  }
  cudaMemsetAsync(c->gp, 0xff, sizeof(int32_t) * P * c->kmax, s);
  cudaMemsetAsync(c->tp, 0xff, sizeof(int32_t) * P * (c->kmax + 1), s);
  launches += 1;
  }

  if (c->loop_mode == LSLU_LOOP_CLUSTER) {
    // r0 = b (x0 = 0), then the whole basis loop on one thread-block cluster
    launch_residual0(db, nullptr, c->r0, m, s);
    launch_cluster_basis(c, c->r0, K, c->loop_blocks, s);
    launches += 2;
  } else if (c->loop_mode == LSLU_LOOP_PERSISTENT) {
    // r0 = b (x0 = 0), then the whole basis loop in one cooperative launch
    launch_residual0(db, nullptr, c->r0, m, s);
    cudaMemsetAsync(c->pq_bar, 0, 3 * sizeof(unsigned), s);
    cudaMemsetAsync(c->pq_err, 0, sizeof(int), s);
    launch_persistent_basis(c, c->r0, K, c->loop_blocks, c->loop_wait_ns, c->loop_stall, s);
    launches += 2;
  } else {
  if (k_begin == 0) {
  // r0 = b - A x0
  if (dx0) {
    launch_spmv<double, double>(c->A, vt, dx0, c->r0, s, c->num_sms);
    launch_residual0(db, c->r0, c->r0, m, s);
    launches += 2;
  } else {
    launch_residual0(db, nullptr, c->r0, m, s);
    launches += 1;
  }
  // beta = signed max-abs entry of r0 (exact, FP64), d_1 = r0 / beta, t(1)
  {
    PivotArgs pa{c->tp, c->kmax + 1, 0, c->tused, nullptr, 0, c->ldt, LSLU_BREAKDOWN_BETA,
                 0, 1, c->TDi, c->t_stride, c->coef, c->c_stride, P, tpm,
                 fixed ? c->fixed_tp : nullptr, samp(0), nsamp, c->rank_m, c->unrank_m};
    launch_init_pivot<BT>(c->r0, m, pa, c->st, s, c->num_sms);
    launch_scale<double, BT>(c->r0, D, m, c->st, P, tpm, s, c->num_sms);
    launches += 3;
  }
  }
  for (int k = k_begin; k < k_end; ++k) {
    // q = A^T d_k (with the coefficients W(0:k, k) from its pivot rows);
    // eliminate l_0..l_{k-1}; pivot; l_k
    cudaEvent_t e0;
    PivotCoef pcw{c->gp,       c->kmax,       k,        L,          c->ldl,
                  c->coef,     c->c_stride,   c->W + k * ldw,       c->w_stride,
                  c->xp,       c->xp_stride,  c->TLi,   c->ldt,     c->t_stride,
                  c->st,       P,             0};
    record_spmv_start(c, s, capturing, &e0);
    if constexpr (std::is_same<BT, float>::value) {
      if (c->shared_rhs) {
        launch_interleave(D + (int64_t)k * c->ldd, c->m1_pad, c->m1, c->shared_rhs, c->xi, s,
                          c->num_sms);
        launch_spmm_pivots(c->AT, vt, c->xi, q, c->n1_pad, c->shared_rhs, pcw, s);
        launches += 1;
      } else {
        launch_spmv_pivots<BT, CT>(c->AT, vt, D + (int64_t)k * c->ldd, q, pcw, s);
      }
    } else {
      launch_spmv_pivots<BT, CT>(c->AT, vt, D + (int64_t)k * c->ldd, q, pcw, s);
    }
    record_spmv_end(c, s, capturing, e0);
    PivotArgs paw{c->gp, c->kmax, k, c->gused, c->W + k + k * ldw, c->w_stride, c->ldt,
                  LSLU_BREAKDOWN_W, k, 0, c->TLi, c->t_stride, c->coef, c->c_stride, P, tpn,
                  fixed ? c->fixed_gp : nullptr, samp(2 * k + 1), nsamp, c->rank_n,
                  c->unrank_n};
    launch_eliminate_argmax<CT, BT, CT>(q, L, c->ldl, k, n, q, paw, c->part_val, c->part_idx,
                                        c->part_cap, c->st, s, c->num_sms);
    launch_scale<CT, BT>(q, L + (int64_t)k * c->ldl, n, c->st, P, tpn, s, c->num_sms);
    // u = A l_k (with H(0:k+1, k)); eliminate d_0..d_k; pivot; d_{k+1}
    PivotCoef pch{c->tp,       c->kmax + 1,   k + 1,    D,          c->ldd,
                  c->coef,     c->c_stride,   c->H + k * ldh,       c->h_stride,
                  c->xp,       c->xp_stride,  c->TDi,   c->ldt,     c->t_stride,
                  c->st,       P,             0};
    record_spmv_start(c, s, capturing, &e0);
    if constexpr (std::is_same<BT, float>::value) {
      if (c->shared_rhs) {
        launch_interleave(L + (int64_t)k * c->ldl, c->n1_pad, c->n1, c->shared_rhs, c->xi, s,
                          c->num_sms);
        launch_spmm_pivots(c->A, vt, c->xi, u, c->m1_pad, c->shared_rhs, pch, s);
        launches += 1;
      } else {
        launch_spmv_pivots<BT, CT>(c->A, vt, L + (int64_t)k * c->ldl, u, pch, s);
      }
    } else {
      launch_spmv_pivots<BT, CT>(c->A, vt, L + (int64_t)k * c->ldl, u, pch, s);
    }
    record_spmv_end(c, s, capturing, e0);
    PivotArgs pah{c->tp, c->kmax + 1, k + 1, c->tused, c->H + (k + 1) + k * ldh, c->h_stride,
                  c->ldt, LSLU_BREAKDOWN_H, k, 0, c->TDi, c->t_stride, c->coef, c->c_stride, P,
                  tpm, fixed ? c->fixed_tp : nullptr, samp(2 * k + 2), nsamp, c->rank_m,
                  c->unrank_m};
    launch_eliminate_argmax<CT, BT, CT>(u, D, c->ldd, k + 1, m, u, pah, c->part_val,
                                        c->part_idx, c->part_cap, c->st, s, c->num_sms);
    launch_scale<CT, BT>(u, D + (int64_t)(k + 1) * c->ldd, m, c->st, P, tpm, s, c->num_sms);
    launches += 6;
  }
  }  // graph-mode basis loop
  if (!finish) return launches;
  // projected problems: every k (histories) or only k = k_done of each problem
  ProjArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.H = c->H;
  pa.ldh = ldh;
  pa.rule = rule;
  pa.lambda = lam;
  pa.m = c->prob_m[0];
  pa.mvec = P > 1 ? c->mvec : nullptr;
  pa.k_first = hist ? 1 : K;
  pa.k_last = K;
  pa.want_y = 1;
  pa.y = c->y;
  pa.ldy = c->kmax;
  pa.nbatch = P;
  pa.strideH = c->h_stride;
  pa.lam_out = c->proj_out;
  pa.res_out = c->proj_out + c->res_off;
  pa.tr_out = hist ? c->proj_out + 2 * c->res_off : nullptr;
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
    w.slot_stride = projected_slot_doubles(c->kmax, c->pw_cluster);
  }
  int nproj = 0;
  launch_projected(pa, w, s, &nproj);
  launch_recombine<BT>(L, c->ldl, c->y, c->kmax, dx0, c->xout, n, c->st, P, tpn, K, s,
                       c->num_sms);
  launches += nproj + 1;
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
                       bool hist, bool fixed = false, int nsamp = 0) {
  if (hist) {
    lslu_status st = ensure_batched_workspace(c);
    if (st != LSLU_OK) return st;
  }
  cudaStream_t s = c->stream;
  int ev_pairs = 0;
  if (c->profile) ensure_events(c, 4 * K + 8);
  if (!c->use_graphs || (c->loop_mode == LSLU_LOOP_PERSISTENT && c->pq_no_graph)) {
    c->launches = enqueue_solve<BT, CT>(c, s, db, dx0, K, rule, lam, hist, false, fixed, nsamp);
    ev_pairs = c->ev_used / 2;
    CK(cudaGetLastError());
  } else {
    const int has_x0 = dx0 != nullptr;
    const int prof = c->profile ? 1 : 0;
    Ctx::GraphEntry* ge = nullptr;
    for (auto& g : c->graphs)
      if (g.K == K && g.rule == rule && g.hist == (int)hist && g.has_x0 == has_x0 &&
          g.lam == lam && g.prof == prof && g.fixed == (int)fixed && g.nsamp == nsamp &&
          g.samples == (nsamp ? (const void*)c->samples : nullptr))
        ge = &g;
    if (!ge) {
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int64_t nl =
          enqueue_solve<BT, CT>(c, c->cap_stream, db, dx0, K, rule, lam, hist, true, fixed, nsamp);
      const int pairs = c->ev_used / 2;
      cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
      cudaGraphExec_t exec = nullptr;
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
      }
      if (e != cudaSuccess && c->loop_mode == LSLU_LOOP_PERSISTENT) {
        // the cooperative launch was not captured: launch this mode directly
        cudaGetLastError();
        c->pq_no_graph = true;
        return solve_impl<BT, CT>(c, db, dx0, K, rule, lam, hist, fixed, nsamp);
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, LSLU_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      }
      if (c->graphs.size() >= 8) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
      }
      c->graphs.push_back({K, rule, (int)hist, has_x0, lam, exec, nl, prof, pairs, (int)fixed,
                           nsamp ? (const void*)c->samples : nullptr, nsamp});
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
  CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevState) * c->nprob, cudaMemcpyDeviceToHost,
                     s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (c->profile) collect_spmv_times(c, ev_pairs);
  if (c->proj_tstamp) {
    const unsigned long long* t = c->proj_tstamp;
    std::fprintf(stderr,
                 "lslu projected k=%d: bidiag %.1f us, singular values + GCV grid %.1f us "
                 "(with launch gaps), lambda %.1f us, lsqr %.1f us, Q %.1f us\n",
                 K, (t[1] - t[0]) * 1e-3, (t[3] - t[1]) * 1e-3, (t[4] - t[3]) * 1e-3,
                 (t[6] - t[5]) * 1e-3, (t[7] - t[6]) * 1e-3);
    std::fprintf(stderr,
                 "  bidiag sections: partial products %.1f, cluster barrier %.1f, "
                 "exchange + reflectors %.1f, column updates %.1f us\n",
                 t[8] * 1e-3, t[9] * 1e-3, t[10] * 1e-3, t[11] * 1e-3);
    std::fprintf(stderr, "  singular values: multisection rounds max %llu, mean %.2f\n", t[13],
                 K > 0 ? (double)t[14] / K : 0.0);
    std::memset(c->proj_tstamp, 0, 16 * sizeof(unsigned long long));
  }
  return LSLU_OK;
}

}  // namespace

namespace {

// lslu_solve, and lslu_solve_fixed_pivots when fix_g / fix_t are given
lslu_status solve_entry(Ctx* c, const double* b, const double* x0, int32_t K, int32_t rule,
                        double lambda, int32_t ptr_location, double* x_out, int32_t* col_pivots,
                        int32_t* row_pivots, double* lambda_hist, double* resid_hist,
                        int32_t* k_done, const int32_t* fix_g, const int32_t* fix_t,
                        const int32_t* samples = nullptr, int32_t nsamp = 0) {
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (c->map_m) return set_err(c, LSLU_ERR_INVALID_ARG, "batched handle: use lslu_solve_batched");
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
  CK(vec_in(c, true, b, host, c->xin));
  const double* db = c->xin;
  const double* dx0 = nullptr;
  if (x0) {
    CK(vec_in(c, false, x0, host, c->xin + m));
    dx0 = c->xin + m;
  }
  const bool ord = c->ord_m != nullptr;
  const bool fixed = fix_g != nullptr;
  if (c->loop_mode != LSLU_LOOP_GRAPH && (x0 || fixed || nsamp > 0))
    return set_err(c, LSLU_ERR_INVALID_ARG,
                   "the persistent and cluster basis loops serve x0 = 0 with searched pivots; "
                   "lslu_set_loop(h, LSLU_LOOP_GRAPH, ...) for x0, replayed or sampled pivots");
  if (fixed) {  // replayed pivots: validate on the host (indices in range, distinct)
    std::vector<int32_t> g(K), t(K + 1);
    if (host) {
      std::memcpy(g.data(), fix_g, (size_t)K * 4);
      std::memcpy(t.data(), fix_t, (size_t)(K + 1) * 4);
    } else {
      CK(cudaMemcpy(g.data(), fix_g, (size_t)K * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(t.data(), fix_t, (size_t)(K + 1) * 4, cudaMemcpyDeviceToHost));
    }
    std::vector<uint8_t> seen_n(n, 0), seen_m(m, 0);
    for (int i = 0; i < K; ++i) {
      if (g[i] < 0 || g[i] >= n || seen_n[g[i]])
        return set_err(c, LSLU_ERR_INVALID_ARG, "col_pivots must be distinct indices in [0, n)");
      seen_n[g[i]] = 1;
    }
    for (int i = 0; i <= K; ++i) {
      if (t[i] < 0 || t[i] >= m || seen_m[t[i]])
        return set_err(c, LSLU_ERR_INVALID_ARG, "row_pivots must be distinct indices in [0, m)");
      seen_m[t[i]] = 1;
    }
    if (ord) {  // to the internal numbering
      for (int i = 0; i < K; ++i) g[i] = c->ord_n_h[g[i]];
      for (int i = 0; i <= K; ++i) t[i] = c->ord_m_h[t[i]];
    }
    CK(cudaMemcpyAsync(c->fixed_gp, g.data(), (size_t)K * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->fixed_tp, t.data(), (size_t)(K + 1) * 4, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // the host vectors go out of scope
  }
  if (nsamp > 0) {  // sample table: validate on the host, stage on the device
    const int64_t rows = 2LL * K + 1;
    std::vector<int32_t> t((size_t)(rows * nsamp));
    if (host)
      std::memcpy(t.data(), samples, t.size() * 4);
    else
      CK(cudaMemcpy(t.data(), samples, t.size() * 4, cudaMemcpyDeviceToHost));
    for (int64_t r = 0; r < rows; ++r) {
      const int64_t lim = (r % 2 == 0) ? m : n;
      for (int j = 0; j < nsamp; ++j) {
        const int32_t v = t[(size_t)(r * nsamp + j)];
        if (v < 0 || v >= lim)
          return set_err(c, LSLU_ERR_INVALID_ARG,
                         "sample indices must lie in [0, m) for even rows, [0, n) for odd rows");
        if (ord) t[(size_t)(r * nsamp + j)] = (r % 2 == 0) ? c->ord_m_h[v] : c->ord_n_h[v];
      }
    }
    if ((int64_t)(2LL * c->kmax + 1) * nsamp > (int64_t)c->samples_cap) {
      if (c->samples) cudaFree(c->samples);
      c->samples = nullptr;
      c->samples_cap = 0;
      const int64_t cap = (2LL * c->kmax + 1) * nsamp;
      CK(cudaMalloc(&c->samples, (size_t)cap * 4));
      c->samples_cap = (int)cap;
    }
    CK(cudaMemcpyAsync(c->samples, t.data(), t.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // the host table goes out of scope
  }
  const bool hist = lambda_hist || resid_hist;
  const double lam = rule == LSLU_LAMBDA_FIXED ? lambda : 0.0;
  lslu_status st =
      c->value_type == LSLU_F64
          ? solve_impl<double, double>(c, db, dx0, K, rule, lam, hist, fixed, nsamp)
          : solve_impl<float, float>(c, db, dx0, K, rule, lam, hist, fixed, nsamp);
  if (st != LSLU_OK) return st;
  const DevState ds = *c->st_host;
  const int kd = ds.k_done < 0 ? 0 : (ds.k_done > K ? K : ds.k_done);
  c->last_k = kd;
  c->last_K = K;
  c->adj_valid = ds.status == LSLU_OK && kd == K;
  const cudaMemcpyKind d2o = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(vec_out(c, false, c->xout, host, x_out));
  // pivot indices of a renumbered handle go back to the caller's numbering
  auto pivots_out = [&](int32_t* dst, const int32_t* src, int cnt,
                        const std::vector<int32_t>& inv) -> cudaError_t {
    if (!ord || cnt <= 0) return cudaMemcpyAsync(dst, src, (size_t)cnt * 4, d2o, s);
    std::vector<int32_t> v(cnt);
    cudaError_t e = cudaMemcpyAsync(v.data(), src, (size_t)cnt * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (int32_t& x : v) x = (x >= 0 && x < (int32_t)inv.size()) ? inv[x] : -1;
    e = cudaMemcpyAsync(dst, v.data(), (size_t)cnt * 4,
                        host ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
  };
  if (col_pivots) {
    CK(pivots_out(col_pivots, c->gp, kd, c->inv_n_h));
    if (K > kd) {
      if (host)
        std::memset(col_pivots + kd, 0xff, (size_t)(K - kd) * 4);
      else
        CK(cudaMemsetAsync(col_pivots + kd, 0xff, (size_t)(K - kd) * 4, s));
    }
  }
  if (row_pivots) {
    const int nt = (ds.status == LSLU_BREAKDOWN_BETA) ? 0 : kd + 1;
    CK(pivots_out(row_pivots, c->tp, nt, c->inv_m_h));
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
    const double* src = c->proj_out + (which == 0 ? 0 : c->res_off);
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
                       : ds.status == LSLU_ERR_TIMEOUT
                           ? "a grid barrier of the persistent basis loop timed out"
                           : "non-finite pivot";
    return set_err(c, (lslu_status)ds.status, what);
  }
  return LSLU_OK;
}


}  // namespace

extern "C" lslu_status lslu_solve(lslu_handle h, const double* b, const double* x0, int32_t K,
                                  int32_t rule, double lambda, int32_t ptr_location,
                                  double* x_out, int32_t* col_pivots, int32_t* row_pivots,
                                  double* lambda_hist, double* resid_hist, int32_t* k_done) {
  return solve_entry(h, b, x0, K, rule, lambda, ptr_location, x_out, col_pivots, row_pivots,
                     lambda_hist, resid_hist, k_done, nullptr, nullptr);
}

extern "C" lslu_status lslu_solve_sampled(lslu_handle h, const double* b, const double* x0,
                                          int32_t K, int32_t rule, double lambda,
                                          const int32_t* samples, int32_t nsamp,
                                          int32_t ptr_location, double* x_out,
                                          int32_t* col_pivots, int32_t* row_pivots,
                                          int32_t* k_done) {
  if (h && (!samples || nsamp < 1 || nsamp > 65536))
    return set_err(h, LSLU_ERR_INVALID_ARG, "samples required, 1 <= nsamp <= 65536");
  return solve_entry(h, b, x0, K, rule, lambda, ptr_location, x_out, col_pivots, row_pivots,
                     nullptr, nullptr, k_done, nullptr, nullptr, samples, nsamp);
}

extern "C" lslu_status lslu_solve_fixed_pivots(lslu_handle h, const double* b, const double* x0,
                                               int32_t K, int32_t rule, double lambda,
                                               int32_t ptr_location, const int32_t* col_pivots,
                                               const int32_t* row_pivots, double* x_out,
                                               int32_t* k_done) {
  if (h && (!col_pivots || !row_pivots))
    return set_err(h, LSLU_ERR_INVALID_ARG, "col_pivots and row_pivots are required");
  return solve_entry(h, b, x0, K, rule, lambda, ptr_location, x_out, nullptr, nullptr, nullptr,
                     nullptr, k_done, col_pivots, row_pivots);
}

namespace {

// Device copies of a batch layout (tile -> problem maps, padding masks,
// caller <-> padded index maps, rows per problem) and the staging buffers.
lslu_status upload_batch_layout(lslu_ctx* c, const std::vector<int32_t>& tpm,
                                const std::vector<int32_t>& tpn,
                                const std::vector<uint8_t>& pad_m,
                                const std::vector<uint8_t>& pad_n,
                                const std::vector<int32_t>& map_m,
                                const std::vector<int32_t>& map_n,
                                const std::vector<int64_t>& mvec) {
  auto up = [&](auto** dst, const auto& v) -> bool {
    using T = typename std::decay<decltype(v[0])>::type;
    if (cudaMalloc((void**)dst, std::max<size_t>(v.size(), 1) * sizeof(T)) != cudaSuccess)
      return false;
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) ==
           cudaSuccess;
  };
  if (!up(&c->tile_prob_m, tpm) || !up(&c->tile_prob_n, tpn) || !up(&c->pad_m, pad_m) ||
      !up(&c->pad_n, pad_n) || !up(&c->map_m, map_m) || !up(&c->map_n, map_n) ||
      !up(&c->mvec, mvec) || cudaMalloc(&c->xin_pad, c->m * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->xout_user, c->n_user * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    lslu::thread_error() = "allocating the batch layout failed";
    destroy_ctx(c);
    return LSLU_ERR_OOM;
  }
  return LSLU_OK;
}

}  // namespace

namespace {

lslu_status create_batched_impl(int32_t nprob, const int64_t* row_off, const int64_t* col_off,
                                const int64_t* row_ptr, const int32_t* col_idx,
                                const double* vals, int32_t value_type, int32_t max_iter,
                                const int32_t* row_order, const int32_t* col_order,
                                void* cuda_stream, lslu_handle* out) {
  if (!out) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nprob < 1 || !row_off || !col_off || !row_ptr)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "invalid nprob or NULL offsets");
  if (value_type != LSLU_F32 && value_type != LSLU_BF16)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "batched solves take FP32 or BF16 values");
  if (max_iter < 1 || max_iter > kMaxIter)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "max_iter must be in [1, 2048]");
  if (row_off[0] != 0 || col_off[0] != 0)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "row_off[0] and col_off[0] must be 0");
  for (int p = 0; p < nprob; ++p)
    if (row_off[p + 1] <= row_off[p] || col_off[p + 1] <= col_off[p])
      return set_err(nullptr, LSLU_ERR_INVALID_ARG, "every problem needs m >= 1 and n >= 1");
  const int64_t mu = row_off[nprob], nu = col_off[nprob];
  const int64_t nnz = row_ptr[mu];
  if (nnz < 0 || nnz >= (int64_t)INT32_MAX || row_ptr[0] != 0 || (nnz > 0 && (!col_idx || !vals)))
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "invalid CSR (row_ptr[0] != 0 or nnz)");
  // renumbering: each problem's rows and columns onto themselves; the rest of
  // the layout is built from the renumbered CSR, and the caller -> padded maps
  // are composed with the orders below
  const bool ordered = row_order || col_order;
  std::vector<int32_t> om, on, im, in;
  std::vector<int64_t> rp_o;
  std::vector<int32_t> ci_o;
  std::vector<double> vv_o;
  if (ordered) {
    lslu_status st0 = read_order(row_order, mu, false, om, im, "row_order");
    if (st0 == LSLU_OK) st0 = read_order(col_order, nu, false, on, in, "col_order");
    if (st0 != LSLU_OK) return st0;
    for (int p = 0; p < nprob; ++p) {
      for (int64_t r = row_off[p]; r < row_off[p + 1]; ++r)
        if (om[r] < row_off[p] || om[r] >= row_off[p + 1])
          return set_err(nullptr, LSLU_ERR_INVALID_ARG,
                         "row_order must map every problem's rows onto themselves");
      for (int64_t j = col_off[p]; j < col_off[p + 1]; ++j)
        if (on[j] < col_off[p] || on[j] >= col_off[p + 1])
          return set_err(nullptr, LSLU_ERR_INVALID_ARG,
                         "col_order must map every problem's columns onto themselves");
    }
    for (int64_t r = 0; r < mu; ++r)
      if (row_ptr[r + 1] < row_ptr[r])
        return set_err(nullptr, LSLU_ERR_INVALID_ARG, "row_ptr is not monotone");
    for (int64_t e = 0; e < nnz; ++e)
      if (col_idx[e] < 0 || col_idx[e] >= nu)
        return set_err(nullptr, LSLU_ERR_INVALID_ARG,
                       "column index outside its problem's column range");
    renumber_csr(mu, row_ptr, col_idx, vals, im, on, rp_o, ci_o, vv_o);
    row_ptr = rp_o.data();
    col_idx = ci_o.data();
    vals = vv_o.data();
  }
  // padded layout: every problem starts on a kTile boundary of both spaces
  std::vector<int64_t> rb(nprob), cb(nprob);
  int64_t mp = 0, np = 0;
  for (int p = 0; p < nprob; ++p) {
    rb[p] = mp;
    cb[p] = np;
    mp = round_up(mp + (row_off[p + 1] - row_off[p]), kTile);
    np = round_up(np + (col_off[p + 1] - col_off[p]), kTile);
  }
  if (mp >= (int64_t)INT32_MAX || np >= (int64_t)INT32_MAX)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "padded sizes must be below 2^31");
  std::vector<int64_t> rp(mp + 1, 0);
  std::vector<int32_t> ci;
  std::vector<double> vv;
  ci.reserve(nnz);
  vv.reserve(nnz);
  std::vector<int32_t> map_m(mu), map_n(nu), tpm(mp / kTile), tpn(np / kTile);
  std::vector<uint8_t> pad_m(mp, 1), pad_n(np, 1);
  std::vector<int64_t> mvec(nprob);
  int64_t prow = 0;
  for (int p = 0; p < nprob; ++p) {
    const int64_t m_p = row_off[p + 1] - row_off[p];
    const int64_t n_p = col_off[p + 1] - col_off[p];
    mvec[p] = m_p;
    for (; prow < rb[p]; ++prow) rp[prow + 1] = (int64_t)ci.size();  // padding rows
    for (int64_t i = 0; i < m_p; ++i, ++prow) {
      const int64_t r = row_off[p] + i;
      if (row_ptr[r + 1] < row_ptr[r])
        return set_err(nullptr, LSLU_ERR_INVALID_ARG, "row_ptr is not monotone");
      for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        const int64_t cglob = col_idx[e];
        if (cglob < col_off[p] || cglob >= col_off[p + 1])
          return set_err(nullptr, LSLU_ERR_INVALID_ARG,
                         "column index outside its problem's column range");
        if (!std::isfinite(vals[e]))
          return set_err(nullptr, LSLU_ERR_INVALID_ARG, "non-finite matrix value");
        ci.push_back((int32_t)(cb[p] + (cglob - col_off[p])));
        vv.push_back(vals[e]);
      }
      rp[prow + 1] = (int64_t)ci.size();
      map_m[r] = (int32_t)prow;
      pad_m[prow] = 0;
    }
    for (int64_t j = 0; j < n_p; ++j) {
      map_n[col_off[p] + j] = (int32_t)(cb[p] + j);
      pad_n[cb[p] + j] = 0;
    }
    const int64_t rend = p + 1 < nprob ? rb[p + 1] : mp;
    for (int64_t t = rb[p] / kTile; t < rend / kTile; ++t) tpm[t] = p;
    const int64_t cend = p + 1 < nprob ? cb[p + 1] : np;
    for (int64_t t = cb[p] / kTile; t < cend / kTile; ++t) tpn[t] = p;
  }
  for (; prow < mp; ++prow) rp[prow + 1] = (int64_t)ci.size();
  if (ordered) {  // caller index -> internal index -> padded position
    std::vector<int32_t> mm(mu), mn(nu);
    for (int64_t r = 0; r < mu; ++r) mm[r] = map_m[om[r]];
    for (int64_t j = 0; j < nu; ++j) mn[j] = map_n[on[j]];
    map_m.swap(mm);
    map_n.swap(mn);
  }

  lslu_ctx* c = new lslu_ctx();
  c->nprob = nprob;
  c->m = mp;
  c->n = np;
  c->m_user = mu;
  c->n_user = nu;
  c->row_base = rb;
  c->col_base = cb;
  for (int p = 0; p < nprob; ++p) {
    c->prob_m.push_back(row_off[p + 1] - row_off[p]);
    c->prob_n.push_back(col_off[p + 1] - col_off[p]);
  }
  c->nnz = nnz;
  c->value_type = value_type;
  c->kmax = max_iter;
  c->stream = (cudaStream_t)cuda_stream;
  lslu_status st = create_common(c, rp.data(), ci.data(), vv.data());
  if (st != LSLU_OK) return st;
  st = upload_batch_layout(c, tpm, tpn, pad_m, pad_n, map_m, map_n, mvec);
  if (st != LSLU_OK) return st;
  if (ordered) {  // pivot ties by the caller's index; pivot indices back to it
    std::vector<int32_t> rm(mp, INT32_MAX), rn(np, INT32_MAX);
    for (int64_t r = 0; r < mu; ++r) rm[map_m[r]] = (int32_t)r;
    for (int64_t j = 0; j < nu; ++j) rn[map_n[j]] = (int32_t)j;
    cudaError_t e = dmalloc(&c->rank_m, mp);
    if (e == cudaSuccess) e = dmalloc(&c->rank_n, np);
    if (e == cudaSuccess) e = cudaMemcpy(c->rank_m, rm.data(), mp * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->rank_n, rn.data(), np * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      destroy_ctx(c);
      return set_err(nullptr, e == cudaErrorMemoryAllocation ? LSLU_ERR_OOM : LSLU_ERR_CUDA,
                     std::string("renumbering ranks: ") + cudaGetErrorString(e));
    }
    c->unrank_m = c->map_m;
    c->unrank_n = c->map_n;
    c->inv_m_h.swap(im);
    c->inv_n_h.swap(in);
  }
  *out = c;
  return LSLU_OK;
}

}  // namespace

extern "C" lslu_status lslu_create_batched(int32_t nprob, const int64_t* row_off,
                                           const int64_t* col_off, const int64_t* row_ptr,
                                           const int32_t* col_idx, const double* vals,
                                           int32_t value_type, int32_t max_iter,
                                           void* cuda_stream, lslu_handle* out) {
  return create_batched_impl(nprob, row_off, col_off, row_ptr, col_idx, vals, value_type,
                             max_iter, nullptr, nullptr, cuda_stream, out);
}

extern "C" lslu_status lslu_create_batched_ordered(int32_t nprob, const int64_t* row_off,
                                                   const int64_t* col_off,
                                                   const int64_t* row_ptr,
                                                   const int32_t* col_idx, const double* vals,
                                                   int32_t value_type, int32_t max_iter,
                                                   const int32_t* row_order,
                                                   const int32_t* col_order,
                                                   void* cuda_stream, lslu_handle* out) {
  return create_batched_impl(nprob, row_off, col_off, row_ptr, col_idx, vals, value_type,
                             max_iter, row_order, col_order, cuda_stream, out);
}

namespace {

lslu_status create_shared_impl(int64_t m, int64_t n, const int64_t* row_ptr,
                               const int32_t* col_idx, const double* vals, int32_t nrhs,
                               int32_t value_type, int32_t max_iter, const int32_t* row_order,
                               const int32_t* col_order, void* cuda_stream, lslu_handle* out) {
  if (!out) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (m < 1 || n < 1 || !row_ptr)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "invalid m, n or row_ptr");
  if (nrhs < 1 || nrhs > 16)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (value_type != LSLU_F32 && value_type != LSLU_BF16)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "shared-matrix solves take FP32 or BF16 values");
  if (max_iter < 1 || max_iter > kMaxIter)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "max_iter must be in [1, 2048]");
  const int64_t nnz = row_ptr[m];
  if (row_ptr[0] != 0 || nnz < 0 || nnz >= (int64_t)INT32_MAX || (nnz > 0 && (!col_idx || !vals)))
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "invalid CSR (row_ptr[0] != 0 or nnz)");
  for (int64_t r = 0; r < m; ++r)
    if (row_ptr[r + 1] < row_ptr[r])
      return set_err(nullptr, LSLU_ERR_INVALID_ARG, "row_ptr is not monotone");
  for (int64_t e = 0; e < nnz; ++e) {
    if (col_idx[e] < 0 || col_idx[e] >= n)
      return set_err(nullptr, LSLU_ERR_INVALID_ARG, "column index out of range");
    if (!std::isfinite(vals[e]))
      return set_err(nullptr, LSLU_ERR_INVALID_ARG, "non-finite matrix value");
  }
  const int64_t m1p = round_up(m, kTile), n1p = round_up(n, kTile);
  const int64_t mp = nrhs * m1p, np = nrhs * n1p;
  if (mp >= (int64_t)INT32_MAX || np >= (int64_t)INT32_MAX)
    return set_err(nullptr, LSLU_ERR_INVALID_ARG, "padded sizes must be below 2^31");
  // renumbering of the one matrix, the same for every right-hand side
  const bool ordered = row_order || col_order;
  std::vector<int32_t> om, on, im, in;
  std::vector<int64_t> rp_o;
  std::vector<int32_t> ci_o;
  std::vector<double> vv_o;
  if (ordered) {
    lslu_status st0 = read_order(row_order, m, false, om, im, "row_order");
    if (st0 == LSLU_OK) st0 = read_order(col_order, n, false, on, in, "col_order");
    if (st0 != LSLU_OK) return st0;
    renumber_csr(m, row_ptr, col_idx, vals, im, on, rp_o, ci_o, vv_o);
    row_ptr = rp_o.data();
    col_idx = ci_o.data();
    vals = vv_o.data();
  }
  std::vector<int32_t> map_m(nrhs * m), map_n(nrhs * n), tpm(mp / kTile), tpn(np / kTile);
  std::vector<uint8_t> pad_m(mp, 1), pad_n(np, 1);
  std::vector<int64_t> mvec(nrhs, m);
  for (int r = 0; r < nrhs; ++r) {
    for (int64_t i = 0; i < m; ++i) {
      map_m[r * m + i] = (int32_t)(r * m1p + (ordered ? om[i] : i));
      pad_m[r * m1p + i] = 0;
    }
    for (int64_t j = 0; j < n; ++j) {
      map_n[r * n + j] = (int32_t)(r * n1p + (ordered ? on[j] : j));
      pad_n[r * n1p + j] = 0;
    }
  }
  for (int64_t t = 0; t < mp / kTile; ++t) tpm[t] = (int32_t)(t / (m1p / kTile));
  for (int64_t t = 0; t < np / kTile; ++t) tpn[t] = (int32_t)(t / (n1p / kTile));
  lslu_ctx* c = new lslu_ctx();
  c->nprob = nrhs;
  c->m = mp;
  c->n = np;
  c->m_user = nrhs * m;
  c->n_user = nrhs * n;
  for (int r = 0; r < nrhs; ++r) {
    c->row_base.push_back(r * m1p);
    c->col_base.push_back(r * n1p);
    c->prob_m.push_back(m);
    c->prob_n.push_back(n);
  }
  c->nnz = nnz;
  c->value_type = value_type;
  c->kmax = max_iter;
  c->stream = (cudaStream_t)cuda_stream;
  c->shared_rhs = nrhs;
  c->m1 = m;
  c->n1 = n;
  c->m1_pad = m1p;
  c->n1_pad = n1p;
  lslu_status st = create_common(c, row_ptr, col_idx, vals, m, n);
  if (st != LSLU_OK) return st;
  st = upload_batch_layout(c, tpm, tpn, pad_m, pad_n, map_m, map_n, mvec);
  if (st != LSLU_OK) return st;
  if (ordered) {  // pivot ties by the caller's index; pivot indices back to it
    std::vector<int32_t> rm(mp, INT32_MAX), rn(np, INT32_MAX), gm(nrhs * m), gn(nrhs * n);
    for (int64_t r = 0; r < nrhs * m; ++r) rm[map_m[r]] = (int32_t)r;
    for (int64_t j = 0; j < nrhs * n; ++j) rn[map_n[j]] = (int32_t)j;
    for (int q = 0; q < nrhs; ++q) {  // caller-global index of internal-global index
      for (int64_t i = 0; i < m; ++i) gm[q * m + i] = (int32_t)(q * m + im[i]);
      for (int64_t j = 0; j < n; ++j) gn[q * n + j] = (int32_t)(q * n + in[j]);
    }
    cudaError_t e = dmalloc(&c->rank_m, mp);
    if (e == cudaSuccess) e = dmalloc(&c->rank_n, np);
    if (e == cudaSuccess) e = cudaMemcpy(c->rank_m, rm.data(), mp * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->rank_n, rn.data(), np * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      destroy_ctx(c);
      return set_err(nullptr, e == cudaErrorMemoryAllocation ? LSLU_ERR_OOM : LSLU_ERR_CUDA,
                     std::string("renumbering ranks: ") + cudaGetErrorString(e));
    }
    c->unrank_m = c->map_m;
    c->unrank_n = c->map_n;
    c->inv_m_h.swap(gm);
    c->inv_n_h.swap(gn);
  }
  *out = c;
  return LSLU_OK;
}

}  // namespace

extern "C" lslu_status lslu_create_shared(int64_t m, int64_t n, const int64_t* row_ptr,
                                          const int32_t* col_idx, const double* vals,
                                          int32_t nrhs, int32_t value_type, int32_t max_iter,
                                          void* cuda_stream, lslu_handle* out) {
  return create_shared_impl(m, n, row_ptr, col_idx, vals, nrhs, value_type, max_iter, nullptr,
                            nullptr, cuda_stream, out);
}

extern "C" lslu_status lslu_create_shared_ordered(int64_t m, int64_t n, const int64_t* row_ptr,
                                                  const int32_t* col_idx, const double* vals,
                                                  int32_t nrhs, int32_t value_type,
                                                  int32_t max_iter, const int32_t* row_order,
                                                  const int32_t* col_order, void* cuda_stream,
                                                  lslu_handle* out) {
  return create_shared_impl(m, n, row_ptr, col_idx, vals, nrhs, value_type, max_iter, row_order,
                            col_order, cuda_stream, out);
}

extern "C" lslu_status lslu_solve_batched(lslu_handle h, const double* b, int32_t K,
                                          int32_t rule, double lambda, int32_t ptr_location,
                                          double* x_out, int32_t* col_pivots,
                                          int32_t* row_pivots, int32_t* k_done,
                                          int32_t* status) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (!c->map_m) return set_err(c, LSLU_ERR_INVALID_ARG, "not a batched handle");
  if (K < 1 || K > c->kmax) return set_err(c, LSLU_ERR_INVALID_ARG, "K must be in [1, max_iter]");
  if (rule < LSLU_LAMBDA_NONE || rule > LSLU_LAMBDA_WGCV)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown lambda rule");
  if (rule == LSLU_LAMBDA_FIXED && !(lambda >= 0.0 && std::isfinite(lambda)))
    return set_err(c, LSLU_ERR_INVALID_ARG, "fixed lambda must be finite and >= 0");
  if (!b || !x_out) return set_err(c, LSLU_ERR_INVALID_ARG, "b and x_out are required");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  const bool host = ptr_location == LSLU_HOST;
  const int P = c->nprob;
  cudaStream_t s = c->stream;
  if (host)
    for (int64_t i = 0; i < c->m_user; ++i)
      if (!std::isfinite(b[i])) return set_err(c, LSLU_ERR_NONFINITE, "b has a non-finite entry");
  CK(cudaMemcpyAsync(c->xin, b, c->m_user * 8,
                     host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(c->xin_pad, 0, c->m * 8, s));
  launch_scatter(c->xin, c->map_m, c->m_user, c->xin_pad, s);
  const double lam = rule == LSLU_LAMBDA_FIXED ? lambda : 0.0;
  lslu_status st = solve_impl<float, float>(c, c->xin_pad, nullptr, K, rule, lam, false);
  if (st != LSLU_OK) return st;
  launch_gather(c->xout, c->map_n, c->n_user, c->xout_user, s);
  const cudaMemcpyKind d2o = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(x_out, c->xout_user, c->n_user * 8, d2o, s));
  // pivots in each problem's own index space; -1 past its k_done
  std::vector<int32_t> g((size_t)P * c->kmax), t((size_t)P * (c->kmax + 1));
  CK(cudaMemcpyAsync(g.data(), c->gp, g.size() * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(t.data(), c->tp, t.size() * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int32_t> go((size_t)P * K), to((size_t)P * (K + 1)), kd(P), sv(P);
  // a renumbered batch: internal local index -> caller local index
  const bool ord = !c->inv_m_h.empty();
  int64_t uro = 0, uco = 0;  // the problem's offsets in the caller's rows and columns
  for (int p = 0; p < P; ++p) {
    const DevState& ds = c->st_host[p];
    const int kdp = ds.k_done < 0 ? 0 : (ds.k_done > K ? K : ds.k_done);
    kd[p] = kdp;
    sv[p] = ds.status;
    const int nt = ds.status == LSLU_BREAKDOWN_BETA ? 0 : kdp + 1;
    for (int j = 0; j < K; ++j) {
      const int32_t v = g[(size_t)p * c->kmax + j];
      int32_t l = (j < kdp && v >= 0) ? (int32_t)(v - c->col_base[p]) : -1;
      if (ord && l >= 0) l = (int32_t)(c->inv_n_h[uco + l] - uco);
      go[(size_t)p * K + j] = l;
    }
    for (int j = 0; j <= K; ++j) {
      const int32_t v = t[(size_t)p * (c->kmax + 1) + j];
      int32_t l = (j < nt && v >= 0) ? (int32_t)(v - c->row_base[p]) : -1;
      if (ord && l >= 0) l = (int32_t)(c->inv_m_h[uro + l] - uro);
      to[(size_t)p * (K + 1) + j] = l;
    }
    uro += c->prob_m[p];
    uco += c->prob_n[p];
  }
  const cudaMemcpyKind h2o = host ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
  if (col_pivots) CK(cudaMemcpyAsync(col_pivots, go.data(), go.size() * 4, h2o, s));
  if (row_pivots) CK(cudaMemcpyAsync(row_pivots, to.data(), to.size() * 4, h2o, s));
  if (k_done) CK(cudaMemcpyAsync(k_done, kd.data(), kd.size() * 4, h2o, s));
  if (status) CK(cudaMemcpyAsync(status, sv.data(), sv.size() * 4, h2o, s));
  CK(cudaStreamSynchronize(s));
  c->last_k = -1;  // lslu_get_state serves single-problem handles only
  for (int p = 0; p < P; ++p)
    if (sv[p] == LSLU_ERR_TIMEOUT)
      return set_err(c, LSLU_ERR_TIMEOUT, "a grid barrier of the persistent basis loop timed out");
  return LSLU_OK;
}

namespace {
void drop_graphs(Ctx* c);
}

extern "C" lslu_status lslu_set_loop(lslu_handle h, int32_t mode, int32_t blocks,
                                     int64_t wait_limit_ns, int32_t stall_first_barrier) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (mode == LSLU_LOOP_GRAPH) {
    CK(cudaStreamSynchronize(c->stream));
    c->loop_mode = LSLU_LOOP_GRAPH;
    c->loop_stall = 0;
    drop_graphs(c);
    return LSLU_OK;
  }
  if (mode == LSLU_LOOP_CLUSTER) {
    if (c->nprob != 1 || c->shared_rhs)
      return set_err(c, LSLU_ERR_INVALID_ARG, "the cluster basis loop serves single problems");
    if (blocks != 0 || stall_first_barrier)
      return set_err(c, LSLU_ERR_INVALID_ARG,
                     "the cluster basis loop takes no block count and no stalled barrier");
    const int C = cluster_loop_setup(c->value_type);
    if (C < 1) return set_err(c, LSLU_ERR_CUDA, "no thread-block cluster can be resident");
    if (!cluster_loop_fits(c->value_type, c->m, c->n, c->kmax, C))
      return set_err(c, LSLU_ERR_INVALID_ARG,
                     "the problem does not fit one cluster's shared memory "
                     "(use LSLU_LOOP_PERSISTENT or LSLU_LOOP_GRAPH)");
    CK(cudaStreamSynchronize(c->stream));
    c->loop_mode = LSLU_LOOP_CLUSTER;
    c->loop_blocks = C;
    c->loop_stall = 0;
    drop_graphs(c);
    return LSLU_OK;
  }
  if (mode != LSLU_LOOP_PERSISTENT) return set_err(c, LSLU_ERR_INVALID_ARG, "unknown loop mode");
  if (c->shared_rhs)
    return set_err(c, LSLU_ERR_INVALID_ARG,
                   "the persistent basis loop does not serve shared-matrix handles");
  if (c->nprob > kMaxPersistProblems)
    return set_err(c, LSLU_ERR_INVALID_ARG, "the persistent basis loop serves at most " +
                                                std::to_string(kMaxPersistProblems) + " problems");
  if (wait_limit_ns < 0 || wait_limit_ns > 60000000000LL)
    return set_err(c, LSLU_ERR_INVALID_ARG, "wait_limit_ns must be in [0, 6e10]");
  if (stall_first_barrier && wait_limit_ns == 0)
    return set_err(c, LSLU_ERR_INVALID_ARG, "a stalled barrier needs an explicit wait limit");
  int coop = 0;
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
  if (!coop) return set_err(c, LSLU_ERR_CUDA, "the device has no cooperative launch");
  const int maxb = persistent_max_blocks(c->value_type, c->kmax, c->nprob, c->num_sms);
  if (maxb < 1)
    return set_err(c, LSLU_ERR_INVALID_ARG,
                   "the persistent kernel cannot be resident for this max_iter and problem count");
  if (blocks < 0 || blocks > maxb)
    return set_err(c, LSLU_ERR_INVALID_ARG, "blocks must be in [0, " + std::to_string(maxb) +
                                                "] (0: automatic)");
  if (blocks == 0) {
    // one block per SM, or fewer when the rows (two per warp in the products)
    // do not fill them
    const int64_t need = (std::max(c->m, c->n) + 15) / 16;
    blocks = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)maxb, (int64_t)c->num_sms,
                                                          need}));
  }
  CK(cudaStreamSynchronize(c->stream));
  const size_t bb = basis_bytes(c->value_type);
  if (!c->pq_v) {
    CK(cudaMalloc(&c->pq_v, (size_t)c->n * bb));
    CK(cudaMalloc(&c->pq_w, (size_t)c->m * bb));
    CK(dmalloc(&c->pq_keys, 2 * (size_t)c->nprob));
    CK(dmalloc(&c->pq_bar, 4));
    CK(dmalloc(&c->pq_err, 1));
    CK(cudaMemset(c->pq_bar, 0, 4 * sizeof(unsigned)));
    CK(cudaMemset(c->pq_err, 0, sizeof(int)));
    if (c->nprob > 1) {
      CK(dmalloc(&c->pq_row0, (size_t)c->nprob));
      CK(dmalloc(&c->pq_col0, (size_t)c->nprob));
      CK(cudaMemcpy(c->pq_row0, c->row_base.data(), c->nprob * 8, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->pq_col0, c->col_base.data(), c->nprob * 8, cudaMemcpyHostToDevice));
    }
  }
  if (c->pq_slot_val) {
    cudaFree(c->pq_slot_val);
    cudaFree(c->pq_slot_idx);
    c->pq_slot_val = nullptr;
    c->pq_slot_idx = nullptr;
  }
  CK(dmalloc(&c->pq_slot_val, (size_t)blocks));
  CK(dmalloc(&c->pq_slot_idx, (size_t)blocks));
  c->loop_mode = LSLU_LOOP_PERSISTENT;
  c->loop_blocks = blocks;
  c->loop_wait_ns = wait_limit_ns ? (unsigned long long)wait_limit_ns : 1000000000ull;
  c->loop_stall = stall_first_barrier ? 1 : 0;
  drop_graphs(c);  // captured solves hold the launch sequence of the old mode
  return LSLU_OK;
}

extern "C" lslu_status lslu_loop_config(lslu_handle h, int32_t* mode, int32_t* blocks,
                                        int32_t* max_blocks) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (mode) *mode = c->loop_mode;
  if (blocks) *blocks = c->loop_mode != LSLU_LOOP_GRAPH ? c->loop_blocks : 0;
  if (max_blocks) {
    *max_blocks = c->shared_rhs ? 0
                                : persistent_max_blocks(c->value_type, c->kmax, c->nprob,
                                                        c->num_sms);
  }
  return LSLU_OK;
}

// The stopping rule online (graph loop mode): the basis in chunks of
// kStopChunk iterations launched directly; after each chunk the projected
// problems of its sizes (one batched launch: residual and trace of each),
// G^(k) for every k so far and the first k that meets Eq. (tol); the host
// reads it and stops as soon as the criterion, a breakdown or K_max decides.
// Each G^(k) and the basis are those of the whole run to K_max, bit for bit.
constexpr int kStopChunk = 8;

template <typename BT, typename CT>
lslu_status stopping_online(Ctx* c, const double* db, const double* dx0, int K_max, int rule,
                            double lam, double tol, double* G, int32_t* dk, int* ks_out) {
  lslu_status st = ensure_batched_workspace(c);
  if (st != LSLU_OK) return st;
  cudaStream_t s = c->stream;
  const int64_t m = c->m, n = c->n;
  CK(cudaMemsetAsync(G, 0, (size_t)K_max * 8, s));
  int64_t launches = 1;
  int ks = 0;
  for (int k0 = 0; k0 < K_max;) {
    const int k1 = std::min(K_max, k0 + kStopChunk);
    launches += enqueue_solve<BT, CT>(c, s, db, dx0, K_max, rule, lam, false, false, false, 0,
                                      k0, k1, false);
    ProjArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.H = c->H;
    pa.ldh = c->kmax + 1;
    pa.rule = rule;
    pa.lambda = lam;
    pa.m = c->prob_m[0];
    pa.k_first = k0 + 1;
    pa.k_last = k1;
    pa.want_y = 0;
    pa.y = c->y;
    pa.ldy = c->kmax;
    pa.nbatch = 1;
    pa.strideH = c->h_stride;
    pa.lam_out = c->proj_out;
    pa.res_out = c->proj_out + c->res_off;
    pa.tr_out = c->proj_out + 2 * c->res_off;
    pa.st = c->st;
    ProjWork w;
    w.cluster = c->pw_cluster;
    w.base = c->pw_batched;
    w.offsets = c->pw_offsets;
    w.packed = 1;
    int nproj = 0;
    CK(launch_projected(pa, w, s, &nproj));
    launch_stop_select(pa.res_out, pa.tr_out, G, k1, (double)n, (double)m, tol, c->st, dk, s);
    launches += nproj + 1;  // projected kernels and the selection
    int32_t r = 0;
    CK(cudaMemcpyAsync(&r, dk, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    // r < k1: the criterion (or a breakdown at k_done = r) decided; a breakdown
    // at k_done = k1 or the last chunk ends the run with r = min(k1, k_done)
    if (r < k1 || c->st_host[0].status != LSLU_OK || k1 == K_max) {
      ks = r;
      break;
    }
    k0 = k1;
  }
  c->launches = launches;
  *ks_out = ks;
  return LSLU_OK;
}

extern "C" lslu_status lslu_solve_stopping(lslu_handle h, const double* b, const double* x0,
                                           int32_t K_max, int32_t rule, double lambda,
                                           double tol, int32_t ptr_location, double* x_out,
                                           int32_t* k_stop, double* g_hist) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (c->map_m) return set_err(c, LSLU_ERR_INVALID_ARG, "single-problem handles only");
  if (K_max < 2 || K_max > c->kmax)
    return set_err(c, LSLU_ERR_INVALID_ARG, "K_max must be in [2, max_iter]");
  if (rule < LSLU_LAMBDA_NONE || rule > LSLU_LAMBDA_WGCV)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown lambda rule");
  if (rule == LSLU_LAMBDA_FIXED && !(lambda >= 0.0 && std::isfinite(lambda)))
    return set_err(c, LSLU_ERR_INVALID_ARG, "fixed lambda must be finite and >= 0");
  if (!(tol > 0.0) || !std::isfinite(tol))
    return set_err(c, LSLU_ERR_INVALID_ARG, "tol must be finite and > 0");
  if (!b || !x_out) return set_err(c, LSLU_ERR_INVALID_ARG, "b and x_out are required");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  if (x0 && c->loop_mode != LSLU_LOOP_GRAPH)
    return set_err(c, LSLU_ERR_INVALID_ARG,
                   "the persistent and cluster basis loops serve x0 = 0 only");
  const bool host = ptr_location == LSLU_HOST;
  const int64_t m = c->m, n = c->n;
  cudaStream_t s = c->stream;
  if (host)
    for (int64_t i = 0; i < m; ++i)
      if (!std::isfinite(b[i])) return set_err(c, LSLU_ERR_NONFINITE, "b has a non-finite entry");
  CK(vec_in(c, true, b, host, c->xin));
  const double* dx0 = nullptr;
  if (x0) {
    CK(vec_in(c, false, x0, host, c->xin + m));
    dx0 = c->xin + m;
  }
  const double lam = rule == LSLU_LAMBDA_FIXED ? lambda : 0.0;
  int32_t* dk = reinterpret_cast<int32_t*>(c->part_idx);
  double* G = nullptr;
  int32_t ks = 0;
  if (c->loop_mode == LSLU_LOOP_GRAPH) {
    // online: the basis in chunks, stopped once k_stop is known
    if (!c->gstop) CK(dmalloc(&c->gstop, (size_t)c->kmax + 1));
    G = c->gstop;
    int ksi = 0;
    lslu_status st =
        c->value_type == LSLU_F64
            ? stopping_online<double, double>(c, c->xin, dx0, K_max, rule, lam, tol, G, dk, &ksi)
            : stopping_online<float, float>(c, c->xin, dx0, K_max, rule, lam, tol, G, dk, &ksi);
    if (st != LSLU_OK) return st;
    ks = ksi;
  } else {
    // the basis for K_max iterations and the projected problem of every k
    lslu_status st = c->value_type == LSLU_F64
                         ? solve_impl<double, double>(c, c->xin, dx0, K_max, rule, lam, true)
                         : solve_impl<float, float>(c, c->xin, dx0, K_max, rule, lam, true);
    if (st != LSLU_OK) return st;
    // G^(k) for every k and the stopping iteration (Eqs. stop2, tol)
    G = c->proj_out + 2 * c->res_off;  // G overwrites the trace in place
    launch_stop_select(c->proj_out + c->res_off, G, G, K_max, (double)n, (double)m, tol, c->st,
                       dk, s);
    CK(cudaMemcpyAsync(&ks, dk, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
  }
  c->adj_valid = false;
  c->last_k = std::min<int>(std::max(c->st_host[0].k_done, 0), K_max);
  c->last_K = K_max;
  if (ks > 0) {  // y_k and x_k at the stopping iteration
    ProjArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.H = c->H;
    pa.ldh = c->kmax + 1;
    pa.rule = rule;
    pa.lambda = lam;
    pa.m = c->prob_m[0];
    pa.k_first = ks;
    pa.k_last = ks;
    pa.want_y = 1;
    pa.y = c->y;
    pa.ldy = c->kmax;
    pa.nbatch = 1;
    pa.st = c->st;
    ProjWork w;
    w.base = c->pw_single;
    w.cluster = c->pw_cluster;
    w.slot_stride = projected_slot_doubles(c->kmax, c->pw_cluster);
    int nproj = 0;
    CK(launch_projected(pa, w, s, &nproj));
    c->launches += nproj + 1;
    if (c->value_type == LSLU_F64)
      launch_recombine<double>((const double*)c->L, c->ldl, c->y, c->kmax, dx0, c->xout, n,
                               nullptr, 1, nullptr, ks, s, c->num_sms);
    else
      launch_recombine<float>((const float*)c->L, c->ldl, c->y, c->kmax, dx0, c->xout, n,
                              nullptr, 1, nullptr, ks, s, c->num_sms);
  } else {
    CK(cudaMemsetAsync(c->xout, 0, n * 8, s));
    if (dx0) CK(cudaMemcpyAsync(c->xout, dx0, n * 8, cudaMemcpyDeviceToDevice, s));
  }
  const cudaMemcpyKind d2o = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(vec_out(c, false, c->xout, host, x_out));
  if (g_hist) CK(cudaMemcpyAsync(g_hist, G, (size_t)K_max * 8, d2o, s));
  if (k_stop) {
    if (host)
      *k_stop = ks;
    else
      CK(cudaMemcpyAsync(k_stop, dk, 4, cudaMemcpyDeviceToDevice, s));
  }
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return LSLU_OK;
}

namespace {

void drop_graphs(Ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

}  // namespace

extern "C" lslu_status lslu_set_spmv_shape(lslu_handle h, int32_t shape_A, int32_t shape_AT) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (shape_A < 0 || shape_A >= kNumShapes || shape_AT < 0 || shape_AT >= kNumShapes)
    return set_err(c, LSLU_ERR_INVALID_ARG, "shape must be in [0, 16)");
  if ((shape_cmp(shape_A) && !c->A.compressed) || (shape_cmp(shape_AT) && !c->AT.compressed))
    return set_err(c, LSLU_ERR_INVALID_ARG,
                   "16-bit offset shapes need a matrix whose 8-entry units span < 2^16 columns");
  CK(cudaStreamSynchronize(c->stream));
  c->A.shape = shape_A;
  c->AT.shape = shape_AT;
  c->A.use_cmp = shape_cmp(shape_A);
  c->AT.use_cmp = shape_cmp(shape_AT);
  drop_graphs(c);  // captured solves hold the kernels of the old shapes
  return LSLU_OK;
}

extern "C" lslu_status lslu_spmv_config(lslu_handle h, int32_t* shape_A, int32_t* shape_AT,
                                        int32_t* compressed_A, int32_t* compressed_AT) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (shape_A) *shape_A = c->A.shape;
  if (shape_AT) *shape_AT = c->AT.shape;
  if (compressed_A) *compressed_A = c->A.compressed;
  if (compressed_AT) *compressed_AT = c->AT.compressed;
  return LSLU_OK;
}

extern "C" lslu_status lslu_tune_spmv(lslu_handle h, int32_t reps, int32_t* shape_A,
                                      int32_t* shape_AT, double* us) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (reps < 1 || reps > 1000) return set_err(c, LSLU_ERR_INVALID_ARG, "reps must be in [1, 1000]");
  cudaStream_t s = c->stream;
  const size_t bb = basis_bytes(c->value_type);
  // the products read q (n) or u (m) and write the other; their contents do
  // not change the time
  CK(cudaMemsetAsync(c->q, 0, (size_t)c->n * bb, s));
  CK(cudaMemsetAsync(c->u, 0, (size_t)c->m * bb, s));
  // in a solve every product follows an elimination that streams the basis
  // through L2; reading twice the L2 size before each timed product leaves
  // the cache in a comparable state (clean lines; the buffer's contents do
  // not matter)
  int l2 = 0;
  CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device));
  const size_t flush_bytes = (size_t)std::max(l2, 1 << 20) * 2;
  void* flush = nullptr;
  if (cudaMalloc(&flush, flush_bytes + 16) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, LSLU_ERR_OOM, "tuning: no room for the L2 flush buffer");
  }
  int* sink = reinterpret_cast<int*>(static_cast<char*>(flush) + flush_bytes);
  std::vector<cudaEvent_t> ev(4 * reps);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  const int saved[2] = {c->A.shape, c->AT.shape};
  const int saved_cmp[2] = {c->A.use_cmp, c->AT.use_cmp};
  int best[2] = {saved[0], saved[1]};
  float best_ms[2] = {0.f, 0.f}, def_ms[2] = {0.f, 0.f};
  bool have[2] = {false, false};
  auto run = [&](DevCsr& M, const void* x, void* y) {
    if (c->value_type == LSLU_F64)
      launch_spmv<double, double>(M, c->value_type, (const double*)x, (double*)y, s, c->num_sms);
    else
      launch_spmv<float, float>(M, c->value_type, (const float*)x, (float*)y, s, c->num_sms);
  };
  lslu_status st = LSLU_OK;
  for (int sh = 0; sh < kNumShapes && st == LSLU_OK; ++sh) {
    const bool cmp = shape_cmp(sh);
    if (cmp && !(c->A.compressed && c->AT.compressed)) {
      if (us) us[sh] = us[kNumShapes + sh] = -1.0;  // not available
      continue;
    }
    c->A.shape = c->AT.shape = sh;
    c->A.use_cmp = c->AT.use_cmp = cmp;
    // A and A^T alternate, as in a solve; each timed launch follows an L2 flush
    run(c->A, c->q, c->u);
    run(c->AT, c->u, c->q);
    for (int r = 0; r < reps; ++r) {
      launch_l2_flush(flush, flush_bytes, sink, s, c->num_sms);
      cudaEventRecord(ev[4 * r], s);
      run(c->A, c->q, c->u);
      cudaEventRecord(ev[4 * r + 1], s);
      launch_l2_flush(flush, flush_bytes, sink, s, c->num_sms);
      cudaEventRecord(ev[4 * r + 2], s);
      run(c->AT, c->u, c->q);
      cudaEventRecord(ev[4 * r + 3], s);
    }
    cudaError_t e = cudaEventSynchronize(ev[4 * reps - 1]);
    float t[2] = {0.f, 0.f};
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      float a = 0.f, b = 0.f;
      e = cudaEventElapsedTime(&a, ev[4 * r], ev[4 * r + 1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[4 * r + 2], ev[4 * r + 3]);
      t[0] += a;
      t[1] += b;
    }
    if (e != cudaSuccess) {
      st = set_err(c, LSLU_ERR_CUDA, std::string("tuning: ") + cudaGetErrorString(e));
      break;
    }
    for (int w = 0; w < 2; ++w) {
      if (sh == default_shape(c->value_type)) def_ms[w] = t[w];
      if (us) us[w * kNumShapes + sh] = 1e3 * t[w] / reps;
      if (!have[w] || t[w] < best_ms[w]) {
        best_ms[w] = t[w];
        best[w] = sh;
        have[w] = true;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  cudaFree(flush);
  if (st != LSLU_OK) {
    c->A.shape = saved[0];
    c->AT.shape = saved[1];
    c->A.use_cmp = saved_cmp[0];
    c->AT.use_cmp = saved_cmp[1];
    return st;
  }
  // shapes within a few per cent of each other swap places from run to run:
  // keep the default unless another is clearly faster
  const int def = default_shape(c->value_type);
  for (int w = 0; w < 2; ++w)
    if (best[w] != def && def_ms[w] > 0.f && best_ms[w] > 0.97f * def_ms[w]) best[w] = def;
  c->A.shape = best[0];
  c->AT.shape = best[1];
  c->A.use_cmp = shape_cmp(best[0]);
  c->AT.use_cmp = shape_cmp(best[1]);
  drop_graphs(c);
  if (shape_A) *shape_A = best[0];
  if (shape_AT) *shape_AT = best[1];
  return LSLU_OK;
}

extern "C" lslu_status lslu_solve_optimal(lslu_handle h, const double* b, int32_t K,
                                          const double* x_true, int32_t ptr_location,
                                          double* x_out, double* lambda_out) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (c->map_m) return set_err(c, LSLU_ERR_INVALID_ARG, "single-problem handles only");
  if (K < 1 || K > c->kmax) return set_err(c, LSLU_ERR_INVALID_ARG, "K must be in [1, max_iter]");
  if (!b || !x_true || !x_out)
    return set_err(c, LSLU_ERR_INVALID_ARG, "b, x_true and x_out are required");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  const bool host = ptr_location == LSLU_HOST;
  const int64_t m = c->m, n = c->n;
  cudaStream_t s = c->stream;
  CK(vec_in(c, true, b, host, c->xin));
  // x_true is staged behind b (the staging buffer holds m + n doubles)
  CK(vec_in(c, false, x_true, host, c->xin + m));
  // the basis and the factorisation of the final projected problem
  lslu_status st = c->value_type == LSLU_F64
                       ? solve_impl<double, double>(c, c->xin, nullptr, K, LSLU_LAMBDA_NONE, 0.0, false)
                       : solve_impl<float, float>(c, c->xin, nullptr, K, LSLU_LAMBDA_NONE, 0.0, false);
  if (st != LSLU_OK) return st;
  c->adj_valid = false;
  if (c->st_host[0].status != LSLU_OK)
    return set_err(c, (lslu_status)c->st_host[0].status, "breakdown before iteration K");
  c->last_k = K;
  c->last_K = K;
  double* G = nullptr;
  CK(cudaMalloc(&G, ((size_t)K * K + K + 260 + optimal_lambda_work_doubles()) * sizeof(double)));
  double* g = G + (size_t)K * K;
  double* Eg = g + K;
  double* dl = Eg + 257;
  double* Er = dl + 3;
  st = basis_gram_products(c, K, c->xin + m, G, g);
  if (st == LSLU_OK) {
    ProjWork w;
    w.base = c->pw_single;
    w.cluster = c->pw_cluster;
    cudaError_t e = launch_optimal_lambda(w, K, c->st, G, g, Eg, Er, dl, s);
    double lam = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lam, dl, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      // y and x for that lambda: the FIXED-rule projected solve
      ProjArgs pa;
      std::memset(&pa, 0, sizeof(pa));
      pa.H = c->H;
      pa.ldh = c->kmax + 1;
      pa.rule = LSLU_LAMBDA_FIXED;
      pa.lambda = lam;
      pa.m = c->prob_m[0];
      pa.k_first = K;
      pa.k_last = K;
      pa.want_y = 1;
      pa.y = c->y;
      pa.ldy = c->kmax;
      pa.nbatch = 1;
      pa.st = c->st;
      ProjWork w2;
      w2.base = c->pw_single;
      w2.cluster = c->pw_cluster;
      w2.slot_stride = projected_slot_doubles(c->kmax, c->pw_cluster);
      e = launch_projected(pa, w2, s);
      if (e == cudaSuccess) {
        if (c->value_type == LSLU_F64)
          launch_recombine<double>((const double*)c->L, c->ldl, c->y, c->kmax, nullptr, c->xout,
                                   n, nullptr, 1, nullptr, K, s, c->num_sms);
        else
          launch_recombine<float>((const float*)c->L, c->ldl, c->y, c->kmax, nullptr, c->xout,
                                  n, nullptr, 1, nullptr, K, s, c->num_sms);
        e = vec_out(c, false, c->xout, host, x_out);
        if (e == cudaSuccess && lambda_out) {
          if (host)
            *lambda_out = lam;
          else
            e = cudaMemcpyAsync(lambda_out, dl, 8, cudaMemcpyDeviceToDevice, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      }
    }
    if (e != cudaSuccess) st = set_err(c, LSLU_ERR_CUDA, std::string("optimal lambda: ") +
                                                           cudaGetErrorString(e));
  }
  cudaFree(G);
  return st;
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
  if (c->ord_m) {  // bases back to the caller's numbering: row gathers
    for (int which = 0; which < 2; ++which) {
      void* dst = which == 0 ? L : D;
      const int64_t rows = which == 0 ? c->n : c->m;
      const int cols = which == 0 ? k : k + 1;
      if (!dst || cols == 0) continue;
      void* tmp = dst;
      if (ptr_location == LSLU_HOST) CK(cudaMalloc(&tmp, (size_t)rows * cols * bb));
      launch_gather_rows(which == 0 ? c->L : c->D, which == 0 ? c->ldl : c->ldd,
                         which == 0 ? c->ord_n : c->ord_m, rows, cols, tmp, rows, (int)bb, s);
      cudaError_t e = cudaGetLastError();
      if (ptr_location == LSLU_HOST) {
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(dst, tmp, (size_t)rows * cols * bb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(tmp);
      }
      CK(e);
    }
  } else {
    if (L && k > 0)
      CK(cudaMemcpy2DAsync(L, c->n * bb, c->L, c->ldl * bb, c->n * bb, k, kind, s));
    if (D)
      CK(cudaMemcpy2DAsync(D, c->m * bb, c->D, c->ldd * bb, c->m * bb, k + 1, kind, s));
  }
  CK(cudaStreamSynchronize(s));
  return LSLU_OK;
}

extern "C" lslu_status lslu_spmv(lslu_handle h, int32_t transpose, const void* x, void* y) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (!x || !y) return set_err(c, LSLU_ERR_INVALID_ARG, "NULL vector");
  if (c->map_m) return set_err(c, LSLU_ERR_INVALID_ARG, "lslu_spmv takes single-problem handles");
  if (c->ord_m)
    return set_err(c, LSLU_ERR_INVALID_ARG, "lslu_spmv takes handles without a renumbering");
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
  c->adj_valid = false;  // the projected work space and y are reused below
  if (k < 1 || k > c->kmax || ldh < k + 1 || !H)
    return set_err(c, LSLU_ERR_INVALID_ARG, "invalid k, ldh or H");
  if (rule < LSLU_LAMBDA_NONE || rule > LSLU_LAMBDA_WGCV || m < 1)
    return set_err(c, LSLU_ERR_INVALID_ARG, "invalid rule or m");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  cudaStream_t s = c->stream;
  const double* dH = H;
  // staging copy of a host H, freed on every exit (cudaFree waits for the
  // work queued on it)
  struct StageGuard {
    double* p = nullptr;
    ~StageGuard() {
      if (p) cudaFree(p);
    }
  } stage;
  if (ptr_location == LSLU_HOST) {
    CK(dmalloc(&stage.p, (size_t)(k + 1) * k));
    CK(cudaMemcpy2DAsync(stage.p, (k + 1) * 8, H, (size_t)ldh * 8, (k + 1) * 8, k,
                         cudaMemcpyHostToDevice, s));
    dH = stage.p;
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
  pa.res_out = c->proj_out + c->res_off;
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
  if (resid_out) CK(cudaMemcpyAsync(resid_out, c->proj_out + c->res_off + (k - 1), 8, kind, s));
  CK(cudaStreamSynchronize(s));
  return LSLU_OK;
}

extern "C" lslu_status lslu_projected_history(lslu_handle h, int32_t K, const double* H,
                                              int32_t ldh, double beta, int32_t rule,
                                              double lambda, int64_t m, int32_t ptr_location,
                                              double* lambda_hist, double* resid_hist) {
  Ctx* c = h;
  if (!c) return set_err(nullptr, LSLU_ERR_INVALID_ARG, "NULL handle");
  if (K < 1 || K > c->kmax || ldh < K + 1 || !H)
    return set_err(c, LSLU_ERR_INVALID_ARG, "invalid K, ldh or H");
  if (rule < LSLU_LAMBDA_NONE || rule > LSLU_LAMBDA_WGCV || m < 1)
    return set_err(c, LSLU_ERR_INVALID_ARG, "invalid rule or m");
  if (rule == LSLU_LAMBDA_FIXED && !(lambda >= 0.0))
    return set_err(c, LSLU_ERR_INVALID_ARG, "fixed lambda must be >= 0");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return set_err(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  c->adj_valid = false;  // the projected work space is reused below
  lslu_status st = ensure_batched_workspace(c);
  if (st != LSLU_OK) return st;
  cudaStream_t s = c->stream;
  const double* dH = H;
  struct StageGuard {  // staging copy of a host H, freed on every exit
    double* p = nullptr;
    ~StageGuard() {
      if (p) cudaFree(p);
    }
  } stage;
  if (ptr_location == LSLU_HOST) {
    CK(dmalloc(&stage.p, (size_t)(K + 1) * K));
    CK(cudaMemcpy2DAsync(stage.p, (K + 1) * 8, H, (size_t)ldh * 8, (K + 1) * 8, K,
                         cudaMemcpyHostToDevice, s));
    dH = stage.p;
    ldh = K + 1;
  }
  ProjArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.H = dH;
  pa.ldh = ldh;
  pa.beta_val = beta;
  pa.rule = rule;
  pa.lambda = rule == LSLU_LAMBDA_FIXED ? lambda : 0.0;
  pa.m = m;
  pa.nbatch = 1;
  pa.k_first = 1;
  pa.k_last = K;
  pa.want_y = 0;
  pa.lam_out = c->proj_out;
  pa.res_out = c->proj_out + c->res_off;
  ProjWork w;
  w.base = c->pw_batched;
  w.offsets = c->pw_offsets;
  w.packed = 1;
  w.cluster = c->pw_cluster;
  CK(launch_projected(pa, w, s));
  const cudaMemcpyKind kind =
      ptr_location == LSLU_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (lambda_hist) CK(cudaMemcpyAsync(lambda_hist, c->proj_out, (size_t)K * 8, kind, s));
  if (resid_hist)
    CK(cudaMemcpyAsync(resid_hist, c->proj_out + c->res_off, (size_t)K * 8, kind, s));
  CK(cudaStreamSynchronize(s));
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
