// Hessenberg step of Algorithm 4 for one new vector x (q = A^T d_k or
// u = A l_k) against the basis B (L_k or D_{k+1}) with pivot rows piv:
//
//   coefficients  c_j = x(piv_j) - sum_{i<j} B_i(piv_j) c_i   (the sequential
//                 elimination "W(j,k) = q(g(j)); q = q - W(j,k) l_j" read at
//                 the pivot rows: a forward substitution with the unit lower
//                 triangular T(j,i) = B_i(piv_j));
//   elimination   v = x - B c, with v = 0 exactly on pivoted rows;
//   pivot         i* = argmax |v| over unpivoted rows (ties: lowest index),
//                 the new Hessenberg entry v(i*), new row of T;
//   scale         b_new = v / v(i*) (1 at i*, 0 on earlier pivots).
//
// The argmax is a grid reduction: every block writes its best candidate and
// the last block to finish (ticket counter) reduces the partials in block
// order and records the pivot, so the result does not depend on timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "lslu_internal.cuh"

namespace lslu {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool better(double va, int ia, double vb, int ib) {
  // larger value wins; equal values: lower index wins; index -1 = no candidate
  if (ia < 0) return false;
  if (ib < 0) return true;
  return va > vb || (va == vb && ia < ib);
}

__device__ __forceinline__ void warp_argmax(double& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(ov, oi, v, i)) {
      v = ov;
      i = oi;
    }
  }
}

// Block-wide argmax; result valid in every thread.
__device__ void block_argmax(double& v, int& i) {
  __shared__ double sv[32];
  __shared__ int si[32];
  warp_argmax(v, i);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sv[w] = v;
    si[w] = i;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = lane < nw ? sv[lane] : 0.0;
  i = lane < nw ? si[lane] : -1;
  warp_argmax(v, i);
  __syncthreads();
}

template <typename XT>
__global__ void k_coefficients(const XT* __restrict__ x, const int32_t* __restrict__ piv, int cnt,
                               const double* __restrict__ T, int64_t ldt, double* __restrict__ coef,
                               double* __restrict__ hess_col, const DevState* st) {
  extern __shared__ double r[];
  if (st->status != LSLU_OK) return;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) r[i] = (double)x[piv[i]];
  for (int j = 0; j < cnt; ++j) {
    __syncthreads();
    const double cj = r[j];
    for (int i = j + 1 + threadIdx.x; i < cnt; i += blockDim.x)
      r[i] = fma(-T[i + j * ldt], cj, r[i]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    coef[i] = r[i];
    if (hess_col) hess_col[i] = r[i];
  }
}

template <typename XT, typename BT, typename CT>
__global__ void __launch_bounds__(kThreads)
    k_eliminate_argmax(const XT* x, const BT* __restrict__ B, int64_t ld, int cnt,
                       const double* __restrict__ coef, int64_t rows, CT* v, PivotArgs pa,
                       double* __restrict__ part_val, int32_t* __restrict__ part_idx,
                       DevState* st) {
  extern __shared__ unsigned char smem_raw[];
  CT* c = reinterpret_cast<CT*>(smem_raw);
  __shared__ bool is_last;
  if (st->status != LSLU_OK) return;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) c[j] = (CT)coef[j];
  __syncthreads();

  double best = 0.0;
  int besti = -1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    CT acc = 0;
    if (!pa.used[i]) {
      acc = (CT)x[i];
      const BT* bp = B + i;
      int j = 0;
      for (; j + 8 <= cnt; j += 8) {
        BT b[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) b[t] = __ldg(bp + (int64_t)(j + t) * ld);
#pragma unroll
        for (int t = 0; t < 8; ++t) acc = fma(-c[j + t], (CT)b[t], acc);
      }
      for (; j < cnt; ++j) acc = fma(-c[j], (CT)__ldg(bp + (int64_t)j * ld), acc);
      double a = fabs((double)acc);
      if (isnan(a)) a = INFINITY;  // a NaN must win so that it is reported
      if (better(a, (int)i, best, besti)) {
        best = a;
        besti = (int)i;
      }
    }
    v[i] = acc;
  }
  block_argmax(best, besti);
  if (threadIdx.x == 0) {
    part_val[blockIdx.x] = best;
    part_idx[blockIdx.x] = besti;
    __threadfence();
    const int t = atomicAdd(&st->ticket, 1);
    is_last = (t == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  best = 0.0;
  besti = -1;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double pv = ((volatile double*)part_val)[b];
    const int pi = ((volatile int32_t*)part_idx)[b];
    if (better(pv, pi, best, besti)) {
      best = pv;
      besti = pi;
    }
  }
  block_argmax(best, besti);
  __shared__ double pval_s;
  if (threadIdx.x == 0) {
    st->ticket = 0;
    if (besti < 0 || best == 0.0) {
      st->status = pa.breakdown_code;
      st->k_done = pa.k_on_breakdown;
      pval_s = 0.0;
    } else if (!isfinite(best)) {
      st->status = LSLU_ERR_NONFINITE;
      st->k_done = pa.k_on_breakdown;
      pval_s = 0.0;
    } else {
      const CT pv = ((volatile CT*)v)[besti];
      pval_s = (double)pv;
      st->pivot = (double)pv;
      st->pivot_f = (float)pv;
      pa.piv_list[pa.piv_slot] = besti;
      pa.used[besti] = 1;
      if (pa.hess_entry) *pa.hess_entry = (double)pv;
      if (pa.is_init) st->beta = (double)pv;
      pa.T[pa.piv_slot + pa.piv_slot * pa.ldt] = 1.0;
    }
    is_last = (pval_s != 0.0);
  }
  __syncthreads();
  if (!is_last) return;
  // new row of T: entries of the earlier basis vectors at the new pivot row
  for (int j = threadIdx.x; j < cnt; j += blockDim.x)
    pa.T[pa.piv_slot + j * pa.ldt] = (double)B[besti + (int64_t)j * ld];
}

template <typename CT, typename BT>
__global__ void k_scale(const CT* __restrict__ v, BT* __restrict__ out, int64_t rows,
                        const DevState* st) {
  if (st->status != LSLU_OK) return;
  const CT p = sizeof(CT) == 8 ? (CT)st->pivot : (CT)st->pivot_f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (BT)(v[i] / p);
}

__global__ void k_residual0(const double* b, const double* Ax0, double* r0, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    r0[i] = Ax0 ? b[i] - Ax0[i] : b[i];
}

template <typename BT>
__global__ void __launch_bounds__(kThreads)
    k_recombine(const BT* __restrict__ L, int64_t ldl, const double* __restrict__ y,
                const double* __restrict__ x0, double* __restrict__ x, int64_t n,
                const DevState* st, int K) {
  extern __shared__ double ys[];
  const int k = st ? min(K, st->k_done) : K;
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma((double)__ldg(L + i + (int64_t)j * ldl), ys[j], acc);
    x[i] = (x0 ? x0[i] : 0.0) + acc;
  }
}

int grid_for(int64_t rows, int num_sms, int per_sm) {
  int64_t b = (rows + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

template <typename BT>
void launch_coefficients(const void* x, int x_is_double, const BT*, const int32_t* piv, int cnt,
                         const double* T, int64_t ldt, double* coef, double* hess_col,
                         DevState* st, cudaStream_t s) {
  if (cnt == 0) return;
  const size_t sm = (size_t)cnt * sizeof(double);
  if (x_is_double)
    k_coefficients<double><<<1, 256, sm, s>>>((const double*)x, piv, cnt, T, ldt, coef,
                                               hess_col, st);
  else
    k_coefficients<float><<<1, 256, sm, s>>>((const float*)x, piv, cnt, T, ldt, coef, hess_col,
                                              st);
}

template <typename XT, typename BT, typename CT>
void launch_eliminate_argmax(const XT* x, const BT* B, int64_t ld, int cnt, const double* coef,
                             int64_t rows, CT* v, const PivotArgs& pa, double* part_val,
                             int32_t* part_idx, int part_cap, DevState* st, cudaStream_t s,
                             int num_sms) {
  int g = grid_for(rows, num_sms, 8);
  if (g > part_cap) g = part_cap;
  const size_t sm = (size_t)(cnt > 0 ? cnt : 1) * sizeof(CT);
  k_eliminate_argmax<XT, BT, CT><<<g, kThreads, sm, s>>>(x, B, ld, cnt, coef, rows, v, pa,
                                                         part_val, part_idx, st);
}

template <typename CT, typename BT>
void launch_scale(const CT* v, BT* out, int64_t rows, DevState* st, cudaStream_t s,
                  int num_sms) {
  k_scale<CT, BT><<<grid_for(rows, num_sms, 8), kThreads, 0, s>>>(v, out, rows, st);
}

void launch_residual0(const double* b, const double* Ax0, double* r0, int64_t m,
                      cudaStream_t s) {
  k_residual0<<<(unsigned)std::min<int64_t>((m + 255) / 256, 4096), 256, 0, s>>>(b, Ax0, r0, m);
}

template <typename BT>
void launch_recombine(const BT* L, int64_t ldl, const double* y, const double* x0, double* x,
                      int64_t n, const DevState* st, int K, cudaStream_t s, int num_sms) {
  k_recombine<BT><<<grid_for(n, num_sms, 8), kThreads, (size_t)(K > 0 ? K : 1) * 8, s>>>(
      L, ldl, y, x0, x, n, st, K);
}

// explicit instantiations: FP64 mode (basis double) and FP32 mode (basis float)
template void launch_coefficients<double>(const void*, int, const double*, const int32_t*, int,
                                          const double*, int64_t, double*, double*, DevState*,
                                          cudaStream_t);
template void launch_coefficients<float>(const void*, int, const float*, const int32_t*, int,
                                         const double*, int64_t, double*, double*, DevState*,
                                         cudaStream_t);
template void launch_eliminate_argmax<double, double, double>(
    const double*, const double*, int64_t, int, const double*, int64_t, double*,
    const PivotArgs&, double*, int32_t*, int, DevState*, cudaStream_t, int);
template void launch_eliminate_argmax<float, float, float>(const float*, const float*, int64_t,
                                                           int, const double*, int64_t, float*,
                                                           const PivotArgs&, double*, int32_t*,
                                                           int, DevState*, cudaStream_t, int);
template void launch_eliminate_argmax<double, float, double>(
    const double*, const float*, int64_t, int, const double*, int64_t, double*,
    const PivotArgs&, double*, int32_t*, int, DevState*, cudaStream_t, int);
template void launch_scale<double, double>(const double*, double*, int64_t, DevState*,
                                           cudaStream_t, int);
template void launch_scale<float, float>(const float*, float*, int64_t, DevState*, cudaStream_t,
                                         int);
template void launch_scale<double, float>(const double*, float*, int64_t, DevState*,
                                          cudaStream_t, int);
template void launch_recombine<double>(const double*, int64_t, const double*, const double*,
                                       double*, int64_t, const DevState*, int, cudaStream_t, int);
template void launch_recombine<float>(const float*, int64_t, const double*, const double*,
                                      double*, int64_t, const DevState*, int, cudaStream_t, int);

}  // namespace lslu
