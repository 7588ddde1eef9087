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

// Tiles of rows x all basis columns: a tile of 32*VEC consecutive rows is read
// by every warp of the block as 16-byte vectors (VEC rows per lane); warp w
// takes the columns j = w, w+8, ...  The eight per-warp partial sums of each
// row are combined in warp order, then subtracted from x.
template <typename BT>
struct Vec16;
template <>
struct Vec16<float> {
  static constexpr int N = 4;
  __device__ static void load(const float* p, float (&o)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct Vec16<double> {
  static constexpr int N = 2;
  __device__ static void load(const double* p, double (&o)[2]) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = v.x; o[1] = v.y;
  }
};

// Pivot search.  FP32 compute: each candidate becomes the 64-bit key
// (bits of |v| << 32) | (2^32 - 1 - i), so one unsigned max gives the
// largest |v| with ties to the lowest index (a NaN has larger bits than any
// number and wins, so it is reported); blocks combine with one atomicMax.
// FP64 compute: (|v|, i) pairs are reduced per block and the partials are
// reduced in block order by the last block.
__device__ __forceinline__ unsigned long long argkey(float a, int i) {
  return ((unsigned long long)__float_as_uint(a) << 32) | (unsigned long long)(0xffffffffu - (unsigned)i);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
    k = ok > k ? ok : k;
  }
  return k;
}

template <typename XT, typename BT, typename CT>
__global__ void __launch_bounds__(kThreads)
    k_eliminate_argmax(const XT* x, const BT* __restrict__ B, int64_t ld, int cnt,
                       const double* __restrict__ coef, int64_t rows, CT* v, PivotArgs pa,
                       double* __restrict__ part_val, int32_t* __restrict__ part_idx,
                       DevState* st) {
  constexpr bool kKey = sizeof(CT) == 4;
  constexpr int VEC = Vec16<BT>::N;
  constexpr int TILE = 32 * VEC;
  constexpr int NW = kThreads / 32;
  extern __shared__ unsigned char smem_raw[];
  CT* c = reinterpret_cast<CT*>(smem_raw);
  __shared__ CT part[NW][TILE];
  __shared__ unsigned long long kred[NW];
  __shared__ bool is_last;
  if (st->status != LSLU_OK) return;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) c[j] = (CT)coef[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (rows + TILE - 1) / TILE;
  double best = 0.0;
  int besti = -1;
  unsigned long long bkey = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * TILE;
    CT acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0;
    const BT* bp = B + r0 + lane * VEC;
    int j = warp;
    for (; j + 7 * NW < cnt; j += 8 * NW) {
      BT b[8][VEC];
#pragma unroll
      for (int u = 0; u < 8; ++u) Vec16<BT>::load(bp + (int64_t)(j + u * NW) * ld, b[u]);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const CT cu = c[j + u * NW];
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = fma(cu, (CT)b[u][e], acc[e]);
      }
    }
    for (; j < cnt; j += NW) {
      BT b0[VEC];
      Vec16<BT>::load(bp + (int64_t)j * ld, b0);
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = fma(c[j], (CT)b0[e], acc[e]);
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) part[warp][lane * VEC + e] = acc[e];
    __syncthreads();
    if (threadIdx.x < TILE) {
      const int64_t i = r0 + threadIdx.x;
      if (i < rows) {
        CT s = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += part[w][threadIdx.x];
        CT val = 0;
        if (!pa.used[i]) {
          val = (CT)x[i] - s;
          if constexpr (kKey) {
            const unsigned long long kk = argkey(fabsf((float)val), (int)i);
            bkey = kk > bkey ? kk : bkey;
          } else {
            double a = fabs((double)val);
            if (isnan(a)) a = INFINITY;  // a NaN must win so that it is reported
            if (better(a, (int)i, best, besti)) {
              best = a;
              besti = (int)i;
            }
          }
        }
        v[i] = val;
      }
    }
    __syncthreads();
  }
  if constexpr (kKey) {
    bkey = warp_max_u64(bkey);
    if (lane == 0) kred[warp] = bkey;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = 0;
      for (int w = 0; w < NW; ++w) m = kred[w] > m ? kred[w] : m;
      if (m) atomicMax(&st->amax, m);
      __threadfence();
      is_last = (atomicAdd(&st->ticket, 1) == (int)gridDim.x - 1);
    }
  } else {
    block_argmax(best, besti);
    if (threadIdx.x == 0) {
      part_val[blockIdx.x] = best;
      part_idx[blockIdx.x] = besti;
      __threadfence();
      is_last = (atomicAdd(&st->ticket, 1) == (int)gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if constexpr (!kKey) {
    best = 0.0;
    besti = -1;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      const double pv = __ldcg(part_val + b);
      const int pi = __ldcg(part_idx + b);
      if (better(pv, pi, best, besti)) {
        best = pv;
        besti = pi;
      }
    }
    block_argmax(best, besti);
  }
  if (threadIdx.x == 0) {
    st->ticket = 0;
    if constexpr (kKey) {
      const unsigned long long m = atomicExch(&st->amax, 0ull);
      besti = m ? (int)(0xffffffffu - (unsigned)(m & 0xffffffffull)) : -1;
      const float a = __uint_as_float((unsigned)(m >> 32));
      best = (a != a) ? INFINITY : (double)a;
    }
    if (besti < 0 || best == 0.0) {
      st->status = pa.breakdown_code;
      st->k_done = pa.k_on_breakdown;
    } else if (!isfinite(best)) {
      st->status = LSLU_ERR_NONFINITE;
      st->k_done = pa.k_on_breakdown;
    } else {
      const CT pv = __ldcg(v + besti);
      st->pivot = (double)pv;
      st->pivot_f = (float)pv;
      pa.piv_list[pa.piv_slot] = besti;
      pa.used[besti] = 1;
      if (pa.hess_entry) *pa.hess_entry = (double)pv;
      if (pa.is_init) st->beta = (double)pv;
      reinterpret_cast<BT*>(pa.Tinv)[(int64_t)pa.piv_slot * pa.ldt + pa.piv_slot] = (BT)1;
    }
  }
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

__global__ void k_init_state(DevState* st, int K) {
  st->status = LSLU_OK;
  st->k_done = K;
  st->ticket = 0;
  st->ticket2 = 0;
  st->beta = 0.0;
  st->pivot = 0.0;
  st->pivot_f = 0.0f;
  st->amax = 0ull;
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

template <typename XT, typename BT, typename CT>
void launch_eliminate_argmax(const XT* x, const BT* B, int64_t ld, int cnt, const double* coef,
                             int64_t rows, CT* v, const PivotArgs& pa, double* part_val,
                             int32_t* part_idx, int part_cap, DevState* st, cudaStream_t s,
                             int) {
  constexpr int TILE = 32 * Vec16<BT>::N;
  int64_t g = (rows + TILE - 1) / TILE;
  if (g > part_cap) g = part_cap;
  if (g < 1) g = 1;
  const size_t sm = (size_t)(cnt > 0 ? cnt : 1) * sizeof(CT);
  k_eliminate_argmax<XT, BT, CT><<<(unsigned)g, kThreads, sm, s>>>(x, B, ld, cnt, coef, rows, v,
                                                                   pa, part_val, part_idx, st);
}

template <typename CT, typename BT>
void launch_scale(const CT* v, BT* out, int64_t rows, DevState* st, cudaStream_t s,
                  int num_sms) {
  k_scale<CT, BT><<<grid_for(rows, num_sms, 8), kThreads, 0, s>>>(v, out, rows, st);
}

void launch_init_state(DevState* st, int K, cudaStream_t s) { k_init_state<<<1, 1, 0, s>>>(st, K); }

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
