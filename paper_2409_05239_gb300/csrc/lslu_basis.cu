// Hessenberg step of Algorithm 4 for one new vector x (q = A^T d_k or
// u = A l_k) against the basis B (L_k or D_{k+1}) with pivot rows piv:
//
//   coefficients  c = T^-1 x(piv), T(i,j) = b_j(piv_i) unit lower triangular
//                 (the sequential elimination "W(j,k) = q(g(j)); q = q -
//                 W(j,k) l_j" read at the pivot rows; computed inside the
//                 sparse product, lslu_spmv.cu);
//   elimination   v = x - B c, with v = 0 exactly on pivoted rows;
//   pivot         i* = argmax |v| over unpivoted rows (ties: lowest index),
//                 the new Hessenberg entry v(i*);
//   scale         b_new = v / v(i*) (1 at i*, 0 on earlier pivots).
//
// A launch serves every problem of a batch: problem p owns whole kTile-row
// tiles, its coefficients, pivot list, T^-1 and state sit at base + p * stride.
// The argmax is a grid reduction that does not depend on timing: FP32 keys
// combine with an integer atomicMax; FP64 (single problem) candidates are
// reduced per block and the partials in block order by the last block.
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

// FP32 pivot key: (bits of |v| << 32) | ((2^31 - 1 - i) << 1) | sign of v.
// One unsigned max gives the largest |v| with ties to the lowest index i
// (0 <= i < 2^31; the sign bit never decides, as i is unique); a NaN has
// larger bits than any number, wins and is reported.  The key holds the
// pivot's value exactly, so the pivot is recorded without reading v again.
__device__ __forceinline__ unsigned long long argkey(float a, int i, bool neg) {
  return ((unsigned long long)__float_as_uint(a) << 32) |
         ((unsigned long long)(0x7fffffffu - (unsigned)i) << 1) | (neg ? 1ull : 0ull);
}
__device__ __forceinline__ int key_index(unsigned long long m) {
  return (int)(0x7fffffffu - (unsigned)((m & 0xffffffffull) >> 1));
}
__device__ __forceinline__ float key_value(unsigned long long m) {
  const float a = __uint_as_float((unsigned)(m >> 32));
  return (m & 1ull) ? -a : a;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
    k = ok > k ? ok : k;
  }
  return k;
}

__device__ __forceinline__ int tile_problem(const int32_t* tile_prob, int64_t row) {
  return tile_prob ? tile_prob[row / kTile] : 0;
}

// The index a pivot search compares on ties (Algorithm 4, lowest index): the
// caller's index of a row on a renumbered handle, the row itself otherwise;
// unrank_of maps the winner back to its stored row.
__device__ __forceinline__ int rank_of(const PivotArgs& pa, int64_t i) {
  return pa.rank ? __ldg(pa.rank + i) : (int)i;
}
__device__ __forceinline__ int unrank_of(const PivotArgs& pa, int r) {
  return (pa.unrank && r >= 0) ? __ldg(pa.unrank + r) : r;
}

// Records the pivot of problem p (one thread).
// have_val: pv_known is v(besti) (from an FP32 key), so v is not read again.
template <typename CT, typename BT>
__device__ void record_pivot(const PivotArgs& pa, DevState& s, int p, int besti, double best,
                             const CT* v, bool have_val = false, CT pv_known = 0) {
  if (pa.fixed) {  // replay: the given row, whatever the search found
    besti = pa.fixed[(int64_t)p * pa.piv_stride + pa.piv_slot];
    best = fabs((double)__ldcg(v + besti));
    if (best != best) best = INFINITY;
    have_val = false;
  }
  if (besti < 0 || best == 0.0) {
    s.status = pa.breakdown_code;
    s.k_done = pa.k_on_breakdown;
  } else if (!isfinite(best)) {
    s.status = LSLU_ERR_NONFINITE;
    s.k_done = pa.k_on_breakdown;
  } else {
    const CT pv = have_val ? pv_known : __ldcg(v + besti);
    s.pivot = (double)pv;
    s.pivot_f = (float)pv;
    pa.piv_list[(int64_t)p * pa.piv_stride + pa.piv_slot] = besti;
    pa.used[besti] = 1;
    if (pa.hess_entry) pa.hess_entry[(int64_t)p * pa.hess_stride] = (double)pv;
    if (pa.is_init) s.beta = (double)pv;
    reinterpret_cast<BT*>(pa.Tinv)[(int64_t)p * pa.tinv_stride +
                                   (int64_t)pa.piv_slot * pa.ldt + pa.piv_slot] = (BT)1;
  }
}

// Sampled pivoting (Section 2.2): the largest |v| among the unpivoted rows of
// the sample (ties to the lowest index) as an FP32 key (0 when none is
// non-zero); every thread of the block calls it, the result is valid in all.
template <typename CT>
__device__ unsigned long long sampled_key(const PivotArgs& pa, const CT* v) {
  __shared__ unsigned long long sk[kThreads / 32];
  unsigned long long k = 0;
  for (int j = threadIdx.x; j < pa.nsamp; j += blockDim.x) {
    const int32_t i = pa.samples[j];
    if (!pa.used[i]) {
      const float vi = (float)__ldcg(v + i);
      const float a = fabsf(vi);
      if (a != 0.0f) {
        const unsigned long long kk = argkey(a, rank_of(pa, i), vi < 0.0f);
        k = kk > k ? kk : k;
      }
    }
  }
  k = warp_max_u64(k);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sk[threadIdx.x >> 5] = k;
  __syncthreads();
  unsigned long long r = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = sk[w] > r ? sk[w] : r;
  __syncthreads();
  return r;
}

// The same in FP64 (value, index) form; best = 0 when none is non-zero.
// besti is the winner's rank (rank_of).
template <typename CT>
__device__ void sampled_best(const PivotArgs& pa, const CT* v, double& best, int& besti) {
  best = 0.0;
  besti = -1;
  for (int j = threadIdx.x; j < pa.nsamp; j += blockDim.x) {
    const int32_t i = pa.samples[j];
    if (pa.used[i]) continue;
    double a = fabs((double)__ldcg(v + i));
    if (isnan(a)) a = INFINITY;
    const int ri = rank_of(pa, i);
    if (a != 0.0 && better(a, ri, best, besti)) {
      best = a;
      besti = ri;
    }
  }
  block_argmax(best, besti);
  if (besti < 0) best = 0.0;
}

// One warp per block and per tile of 32*VEC rows: lane l owns rows
// r0 + l*VEC .. r0 + l*VEC + VEC-1 and eliminates them against all cnt basis
// columns in order, v = fma(-c_j, b_j, v) for j = 0 .. cnt-1 (the sequential
// order of Algorithm 4), reading each column as one 16-byte vector with
// UJ = 8 columns in flight.  No block-level combination is needed, and the
// small blocks spread evenly over the SMs.  The pivot search is a grid
// reduction that does not depend on timing: FP32 keys combine with an
// integer atomicMax; FP64 (single problem) candidates are reduced per block
// and the partials in block order by the last block.
template <typename XT, typename BT, typename CT>
__global__ void __launch_bounds__(32)
    k_eliminate_argmax(const XT* x, const BT* __restrict__ B, int64_t ld, int cnt, int64_t rows,
                       CT* v, PivotArgs pa, double* __restrict__ part_val,
                       int32_t* __restrict__ part_idx, DevState* st) {
  constexpr bool kKey = sizeof(CT) == 4;
  constexpr int VEC = Vec16<BT>::N;
  constexpr int TILE = 32 * VEC;
  constexpr int UJ = 8;  // basis columns in flight per lane
  static_assert(kTile % TILE == 0, "problem tiles must hold whole elimination tiles");
  extern __shared__ unsigned char smem_raw[];
  CT* c = reinterpret_cast<CT*>(smem_raw);
  __shared__ bool is_last;
  pdl_wait();  // x, the coefficients and the state come from the kernels before
  pdl_trigger();
  // A single problem that has broken down writes nothing.  Its status is only
  // needed at the first store, so its read overlaps the tile's first reads
  // (x, the pivot flags, the coefficients, the basis).
  const int status0 = pa.nprob == 1 ? st[0].status : (int)LSLU_OK;
  const int lane = threadIdx.x;
  const int64_t ntiles = (rows + TILE - 1) / TILE;
  double best = 0.0;
  int besti = -1;
  unsigned long long bkey = 0;
  int cur_p = -1;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * TILE;
    const int p = tile_problem(pa.tile_prob, r0);
    const int64_t i0 = r0 + lane * VEC;
    const bool full = i0 + VEC <= rows;
    CT val[VEC];
    if constexpr (sizeof(XT) == sizeof(CT) && VEC * sizeof(CT) == 16) {
      if (full) {  // one 16-byte load of x (x may alias v: a coherent load)
        if constexpr (sizeof(CT) == 4) {
          const float4 w = *reinterpret_cast<const float4*>(x + i0);
          val[0] = w.x; val[1] = w.y; val[2] = w.z; val[3] = w.w;
        } else {
          const double2 w = *reinterpret_cast<const double2*>(x + i0);
          val[0] = w.x; val[1] = w.y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) val[e] = (i0 + e < rows) ? (CT)x[i0 + e] : (CT)0;
      }
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) val[e] = (i0 + e < rows) ? (CT)x[i0 + e] : (CT)0;
    }
    // pivoted-row flags of the lane's rows (one 32-bit load when VEC == 4)
    uint8_t usedf[VEC];
    if (VEC == 4 && full) {
      const uint32_t w = *reinterpret_cast<const uint32_t*>(pa.used + i0);
#pragma unroll
      for (int e = 0; e < VEC; ++e) usedf[e] = (uint8_t)((w >> (8 * e)) & 0xffu);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) usedf[e] = (i0 + e < rows) ? pa.used[i0 + e] : (uint8_t)1;
    }
    if (p != cur_p) {  // the problem's coefficients (x and the flags are in flight meanwhile)
      __syncwarp();
      for (int j = lane; j < cnt; j += 32) c[j] = (CT)pa.coef[(int64_t)p * pa.coef_stride + j];
      __syncwarp();
      cur_p = p;
    }
    const BT* bp = B + i0;  // the basis has whole tiles of rows
    int j = 0;
    for (; j + UJ <= cnt; j += UJ) {
      BT b[UJ][VEC];
#pragma unroll
      for (int u = 0; u < UJ; ++u) Vec16<BT>::load(bp + (int64_t)(j + u) * ld, b[u]);
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
        const CT cu = c[j + u];
#pragma unroll
        for (int e = 0; e < VEC; ++e) val[e] = fma(-cu, (CT)b[u][e], val[e]);
      }
    }
    for (; j < cnt; ++j) {
      BT b0[VEC];
      Vec16<BT>::load(bp + (int64_t)j * ld, b0);
#pragma unroll
      for (int e = 0; e < VEC; ++e) val[e] = fma(-c[j], (CT)b0[e], val[e]);
    }
    // tie-breaking index of the lane's rows: the row itself, or (renumbered
    // handle, FP64 comparisons) its rank in one vector load; FP32 keys read
    // the ranks of the few rows that can win after the warp's maximum below
    int rk[VEC];
    if (!kKey && pa.rank) {
      if constexpr (VEC == 4) {
        if (full) {
          const int4 w = __ldg(reinterpret_cast<const int4*>(pa.rank + i0));
          rk[0] = w.x; rk[1] = w.y; rk[2] = w.z; rk[3] = w.w;
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) rk[e] = (i0 + e < rows) ? __ldg(pa.rank + i0 + e) : 0;
        }
      } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) rk[e] = (i0 + e < rows) ? __ldg(pa.rank + i0 + e) : 0;
      }
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) rk[e] = (int)(i0 + e);
    }
    if (status0 != LSLU_OK) return;
    unsigned long long tkey = 0;
    CT outv[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int64_t i = i0 + e;
      outv[e] = 0;
      if (i >= rows) continue;
      CT out = 0;
      if (!usedf[e]) {
        out = val[e];
        if constexpr (kKey) {
          const unsigned long long kk = argkey(fabsf((float)out), rk[e], (float)out < 0.0f);
          tkey = kk > tkey ? kk : tkey;
        } else {
          double a = fabs((double)out);
          if (isnan(a)) a = INFINITY;  // a NaN must win so that it is reported
          if (better(a, rk[e], best, besti)) {
            best = a;
            besti = rk[e];
          }
        }
      }
      outv[e] = out;
    }
    if (full && VEC * sizeof(CT) == 16) {
      if constexpr (sizeof(CT) == 4)
        *reinterpret_cast<float4*>(v + i0) = make_float4(outv[0], outv[1], outv[2], outv[3]);
      else
        *reinterpret_cast<double2*>(v + i0) = make_double2(outv[0], outv[1]);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e)
        if (i0 + e < rows) v[i0 + e] = outv[e];
    }
    if constexpr (kKey) {
      if (pa.rank) {
        // only rows holding the warp's largest |v| can win here: their keys
        // are rebuilt on the rank, the rest drop out (same maximum key as
        // keying every row on its rank)
        const unsigned wb = __reduce_max_sync(0xffffffffu, (unsigned)(tkey >> 32));
        unsigned long long rkey = 0;
        if (wb != 0u && (unsigned)(tkey >> 32) == wb) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const float a = fabsf((float)outv[e]);
            if (i0 + e < rows && !usedf[e] && __float_as_uint(a) == wb) {
              const unsigned long long kk =
                  argkey(a, __ldg(pa.rank + i0 + e), (float)outv[e] < 0.0f);
              rkey = kk > rkey ? kk : rkey;
            }
          }
        }
        tkey = rkey;
      }
      tkey = warp_max_u64(tkey);
      if (pa.nprob == 1) {
        bkey = tkey > bkey ? tkey : bkey;
      } else if (lane == 0 && tkey) {  // batch: one atomicMax per tile on its problem
        atomicMax(&st[p].amax, tkey);
      }
    }
  }
  if constexpr (kKey) {
    if (pa.nprob == 1 && lane == 0 && bkey) atomicMax(&st[0].amax, bkey);
    if (lane == 0) {
      __threadfence();
      is_last = (atomicAdd(&st[0].ticket, 1) == (int)gridDim.x - 1);
    }
  } else {
    warp_argmax(best, besti);
    if (lane == 0) {
      part_val[blockIdx.x] = best;
      part_idx[blockIdx.x] = besti;
      __threadfence();
      is_last = (atomicAdd(&st[0].ticket, 1) == (int)gridDim.x - 1);
    }
  }
  __syncwarp();
  if (!is_last) return;
  __threadfence();
  if constexpr (kKey) {
    if (lane == 0) st[0].ticket = 0;
    const unsigned long long skey = pa.samples ? sampled_key<CT>(pa, v) : 0ull;
    for (int p = lane; p < pa.nprob; p += 32) {
      unsigned long long m = atomicExch(&st[p].amax, 0ull);
      if (p == 0 && (skey >> 32) != 0) m = skey;  // sampled pivot (full search as fallback)
      if (st[p].status != LSLU_OK) continue;
      const int bi = m ? unrank_of(pa, key_index(m)) : -1;
      const float a = __uint_as_float((unsigned)(m >> 32));
      record_pivot<CT, BT>(pa, st[p], p, bi, (a != a) ? INFINITY : (double)a, v, true,
                           (CT)key_value(m));
    }
  } else {
    best = 0.0;
    besti = -1;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const double pv = __ldcg(part_val + b);
      const int pi = __ldcg(part_idx + b);
      if (better(pv, pi, best, besti)) {
        best = pv;
        besti = pi;
      }
    }
    warp_argmax(best, besti);
    if (pa.samples) {  // sampled pivot, the full search as fallback
      double sb;
      int si;
      sampled_best<CT>(pa, v, sb, si);
      if (sb > 0.0) {
        best = sb;
        besti = si;
      }
    }
    if (lane == 0) {
      st[0].ticket = 0;
      record_pivot<CT, BT>(pa, st[0], 0, unrank_of(pa, besti), best, v);
    }
  }
}

// Exact pivot of r0 for every problem, in two passes over FP64 values: the
// largest |r0| (non-negative doubles order like their bit patterns), then the
// lowest index attaining it; the last block of the second pass records it.
__global__ void k_r0_max(const double* __restrict__ r0, int64_t rows, const uint8_t* used,
                         const int32_t* tile_prob, DevState* st) {
  // warp-uniform trip count: the 32 rows of a warp lie in one kTile tile, so
  // one problem; the warp's maximum goes to that problem with one atomic
  const int lane = threadIdx.x & 31;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x - lane); i0 < rows;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + lane;
    unsigned long long bits = 0;
    if (i < rows && !used[i]) {
      const double a = fabs(r0[i]);
      bits = (unsigned long long)__double_as_longlong(a);
      if (a != a) bits = 0x7ff0000000000001ull;  // NaN above every number
    }
    bits = warp_max_u64(bits);
    if (lane == 0 && bits) atomicMax(&st[tile_problem(tile_prob, i0)].amax, bits);
  }
}

template <typename BT>
__global__ void k_r0_argmin(const double* __restrict__ r0, int64_t rows, PivotArgs pa,
                            DevState* st) {
  __shared__ bool is_last;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (pa.used[i]) continue;
    const int p = tile_problem(pa.tile_prob, i);
    const double a = fabs(r0[i]);
    unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    if (a != a) bits = 0x7ff0000000000001ull;
    if (bits && bits == __ldcg(&st[p].amax)) atomicMin(&st[p].amin, rank_of(pa, i));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(&st[0].ticket, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (threadIdx.x == 0) st[0].ticket = 0;
  double sb = 0.0;
  int si = -1;
  if (pa.samples) sampled_best<double>(pa, r0, sb, si);
  for (int p = threadIdx.x; p < pa.nprob; p += blockDim.x) {
    const unsigned long long m = atomicExch(&st[p].amax, 0ull);
    const int bi = atomicExch(&st[p].amin, 0x7fffffff);
    if (st[p].status != LSLU_OK) continue;
    double best = m == 0x7ff0000000000001ull ? INFINITY : __longlong_as_double((long long)m);
    int besti = (m && bi != 0x7fffffff) ? unrank_of(pa, bi) : -1;
    if (p == 0 && sb > 0.0) {  // sampled pivot, the full search as fallback
      best = sb;
      besti = unrank_of(pa, si);
    }
    record_pivot<double, BT>(pa, st[p], p, besti, best, r0);
  }
}

template <typename CT, typename BT>
__global__ void k_scale(const CT* __restrict__ v, BT* __restrict__ out, int64_t rows,
                        const DevState* st, int nprob, const int32_t* tile_prob) {
  // four consecutive rows per thread (one problem: kTile is a multiple of 4),
  // the vector read issued before the dependent pivot read
  pdl_wait();  // v and the pivot come from the elimination before
  pdl_trigger();
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i0 >= rows) return;
  const bool full = i0 + 4 <= rows;
  CT a[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) a[e] = (full || i0 + e < rows) ? v[i0 + e] : (CT)0;
  const DevState& s = st[tile_problem(tile_prob, i0)];
  if (s.status != LSLU_OK) return;
  const CT p = sizeof(CT) == 8 ? (CT)s.pivot : (CT)s.pivot_f;
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (full || i0 + e < rows) out[i0 + e] = (BT)(a[e] / p);
}

__global__ void k_init_state(DevState* st, int nprob, int K) {
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    DevState& s = st[p];
    s.status = LSLU_OK;
    s.k_done = K;
    s.ticket = 0;
    s.ticket2 = 0;
    s.beta = 0.0;
    s.pivot = 0.0;
    s.pivot_f = 0.0f;
    s.amin = 0x7fffffff;
    s.amax = 0ull;
  }
}

__global__ void k_residual0(const double* b, const double* Ax0, double* r0, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    r0[i] = Ax0 ? b[i] - Ax0[i] : b[i];
}

__global__ void k_scatter(const double* __restrict__ src, const int32_t* __restrict__ map,
                          int64_t count, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[map[i]] = src[i];
}

__global__ void k_gather(const double* __restrict__ src, const int32_t* __restrict__ map,
                         int64_t count, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[map[i]];
}

template <typename T>
__global__ void k_gather_rows(const T* __restrict__ src, int64_t lds,
                              const int32_t* __restrict__ map, int64_t rows, int64_t cols,
                              T* __restrict__ dst, int64_t ldd) {
  for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x)
      dst[j * ldd + i] = src[j * lds + map[i]];
}

// x = x0 + L y for every problem; tiles of kTile rows (one problem each),
// FP64 accumulation.
template <typename BT>
__global__ void __launch_bounds__(kTile)
    k_recombine(const BT* __restrict__ L, int64_t ldl, const double* __restrict__ y, int64_t ldy,
                const double* __restrict__ x0, double* __restrict__ x, int64_t n,
                const DevState* st, int nprob, const int32_t* tile_prob, int K) {
  extern __shared__ double ys[];
  const int64_t ntiles = (n + kTile - 1) / kTile;
  int cur_p = -1, k = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int p = tile_problem(tile_prob, t * kTile);
    if (p != cur_p) {
      __syncthreads();
      k = st ? min(K, st[p].k_done) : K;
      for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[(int64_t)p * ldy + j];
      __syncthreads();
      cur_p = p;
    }
    const int64_t i = t * kTile + threadIdx.x;
    if (i < n) {
      double acc = 0.0;
      for (int j = 0; j < k; ++j) acc = fma((double)__ldg(L + i + (int64_t)j * ldl), ys[j], acc);
      x[i] = (x0 ? x0[i] : 0.0) + acc;
    }
  }
}

// G^(k) = n res_k^2 / ((m - k) + tr_k)^2 for k = 1..k_done (Eq. stop2; tr may
// be G itself), zero past k_done, and the first k with
// |G(k+1) - G(k)| / G(1) < tol (Eq. tol), else min(K, k_done).  One block.
__global__ void k_stop_select(const double* __restrict__ res, const double* tr, double* G, int K,
                              double n, double m, double tol, const DevState* st,
                              int32_t* k_stop) {
  __shared__ int first;
  const int kd = min(K, max(st->k_done, 0));
  if (threadIdx.x == 0) first = kd;
  for (int k = 1 + threadIdx.x; k <= K; k += blockDim.x) {
    double g = 0.0;
    if (k <= kd) {
      const double den = (m - k) + tr[k - 1];
      g = n * res[k - 1] * res[k - 1] / (den * den);
    }
    G[k - 1] = g;
  }
  __syncthreads();
  const double g1 = G[0];
  for (int k = 1 + threadIdx.x; k < kd; k += blockDim.x)
    if (fabs((G[k] - G[k - 1]) / g1) < tol) atomicMin(&first, k);
  __syncthreads();
  if (threadIdx.x == 0) *k_stop = first;
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
void launch_eliminate_argmax(const XT* x, const BT* B, int64_t ld, int cnt, int64_t rows, CT* v,
                             const PivotArgs& pa, double* part_val, int32_t* part_idx,
                             int part_cap, DevState* st, cudaStream_t s, int) {
  constexpr int TILE = 32 * Vec16<BT>::N;
  int64_t g = (rows + TILE - 1) / TILE;  // one warp per tile
  if (sizeof(CT) == 8 && g > part_cap) g = part_cap;  // FP64 partials: one per block
  if (g > (1LL << 30)) g = 1LL << 30;
  if (g < 1) g = 1;
  const size_t sm = (size_t)(cnt > 0 ? cnt : 1) * sizeof(CT);
  launch_pdl(k_eliminate_argmax<XT, BT, CT>, dim3((unsigned)g), dim3(32), sm, s, x, B, ld, cnt,
             rows, v, pa, part_val, part_idx, st);
}

template <typename BT>
void launch_init_pivot(const double* r0, int64_t rows, const PivotArgs& pa, DevState* st,
                       cudaStream_t s, int num_sms) {
  const int g = grid_for(rows, num_sms, 4);
  k_r0_max<<<g, kThreads, 0, s>>>(r0, rows, pa.used, pa.tile_prob, st);
  k_r0_argmin<BT><<<g, kThreads, 0, s>>>(r0, rows, pa, st);
}

template <typename CT, typename BT>
void launch_scale(const CT* v, BT* out, int64_t rows, DevState* st, int nprob,
                  const int32_t* tile_prob, cudaStream_t s, int num_sms) {
  const int64_t g = (rows + 4 * kThreads - 1) / (4 * kThreads);
  if (g < 1) return;
  launch_pdl(k_scale<CT, BT>, dim3((unsigned)g), dim3(kThreads), 0, s, v, out, rows, st, nprob,
             tile_prob);
}

void launch_init_state(DevState* st, int nprob, int K, cudaStream_t s) {
  k_init_state<<<1, 256, 0, s>>>(st, nprob, K);
}

void launch_stop_select(const double* res, const double* tr, double* G, int K, double n,
                        double m, double tol, const DevState* st, int32_t* k_stop,
                        cudaStream_t s) {
  k_stop_select<<<1, 256, 0, s>>>(res, tr, G, K, n, m, tol, st, k_stop);
}

void launch_residual0(const double* b, const double* Ax0, double* r0, int64_t m,
                      cudaStream_t s) {
  k_residual0<<<(unsigned)std::min<int64_t>((m + 255) / 256, 4096), 256, 0, s>>>(b, Ax0, r0, m);
}

void launch_scatter(const double* src, const int32_t* map, int64_t count, double* dst,
                    cudaStream_t s) {
  if (count <= 0) return;
  k_scatter<<<(unsigned)std::min<int64_t>((count + 255) / 256, 4096), 256, 0, s>>>(src, map,
                                                                                 count, dst);
}

void launch_gather(const double* src, const int32_t* map, int64_t count, double* dst,
                   cudaStream_t s) {
  if (count <= 0) return;
  k_gather<<<(unsigned)std::min<int64_t>((count + 255) / 256, 4096), 256, 0, s>>>(src, map,
                                                                                count, dst);
}

void launch_gather_rows(const void* src, int64_t lds, const int32_t* map, int64_t rows,
                        int64_t cols, void* dst, int64_t ldd, int elem_bytes, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  const dim3 grid((unsigned)std::min<int64_t>((rows + 255) / 256, 1024),
                  (unsigned)std::min<int64_t>(cols, 4096));
  if (elem_bytes == 8)
    k_gather_rows<double><<<grid, 256, 0, s>>>((const double*)src, lds, map, rows, cols,
                                               (double*)dst, ldd);
  else
    k_gather_rows<float><<<grid, 256, 0, s>>>((const float*)src, lds, map, rows, cols,
                                              (float*)dst, ldd);
}

template <typename BT>
void launch_recombine(const BT* L, int64_t ldl, const double* y, int64_t ldy, const double* x0,
                      double* x, int64_t n, const DevState* st, int nprob,
                      const int32_t* tile_prob, int K, cudaStream_t s, int num_sms) {
  int64_t g = (n + kTile - 1) / kTile;
  if (g > (int64_t)num_sms * 16) g = (int64_t)num_sms * 16;
  k_recombine<BT><<<(unsigned)g, kTile, (size_t)(K > 0 ? K : 1) * 8, s>>>(
      L, ldl, y, ldy, x0, x, n, st, nprob, tile_prob, K);
}

// explicit instantiations: FP64 mode (basis double) and FP32 mode (basis float)
template void launch_eliminate_argmax<double, double, double>(const double*, const double*,
                                                              int64_t, int, int64_t, double*,
                                                              const PivotArgs&, double*,
                                                              int32_t*, int, DevState*,
                                                              cudaStream_t, int);
template void launch_eliminate_argmax<float, float, float>(const float*, const float*, int64_t,
                                                           int, int64_t, float*,
                                                           const PivotArgs&, double*, int32_t*,
                                                           int, DevState*, cudaStream_t, int);
template void launch_init_pivot<double>(const double*, int64_t, const PivotArgs&, DevState*,
                                        cudaStream_t, int);
template void launch_init_pivot<float>(const double*, int64_t, const PivotArgs&, DevState*,
                                       cudaStream_t, int);
template void launch_scale<double, double>(const double*, double*, int64_t, DevState*, int,
                                           const int32_t*, cudaStream_t, int);
template void launch_scale<float, float>(const float*, float*, int64_t, DevState*, int,
                                         const int32_t*, cudaStream_t, int);
template void launch_scale<double, float>(const double*, float*, int64_t, DevState*, int,
                                          const int32_t*, cudaStream_t, int);
template void launch_recombine<double>(const double*, int64_t, const double*, int64_t,
                                       const double*, double*, int64_t, const DevState*, int,
                                       const int32_t*, int, cudaStream_t, int);
template void launch_recombine<float>(const float*, int64_t, const double*, int64_t,
                                      const double*, double*, int64_t, const DevState*, int,
                                      const int32_t*, int, cudaStream_t, int);

}  // namespace lslu
