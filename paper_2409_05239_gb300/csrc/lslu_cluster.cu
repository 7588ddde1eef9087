// Basis loop of Hybrid LSLU (Algorithm 5, basis steps of Algorithm 4) for one
// small problem on one thread-block cluster (lslu_set_loop LSLU_LOOP_CLUSTER).
//
// The cluster's C CTAs (16 where the device allows, else 8) own contiguous
// ranges of the rows of A (m-space) and of A^T (n-space).  Every CTA keeps in
// shared memory a copy of the whole current basis vector (the input of the
// next sparse product), its own rows of the product and of the eliminated
// vector, its own rows of both bases (row-major, so the elimination reads
// them without touching global memory), its own row pointers, and its own
// copies of T_L^-1 and T_D^-1.
// Cross-CTA data moves through distributed shared memory, and the three
// synchronisation points of a half iteration are hardware cluster barriers
// (release / acquire):
//
//   P1  y = A^T d_k (or A l_k) on the CTA's own rows, gathering from its copy
//       of the input vector;                                   cluster barrier
//   P2  coefficients c = T^-1 y(piv): y at the pivot rows read from the owning
//       CTAs; P3  eliminate the own rows, v = y - B c (0 on pivoted rows), and
//       send the CTA's largest |v| (value, rank) to every CTA;  cluster barrier
//   P4  every CTA reduces the C candidates in CTA order (the same pivot
//       everywhere), extends its T^-1, stores b_new = v / pivot on its own rows
//       and writes them into every CTA's copy of the input vector;
//                                                               cluster barrier
//
// The matrix stays in global memory (L2-resident at these sizes); the bases
// are also written there, for the projected solve and lslu_get_state.  The
// cluster's CTAs are co-scheduled by the hardware, so no barrier can wait on a
// CTA that is not running.  Summation orders are fixed (lane groups and
// shuffle trees), so results are bitwise reproducible.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "lslu_internal.cuh"

namespace lslu {

namespace {

namespace cg = cooperative_groups;

constexpr int kCT = 512;             // threads per CTA
constexpr int kCW = kCT / 32;        // warps per CTA
constexpr int kLanesPerRow = 4;      // lanes of one row of a product or an elimination
constexpr int kSumLanes = 8;         // lanes of one coefficient or one new T^-1 entry
constexpr int kRowsPerPass = kCT / kLanesPerRow;
constexpr int kMaxClusterCTAs = 16;

struct ClusterArgs {
  int64_t m, n;
  const int32_t* a_rp;
  const int32_t* a_rl;
  const int32_t* a_col;
  const void* a_val;
  const int32_t* t_rp;
  const int32_t* t_rl;
  const int32_t* t_col;
  const void* t_val;
  const double* r0;
  void* L;
  int64_t ldl;
  void* D;
  int64_t ldd;
  double* H;
  int64_t ldh;
  double* W;
  int64_t ldw;
  void* TLi;
  void* TDi;
  int64_t ldt;
  int32_t* gp;
  int32_t* tp;
  uint8_t* gused;
  uint8_t* tused;
  DevState* st;
  const int32_t* rank_m;
  const int32_t* rank_n;
  const int32_t* unrank_m;
  const int32_t* unrank_n;
  int K;
};

// Pivot candidate as an integer key: hi = bits of |v| (a NaN has larger bits
// than any number, wins and is reported), lo = (2^31 - 1 - rank) << 1 | sign
// of v.  The larger (hi, lo) is the larger |v|, ties to the lowest rank (ranks
// are distinct, so the sign never decides); (0, 0) is no candidate.  Integer
// comparisons keep the reductions off the FP64 pipe.
struct PKey {
  unsigned long long hi;
  unsigned lo;
};
__device__ __forceinline__ bool key_less(const PKey& x, const PKey& y) {
  return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}
template <typename CT>
__device__ __forceinline__ PKey make_key(CT v, int rank) {
  PKey k;
  if constexpr (sizeof(CT) == 8) {
    const unsigned long long b = (unsigned long long)__double_as_longlong((double)v);
    k.hi = b & 0x7fffffffffffffffull;
    k.lo = ((0x7fffffffu - (unsigned)rank) << 1) | (unsigned)(b >> 63);
  } else {
    const unsigned b = __float_as_uint((float)v);
    k.hi = b & 0x7fffffffu;
    k.lo = ((0x7fffffffu - (unsigned)rank) << 1) | (b >> 31);
  }
  return k;
}
template <typename CT>
__device__ __forceinline__ CT key_value(const PKey& k) {
  if constexpr (sizeof(CT) == 8)
    return (CT)__longlong_as_double((long long)(k.hi | ((unsigned long long)(k.lo & 1u) << 63)));
  else
    return (CT)__uint_as_float((unsigned)k.hi | ((k.lo & 1u) << 31));
}
__device__ __forceinline__ int key_rank(const PKey& k) {
  return (int)(0x7fffffffu - (k.lo >> 1));
}
__device__ __forceinline__ PKey warp_max_key(PKey k, unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    PKey x;
    x.hi = __shfl_xor_sync(mask, k.hi, o);
    x.lo = __shfl_xor_sync(mask, k.lo, o);
    if (key_less(k, x)) k = x;
  }
  return k;
}

template <typename VT>
__device__ __forceinline__ double val_at(const VT* p, int64_t i);
template <>
__device__ __forceinline__ double val_at<double>(const double* p, int64_t i) {
  return __ldg(p + i);
}
template <>
__device__ __forceinline__ double val_at<float>(const float* p, int64_t i) {
  return (double)__ldg(p + i);
}
template <>
__device__ __forceinline__ double val_at<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return (double)__bfloat162float(p[i]);
}

// Row range [lo, hi) of CTA c among C over `rows` rows.
__device__ __forceinline__ int64_t range_lo(int64_t rows, int c, int C) {
  return rows * c / C;
}
__device__ __forceinline__ int owner_of(int64_t row, int64_t rows, int C) {
  // largest c with rows * c / C <= row
  int c = (int)(((row + 1) * C - 1) / rows);
  return c < C ? c : C - 1;
}

// Shared-memory layout of one CTA (offsets in bytes).
template <typename CT>
struct CLayout {
  size_t xv, rows_max, yown, vown, rp, rl, used, cs, xs, trow, slots_h, slots_l, gps, tps, tl, td,
      lrows, drows, total;
  int ldr;  // leading dimension of the own basis rows (row-major, columns 0..K)
  int lds;
  __host__ __device__ CLayout(int64_t m, int64_t n, int K, int C) {
    const size_t nmax = (size_t)(m > n ? m : n);
    rows_max = (nmax + C - 1) / C + 1;
    const size_t kc = (size_t)K + 2;
    lds = K + 1 + (((K + 1) & 1) ? 0 : 1);
    size_t o = 0;
    auto take = [&](size_t bytes) {
      const size_t at = o;
      o += (bytes + 15) / 16 * 16;
      return at;
    };
    xv = take(nmax * sizeof(CT));
    yown = take(rows_max * sizeof(CT));
    vown = take(rows_max * sizeof(CT));
    rp = take(2 * rows_max * sizeof(int32_t));  // own rows of A and of A^T
    rl = take(2 * rows_max * sizeof(int32_t));
    used = take(2 * rows_max);
    cs = take(kc * sizeof(CT));
    xs = take(kc * sizeof(CT));
    trow = take(kc * sizeof(CT));
    slots_h = take(kMaxClusterCTAs * sizeof(unsigned long long));
    slots_l = take(kMaxClusterCTAs * sizeof(unsigned));
    gps = take(kc * sizeof(int32_t));
    tps = take(kc * sizeof(int32_t));
    tl = take((size_t)(K + 1) * lds * sizeof(CT));
    td = take((size_t)(K + 1) * lds * sizeof(CT));
    ldr = K + 1 + (((K + 1) & 1) ? 0 : 1);
    lrows = take(rows_max * ldr * sizeof(CT));  // own rows of L (columns 0..K-1)
    drows = take(rows_max * ldr * sizeof(CT));  // own rows of D (columns 0..K)
    total = o;
  }
};

template <typename VT, typename BT, typename CT>
__global__ void __launch_bounds__(kCT, 1) k_cluster_basis(ClusterArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int me = (int)cluster.block_rank();
  const CLayout<CT> lay(a.m, a.n, a.K, C);
  CT* xv = reinterpret_cast<CT*>(smem + lay.xv);
  CT* yown = reinterpret_cast<CT*>(smem + lay.yown);
  CT* vown = reinterpret_cast<CT*>(smem + lay.vown);
  int32_t* rp_s = reinterpret_cast<int32_t*>(smem + lay.rp);
  int32_t* rl_s = reinterpret_cast<int32_t*>(smem + lay.rl);
  uint8_t* used_s = smem + lay.used;
  CT* cs = reinterpret_cast<CT*>(smem + lay.cs);
  CT* xs = reinterpret_cast<CT*>(smem + lay.xs);
  CT* trow = reinterpret_cast<CT*>(smem + lay.trow);
  unsigned long long* slot_h = reinterpret_cast<unsigned long long*>(smem + lay.slots_h);
  unsigned* slot_l = reinterpret_cast<unsigned*>(smem + lay.slots_l);
  CT* lrows = reinterpret_cast<CT*>(smem + lay.lrows);  // own rows of the bases, kept in
  CT* drows = reinterpret_cast<CT*>(smem + lay.drows);  // shared memory (row-major)
  const int ldr = lay.ldr;
  int32_t* gps = reinterpret_cast<int32_t*>(smem + lay.gps);  // pivot lists, the same in
  int32_t* tps = reinterpret_cast<int32_t*>(smem + lay.tps);  // every CTA
  CT* TLs = reinterpret_cast<CT*>(smem + lay.tl);
  CT* TDs = reinterpret_cast<CT*>(smem + lay.td);
  const int lds = lay.lds;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int s_idx;
  __shared__ CT s_piv;

  // own rows: m-space [m0, m1), n-space [n0, n1)
  const int64_t m0 = range_lo(a.m, me, C), m1 = range_lo(a.m, me + 1, C);
  const int64_t n0 = range_lo(a.n, me, C), n1 = range_lo(a.n, me + 1, C);
  const int nm = (int)(m1 - m0), nn = (int)(n1 - n0);
  const size_t rmax = lay.rows_max;
  for (int i = tid; i < nm; i += kCT) {
    rp_s[i] = __ldg(a.a_rp + m0 + i);
    rl_s[i] = __ldg(a.a_rl + m0 + i);
    used_s[i] = 0;
  }
  for (int i = tid; i < nn; i += kCT) {
    rp_s[rmax + i] = __ldg(a.t_rp + n0 + i);
    rl_s[rmax + i] = __ldg(a.t_rl + n0 + i);
    used_s[rmax + i] = 0;
  }
  BT* Lb = reinterpret_cast<BT*>(a.L);
  BT* Db = reinterpret_cast<BT*>(a.D);
  const VT* aval = reinterpret_cast<const VT*>(a.a_val);
  const VT* tval = reinterpret_cast<const VT*>(a.t_val);
  __syncthreads();

  // the CTA's largest key over the keys every thread holds, written into
  // slot `me` of every CTA of the cluster
  __shared__ unsigned long long w_hi[kCW];
  __shared__ unsigned w_lo[kCW];
  auto publish_key = [&](PKey k) {
    k = warp_max_key(k);
    if (lane == 0) {
      w_hi[warp] = k.hi;
      w_lo[warp] = k.lo;
    }
    __syncthreads();
    if (warp == 0) {
      PKey b;
      b.hi = lane < kCW ? w_hi[lane] : 0ull;
      b.lo = lane < kCW ? w_lo[lane] : 0u;
      b = warp_max_key(b);
      if (lane < C) {  // lane q sends the CTA's best to CTA q
        *cluster.map_shared_rank(slot_h + me, lane) = b.hi;
        *cluster.map_shared_rank(slot_l + me, lane) = b.lo;
      }
    }
  };
  // the cluster-wide pivot from the C slots (after a cluster barrier), the
  // same in every CTA: rank into s_idx (-1: none), value into s_piv
  auto resolve_slots = [&]() {
    if (warp == 0) {
      PKey b;
      b.hi = lane < C ? slot_h[lane] : 0ull;
      b.lo = lane < C ? slot_l[lane] : 0u;
      b = warp_max_key(b);
      if (lane == 0) {
        s_idx = (b.hi | b.lo) ? key_rank(b) : -1;
        s_piv = key_value<CT>(b);
      }
    }
    __syncthreads();
  };

  // ---- pivot of r0 (exact, FP64) and d_1 = r0 / beta
  {
    PKey best = {0ull, 0u};
    for (int i = tid; i < nm; i += kCT) {
      if (__ldg(a.tused + m0 + i)) {  // (single problem: nothing is pivoted yet)
        used_s[i] = 1;
        continue;
      }
      const int r = a.rank_m ? __ldg(a.rank_m + m0 + i) : (int)(m0 + i);
      const PKey kk = make_key<double>(__ldg(a.r0 + m0 + i), r);
      if (key_less(best, kk)) best = kk;
    }
    publish_key(best);
    cluster.sync();
    // the exact FP64 pivot of r0 (resolve_slots gives the compute type)
    __shared__ double s_beta;
    if (warp == 0) {
      PKey b;
      b.hi = lane < C ? slot_h[lane] : 0ull;
      b.lo = lane < C ? slot_l[lane] : 0u;
      b = warp_max_key(b);
      if (lane == 0) {
        s_idx = (b.hi | b.lo) ? key_rank(b) : -1;
        s_beta = key_value<double>(b);
      }
    }
    __syncthreads();
    const int rk = s_idx;
    const double beta = s_beta;
    const int idx = rk >= 0 ? (a.unrank_m ? __ldg(a.unrank_m + rk) : rk) : -1;
    if (idx < 0 || beta == 0.0 || !isfinite(beta)) {
      if (me == 0 && tid == 0) {
        a.st[0].status = (idx >= 0 && !isfinite(beta)) ? LSLU_ERR_NONFINITE : LSLU_BREAKDOWN_BETA;
        a.st[0].k_done = 0;
      }
      return;  // every CTA takes the same branch: no barrier is left waiting
    }
    if (me == 0 && tid == 0) {
      a.tp[0] = idx;
      a.st[0].beta = beta;
      a.st[0].pivot = beta;
      reinterpret_cast<CT*>(a.TDi)[0] = (CT)1;
    }
    if (tid == 0) {
      TDs[0] = (CT)1;
      tps[0] = idx;
      if (idx >= m0 && idx < m1) {
        used_s[idx - m0] = 1;
        a.tused[idx] = 1;
      }
    }
    // d_1 on the own rows: the global basis, the own rows of D and every
    // CTA's input copy
    for (int i = tid; i < nm; i += kCT) {
      const BT d = (BT)(__ldg(a.r0 + m0 + i) / beta);
      Db[m0 + i] = d;
      drows[(size_t)i * ldr] = (CT)d;
      for (int q = 0; q < C; ++q) *cluster.map_shared_rank(xv + m0 + i, q) = (CT)d;
    }
    cluster.sync();
  }

  for (int k = 0; k < a.K; ++k) {
    for (int side = 0; side < 2; ++side) {
      // side 0: q = A^T d_k against L (n-space rows); side 1: u = A l_k
      // against D (m-space rows)
      const bool Ls = side == 0;
      const int nr = Ls ? nn : nm;
      const int64_t r0 = Ls ? n0 : m0;
      const int64_t rows = Ls ? a.n : a.m;
      const int32_t* rps = Ls ? rp_s + rmax : rp_s;
      const int32_t* rls = Ls ? rl_s + rmax : rl_s;
      uint8_t* us = Ls ? used_s + rmax : used_s;
      const int32_t* col = Ls ? a.t_col : a.a_col;
      const VT* val = Ls ? tval : aval;
      const int cnt = Ls ? k : k + 1;  // earlier basis vectors of this side
      const int32_t* piv = Ls ? gps : tps;
      CT* brows = Ls ? lrows : drows;  // own rows of this side's basis
      CT* Ts = Ls ? TLs : TDs;
      // ---- P1: own rows of the product, gathering from the input copy
      for (int base = 0; base < nr; base += kRowsPerPass) {
        const int rr = base + tid / kLanesPerRow;
        const int gl = tid & (kLanesPerRow - 1);
        CT acc = 0, acc2 = 0;
        if (rr < nr) {
          const int32_t st = rps[rr], len = rls[rr];
          // eight entries per lane in flight: loads first, then the gathers
          for (int32_t e = gl; e < len; e += 8 * kLanesPerRow) {
            int32_t cc[8];
            CT vv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int32_t q = e + u * kLanesPerRow;
              cc[u] = q < len ? __ldg(col + st + q) : -1;
              vv[u] = q < len ? (CT)val_at<VT>(val, st + q) : (CT)0;
            }
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
              if (cc[u] >= 0) acc = fma(vv[u], xv[cc[u]], acc);
              if (cc[u + 1] >= 0) acc2 = fma(vv[u + 1], xv[cc[u + 1]], acc2);
            }
          }
        }
        acc += acc2;
#pragma unroll
        for (int o = kLanesPerRow / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (rr < nr && gl == 0) yown[rr] = acc;
      }
      cluster.sync();
      // ---- P2: coefficients c = T^-1 y(piv), y at the pivot rows from their owners
      for (int j = tid; j < cnt; j += kCT) {
        const int64_t pr = piv[j];
        const int o = owner_of(pr, rows, C);
        xs[j] = *cluster.map_shared_rank(yown + (pr - range_lo(rows, o, C)), o);
      }
      __syncthreads();
      // (kSumLanes lanes per coefficient, each a strided part of its sum, then
      // a fixed shuffle tree: the dependent FP64 chains are kSumLanes times
      // shorter and spread over the CTA's warps)
      for (int b0 = 0; b0 < cnt; b0 += kCT / kSumLanes) {
        const int i = b0 + tid / kSumLanes, part = tid & (kSumLanes - 1);
        CT sum = 0;
        if (i < cnt)
          for (int j = part; j <= i; j += kSumLanes) sum = fma(Ts[j * lds + i], xs[j], sum);
#pragma unroll
        for (int o = kSumLanes / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (i < cnt && part == 0) cs[i] = sum;
      }
      __syncthreads();
      if (me == 0) {
        double* hess = Ls ? a.W + (int64_t)k * a.ldw : a.H + (int64_t)k * a.ldh;
        for (int j = tid; j < cnt; j += kCT) hess[j] = (double)cs[j];
      }
      // ---- P3: eliminate the own rows (lane group per row, columns split
      // over the group's lanes in a fixed order), then the CTA's best
      PKey best = {0ull, 0u};
      for (int base = 0; base < nr; base += kRowsPerPass) {
        const int rr = base + tid / kLanesPerRow;
        const int gl = tid & (kLanesPerRow - 1);
        CT acc = 0, acc2 = 0;
        if (rr < nr) {
          const CT* bp = brows + (size_t)rr * ldr;
          int j = gl;
          for (; j + kLanesPerRow < cnt; j += 2 * kLanesPerRow) {
            acc = fma(cs[j], bp[j], acc);
            acc2 = fma(cs[j + kLanesPerRow], bp[j + kLanesPerRow], acc2);
          }
          if (j < cnt) acc = fma(cs[j], bp[j], acc);
        }
        acc += acc2;
#pragma unroll
        for (int o = kLanesPerRow / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (rr < nr && gl == 0) {
          const CT v = us[rr] ? (CT)0 : yown[rr] - acc;
          vown[rr] = v;
          if (!us[rr]) {
            const int64_t row = r0 + rr;
            const int rk = Ls ? (a.rank_n ? __ldg(a.rank_n + row) : (int)row)
                              : (a.rank_m ? __ldg(a.rank_m + row) : (int)row);
            const PKey kk = make_key<CT>(v, rk);
            if (key_less(best, kk)) best = kk;
          }
        }
      }
      publish_key(best);
      cluster.sync();
      // ---- P4: the pivot, T^-1, the new basis vector
      resolve_slots();
      const int rk = s_idx;
      const int32_t* unrank = Ls ? a.unrank_n : a.unrank_m;
      const int idx = rk >= 0 ? (unrank ? __ldg(unrank + rk) : rk) : -1;
      const CT pv = s_piv;
      const int slot = cnt;
      if (idx < 0 || pv == (CT)0 || !isfinite((double)pv)) {
        if (me == 0 && tid == 0) {
          a.st[0].status = (idx >= 0 && pv != (CT)0) ? LSLU_ERR_NONFINITE
                                                      : (Ls ? LSLU_BREAKDOWN_W : LSLU_BREAKDOWN_H);
          a.st[0].k_done = k;
        }
        return;  // the same decision in every CTA
      }
      if (me == 0 && tid == 0) {
        if (Ls) {
          a.gp[k] = idx;
          a.W[(int64_t)k * a.ldw + k] = (double)pv;
        } else {
          a.tp[k + 1] = idx;
          a.H[(int64_t)k * a.ldh + k + 1] = (double)pv;
        }
        a.st[0].pivot = (double)pv;
        a.st[0].pivot_f = (float)pv;
      }
      if (tid == 0) {
        (Ls ? gps : tps)[slot] = idx;
        if (idx >= r0 && idx < r0 + nr) {
          us[idx - r0] = 1;
          (Ls ? a.gused : a.tused)[idx] = 1;
        }
      }
      // new row `slot` of T^-1: T(slot, l) = b_l(idx), from the owner's rows
      {
        const int o = owner_of(idx, rows, C);
        const CT* orow =
            cluster.map_shared_rank(brows, o) + (size_t)(idx - range_lo(rows, o, C)) * ldr;
        for (int l = tid; l < slot; l += kCT) trow[l] = orow[l];
      }
      __syncthreads();
      // (kSumLanes lanes per entry j, each a strided part of the sum over
      // l = j .. slot-1, then a fixed shuffle tree; the terms l < j are zero)
      for (int b0 = 0; b0 < slot; b0 += kCT / kSumLanes) {
        const int j = b0 + tid / kSumLanes, part = tid & (kSumLanes - 1);
        CT sum = 0;
        if (j < slot)
          for (int l = j + part; l < slot; l += kSumLanes) sum = fma(trow[l], Ts[j * lds + l], sum);
#pragma unroll
        for (int o = kSumLanes / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (j < slot && part == 0) Ts[j * lds + slot] = -sum;
      }
      if (tid == 0) Ts[slot * lds + slot] = (CT)1;
      __syncthreads();
      if (me == 0) {
        CT* Tg = reinterpret_cast<CT*>(Ls ? a.TLi : a.TDi);
        for (int j = tid; j <= slot; j += kCT) Tg[(int64_t)j * a.ldt + slot] = Ts[j * lds + slot];
      }
      // b_new = v / pivot on the own rows: the global basis (column k of L, or
      // k+1 of D) and every CTA's input copy for the next product
      BT* out = Ls ? Lb + (int64_t)k * a.ldl : Db + (int64_t)(k + 1) * a.ldd;
      const int ocol = Ls ? k : k + 1;
      for (int i = tid; i < nr; i += kCT) {
        const BT b = (BT)(vown[i] / pv);
        out[r0 + i] = b;
        brows[(size_t)i * ldr + ocol] = (CT)b;
        for (int q = 0; q < C; ++q) *cluster.map_shared_rank(xv + r0 + i, q) = (CT)b;
      }
      cluster.sync();
    }
  }
}

// Per device: the cluster size the kernels run with (16 where allowed, else
// 8) and the attributes they need, set once under a mutex.
constexpr int kClusterMaxDevices = 64;
constexpr size_t kClusterSmemCap = 200 * 1024;
int g_cluster_size[kClusterMaxDevices] = {0};
std::mutex g_cluster_mutex;

template <typename VT, typename BT, typename CT>
int setup_typed() {
  auto kern = k_cluster_basis<VT, BT, CT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kClusterSmemCap) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int cand : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cand);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = kClusterSmemCap;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cand;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0)
      return cand;
    cudaGetLastError();
  }
  return 0;
}

template <typename CT>
size_t smem_need(int64_t m, int64_t n, int K, int C) {
  return CLayout<CT>(m, n, K, C).total;
}

}  // namespace

int cluster_loop_setup(int vt) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kClusterMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(g_cluster_mutex);
  // the three instantiations share one size; every one is set up
  const int a = setup_typed<double, double, double>();
  const int b = setup_typed<float, float, float>();
  const int c = setup_typed<__nv_bfloat16, float, float>();
  const int cs = std::min(a, std::min(b, c));
  g_cluster_size[dev] = cs;
  (void)vt;
  return cs;
}

bool cluster_loop_fits(int vt, int64_t m, int64_t n, int K, int C) {
  const size_t need = vt == LSLU_F64 ? smem_need<double>(m, n, K, C) : smem_need<float>(m, n, K, C);
  return C > 0 && need <= kClusterSmemCap;
}

cudaError_t launch_cluster_basis(Ctx* c, const double* r0, int K, int C, cudaStream_t s) {
  ClusterArgs a = {};
  a.m = c->m;
  a.n = c->n;
  a.a_rp = c->A.row_ptr;
  a.a_rl = c->A.row_len;
  a.a_col = c->A.col;
  a.a_val = c->A.val;
  a.t_rp = c->AT.row_ptr;
  a.t_rl = c->AT.row_len;
  a.t_col = c->AT.col;
  a.t_val = c->AT.val;
  a.r0 = r0;
  a.L = c->L;
  a.ldl = c->ldl;
  a.D = c->D;
  a.ldd = c->ldd;
  a.H = c->H;
  a.ldh = c->kmax + 1;
  a.W = c->W;
  a.ldw = c->kmax;
  a.TLi = c->TLi;
  a.TDi = c->TDi;
  a.ldt = c->ldt;
  a.gp = c->gp;
  a.tp = c->tp;
  a.gused = c->gused;
  a.tused = c->tused;
  a.st = c->st;
  a.rank_m = c->rank_m;
  a.rank_n = c->rank_n;
  a.unrank_m = c->rank_m ? c->unrank_m : nullptr;
  a.unrank_n = c->rank_n ? c->unrank_n : nullptr;
  a.K = K;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(kCT);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (c->value_type == LSLU_F64) {
    cfg.dynamicSmemBytes = smem_need<double>(a.m, a.n, K, C);
    return cudaLaunchKernelEx(&cfg, k_cluster_basis<double, double, double>, a);
  }
  cfg.dynamicSmemBytes = smem_need<float>(a.m, a.n, K, C);
  if (c->value_type == LSLU_F32) return cudaLaunchKernelEx(&cfg, k_cluster_basis<float, float, float>, a);
  return cudaLaunchKernelEx(&cfg, k_cluster_basis<__nv_bfloat16, float, float>, a);
}

}  // namespace lslu
