// Persistent basis loop of Hybrid LSLU (Algorithm 5, basis steps of
// Algorithm 4) for latency-bound workloads: one cooperative launch runs the
// pivot of r0 and all K iterations of
//
//   q = A^T d_k;  W(0:k, k) = T_L^-1 q(g);  v = q - L_k W(0:k, k);
//   g_k = argmax |v| (unpivoted rows);  l_k = v / v(g_k);
//   u = A l_k;    H(0:k+1, k) = T_D^-1 u(t);  w = u - D_{k+1} H(0:k+1, k);
//   t_{k+1} = argmax |w|;  d_{k+1} = w / w(t_{k+1})
//
// with grid-wide barriers between the dependent phases instead of six kernel
// launches per iteration.  The coefficients are the sequential elimination of
// Algorithm 4 read at the pivot rows, c = T^-1 x(piv) with the unit lower
// triangular pivot-row matrix T(i, j) = b_j(piv_i) (kept as an explicit
// inverse, as the launched kernels do).
//
// Phases of one iteration and the barrier after each (4 per iteration):
//   S1  q = A^T d_k.  The gather reads the previous eliminated vector w and
//       divides by its pivot on the fly (IEEE division: the same bits as the
//       stored d_k = w / w(t_k)), so d_k need not be complete before the
//       product starts; the block also stores d_k on the rows it owns.
//   E1  every block forms the coefficients of the problems of its rows from
//       q at the pivot rows, eliminates its rows (v = 0 on pivoted rows) and
//       publishes its largest |v|.
//   R1  (no barrier) every block finds the pivot g_k from the published
//       maxima, identically; the block owning the problem's first rows
//       records it, W(k, k) and the new row of T_L^-1.
//   S2, E2, R2: the same for u = A l_k and the D side.
//
// Barriers are counters in global memory with a bounded wait on %globaltimer:
// a block that waits longer than the limit records LSLU_ERR_TIMEOUT, every
// other block leaves at its next barrier, and the host reads the status (the
// context stays usable).  A test-only flag makes the first barrier wait on a
// word that nothing writes.  The launch is cooperative, so every block is
// resident and a barrier can only fail by that limit.
//
// Data written by another block during the kernel is read with plain loads
// after a barrier (its fences order them); only the matrices and r0, constant
// for the whole launch, use the non-coherent read-only path.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "lslu_internal.cuh"

namespace lslu {

namespace {

constexpr int kPT = 256;           // threads per block
constexpr int kSumLanes = 8;       // lanes of one coefficient or one new T^-1 entry
constexpr int kPWarps = kPT / 32;  // warps per block

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}

// Grid barrier; false when the launch must stop (a wait ran out here or in
// another block).  bar[0] counts arrivals and is never reset during a launch
// (the host clears it before every launch): the n-th barrier completes when
// it reaches n * gridDim.x.  Each block's thread 0 arrives with a release
// add, after the block's __syncthreads, and waits with acquire loads, so
// every write made before the barrier by any block is visible to every
// thread after it.  bar[2] is a word nothing writes (the test-only stall
// waits on it).
__device__ bool grid_barrier(unsigned* bar, int* err, unsigned long long limit_ns, bool stall) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned old = atom_add_release(bar, 1u);
    const unsigned target = (old / gridDim.x + 1) * gridDim.x;
    const unsigned* word = stall ? bar + 2 : bar;
    // bounded by the clock, and by a poll count as a second guard (a poll
    // takes well over 64 ns, so the count cannot end a wait early)
    const unsigned long long t0 = global_ns();
    const unsigned long long max_polls = limit_ns / 64 + 1000;
    unsigned long long polls = 0;
    while (stall ? ld_acquire(word) == 0u : (int)(ld_acquire(word) - target) < 0) {
      if (ld_volatile(err)) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > limit_ns || ++polls > max_polls) {
        atomicExch(err, (int)LSLU_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    s_ok = ok && ld_volatile(err) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

struct PersistArgs {
  int64_t m, n;  // rows of A (m-space) and of A^T (n-space), padded totals
  const int32_t* a_rp;
  const int32_t* a_rl;
  const int32_t* a_col;
  const void* a_val;
  const int32_t* t_rp;
  const int32_t* t_rl;
  const int32_t* t_col;
  const void* t_val;
  const double* r0;  // m, FP64
  void* L;
  int64_t ldl;
  void* D;
  int64_t ldd;
  double* H;
  int64_t ldh, h_stride;
  double* W;
  int64_t ldw, w_stride;
  void* TLi;
  void* TDi;
  int64_t ldt, t_stride;
  int32_t* gp;
  int64_t gp_stride;
  int32_t* tp;
  int64_t tp_stride;
  uint8_t* gused;
  uint8_t* tused;
  void* qx;  // n: q = A^T d_k
  void* qv;  // n: eliminated q
  void* ux;  // m: u = A l_k
  void* uv;  // m: eliminated u
  DevState* st;
  int nprob;
  const int32_t* tile_prob_m;  // problem of each kTile rows (null: one problem)
  const int32_t* tile_prob_n;
  const int64_t* row0;  // first m-space row of every problem
  const int64_t* col0;  // first n-space row of every problem
  const int32_t* rank_m;
  const int32_t* rank_n;
  const int32_t* unrank_m;
  const int32_t* unrank_n;
  unsigned long long* keys;  // 2 * nprob pivot keys (FP32), two parities
  double* slot_val;          // gridDim.x partial maxima (FP64, one problem)
  int32_t* slot_idx;
  unsigned* bar;
  int* err;
  int K;
  unsigned long long wait_ns;
  int stall;
};

template <typename VT>
__device__ __forceinline__ void ld_vals4(const VT* p, double (&v)[4]);
template <>
__device__ __forceinline__ void ld_vals4<double>(const double* p, double (&v)[4]) {
  double a0, a1, a2, a3;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(a0), "=d"(a1) : "l"(p));
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
               : "=d"(a2), "=d"(a3)
               : "l"(p + 2));
  v[0] = a0; v[1] = a1; v[2] = a2; v[3] = a3;
}
template <typename VT>
__device__ __forceinline__ void ld_vals4f(const VT* p, float (&v)[4]);
template <>
__device__ __forceinline__ void ld_vals4f<float>(const float* p, float (&v)[4]) {
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
               : "l"(p));
}
template <>
__device__ __forceinline__ void ld_vals4f<__nv_bfloat16>(const __nv_bfloat16* p, float (&v)[4]) {
  uint32_t w0, w1;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(w0), "=r"(w1) : "l"(p));
  v[0] = __uint_as_float(w0 << 16);
  v[1] = __uint_as_float(w0 & 0xffff0000u);
  v[2] = __uint_as_float(w1 << 16);
  v[3] = __uint_as_float(w1 & 0xffff0000u);
}
__device__ __forceinline__ int4 ld_cols4(const int32_t* p) {
  int4 c;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(c.x), "=r"(c.y), "=r"(c.z), "=r"(c.w)
               : "l"(p));
  return c;
}
template <typename VT, typename CT>
__device__ __forceinline__ void ld_vals(const VT* p, CT (&v)[4]) {
  if constexpr (sizeof(CT) == 8) {
    ld_vals4<VT>(p, v);
  } else {
    ld_vals4f<VT>(p, v);
  }
}

__device__ __forceinline__ int prob_of(const int32_t* tile_prob, int64_t row) {
  return tile_prob ? __ldg(tile_prob + row / kTile) : 0;
}

// FP32 pivot key: bits of |v| << 32 | (2^31 - 1 - rank) << 1 | sign of v.
// One unsigned max gives the largest |v| with ties to the lowest rank (ranks
// are distinct, so the sign bit never decides), and the key carries the
// pivot's value itself; a NaN has larger bits than any number, wins and is
// reported.
__device__ __forceinline__ unsigned long long pkey(float v, int r) {
  const unsigned lo = ((0x7fffffffu - (unsigned)r) << 1) | (__float_as_uint(v) >> 31);
  return ((unsigned long long)(__float_as_uint(v) & 0x7fffffffu) << 32) | lo;
}
__device__ __forceinline__ int pkey_rank(unsigned long long k) {
  return (int)(0x7fffffffu - (((unsigned)k >> 1) & 0x7fffffffu));
}
__device__ __forceinline__ float pkey_value(unsigned long long k) {
  return __uint_as_float((unsigned)(k >> 32) | ((unsigned)k << 31));
}

// larger |value| wins, equal |value|: lower rank; rank -1 = no candidate
__device__ __forceinline__ bool better(double va, int ia, double vb, int ib) {
  if (ia < 0) return false;
  if (ib < 0) return true;
  double a = fabs(va), b = fabs(vb);
  if (a != a) a = INFINITY;  // a NaN must win so that it is reported
  if (b != b) b = INFINITY;
  return a > b || (a == b && ia < ib);
}

// One sparse product over all rows of a matrix (16 lanes per row, two rows
// per warp, warps of the whole grid in turn).  The input entry j is
// src(j) / div(problem), rounded to the basis type, computed at the gather.
// Rows of stopped problems are skipped.
template <typename VT, typename BT, typename CT, bool INIT>
__device__ void product_phase(int64_t rows, const int32_t* __restrict__ rp,
                              const int32_t* __restrict__ rl, const int32_t* __restrict__ col,
                              const VT* __restrict__ val, const void* src, const CT* div_tab,
                              const double* beta_tab, const int* stat,
                              const int32_t* tile_prob, CT* out) {
  const int lane = threadIdx.x & 31;
  const int gl = lane & 15;
  const int64_t nwarps = (int64_t)gridDim.x * kPWarps;
  const int64_t gw = (int64_t)blockIdx.x * kPWarps + (threadIdx.x >> 5);
  for (int64_t r0 = 2 * gw; r0 < rows; r0 += 2 * nwarps) {
    const int64_t row = r0 + (lane >> 4);
    const bool valid = row < rows;
    const int p = valid ? prob_of(tile_prob, row) : 0;
    const bool live = valid && stat[p] == LSLU_OK;
    const int32_t start = live ? __ldg(rp + row) : 0;
    const int32_t len = live ? __ldg(rl + row) : 0;
    CT acc = 0;
    if constexpr (INIT) {
      const double bt = live ? beta_tab[p] : 1.0;
      const double* s = reinterpret_cast<const double*>(src);
      for (int32_t e = gl * 4; e < len; e += 64) {
        const int4 c = ld_cols4(col + start + e);
        CT a[4];
        ld_vals<VT, CT>(val + start + e, a);
        const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const CT x = (CT)(BT)(__ldg(s + cc[i]) / bt);
          acc = fma(a[i], x, acc);
        }
      }
    } else {
      const CT dv = live ? div_tab[p] : (CT)1;
      const CT* s = reinterpret_cast<const CT*>(src);
      for (int32_t e = gl * 4; e < len; e += 64) {
        const int4 c = ld_cols4(col + start + e);
        CT a[4];
        ld_vals<VT, CT>(val + start + e, a);
        const int cc[4] = {c.x, c.y, c.z, c.w};
        CT xs[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xs[i] = s[cc[i]];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc = fma(a[i], (CT)(BT)(xs[i] / dv), acc);
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (live && gl == 0) out[row] = acc;
  }
}

// Tiles of the elimination: TILE rows, lane l owns rows l*VEC .. l*VEC+VEC-1
// (16 bytes of the compute type).  Block b owns tiles [b T / G, (b+1) T / G).
template <typename CT>
struct TileGeom {
  static constexpr int VEC = 16 / sizeof(CT);
  static constexpr int TILE = 32 * VEC;
};

__device__ __forceinline__ int64_t tile_begin(int64_t T, int b) {
  return (int64_t)b * T / gridDim.x;
}
__device__ __forceinline__ int tile_owner(int64_t t, int64_t T) {
  const int64_t b = ((t + 1) * (int64_t)gridDim.x - 1) / T;
  return (int)(b < gridDim.x ? b : gridDim.x - 1);
}

// Stores b_new = v / pivot (the scale step) on the rows of the block's tiles.
template <typename BT, typename CT>
__device__ void scale_own_rows(int64_t rows, const CT* v, const CT* div_tab, const int* stat,
                               const int32_t* tile_prob, BT* out) {
  constexpr int TILE = TileGeom<CT>::TILE;
  const int64_t T = (rows + TILE - 1) / TILE;
  const int64_t r_begin = tile_begin(T, blockIdx.x) * TILE;
  const int64_t r_end = min(tile_begin(T, blockIdx.x + 1) * TILE, rows);
  for (int64_t i = r_begin + threadIdx.x; i < r_end; i += kPT) {
    const int p = prob_of(tile_prob, i);
    if (stat[p] != LSLU_OK) continue;
    out[i] = (BT)(v[i] / div_tab[p]);
  }
}

// d_1 = r0 / beta on the block's rows (FP64 division, then the basis type).
template <typename BT, typename CT>
__device__ void scale_own_rows_init(int64_t rows, const double* r0, const double* beta_tab,
                                    const int* stat, const int32_t* tile_prob, BT* out) {
  constexpr int TILE = TileGeom<CT>::TILE;
  const int64_t T = (rows + TILE - 1) / TILE;
  const int64_t r_begin = tile_begin(T, blockIdx.x) * TILE;
  const int64_t r_end = min(tile_begin(T, blockIdx.x + 1) * TILE, rows);
  for (int64_t i = r_begin + threadIdx.x; i < r_end; i += kPT) {
    const int p = prob_of(tile_prob, i);
    if (stat[p] != LSLU_OK) continue;
    out[i] = (BT)(__ldg(r0 + i) / beta_tab[p]);
  }
}

// Side of one half-iteration: the new vector x (n- or m-space), the basis B it
// is eliminated against, its pivot list and mask, T^-1, the Hessenberg column.
template <typename BT, typename CT>
struct Side {
  int64_t rows;
  const CT* x;      // product output
  CT* v;            // eliminated vector
  const BT* B;      // basis, column-major
  int64_t ldb;
  int32_t* piv;     // pivot list of problem 0 (stride piv_stride)
  int64_t piv_stride;
  uint8_t* used;
  CT* Tinv;         // of problem 0 (stride t_stride), column-major ld ldt (global)
  CT* Ts;           // the block's copy of T^-1 (one problem), ld lds; null: use Tinv
  int lds;
  double* hess;     // Hessenberg column of problem 0 (W(:, k) or H(:, k)), stride hess_stride
  int64_t hess_stride;
  const int32_t* tile_prob;
  const int64_t* first_row;  // first row of every problem in this space
  const int32_t* rank;
  const int32_t* unrank;
  int cnt;          // earlier basis vectors (= coefficients)
};

// Coefficients c = T^-1 x(piv) of problem p into cs (every thread of the
// block calls it): x at the pivot rows into xs, then one coefficient per
// thread from the block's shared copy of T^-1, or from global memory.
template <typename BT, typename CT>
__device__ void coefficients(const Side<BT, CT>& sd, const PersistArgs& a, int p, CT* cs,
                             CT* xs) {
  const int cnt = sd.cnt;
  const int32_t* piv = sd.piv + (int64_t)p * sd.piv_stride;
  for (int j = threadIdx.x; j < cnt; j += kPT) xs[j] = sd.x[piv[j]];
  __syncthreads();
  const CT* Ti = sd.Ts ? sd.Ts : sd.Tinv + (int64_t)p * a.t_stride;
  const int64_t ld = sd.Ts ? sd.lds : a.ldt;
  // kSumLanes lanes per coefficient, each a strided part of its sum, then a
  // fixed shuffle tree (short FP64 chains spread over the block's warps)
  for (int b0 = 0; b0 < cnt; b0 += kPT / kSumLanes) {
    const int i = b0 + (int)threadIdx.x / kSumLanes, part = threadIdx.x & (kSumLanes - 1);
    CT sum = 0;
    if (i < cnt)
      for (int j = part; j <= i; j += kSumLanes) sum = fma(Ti[(int64_t)j * ld + i], xs[j], sum);
#pragma unroll
    for (int o = kSumLanes / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (i < cnt && part == 0) cs[i] = sum;
  }
  __syncthreads();
}

// acc += sum_{j in [j0, j1)} c_j b_j on the lane's VEC rows (from bp)
template <typename BT, typename CT, int VEC>
__device__ __forceinline__ void column_sum(const BT* bp, int64_t ldb, const CT* cs, int j0,
                                           int j1, CT (&acc)[VEC]) {
  int j = j0;
  for (; j + 8 <= j1; j += 8) {
    BT b[8][VEC];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if constexpr (VEC == 4) {
        const float4 w = *reinterpret_cast<const float4*>(bp + (int64_t)(j + u) * ldb);
        b[u][0] = w.x; b[u][1] = w.y; b[u][2] = w.z; b[u][3] = w.w;
      } else {
        const double2 w = *reinterpret_cast<const double2*>(bp + (int64_t)(j + u) * ldb);
        b[u][0] = w.x; b[u][1] = w.y;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const CT cu = cs[j + u];
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = fma(cu, (CT)b[u][e], acc[e]);
    }
  }
  for (; j < j1; ++j) {
    const CT cu = cs[j];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = fma(cu, (CT)bp[(int64_t)j * ldb + e], acc[e]);
  }
}

// Masks pivoted rows, stores v and folds the lane's rows into its pivot key
// (FP32) or best (value, rank) (FP64).
template <typename BT, typename CT, int VEC>
__device__ __forceinline__ void finish_rows(const Side<BT, CT>& sd, int64_t i0,
                                            const CT (&val)[VEC], unsigned long long& wkey,
                                            double& best, int& besti) {
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    const int64_t i = i0 + e;
    if (i >= sd.rows) continue;
    CT out = 0;
    if (!sd.used[i]) {
      out = val[e];
      const int r = sd.rank ? __ldg(sd.rank + i) : (int)i;
      if constexpr (sizeof(CT) == 4) {
        const unsigned long long kk = pkey((float)out, r);
        wkey = kk > wkey ? kk : wkey;
      } else {
        if (better((double)out, r, best, besti)) {
          best = (double)out;
          besti = r;
        }
      }
    }
    sd.v[i] = out;
  }
}

// Elimination of the block's tiles with the pivot search: v = x - B c on
// every row of a live problem, 0 on pivoted rows; the block's largest |v|
// per problem goes to keys (FP32) or to its slot (FP64, one problem).  The
// columns are summed in eight ranges, each from zero, and the eight partial
// sums subtracted from x in range order.  A block with at least as many
// tiles of a problem as warps gives each warp whole tiles (the warp runs the
// ranges one after another); with fewer tiles the eight warps take one range
// each of every tile (the dependent chain shrinks eightfold for small
// problems).  Both forms give the same bits, so the result does not depend
// on the block count.
template <typename BT, typename CT>
__device__ void eliminate_phase(const Side<BT, CT>& sd, const PersistArgs& a, const int* stat,
                                CT* cs, CT* xs, CT* part, unsigned long long* keys,
                                bool record_hess) {
  constexpr int VEC = TileGeom<CT>::VEC;
  constexpr int TILE = TileGeom<CT>::TILE;
  constexpr bool kKey = sizeof(CT) == 4;
  __shared__ double s_best[kPWarps];
  __shared__ int s_bi[kPWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t T = (sd.rows + TILE - 1) / TILE;
  const int64_t t0 = tile_begin(T, blockIdx.x), t1 = tile_begin(T, blockIdx.x + 1);
  double best = 0.0;
  int besti = -1;
  int64_t t = t0;
  while (t < t1) {
    const int p = prob_of(sd.tile_prob, t * TILE);
    // the block's tiles of problem p
    int64_t te = t + 1;
    while (te < t1 && prob_of(sd.tile_prob, te * TILE) == p) ++te;
    if (stat[p] == LSLU_OK) {
      coefficients<BT, CT>(sd, a, p, cs, xs);
      const int64_t first_tile = sd.first_row ? sd.first_row[p] / TILE : 0;
      if (record_hess && t == first_tile) {  // the owner of p's first tile records them
        double* h = sd.hess + (int64_t)p * sd.hess_stride;
        for (int j = threadIdx.x; j < sd.cnt; j += kPT) h[j] = (double)cs[j];
      }
      unsigned long long wkey = 0;
      if (te - t >= kPWarps) {
        for (int64_t tt = t + warp; tt < te; tt += kPWarps) {
          const int64_t i0 = tt * TILE + lane * VEC;
          CT val[VEC];
#pragma unroll
          for (int e = 0; e < VEC; ++e) val[e] = (i0 + e < sd.rows) ? sd.x[i0 + e] : (CT)0;
          // the eight column ranges of the split form, in the same order
          for (int w = 0; w < kPWarps; ++w) {
            CT acc[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[e] = 0;
            column_sum<BT, CT, VEC>(sd.B + i0, sd.ldb, cs, (int)((int64_t)w * sd.cnt / kPWarps),
                                    (int)((int64_t)(w + 1) * sd.cnt / kPWarps), acc);
#pragma unroll
            for (int e = 0; e < VEC; ++e) val[e] -= acc[e];
          }
          finish_rows<BT, CT, VEC>(sd, i0, val, wkey, best, besti);
        }
      } else {
        const int j0 = (int)((int64_t)warp * sd.cnt / kPWarps);
        const int j1 = (int)((int64_t)(warp + 1) * sd.cnt / kPWarps);
        for (int64_t tt = t; tt < te; ++tt) {
          const int64_t i0 = tt * TILE + lane * VEC;
          CT acc[VEC];
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[e] = 0;
          column_sum<BT, CT, VEC>(sd.B + i0, sd.ldb, cs, j0, j1, acc);
#pragma unroll
          for (int e = 0; e < VEC; ++e) part[(warp * 32 + lane) * VEC + e] = acc[e];
          __syncthreads();
          if (warp == 0) {
            CT val[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
              val[e] = (i0 + e < sd.rows) ? sd.x[i0 + e] : (CT)0;
              for (int w = 0; w < kPWarps; ++w) val[e] -= part[(w * 32 + lane) * VEC + e];
            }
            finish_rows<BT, CT, VEC>(sd, i0, val, wkey, best, besti);
          }
          __syncthreads();
        }
      }
      if constexpr (kKey) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long ok = __shfl_xor_sync(0xffffffffu, wkey, o);
          wkey = ok > wkey ? ok : wkey;
        }
        if (lane == 0 && wkey) atomicMax(keys + p, wkey);
      }
    }
    t = te;
    __syncthreads();  // cs and xs are reused by the next problem
  }
  if constexpr (!kKey) {
    // one problem: the block's best (value, rank) to its slot, warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
      if (better(ov, oi, best, besti)) {
        best = ov;
        besti = oi;
      }
    }
    if (lane == 0) {
      s_best[warp] = best;
      s_bi[warp] = besti;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bb = 0.0;
      int bi = -1;
      for (int w = 0; w < kPWarps; ++w)
        if (better(s_best[w], s_bi[w], bb, bi)) {
          bb = s_best[w];
          bi = s_bi[w];
        }
      a.slot_val[blockIdx.x] = bb;
      a.slot_idx[blockIdx.x] = bi;
    }
  }
}

// New row `slot` of T^-1 for the pivot row idx: T(slot, l) = b_l(idx),
// Tinv(slot, j) = -sum_{l=j}^{slot-1} T(slot, l) Tinv(l, j), Tinv(slot, slot) = 1,
// into Ti (column-major, leading dimension ld).  Every thread of the block
// calls it; trow is scratch of slot entries.
template <typename BT, typename CT>
__device__ void tinv_new_row(const BT* B, int64_t ldb, int idx, int slot, CT* Ti, int64_t ld,
                             CT* trow) {
  for (int l = threadIdx.x; l < slot; l += kPT) trow[l] = (CT)B[(int64_t)l * ldb + idx];
  __syncthreads();
  // kSumLanes lanes per entry, as in coefficients()
  for (int b0 = 0; b0 < slot; b0 += kPT / kSumLanes) {
    const int j = b0 + (int)threadIdx.x / kSumLanes, part = threadIdx.x & (kSumLanes - 1);
    CT sum = 0;
    if (j < slot)
      for (int l = j + part; l < slot; l += kSumLanes)
        sum = fma(trow[l], Ti[(int64_t)j * ld + l], sum);
#pragma unroll
    for (int o = kSumLanes / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (j < slot && part == 0) Ti[(int64_t)j * ld + slot] = -sum;
  }
  if (threadIdx.x == 0) Ti[(int64_t)slot * ld + slot] = (CT)1;
  __syncthreads();
}

// Pivot of every problem from the published maxima (every block, the same
// result): updates the block's status table and pivot values (and its copy
// of T^-1); the owner of the problem's first tile records the pivot, the
// Hessenberg entry, the status of a breakdown and the new row of T^-1.
template <typename BT, typename CT>
__device__ void resolve_phase(const Side<BT, CT>& sd, const PersistArgs& a, int* stat,
                              CT* piv_tab, const unsigned long long* keys, int bcode, int k_on_bd,
                              CT* trow) {
  constexpr int TILE = TileGeom<CT>::TILE;
  constexpr bool kKey = sizeof(CT) == 4;
  __shared__ int s_idx[1];
  __shared__ double s_val[1];
  const int64_t T = (sd.rows + TILE - 1) / TILE;
  if constexpr (!kKey) {  // one problem: reduce the slots in block order (warp 0)
    if (threadIdx.x < 32) {
      double best = 0.0;
      int besti = -1;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
        const double pv = a.slot_val[b];
        const int pi = a.slot_idx[b];
        if (better(pv, pi, best, besti)) {
          best = pv;
          besti = pi;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
        if (better(ov, oi, best, besti)) {
          best = ov;
          besti = oi;
        }
      }
      if (threadIdx.x == 0) {
        s_idx[0] = besti;
        s_val[0] = best;
      }
    }
    __syncthreads();
  }
  for (int p = 0; p < a.nprob; ++p) {
    if (stat[p] != LSLU_OK) continue;  // uniform across the block
    int idx = -1;
    CT pv = 0;
    if constexpr (kKey) {
      const unsigned long long key = keys[p];
      if (key >> 32) {
        idx = pkey_rank(key);
        idx = sd.unrank ? __ldg(sd.unrank + idx) : idx;
        pv = pkey_value(key);
      }
    } else {
      idx = s_idx[0] >= 0 ? (sd.unrank ? __ldg(sd.unrank + s_idx[0]) : s_idx[0]) : -1;
      pv = (CT)s_val[0];
    }
    const bool owner =
        tile_owner(sd.first_row ? sd.first_row[p] / TILE : 0, T) == (int)blockIdx.x;
    int code = LSLU_OK;
    if (idx < 0 || pv == (CT)0)
      code = bcode;
    else if (!isfinite((double)pv))
      code = LSLU_ERR_NONFINITE;
    if (code != LSLU_OK) {
      __syncthreads();
      if (threadIdx.x == 0) {
        stat[p] = code;
        if (owner) {
          a.st[p].status = code;
          a.st[p].k_done = k_on_bd;
        }
      }
      __syncthreads();
      continue;
    }
    const int slot = sd.cnt;  // the new pivot's index in the list
    if (threadIdx.x == 0) piv_tab[p] = pv;
    if (owner && threadIdx.x == 0) {
      sd.piv[(int64_t)p * sd.piv_stride + slot] = idx;
      sd.used[idx] = 1;
      sd.hess[(int64_t)p * sd.hess_stride + slot] = (double)pv;
      a.st[p].pivot = (double)pv;
      a.st[p].pivot_f = (float)pv;
    }
    CT* Tg = sd.Tinv + (int64_t)p * a.t_stride;
    if (sd.Ts) {
      // every block extends its own copy; the owner also stores the new row
      tinv_new_row<BT, CT>(sd.B, sd.ldb, idx, slot, sd.Ts, sd.lds, trow);
      if (owner)
        for (int j = threadIdx.x; j <= slot; j += kPT)
          Tg[(int64_t)j * a.ldt + slot] = sd.Ts[(int64_t)j * sd.lds + slot];
    } else if (owner) {
      tinv_new_row<BT, CT>(sd.B, sd.ldb, idx, slot, Tg, a.ldt, trow);
    }
    __syncthreads();
  }
}

// Shared memory of the kernel: coefficient, pivot-row and T-row scratch
// (kcap = K + 2 entries each), the column-split partial sums (8 warps x one
// tile), the per-problem tables (pivot values of both sides, beta, status)
// and, with SMT, the block's copies of T_L^-1 and T_D^-1 ((K+1) x lds each).
template <typename CT>
struct SmemLayout {
  size_t kcap, part, ts_ld, ts_elems;
  size_t off_tables, off_beta, off_stat, off_ts, total;
  __host__ __device__ SmemLayout(int K, int nprob, bool smt) {
    kcap = (size_t)K + 2;
    part = (size_t)kPWarps * TileGeom<CT>::TILE;
    ts_ld = (size_t)K + 1 + (((K + 1) & 1) ? 0 : 1);  // odd leading dimension
    ts_elems = smt ? (size_t)(K + 1) * ts_ld : 0;
    off_tables = (3 * kcap + part) * sizeof(CT);
    off_beta = ((off_tables + 2 * (size_t)nprob * sizeof(CT) + 7) / 8) * 8;
    off_stat = off_beta + (size_t)nprob * 8;
    off_ts = ((off_stat + (size_t)nprob * 4 + 15) / 16) * 16;
    total = off_ts + 2 * ts_elems * sizeof(CT);
  }
};

template <typename VT, typename BT, typename CT, bool SMT>
__global__ void __launch_bounds__(kPT, 1) k_persistent_basis(PersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = a.nprob;
  const SmemLayout<CT> lay(a.K, P, SMT);
  CT* cs = reinterpret_cast<CT*>(smem_raw);
  CT* xs = cs + lay.kcap;
  CT* trow = xs + lay.kcap;
  CT* part = trow + lay.kcap;
  CT* piv_l = reinterpret_cast<CT*>(smem_raw + lay.off_tables);
  CT* piv_d = piv_l + P;
  double* beta = reinterpret_cast<double*>(smem_raw + lay.off_beta);
  int* stat = reinterpret_cast<int*>(smem_raw + lay.off_stat);
  CT* TLs = SMT ? reinterpret_cast<CT*>(smem_raw + lay.off_ts) : nullptr;
  CT* TDs = SMT ? TLs + lay.ts_elems : nullptr;
  const int lds = (int)lay.ts_ld;
  for (int p = threadIdx.x; p < P; p += kPT) {
    stat[p] = LSLU_OK;
    piv_l[p] = (CT)1;
    piv_d[p] = (CT)1;
    beta[p] = 1.0;
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < 2 * P; i += kPT) a.keys[i] = 0ull;
  __syncthreads();
  const unsigned long long lim = a.wait_ns;
  bool stall = a.stall != 0;
  auto sync = [&]() -> bool {
    const bool ok = grid_barrier(a.bar, a.err, lim, stall);
    stall = false;
    return ok;
  };
  auto any_live = [&]() -> bool {
    for (int p = 0; p < P; ++p)
      if (stat[p] == LSLU_OK) return true;
    return false;
  };
  BT* Lb = reinterpret_cast<BT*>(a.L);
  BT* Db = reinterpret_cast<BT*>(a.D);
  CT* qx = reinterpret_cast<CT*>(a.qx);
  CT* qv = reinterpret_cast<CT*>(a.qv);
  CT* ux = reinterpret_cast<CT*>(a.ux);
  CT* uv = reinterpret_cast<CT*>(a.uv);
  const VT* aval = reinterpret_cast<const VT*>(a.a_val);
  const VT* tval = reinterpret_cast<const VT*>(a.t_val);
  constexpr int TILE = TileGeom<CT>::TILE;

  // ---- pivot of r0: the largest |r0| (FP64 bits), then the lowest rank
  {
    const int64_t nthreads = (int64_t)gridDim.x * kPT;
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = (int64_t)blockIdx.x * kPT + (threadIdx.x - lane); i0 < a.m; i0 += nthreads) {
      const int64_t i = i0 + lane;
      unsigned long long bits = 0;
      if (i < a.m && !a.tused[i]) {
        const double av = fabs(__ldg(a.r0 + i));
        bits = (unsigned long long)__double_as_longlong(av);
        if (av != av) bits = 0x7ff0000000000001ull;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = ob > bits ? ob : bits;
      }
      // a warp's 32 rows lie in one kTile tile, so in one problem
      if (lane == 0 && bits) atomicMax(&a.st[prob_of(a.tile_prob_m, i0)].amax, bits);
    }
  }
  if (!sync()) goto out;
  for (int64_t i = (int64_t)blockIdx.x * kPT + threadIdx.x; i < a.m;
       i += (int64_t)gridDim.x * kPT) {
    if (a.tused[i]) continue;
    const int p = prob_of(a.tile_prob_m, i);
    const double av = fabs(__ldg(a.r0 + i));
    unsigned long long bits = (unsigned long long)__double_as_longlong(av);
    if (av != av) bits = 0x7ff0000000000001ull;
    const unsigned long long mx = *reinterpret_cast<volatile unsigned long long*>(&a.st[p].amax);
    if (bits && bits == mx) atomicMin(&a.st[p].amin, a.rank_m ? __ldg(a.rank_m + i) : (int)i);
  }
  if (!sync()) goto out;
  {
    const int64_t Tm = (a.m + TILE - 1) / TILE;
    for (int p = 0; p < P; ++p) {
      const unsigned long long mx = *reinterpret_cast<volatile unsigned long long*>(&a.st[p].amax);
      const int rk = *reinterpret_cast<volatile int*>(&a.st[p].amin);
      const bool owner = tile_owner(a.row0 ? a.row0[p] / TILE : 0, Tm) == (int)blockIdx.x;
      int code = LSLU_OK;
      int idx = -1;
      if (mx == 0 || rk == 0x7fffffff) {
        code = LSLU_BREAKDOWN_BETA;
      } else if (mx >= 0x7ff0000000000000ull) {
        code = LSLU_ERR_NONFINITE;
      } else {
        idx = a.unrank_m ? __ldg(a.unrank_m + rk) : rk;
      }
      if (threadIdx.x == 0) {
        if (code != LSLU_OK) {
          stat[p] = code;
          if (owner) {
            a.st[p].status = code;
            a.st[p].k_done = 0;
          }
        } else {
          const double bv = __ldg(a.r0 + idx);
          beta[p] = bv;
          if (owner) {
            a.tp[(int64_t)p * a.tp_stride] = idx;
            a.tused[idx] = 1;
            a.st[p].beta = bv;
            a.st[p].pivot = bv;
            CT* Ti = reinterpret_cast<CT*>(a.TDi) + (int64_t)p * a.t_stride;
            Ti[0] = (CT)1;
          }
        }
      }
    }
    if (SMT && threadIdx.x == 0) TDs[0] = (CT)1;
    __syncthreads();
  }

  for (int k = 0; k < a.K; ++k) {
    if (!any_live()) break;  // every problem stopped (the same in every block)
    // ---- S1: q = A^T d_k; store d_k on the block's rows
    if (k == 0) {
      product_phase<VT, BT, CT, true>(a.n, a.t_rp, a.t_rl, a.t_col, tval, a.r0, piv_d, beta,
                                      stat, a.tile_prob_n, qx);
      scale_own_rows_init<BT, CT>(a.m, a.r0, beta, stat, a.tile_prob_m, Db);
    } else {
      product_phase<VT, BT, CT, false>(a.n, a.t_rp, a.t_rl, a.t_col, tval, uv, piv_d, beta,
                                       stat, a.tile_prob_n, qx);
      scale_own_rows<BT, CT>(a.m, uv, piv_d, stat, a.tile_prob_m, Db + (int64_t)k * a.ldd);
    }
    if (!sync()) goto out;
    // ---- E1: eliminate q against l_0 .. l_{k-1}
    {
      if (blockIdx.x == 0)  // keys of the other parity: everyone read them before the last barrier
        for (int i = threadIdx.x; i < P; i += kPT) a.keys[(int64_t)((2 * k + 1) & 1) * P + i] = 0ull;
      Side<BT, CT> sd{a.n, qx, qv, Lb, a.ldl, a.gp, a.gp_stride, a.gused,
                      reinterpret_cast<CT*>(a.TLi), TLs, lds, a.W + (int64_t)k * a.ldw,
                      a.w_stride, a.tile_prob_n, a.col0, a.rank_n, a.unrank_n, k};
      eliminate_phase<BT, CT>(sd, a, stat, cs, xs, part, a.keys + (int64_t)((2 * k) & 1) * P,
                              true);
      if (!sync()) goto out;
      // ---- R1: pivot g_k, W(k, k), new row of T_L^-1
      resolve_phase<BT, CT>(sd, a, stat, piv_l, a.keys + (int64_t)((2 * k) & 1) * P,
                            LSLU_BREAKDOWN_W, k, trow);
    }
    if (!any_live()) break;
    // ---- S2: u = A l_k; store l_k on the block's rows
    product_phase<VT, BT, CT, false>(a.m, a.a_rp, a.a_rl, a.a_col, aval, qv, piv_l, beta, stat,
                                     a.tile_prob_m, ux);
    scale_own_rows<BT, CT>(a.n, qv, piv_l, stat, a.tile_prob_n, Lb + (int64_t)k * a.ldl);
    if (!sync()) goto out;
    // ---- E2: eliminate u against d_0 .. d_k
    {
      if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < P; i += kPT) a.keys[(int64_t)((2 * k) & 1) * P + i] = 0ull;
      Side<BT, CT> sd{a.m, ux, uv, Db, a.ldd, a.tp, a.tp_stride, a.tused,
                      reinterpret_cast<CT*>(a.TDi), TDs, lds, a.H + (int64_t)k * a.ldh,
                      a.h_stride, a.tile_prob_m, a.row0, a.rank_m, a.unrank_m, k + 1};
      eliminate_phase<BT, CT>(sd, a, stat, cs, xs, part,
                              a.keys + (int64_t)((2 * k + 1) & 1) * P, true);
      if (!sync()) goto out;
      // ---- R2: pivot t_{k+1}, H(k+1, k), new row of T_D^-1
      resolve_phase<BT, CT>(sd, a, stat, piv_d, a.keys + (int64_t)((2 * k + 1) & 1) * P,
                            LSLU_BREAKDOWN_H, k, trow);
    }
    if (k == a.K - 1)  // d_{K+1} on the block's rows
      scale_own_rows<BT, CT>(a.m, uv, piv_d, stat, a.tile_prob_m, Db + (int64_t)a.K * a.ldd);
  }
  return;
out:
  // a barrier wait ran out (here or in another block): the solve stops with
  // LSLU_ERR_TIMEOUT and no completed iteration
  if (threadIdx.x == 0 && ld_volatile(a.err))
    for (int p = 0; p < P; ++p) {
      a.st[p].status = LSLU_ERR_TIMEOUT;
      a.st[p].k_done = 0;
    }
}

// Dynamic shared memory the kernels are set up for (an upper bound; a launch
// asks for what its K and problem count need).
constexpr size_t kPersistSmemCap = 200 * 1024;

template <typename VT, typename BT, typename CT, bool SMT>
cudaError_t launch_typed(const PersistArgs& a, int blocks, size_t smem, cudaStream_t s) {
  auto kern = k_persistent_basis<VT, BT, CT, SMT>;
  if (smem > kPersistSmemCap) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kPT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// Sets one instantiation up on the current device (its shared-memory bound)
// and returns its co-resident block count at the largest shared memory a
// launch may ask for.
template <typename VT, typename BT, typename CT, bool SMT>
int max_resident_one(int num_sms) {
  auto kern = k_persistent_basis<VT, BT, CT, SMT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kPersistSmemCap) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPT, kPersistSmemCap) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * num_sms;
}

template <typename VT, typename BT, typename CT>
int max_resident_typed(int num_sms) {
  return std::min(max_resident_one<VT, BT, CT, false>(num_sms),
                  max_resident_one<VT, BT, CT, true>(num_sms));
}

template <typename CT>
size_t smem_bytes(int K, int nprob, bool smt) {
  return SmemLayout<CT>(K, nprob, smt).total;
}

// The block keeps its own T^-1 copies when one problem's two fit.
template <typename CT>
bool use_smem_tinv(int K, int nprob) {
  return nprob == 1 && smem_bytes<CT>(K, nprob, true) <= kPersistSmemCap;
}

}  // namespace

int persistent_max_blocks(int vt, int K, int nprob, int num_sms) {
  const size_t need = vt == LSLU_F64 ? smem_bytes<double>(K, nprob, false)
                                     : smem_bytes<float>(K, nprob, false);
  if (need > kPersistSmemCap) return 0;
  if (vt == LSLU_F64) return max_resident_typed<double, double, double>(num_sms);
  if (vt == LSLU_F32) return max_resident_typed<float, float, float>(num_sms);
  return max_resident_typed<__nv_bfloat16, float, float>(num_sms);
}

cudaError_t launch_persistent_basis(Ctx* c, const double* r0, int K, int blocks,
                                    unsigned long long wait_ns, int stall, cudaStream_t s) {
  PersistArgs a = {};
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
  a.h_stride = c->h_stride;
  a.W = c->W;
  a.ldw = c->kmax;
  a.w_stride = c->w_stride;
  a.TLi = c->TLi;
  a.TDi = c->TDi;
  a.ldt = c->ldt;
  a.t_stride = c->t_stride;
  a.gp = c->gp;
  a.gp_stride = c->kmax;
  a.tp = c->tp;
  a.tp_stride = c->kmax + 1;
  a.gused = c->gused;
  a.tused = c->tused;
  a.qx = c->q;
  a.qv = c->pq_v;
  a.ux = c->u;
  a.uv = c->pq_w;
  a.st = c->st;
  a.nprob = c->nprob;
  a.tile_prob_m = c->tile_prob_m;
  a.tile_prob_n = c->tile_prob_n;
  a.row0 = c->nprob > 1 ? c->pq_row0 : nullptr;
  a.col0 = c->nprob > 1 ? c->pq_col0 : nullptr;
  a.rank_m = c->rank_m;
  a.rank_n = c->rank_n;
  a.unrank_m = c->rank_m ? c->unrank_m : nullptr;
  a.unrank_n = c->rank_n ? c->unrank_n : nullptr;
  a.keys = c->pq_keys;
  a.slot_val = c->pq_slot_val;
  a.slot_idx = c->pq_slot_idx;
  a.bar = c->pq_bar;
  a.err = c->pq_err;
  a.K = K;
  a.wait_ns = wait_ns;
  a.stall = stall;
  if (c->value_type == LSLU_F64) {
    const bool smt = use_smem_tinv<double>(K, c->nprob);
    const size_t smem = smem_bytes<double>(K, c->nprob, smt);
    return smt ? launch_typed<double, double, double, true>(a, blocks, smem, s)
               : launch_typed<double, double, double, false>(a, blocks, smem, s);
  }
  const bool smt = use_smem_tinv<float>(K, c->nprob);
  const size_t smem = smem_bytes<float>(K, c->nprob, smt);
  if (c->value_type == LSLU_F32)
    return smt ? launch_typed<float, float, float, true>(a, blocks, smem, s)
               : launch_typed<float, float, float, false>(a, blocks, smem, s);
  return smt ? launch_typed<__nv_bfloat16, float, float, true>(a, blocks, smem, s)
             : launch_typed<__nv_bfloat16, float, float, false>(a, blocks, smem, s);
}

}  // namespace lslu
