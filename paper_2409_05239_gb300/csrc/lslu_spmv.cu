// Sparse products of Algorithm 4: u = A l_k and q = A^T d_k.
//
// Both run on a row-major CSR: A^T is stored as its own (transposed) CSR, so
// every output entry is one row dot product and no atomics are needed.  A
// group of 16 lanes (half a warp) owns one row; lane j of the group reads the
// 4-entry chunks j, j+16, j+32, ... of the row with vector loads (rows are
// padded to a multiple of kRowAlign entries), two chunks per step so that
// more loads are in flight, keeps a private partial sum in chunk order, and
// the group adds its 16 partials with a fixed butterfly, so results are
// bitwise reproducible run to run.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lslu_internal.cuh"

namespace lslu {

namespace {

// Lanes per row and chunks per step; kMinBlocks bounds the registers so that
// that many 256-thread blocks stay resident per SM.
constexpr int kGroup = 16;
constexpr int kRowsPerBlock = 256 / kGroup;
template <typename VT>
struct ValTraits;
template <>
struct ValTraits<double> {
  static constexpr int kChunk = 4;  // entries per chunk
  static constexpr int kUnroll = 1;
  static constexpr int kMinBlocks = 6;
};
template <>
struct ValTraits<float> {
  static constexpr int kChunk = 4;
  static constexpr int kUnroll = 2;
  static constexpr int kMinBlocks = 6;
};
template <>
struct ValTraits<__nv_bfloat16> {
  static constexpr int kChunk = 4;
  static constexpr int kUnroll = 2;
  static constexpr int kMinBlocks = 6;
};

template <typename AT>
__device__ __forceinline__ AT warp_sum(AT v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over each group of kGroup lanes (every lane of the warp must call it).
template <typename AT>
__device__ __forceinline__ AT group_sum(AT v) {
#pragma unroll
  for (int o = kGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Matrix stream: 16-byte loads through the non-coherent path without L1
// allocation (ld.global.nc.L1::no_allocate), so L1 keeps the gathered x.
__device__ __forceinline__ int4 ld_stream(const int32_t* p) {
  int4 c;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(c.x), "=r"(c.y), "=r"(c.z), "=r"(c.w)
               : "l"(p));
  return c;
}
template <typename AT>
__device__ __forceinline__ void load_vals_cs(const double* p, AT (&v)[4]) {
  double a0, a1, a2, a3;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(a0), "=d"(a1) : "l"(p));
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
               : "=d"(a2), "=d"(a3)
               : "l"(p + 2));
  v[0] = (AT)a0; v[1] = (AT)a1; v[2] = (AT)a2; v[3] = (AT)a3;
}
template <typename AT>
__device__ __forceinline__ void load_vals_cs(const float* p, AT (&v)[4]) {
  float a0, a1, a2, a3;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(a0), "=f"(a1), "=f"(a2), "=f"(a3)
               : "l"(p));
  v[0] = (AT)a0; v[1] = (AT)a1; v[2] = (AT)a2; v[3] = (AT)a3;
}
template <typename AT>
__device__ __forceinline__ void load_vals_cs(const __nv_bfloat16* p, AT (&v)[4]) {
  uint32_t w[2];
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];"
               : "=r"(w[0]), "=r"(w[1])
               : "l"(p));
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    v[2 * i] = (AT)__uint_as_float(w[i] << 16);
    v[2 * i + 1] = (AT)__uint_as_float(w[i] & 0xffff0000u);
  }
}

// Dot product of one CSR row with x, computed by one group of kGroup lanes
// (result in every lane of the group; gl = lane index within the group; a
// lane with len = 0 contributes nothing).  Lane gl takes chunks gl, gl+16,
// ... in order (kUnroll chunks per step); the 16 partial sums are combined by
// a fixed butterfly, so a row always gets the same bits.  Every lane of the
// warp must call it (the butterfly is a full-warp shuffle).
template <typename VT, typename XT, typename YT>
__device__ __forceinline__ YT row_dot_len(int32_t start, int32_t len,
                                          const int32_t* __restrict__ col,
                                          const VT* __restrict__ val, const XT* __restrict__ x,
                                          int gl) {
  constexpr int C = ValTraits<VT>::kChunk;
  constexpr int U = ValTraits<VT>::kUnroll;
  constexpr int S = kGroup * C;  // entries between a lane's consecutive chunks
  YT acc = 0;
  for (int32_t e = gl * C; e < len; e += U * S) {
    int32_t cidx[U][C];
    YT v[U][C];
    bool has[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      has[u] = u == 0 || e + u * S < len;
      if (has[u]) {
        const int4 c4 = ld_stream(col + start + e + u * S);
        cidx[u][0] = c4.x; cidx[u][1] = c4.y; cidx[u][2] = c4.z; cidx[u][3] = c4.w;
        load_vals_cs<YT>(val + start + e + u * S, v[u]);
      } else {
#pragma unroll
        for (int i = 0; i < C; ++i) v[u][i] = 0;
      }
    }
    XT xv[U][C];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int i = 0; i < C; ++i) xv[u][i] = has[u] ? __ldg(x + cidx[u][i]) : (XT)0;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int i = 0; i < C; ++i) acc = fma(v[u][i], (YT)xv[u][i], acc);
  }
  return group_sum(acc);
}

template <typename VT, typename XT, typename YT>
__device__ __forceinline__ YT row_dot(int64_t row, bool valid, const int32_t* __restrict__ rp,
                                      const int32_t* __restrict__ rl,
                                      const int32_t* __restrict__ col,
                                      const VT* __restrict__ val, const XT* __restrict__ x,
                                      int gl) {
  const int32_t start = valid ? __ldg(rp + row) : 0;
  const int32_t len = valid ? __ldg(rl + row) : 0;
  return row_dot_len<VT, XT, YT>(start, len, col, val, x, gl);
}

template <typename VT, typename XT, typename YT>
__global__ void __launch_bounds__(256, ValTraits<VT>::kMinBlocks)
    k_spmv(int64_t rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ rl,
           const int32_t* __restrict__ col, const VT* __restrict__ val, const XT* __restrict__ x,
           YT* __restrict__ y) {
  const int gl = threadIdx.x & (kGroup - 1);
  const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x / kGroup;
  if ((int64_t)blockIdx.x * kRowsPerBlock + (threadIdx.x & ~31) / kGroup >= rows)
    return;  // the whole warp is past the last row
  const bool valid = row < rows;
  const YT acc = row_dot<VT, XT, YT>(row, valid, rp, rl, col, val, x, gl);
  if (valid && gl == 0) y[row] = acc;
}

// y = A x plus the elimination coefficients of the next Hessenberg step,
// c = T^-1 y(piv), where T(i,j) = b_j(piv_i) is the unit lower triangular
// pivot-row matrix of the basis b and T^-1 is kept explicitly (column-major,
// accumulation type).  |T| <= 1 under max-abs pivoting keeps
// T^-1 small and well conditioned, so every coefficient becomes a plain
// dot product instead of a step of a sequential forward substitution.
//
// The first npiv blocks own the pivot columns, one warp per column j:
//   a. completes the newest row of T^-1 in its column,
//      Tinv(nr, j) = -sum_{l=j}^{nr-1} T(nr, l) Tinv(l, j),  nr = cnt-1;
//   b. computes y(piv_j) with the same warp reduction as every other row
//      (so the two agree bit for bit);
//   c. the block adds Tinv(i, j) y(piv_j) over its 8 columns into a partial
//      vector; the last pivot block to finish adds the partials in block order.
// The remaining blocks compute the other rows of y meanwhile.
// Pivot blocks (steps a-c above) for problem p = blockIdx.x / npiv_blocks;
// rowdot(p, row, gl) is the product of the output row `row` for problem p,
// computed exactly as the streaming blocks compute it.
template <typename YT, typename RowDot>
__device__ __forceinline__ void pivot_blocks(const PivotCoef& pc, RowDot rowdot) {
  __shared__ int last;
  __shared__ YT xs[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = blockIdx.x / pc.npiv_blocks;  // problem of this pivot block
  const int bb = blockIdx.x - p * pc.npiv_blocks;
  DevState& sp = pc.st[p];
  if (sp.status != LSLU_OK) return;
  YT* Tinv = reinterpret_cast<YT*>(pc.Tinv) + (int64_t)p * pc.tinv_stride;
  YT* part = reinterpret_cast<YT*>(pc.xp) + (int64_t)p * pc.xp_stride;
  const int32_t* piv = pc.piv + (int64_t)p * pc.piv_stride;
  const int cnt = pc.cnt, nr = cnt - 1;
  const int j0 = bb * 8;
  const int j = j0 + warp;
  if (j < cnt) {
    if (j < nr) {
      YT a = 0;
      // T(nr, l) = b_l(piv_nr): the newest pivot row of the earlier basis vectors
      const YT* brow = reinterpret_cast<const YT*>(pc.B) + piv[nr];
      const YT* tcol = Tinv + (int64_t)j * pc.ldi;
      for (int l = j + lane; l < nr; l += 32)
        a = fma(__ldcg(brow + (int64_t)l * pc.ldb), __ldcg(tcol + l), a);
      a = warp_sum(a);
      if (lane == 0) __stcg(Tinv + (int64_t)j * pc.ldi + nr, -a);
    }
    // both half-warps compute the pivot row (the same bits as its y entry)
    const YT yp = rowdot(p, piv[j], lane & (kGroup - 1));
    if (lane == 0) xs[warp] = yp;
  } else if (lane == 0) {
    xs[warp] = 0;
  }
  __threadfence_block();
  __syncthreads();
  const int jn = min(8, cnt - j0);
  for (int i = j0 + threadIdx.x; i < cnt; i += blockDim.x) {
    YT acc = 0;
    for (int w = 0; w < jn; ++w)
      if (i >= j0 + w) acc = fma(__ldcg(Tinv + (int64_t)(j0 + w) * pc.ldi + i), xs[w], acc);
    __stcg(part + (int64_t)bb * pc.ldi + i, acc);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&sp.ticket2, 1) == pc.npiv_blocks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) sp.ticket2 = 0;
  double* coef = pc.coef + (int64_t)p * pc.coef_stride;
  double* hess = pc.hess_col ? pc.hess_col + (int64_t)p * pc.hess_stride : nullptr;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    YT acc = 0;
    const int bmax = i / 8;  // blocks whose columns start at or before row i
    for (int b2 = 0; b2 <= bmax; ++b2) acc += __ldcg(part + (int64_t)b2 * pc.ldi + i);
    coef[i] = (double)acc;
    if (hess) hess[i] = (double)acc;
  }
}

template <typename VT, typename XT, typename YT>
__global__ void __launch_bounds__(256, ValTraits<VT>::kMinBlocks)
    k_spmv_pivots(int64_t rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ rl,
                  const int32_t* __restrict__ col, const VT* __restrict__ val,
                  const XT* __restrict__ x, YT* __restrict__ y, PivotCoef pc) {
  const int lane = threadIdx.x & 31;
  const int npiv_all = pc.npiv_blocks * pc.nprob;
  if ((int)blockIdx.x < npiv_all) {
    pivot_blocks<YT>(pc, [=](int, int32_t row, int gl) {
      return row_dot<VT, XT, YT>(row, true, rp, rl, col, val, x, gl);
    });
    return;
  }
  const int64_t b0 = (int64_t)(blockIdx.x - npiv_all) * kRowsPerBlock;
  if (b0 + (threadIdx.x & ~31) / kGroup >= rows) return;  // whole warp past the end
  const int64_t row = b0 + threadIdx.x / kGroup;
  const bool valid = row < rows;
  const YT acc = row_dot<VT, XT, YT>(row, valid, rp, rl, col, val, x, lane & (kGroup - 1));
  if (valid && (lane & (kGroup - 1)) == 0) y[row] = acc;
}

// ---- several right-hand sides sharing one matrix ---------------------------
// The R input vectors are first interleaved, xi[j * RS + r] (RS = R rounded
// up to 4, zero-padded), so each non-zero fetches all R values with RS/4
// 16-byte loads and the matrix is read once for all R products.  Lane gl of a
// row's 16-lane group takes the same chunks in the same order as row_dot_len,
// and each right-hand side keeps its own accumulator, so every output equals
// the single-vector product bit for bit.

// Product of CSR row `row` with right-hand side r of the interleaved xi.
template <typename VT, int RS>
__device__ __forceinline__ float row_dot_rhs(int64_t row, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ rl,
                                             const int32_t* __restrict__ col,
                                             const VT* __restrict__ val,
                                             const float* __restrict__ xi, int r, int gl) {
  constexpr int C = ValTraits<VT>::kChunk;
  constexpr int S = kGroup * C;
  const int32_t start = __ldg(rp + row), len = __ldg(rl + row);
  float acc = 0.f;
  for (int32_t e = gl * C; e < len; e += S) {
    const int4 c4 = ld_stream(col + start + e);
    float v[C];
    load_vals_cs<float>(val + start + e, v);
    acc = fmaf(v[0], __ldg(xi + (int64_t)c4.x * RS + r), acc);
    acc = fmaf(v[1], __ldg(xi + (int64_t)c4.y * RS + r), acc);
    acc = fmaf(v[2], __ldg(xi + (int64_t)c4.z * RS + r), acc);
    acc = fmaf(v[3], __ldg(xi + (int64_t)c4.w * RS + r), acc);
  }
  return group_sum(acc);
}

template <int RS>
__device__ __forceinline__ void gather_rhs(const float* __restrict__ xi, int32_t c, float (&xv)[RS]) {
  const float4* p = reinterpret_cast<const float4*>(xi + (int64_t)c * RS);
#pragma unroll
  for (int q = 0; q < RS / 4; ++q) {
    const float4 t = __ldg(p + q);
    xv[4 * q] = t.x; xv[4 * q + 1] = t.y; xv[4 * q + 2] = t.z; xv[4 * q + 3] = t.w;
  }
}

// y[r * ystride + row] = (A xi_r)(row) for r < R, rows of the shared CSR;
// pivot blocks as in k_spmv_pivots, with output rows of problem p at
// p * ystride + row.
template <typename VT, int RS>
__global__ void __launch_bounds__(256, 4)
    k_spmm_pivots(int64_t rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ rl,
                  const int32_t* __restrict__ col, const VT* __restrict__ val,
                  const float* __restrict__ xi, float* __restrict__ y, int64_t ystride, int R,
                  PivotCoef pc) {
  constexpr int C = ValTraits<VT>::kChunk;
  constexpr int S = kGroup * C;
  const int lane = threadIdx.x & 31;
  const int npiv_all = pc.npiv_blocks * pc.nprob;
  if ((int)blockIdx.x < npiv_all) {
    pivot_blocks<float>(pc, [=](int p, int32_t row, int gl) {
      return row_dot_rhs<VT, RS>((int64_t)row - (int64_t)p * ystride, rp, rl, col, val, xi, p,
                                 gl);
    });
    return;
  }
  const int64_t b0 = (int64_t)(blockIdx.x - npiv_all) * kRowsPerBlock;
  if (b0 + (threadIdx.x & ~31) / kGroup >= rows) return;  // whole warp past the end
  const int64_t row = b0 + threadIdx.x / kGroup;
  const bool valid = row < rows;
  const int gl = lane & (kGroup - 1);
  const int32_t start = valid ? __ldg(rp + row) : 0;
  const int32_t len = valid ? __ldg(rl + row) : 0;
  float acc[RS];
#pragma unroll
  for (int r = 0; r < RS; ++r) acc[r] = 0.f;
  for (int32_t e = gl * C; e < len; e += S) {
    const int4 c4 = ld_stream(col + start + e);
    float v[C];
    load_vals_cs<float>(val + start + e, v);
    const int32_t cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
    for (int i = 0; i < C; ++i) {
      float xv[RS];
      gather_rhs<RS>(xi, cs[i], xv);
#pragma unroll
      for (int r = 0; r < RS; ++r) acc[r] = fmaf(v[i], xv[r], acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < RS; ++r) acc[r] = group_sum(acc[r]);
  if (valid) {
#pragma unroll
    for (int r = 0; r < RS; ++r)
      if (r == gl && r < R) y[(int64_t)r * ystride + row] = acc[r];
  }
}

// xi[j * RS + r] = x[r * xstride + j] (r < R), 0 for R <= r < RS.
template <int RS>
__global__ void k_interleave(const float* __restrict__ x, int64_t xstride, int64_t count, int R,
                             float* __restrict__ xi) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
       j += (int64_t)gridDim.x * blockDim.x) {
    float4* o = reinterpret_cast<float4*>(xi + j * RS);
#pragma unroll
    for (int q = 0; q < RS / 4; ++q) {
      float t[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 4 * q + e;
        t[e] = r < R ? x[(int64_t)r * xstride + j] : 0.f;
      }
      o[q] = make_float4(t[0], t[1], t[2], t[3]);
    }
  }
}

template <typename VT, typename XT, typename YT>
void spmv_typed(const DevCsr& A, const XT* x, YT* y, cudaStream_t s) {
  if (A.rows == 0) return;
  const int64_t blocks = (A.rows + kRowsPerBlock - 1) / kRowsPerBlock;
  k_spmv<VT, XT, YT><<<(unsigned)blocks, 256, 0, s>>>(
      A.rows, A.row_ptr, A.row_len, A.col, reinterpret_cast<const VT*>(A.val), x, y);
}

template <typename VT, typename XT, typename YT>
void spmv_pivots_typed(const DevCsr& A, const XT* x, YT* y, const PivotCoef& pc, cudaStream_t s) {
  const int64_t blocks =
      (int64_t)pc.npiv_blocks * pc.nprob + (A.rows + kRowsPerBlock - 1) / kRowsPerBlock;
  k_spmv_pivots<VT, XT, YT><<<(unsigned)blocks, 256, 0, s>>>(
      A.rows, A.row_ptr, A.row_len, A.col, reinterpret_cast<const VT*>(A.val), x, y, pc);
}

uint16_t f32_to_bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  return (uint16_t)((u + 0x7fffu + lsb) >> 16);
}

// Host-side construction of the padded CSR (values converted to the storage
// type): rows start on multiples of kRowAlign; pad entries repeat the last
// column of their row with value 0.
cudaError_t upload_padded(int64_t rows, int64_t cols, const std::vector<int64_t>& rp,
                          const std::vector<int32_t>& ci, const std::vector<double>& vv, int vt,
                          DevCsr* out, cudaStream_t s) {
  std::vector<int32_t> prp(rows + 1), prl(rows);
  int64_t tot = 0;
  for (int64_t r = 0; r < rows; ++r) {
    const int64_t len = rp[r + 1] - rp[r];
    const int64_t plen = (len + kRowAlign - 1) / kRowAlign * kRowAlign;
    prp[r] = (int32_t)tot;
    prl[r] = (int32_t)plen;
    tot += plen;
    if (tot >= (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  }
  prp[rows] = (int32_t)tot;
  std::vector<int32_t> pc((size_t)tot);
  std::vector<double> pv((size_t)tot);
  for (int64_t r = 0; r < rows; ++r) {
    const int64_t a = rp[r], len = rp[r + 1] - rp[r];
    int32_t* dc = pc.data() + prp[r];
    double* dv = pv.data() + prp[r];
    for (int64_t e = 0; e < len; ++e) {
      dc[e] = ci[a + e];
      dv[e] = vv[a + e];
    }
    for (int64_t e = len; e < prl[r]; ++e) {
      dc[e] = len ? ci[a + len - 1] : 0;
      dv[e] = 0.0;
    }
  }
  out->rows = rows;
  out->cols = cols;
  out->nnz = rp[rows];
  out->nnz_padded = tot;
  size_t vbytes = vt == LSLU_F64 ? 8 : (vt == LSLU_F32 ? 4 : 2);
  cudaError_t e;
  if ((e = cudaMalloc(&out->row_ptr, (rows + 1) * sizeof(int32_t))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&out->row_len, std::max<int64_t>(rows, 1) * sizeof(int32_t))) != cudaSuccess)
    return e;
  if ((e = cudaMalloc(&out->col, std::max<int64_t>(tot, kRowAlign) * sizeof(int32_t))) !=
      cudaSuccess)
    return e;
  if ((e = cudaMalloc(&out->val, std::max<int64_t>(tot, kRowAlign) * vbytes)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(out->row_ptr, prp.data(), (rows + 1) * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if (rows && (e = cudaMemcpyAsync(out->row_len, prl.data(), rows * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if (tot && (e = cudaMemcpyAsync(out->col, pc.data(), tot * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if (tot) {
    if (vt == LSLU_F64) {
      e = cudaMemcpyAsync(out->val, pv.data(), tot * 8, cudaMemcpyHostToDevice, s);
    } else if (vt == LSLU_F32) {
      std::vector<float> f((size_t)tot);
      for (int64_t i = 0; i < tot; ++i) f[i] = (float)pv[i];
      e = cudaMemcpyAsync(out->val, f.data(), tot * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    } else {
      std::vector<uint16_t> h((size_t)tot);
      for (int64_t i = 0; i < tot; ++i) h[i] = f32_to_bf16_rne((float)pv[i]);
      e = cudaMemcpyAsync(out->val, h.data(), tot * 2, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaStreamSynchronize(s);
}

}  // namespace

cudaError_t build_csr_pair(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                           const double* vv, int vt, DevCsr* A, DevCsr* AT, cudaStream_t s) {
  const int64_t nnz = rp[m];
  std::vector<int64_t> rpa(rp, rp + m + 1);
  std::vector<int32_t> cia(ci, ci + nnz);
  std::vector<double> va(vv, vv + nnz);
  cudaError_t e = upload_padded(m, n, rpa, cia, va, vt, A, s);
  if (e != cudaSuccess) return e;
  // stable counting sort by column: rows of A^T list the rows of A in
  // increasing order (entries of one row of A keep their input order)
  std::vector<int64_t> rpt(n + 1, 0);
  for (int64_t i = 0; i < nnz; ++i) rpt[cia[i] + 1]++;
  for (int64_t c = 0; c < n; ++c) rpt[c + 1] += rpt[c];
  std::vector<int64_t> cur(rpt.begin(), rpt.end() - 1);
  std::vector<int32_t> cit((size_t)nnz);
  std::vector<double> vt_((size_t)nnz);
  for (int64_t r = 0; r < m; ++r)
    for (int64_t i = rpa[r]; i < rpa[r + 1]; ++i) {
      const int64_t pos = cur[cia[i]]++;
      cit[pos] = (int32_t)r;
      vt_[pos] = va[i];
    }
  return upload_padded(n, m, rpt, cit, vt_, vt, AT, s);
}

void free_csr(DevCsr* c) {
  cudaFree(c->row_ptr);
  cudaFree(c->row_len);
  cudaFree(c->col);
  cudaFree(c->val);
  *c = DevCsr();
}

template <typename XT, typename YT>
void launch_spmv(const DevCsr& A, int vt, const XT* x, YT* y, cudaStream_t s, int) {
  if (vt == LSLU_F64)
    spmv_typed<double, XT, YT>(A, x, y, s);
  else if (vt == LSLU_F32)
    spmv_typed<float, XT, YT>(A, x, y, s);
  else
    spmv_typed<__nv_bfloat16, XT, YT>(A, x, y, s);
}

template <typename XT, typename YT>
void launch_spmv_pivots(const DevCsr& A, int vt, const XT* x, YT* y, PivotCoef pc,
                        cudaStream_t s) {
  pc.npiv_blocks = (pc.cnt + 7) / 8;
  if (vt == LSLU_F64)
    spmv_pivots_typed<double, XT, YT>(A, x, y, pc, s);
  else if (vt == LSLU_F32)
    spmv_pivots_typed<float, XT, YT>(A, x, y, pc, s);
  else
    spmv_pivots_typed<__nv_bfloat16, XT, YT>(A, x, y, pc, s);
}

template <typename VT, int RS>
void spmm_typed(const DevCsr& A, const float* xi, float* y, int64_t ystride, int R,
                const PivotCoef& pc, cudaStream_t s) {
  const int64_t blocks =
      (int64_t)pc.npiv_blocks * pc.nprob + (A.rows + kRowsPerBlock - 1) / kRowsPerBlock;
  k_spmm_pivots<VT, RS><<<(unsigned)blocks, 256, 0, s>>>(
      A.rows, A.row_ptr, A.row_len, A.col, reinterpret_cast<const VT*>(A.val), xi, y, ystride, R,
      pc);
}

template <typename VT>
void spmm_rs(const DevCsr& A, const float* xi, float* y, int64_t ystride, int R, int RS,
             const PivotCoef& pc, cudaStream_t s) {
  if (RS == 4)
    spmm_typed<VT, 4>(A, xi, y, ystride, R, pc, s);
  else if (RS == 8)
    spmm_typed<VT, 8>(A, xi, y, ystride, R, pc, s);
  else
    spmm_typed<VT, 16>(A, xi, y, ystride, R, pc, s);
}

int rhs_stride(int R) { return R <= 4 ? 4 : (R <= 8 ? 8 : 16); }

void launch_interleave(const float* x, int64_t xstride, int64_t count, int R, float* xi,
                       cudaStream_t s, int num_sms) {
  const int RS = rhs_stride(R);
  const int g = (int)std::min<int64_t>((count + 255) / 256, (int64_t)num_sms * 8);
  if (RS == 4)
    k_interleave<4><<<g, 256, 0, s>>>(x, xstride, count, R, xi);
  else if (RS == 8)
    k_interleave<8><<<g, 256, 0, s>>>(x, xstride, count, R, xi);
  else
    k_interleave<16><<<g, 256, 0, s>>>(x, xstride, count, R, xi);
}

void launch_spmm_pivots(const DevCsr& A, int vt, const float* xi, float* y, int64_t ystride,
                        int R, PivotCoef pc, cudaStream_t s) {
  pc.npiv_blocks = (pc.cnt + 7) / 8;
  const int RS = rhs_stride(R);
  if (vt == LSLU_BF16)
    spmm_rs<__nv_bfloat16>(A, xi, y, ystride, R, RS, pc, s);
  else
    spmm_rs<float>(A, xi, y, ystride, R, RS, pc, s);
}

template void launch_spmv<double, double>(const DevCsr&, int, const double*, double*,
                                          cudaStream_t, int);
template void launch_spmv<float, float>(const DevCsr&, int, const float*, float*, cudaStream_t,
                                        int);
template void launch_spmv_pivots<double, double>(const DevCsr&, int, const double*, double*,
                                                 PivotCoef, cudaStream_t);
template void launch_spmv_pivots<float, float>(const DevCsr&, int, const float*, float*,
                                               PivotCoef, cudaStream_t);

}  // namespace lslu
