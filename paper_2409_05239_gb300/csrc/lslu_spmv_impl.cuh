// Device code of the sparse products of Algorithm 4 (u = A l_k, q = A^T d_k),
// templated on the row shape: G lanes per CSR row (4, 8, 16 or 32) and U
// 4-entry chunks in flight per lane.  Included by the translation units that
// instantiate the shapes (lslu_spmv.cu: the default shapes and the shared-
// matrix products; lslu_spmv_shapes.cu: the others).
//
// Both products run on a row-major CSR: A^T is stored as its own (transposed)
// CSR, so every output entry is one row dot product and no atomics are needed.
// Lane j of a row's group reads the chunks j, j+G, j+2G, ... of the row with
// vector loads (rows are padded to a multiple of kRowAlign entries), keeps a
// private partial sum in chunk order, and the group adds its G partials with
// a fixed butterfly, so results are bitwise reproducible run to run (for a
// given shape).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "lslu_internal.cuh"

namespace lslu {
namespace {

template <typename VT>
struct ValTraits {
  static constexpr int kChunk = 4;  // entries per chunk (16-byte column loads)
};

// Blocks of 256 threads kept resident per SM: bounds the registers per thread
// (E = 4-entry chunks in flight per lane).
template <typename VT, int E>
constexpr int min_blocks() {
  return (E >= 2 || sizeof(VT) == 8) ? 6 : 8;
}

template <typename AT>
__device__ __forceinline__ AT warp_sum(AT v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over each group of G lanes (every lane of the warp must call it).
template <int G, typename AT>
__device__ __forceinline__ AT group_sum(AT v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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

// Compressed columns: 8 16-bit offsets of one 8-entry unit (16 bytes).
__device__ __forceinline__ uint4 ld_stream_off(const uint16_t* p) {
  uint4 c;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(c.x), "=r"(c.y), "=r"(c.z), "=r"(c.w)
               : "l"(p));
  return c;
}
template <typename AT, typename VT>
__device__ __forceinline__ void load_vals8(const VT* p, AT (&v)[8]) {
  AT a[4], b[4];
  load_vals_cs<AT>(p, a);
  load_vals_cs<AT>(p + 4, b);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[i] = a[i];
    v[4 + i] = b[i];
  }
}
template <typename AT>
__device__ __forceinline__ void load_vals8(const __nv_bfloat16* p, AT (&v)[8]) {
  uint32_t w[4];
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
               : "l"(p));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = (AT)__uint_as_float(w[i] << 16);
    v[2 * i + 1] = (AT)__uint_as_float(w[i] & 0xffff0000u);
  }
}

// The column storage a kernel reads: 32-bit indices (chunks of 4 entries) or,
// when every 8-entry unit spans fewer than 2^16 columns, 16-bit offsets from
// the unit's first column (chunks of 8 entries; 2.5 bytes per entry).
struct ColIdx {
  const int32_t* col;     // nnz_padded 32-bit columns
  const uint16_t* off;    // nnz_padded offsets (compressed)
  const int32_t* ubase;   // nnz_padded / 8 unit bases (compressed)
};

// Dot product of one CSR row with x, computed by one group of G lanes (result
// in every lane of the group; gl = lane index within the group; a lane with
// len = 0 contributes nothing).  Lane gl takes chunks gl, gl+G, ... in order
// (U chunks per step); the G partial sums are combined by a fixed butterfly,
// so a row always gets the same bits.  Every lane of the warp must call it.
template <typename VT, typename XT, typename YT, int G, int U>
__device__ __forceinline__ YT row_dot_len_c(int32_t start, int32_t len, const ColIdx ci,
                                            const VT* __restrict__ val,
                                            const XT* __restrict__ x, int gl) {
  constexpr int C = 8;
  constexpr int S = G * C;
  YT acc = 0;
  for (int32_t e = gl * C; e < len; e += U * S) {
    int32_t cidx[U][C];
    YT v[U][C];
    bool has[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      has[u] = u == 0 || e + u * S < len;
      if (has[u]) {
        const int32_t p = start + e + u * S;
        const uint4 o = ld_stream_off(ci.off + p);
        const int32_t b = __ldg(ci.ubase + (p >> 3));
        const uint32_t w[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          cidx[u][2 * q] = b + (int32_t)(w[q] & 0xffffu);
          cidx[u][2 * q + 1] = b + (int32_t)(w[q] >> 16);
        }
        load_vals8<YT>(val + p, v[u]);
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
  return group_sum<G>(acc);
}

template <typename VT, typename XT, typename YT, int G, int U>
__device__ __forceinline__ YT row_dot_len(int32_t start, int32_t len,
                                          const int32_t* __restrict__ col,
                                          const VT* __restrict__ val, const XT* __restrict__ x,
                                          int gl) {
  constexpr int C = ValTraits<VT>::kChunk;
  constexpr int S = G * C;  // entries between a lane's consecutive chunks
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
  return group_sum<G>(acc);
}

// Scalar stream loads (one entry per lane) without L1 allocation.
__device__ __forceinline__ float ld_stream1(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_stream1(const double* p) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream1(const __nv_bfloat16* p) {
  unsigned short h;
  asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(h) : "l"(p));
  return __uint_as_float((uint32_t)h << 16);
}
__device__ __forceinline__ int32_t ld_stream1(const int32_t* p) {
  int32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int32_t ld_stream1(const uint16_t* p) {
  unsigned short h;
  asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(h) : "l"(p));
  return (int32_t)h;
}

// Row dot with the 32 lanes of a warp on consecutive entries: lane l takes
// entries l, l+32, l+64, ... (U per step), so one gather instruction reads 32
// neighbouring entries of the row; where those have nearby columns (a ray
// crossing neighbouring pixels) the gathers of x share sectors.  Each lane
// sums its entries in order; the warp adds the 32 partials by a fixed
// butterfly.
template <typename VT, typename XT, typename YT, int U, bool CMP>
__device__ __forceinline__ YT row_dot_s1(int32_t start, int32_t len, const ColIdx ci,
                                         const VT* __restrict__ val, const XT* __restrict__ x,
                                         int lane) {
  YT acc = 0;
  for (int32_t e = lane; e < len; e += 32 * U) {
    YT v[U];
    int32_t c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t q = e + 32 * u;
      if (q < len) {
        const int32_t p = start + q;
        v[u] = (YT)ld_stream1(val + p);
        c[u] = CMP ? __ldg(ci.ubase + (p >> 3)) + ld_stream1(ci.off + p) : ld_stream1(ci.col + p);
      } else {
        v[u] = 0;
        c[u] = -1;
      }
    }
    XT xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : (XT)0;
#pragma unroll
    for (int u = 0; u < U; ++u) acc = fma(v[u], (YT)xv[u], acc);
  }
  return group_sum<32>(acc);
}

// G = 0 selects the warp-per-row stride-1 form (row_dot_s1) with U entries in
// flight per lane.
template <typename VT, typename XT, typename YT, int G, int U, bool CMP>
__device__ __forceinline__ YT row_dot(int64_t row, bool valid, const int32_t* __restrict__ rp,
                                      const int32_t* __restrict__ rl, const ColIdx ci,
                                      const VT* __restrict__ val, const XT* __restrict__ x,
                                      int gl) {
  const int32_t start = valid ? __ldg(rp + row) : 0;
  const int32_t len = valid ? __ldg(rl + row) : 0;
  if constexpr (G == 0)
    return row_dot_s1<VT, XT, YT, U, CMP>(start, len, ci, val, x, gl);
  else if constexpr (CMP)
    return row_dot_len_c<VT, XT, YT, G, U>(start, len, ci, val, x, gl);
  else
    return row_dot_len<VT, XT, YT, G, U>(start, len, ci.col, val, x, gl);
}

template <typename VT, typename XT, typename YT, int G, int U, bool CMP>
__global__ void __launch_bounds__(256, (G == 0 && sizeof(VT) == 8 && U > 4) ? 4 : min_blocks<VT, G == 0 ? U / 4 : (CMP ? 2 * U : U)>())
    k_spmv(int64_t rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ rl,
           const ColIdx ci, const VT* __restrict__ val, const XT* __restrict__ x,
           YT* __restrict__ y) {
  constexpr int GL = G == 0 ? 32 : G;  // lanes per row
  constexpr int RPB = 256 / GL;        // rows per block
  const int gl = threadIdx.x & (GL - 1);
  const int64_t row = (int64_t)blockIdx.x * RPB + threadIdx.x / GL;
  if ((int64_t)blockIdx.x * RPB + (threadIdx.x & ~31) / GL >= rows)
    return;  // the whole warp is past the last row
  const bool valid = row < rows;
  const YT acc = row_dot<VT, XT, YT, G, U, CMP>(row, valid, rp, rl, ci, val, x, gl);
  if (valid && gl == 0) y[row] = acc;
}

// y = A x plus the elimination coefficients of the next Hessenberg step,
// c = T^-1 y(piv), where T(i,j) = b_j(piv_i) is the unit lower triangular
// pivot-row matrix of the basis b and T^-1 is kept explicitly (column-major,
// accumulation type).  |T| <= 1 under max-abs pivoting keeps
// T^-1 small and well conditioned, so every coefficient becomes a plain
// dot product instead of a step of a sequential forward substitution.
//
// The first npiv blocks per problem own the pivot columns, one warp per
// column j:
//   a. completes the newest row of T^-1 in its column,
//      Tinv(nr, j) = -sum_{l=j}^{nr-1} T(nr, l) Tinv(l, j),  nr = cnt-1;
//   b. computes y(piv_j) with the same row reduction as every other row
//      (so the two agree bit for bit);
//   c. the block adds Tinv(i, j) y(piv_j) over its 8 columns into a partial
//      vector; the last pivot block to finish adds the partials in block order.
// The remaining blocks compute the other rows of y meanwhile.  rowdot(p, row,
// gl) is the product of output row `row` for problem p.
template <typename YT, int G, typename RowDot>
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
    // every lane group of the warp computes the pivot row (the same bits as
    // its y entry)
    const YT yp = rowdot(p, piv[j], lane & (G - 1));
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

template <typename VT, typename XT, typename YT, int G, int U, bool CMP>
__global__ void __launch_bounds__(256, (G == 0 && sizeof(VT) == 8 && U > 4) ? 4 : min_blocks<VT, G == 0 ? U / 4 : (CMP ? 2 * U : U)>())
    k_spmv_pivots(int64_t rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ rl,
                  const ColIdx ci, const VT* __restrict__ val, const XT* __restrict__ x,
                  YT* __restrict__ y, PivotCoef pc) {
  constexpr int GL = G == 0 ? 32 : G;
  constexpr int RPB = 256 / GL;
  pdl_wait();  // x and the pivot rows come from the kernels before
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int npiv_all = pc.npiv_blocks * pc.nprob;
  if ((int)blockIdx.x >= npiv_all) {  // streaming rows (all but the first npiv_all blocks)
    const int64_t b0 = (int64_t)(blockIdx.x - npiv_all) * RPB;
    if (b0 + (threadIdx.x & ~31) / GL >= rows) return;  // whole warp past the end
    const int64_t row = b0 + threadIdx.x / GL;
    const bool valid = row < rows;
    const YT acc =
        row_dot<VT, XT, YT, G, U, CMP>(row, valid, rp, rl, ci, val, x, lane & (GL - 1));
    if (valid && (lane & (GL - 1)) == 0) y[row] = acc;
    return;
  }
  pivot_blocks<YT, GL>(pc, [=](int, int32_t row, int gl) {
    return row_dot<VT, XT, YT, G, U, CMP>(row, true, rp, rl, ci, val, x, gl);
  });
}

// Launch in the matrix's column format: 16-bit offsets when its shape reads
// them (use_cmp) and MAYCMP (native vector types), else 32-bit columns.
template <typename VT, typename XT, typename YT, int G, int U, bool MAYCMP = true>
void spmv_run(const DevCsr& A, const XT* x, YT* y, cudaStream_t s) {
  if (A.rows == 0) return;
  constexpr int GL = G == 0 ? 32 : G;
  const int64_t blocks = (A.rows + 256 / GL - 1) / (256 / GL);
  const ColIdx ci{A.col, A.off, A.ubase};
  const VT* v = reinterpret_cast<const VT*>(A.val);
  if constexpr (MAYCMP) {
    if (A.compressed && A.use_cmp) {
      k_spmv<VT, XT, YT, G, U, true><<<(unsigned)blocks, 256, 0, s>>>(A.rows, A.row_ptr,
                                                                       A.row_len, ci, v, x, y);
      return;
    }
  }
  k_spmv<VT, XT, YT, G, U, false><<<(unsigned)blocks, 256, 0, s>>>(A.rows, A.row_ptr,
                                                                    A.row_len, ci, v, x, y);
}

template <typename VT, typename XT, typename YT, int G, int U, bool MAYCMP = true>
void spmv_pivots_run(const DevCsr& A, const XT* x, YT* y, const PivotCoef& pc, cudaStream_t s) {
  constexpr int GL = G == 0 ? 32 : G;
  const int64_t blocks =
      (int64_t)pc.npiv_blocks * pc.nprob + (A.rows + 256 / GL - 1) / (256 / GL);
  const ColIdx ci{A.col, A.off, A.ubase};
  const VT* v = reinterpret_cast<const VT*>(A.val);
  if constexpr (MAYCMP) {
    if (A.compressed && A.use_cmp) {
      launch_pdl(k_spmv_pivots<VT, XT, YT, G, U, true>, dim3((unsigned)blocks), dim3(256), 0, s,
                 A.rows, A.row_ptr, A.row_len, ci, v, x, y, pc);
      return;
    }
  }
  launch_pdl(k_spmv_pivots<VT, XT, YT, G, U, false>, dim3((unsigned)blocks), dim3(256), 0, s,
             A.rows, A.row_ptr, A.row_len, ci, v, x, y, pc);
}

}  // namespace
}  // namespace lslu
