// Sparse products of Algorithm 4: u = A l_k and q = A^T d_k (host side,
// default row shapes, and the products of right-hand sides sharing one
// matrix).  The device code of the single-vector products is in
// lslu_spmv_impl.cuh; the default shape is 16 lanes per row with two chunks
// in flight (one for FP64 values); other shapes, chosen per matrix by
// lslu_tune_spmv, are instantiated in lslu_spmv_shapes.cu.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "lslu_spmv_impl.cuh"

namespace lslu {

namespace {

constexpr int kGroup = 16;  // lanes per row of the shared-matrix product
constexpr int kRowsPerBlock = 256 / kGroup;

// ---- several right-hand sides sharing one matrix ---------------------------
// The R input vectors are first interleaved, xi[j * RS + r] (RS = R rounded
// up to 4, zero-padded), so each non-zero fetches all R values with RS/4
// 16-byte loads and the matrix is read once for all R products.  Lane gl of a
// row's 16-lane group takes the same chunks in the same order as row_dot_len,
// and each right-hand side keeps its own accumulator, so every output equals
// the single-vector product of the default 16-lane shapes bit for bit (16x2 on
// 32-bit columns, 16x1 on 16-bit offsets).

// Columns of the lane's next chunk (C entries at position p of the row
// storage): 32-bit indices (C = 4) or a unit of 16-bit offsets (C = 8).
template <bool CMP>
__device__ __forceinline__ void chunk_cols(const ColIdx& ci, int32_t p, int32_t (&c)[CMP ? 8 : 4]) {
  if constexpr (CMP) {
    const uint4 o = ld_stream_off(ci.off + p);
    const int32_t b = __ldg(ci.ubase + (p >> 3));
    const uint32_t w[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      c[2 * q] = b + (int32_t)(w[q] & 0xffffu);
      c[2 * q + 1] = b + (int32_t)(w[q] >> 16);
    }
  } else {
    const int4 c4 = ld_stream(ci.col + p);
    c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
  }
}

template <typename VT, bool CMP>
__device__ __forceinline__ void chunk_vals(const VT* val, int32_t p, float (&v)[CMP ? 8 : 4]) {
  if constexpr (CMP)
    load_vals8<float>(val + p, v);
  else
    load_vals_cs<float>(val + p, v);
}

// Product of CSR row `row` with right-hand side r of the interleaved xi, in
// the chunk order of the single-vector default shape (16 lanes).
template <typename VT, int RS, bool CMP>
__device__ __forceinline__ float row_dot_rhs(int64_t row, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ rl, const ColIdx ci,
                                             const VT* __restrict__ val,
                                             const float* __restrict__ xi, int r, int gl) {
  constexpr int C = CMP ? 8 : 4;
  constexpr int S = kGroup * C;
  const int32_t start = __ldg(rp + row), len = __ldg(rl + row);
  float acc = 0.f;
  for (int32_t e = gl * C; e < len; e += S) {
    int32_t c[C];
    float v[C];
    chunk_cols<CMP>(ci, start + e, c);
    chunk_vals<VT, CMP>(val, start + e, v);
#pragma unroll
    for (int i = 0; i < C; ++i) acc = fmaf(v[i], __ldg(xi + (int64_t)c[i] * RS + r), acc);
  }
  return group_sum<kGroup>(acc);
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
template <typename VT, int RS, bool CMP>
__global__ void __launch_bounds__(256, 4)
    k_spmm_pivots(int64_t rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ rl,
                  const ColIdx ci, const VT* __restrict__ val, const float* __restrict__ xi,
                  float* __restrict__ y, int64_t ystride, int R, PivotCoef pc) {
  constexpr int C = CMP ? 8 : 4;
  constexpr int S = kGroup * C;
  const int lane = threadIdx.x & 31;
  const int npiv_all = pc.npiv_blocks * pc.nprob;
  if ((int)blockIdx.x < npiv_all) {
    pivot_blocks<float, kGroup>(pc, [=](int p, int32_t row, int gl) {
      return row_dot_rhs<VT, RS, CMP>((int64_t)row - (int64_t)p * ystride, rp, rl, ci, val, xi,
                                      p, gl);
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
    int32_t cs[C];
    float v[C];
    chunk_cols<CMP>(ci, start + e, cs);
    chunk_vals<VT, CMP>(val, start + e, v);
#pragma unroll
    for (int i = 0; i < C; ++i) {
      float xv[RS];
      gather_rhs<RS>(xi, cs[i], xv);
#pragma unroll
      for (int r = 0; r < RS; ++r) acc[r] = fmaf(v[i], xv[r], acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < RS; ++r) acc[r] = group_sum<kGroup>(acc[r]);
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
    // full kPermBlock-entry blocks stored transposed (4 x 16): position 4 l + i
    // holds entry 16 i + l, so that the 16 lanes of a row group gather 16
    // consecutive entries of the row in each step; the last partial block
    // keeps its order
    const int64_t nfull = prl[r] / kPermBlock;
    for (int64_t b = 0; b < nfull; ++b) {
      int32_t tc[kPermBlock];
      double tv[kPermBlock];
      const int64_t base = b * kPermBlock;
      for (int l = 0; l < 16; ++l)
        for (int i = 0; i < 4; ++i) {
          tc[4 * l + i] = dc[base + 16 * i + l];
          tv[4 * l + i] = dv[base + 16 * i + l];
        }
      for (int q = 0; q < kPermBlock; ++q) {
        dc[base + q] = tc[q];
        dv[base + q] = tv[q];
      }
    }
  }
  out->rows = rows;
  out->cols = cols;
  out->nnz = rp[rows];
  out->nnz_padded = tot;
  size_t vbytes = vt == LSLU_F64 ? 8 : (vt == LSLU_F32 ? 4 : 2);
  cudaError_t e;
  // row pointers padded to a multiple of 4 entries
  const int64_t nrp = (rows + 1 + 3) / 4 * 4;
  prp.resize((size_t)nrp, (int32_t)tot);
  if ((e = cudaMalloc(&out->row_ptr, nrp * sizeof(int32_t))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&out->row_len, std::max<int64_t>(rows, 1) * sizeof(int32_t))) != cudaSuccess)
    return e;
  if ((e = cudaMalloc(&out->col, std::max<int64_t>(tot, kRowAlign) * sizeof(int32_t))) !=
      cudaSuccess)
    return e;
  if ((e = cudaMalloc(&out->val, std::max<int64_t>(tot, kRowAlign) * vbytes)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(out->row_ptr, prp.data(), nrp * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if (rows && (e = cudaMemcpyAsync(out->row_len, prl.data(), rows * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if (tot && (e = cudaMemcpyAsync(out->col, pc.data(), tot * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  // 16-bit column offsets when every 8-entry unit (rows start and end on unit
  // boundaries) spans fewer than 2^16 columns: offset = column - unit minimum
  const int64_t units = tot / kRowAlign;
  std::vector<uint16_t> po;
  std::vector<int32_t> pb;
  bool fits = units > 0;
  if (fits) {
    po.resize((size_t)tot);
    pb.resize((size_t)units);
    for (int64_t u = 0; u < units && fits; ++u) {
      const int32_t* c = pc.data() + u * kRowAlign;
      int32_t lo = c[0], hi = c[0];
      for (int i = 1; i < kRowAlign; ++i) {
        lo = std::min(lo, c[i]);
        hi = std::max(hi, c[i]);
      }
      if ((int64_t)hi - lo > 65535) {
        fits = false;
        break;
      }
      pb[u] = lo;
      for (int i = 0; i < kRowAlign; ++i) po[u * kRowAlign + i] = (uint16_t)(c[i] - lo);
    }
  }
  if (fits) {
    // unit bases readable up to a multiple of 4 units (aligned bulk copies)
    const int64_t nub = (units + 3) / 4 * 4;
    pb.resize((size_t)nub, 0);
    if ((e = cudaMalloc(&out->off, tot * sizeof(uint16_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&out->ubase, nub * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(out->off, po.data(), tot * sizeof(uint16_t), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(out->ubase, pb.data(), nub * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;  // po, pb go out of scope
    out->compressed = 1;
  }
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
  const cudaError_t e2 = upload_padded(n, m, rpt, cit, vt_, vt, AT, s);
  A->shape = AT->shape = default_shape(vt);
  return e2;
}

void free_csr(DevCsr* c) {
  cudaFree(c->row_ptr);
  cudaFree(c->row_len);
  cudaFree(c->col);
  cudaFree(c->val);
  cudaFree(c->off);
  cudaFree(c->ubase);
  *c = DevCsr();
}

// 16 lanes per row with 8 entries in flight per lane (two 4-entry chunks of
// 32-bit columns); FP64 values keep 4 in flight (registers).
int default_shape(int vt) { return vt == LSLU_F64 ? kShapeG16U1 : kShapeG16U2; }

namespace {

// The value type's native vector type: FP64 basis for FP64 values, FP32 basis
// otherwise.  Only native products use the tuned shapes.
template <typename XT, typename YT>
bool native(int vt) {
  if (!std::is_same<XT, YT>::value) return false;
  return (vt == LSLU_F64) == std::is_same<XT, double>::value;
}

}  // namespace

// Native products (FP64 vectors for FP64 values, FP32 otherwise) run in the
// matrix's shape and column format; the others (FP64 vectors on FP32 / BF16
// values: r0 with x0, the adjoint's x0 term) in the default shape.
template <typename XT, typename YT>
void launch_spmv(const DevCsr& A, int vt, const XT* x, YT* y, cudaStream_t s, int) {
  if (native<XT, YT>(vt) && A.shape != default_shape(vt)) {
    launch_spmv_shape(A.shape, A, vt, x, y, s);
    return;
  }
  if (vt == LSLU_F64)
    spmv_run<double, XT, YT, 16, 1, false>(A, x, y, s);
  else if (vt == LSLU_F32)
    spmv_run<float, XT, YT, 16, 2, false>(A, x, y, s);
  else
    spmv_run<__nv_bfloat16, XT, YT, 16, 2, false>(A, x, y, s);
}

template <typename XT, typename YT>
void launch_spmv_pivots(const DevCsr& A, int vt, const XT* x, YT* y, PivotCoef pc,
                        cudaStream_t s) {
  pc.npiv_blocks = (pc.cnt + 7) / 8;
  if (native<XT, YT>(vt) && A.shape != default_shape(vt)) {
    launch_spmv_pivots_shape(A.shape, A, vt, x, y, pc, s);
    return;
  }
  if (vt == LSLU_F64)
    spmv_pivots_run<double, XT, YT, 16, 1, false>(A, x, y, pc, s);
  else if (vt == LSLU_F32)
    spmv_pivots_run<float, XT, YT, 16, 2, false>(A, x, y, pc, s);
  else
    spmv_pivots_run<__nv_bfloat16, XT, YT, 16, 2, false>(A, x, y, pc, s);
}

template <typename VT, int RS>
void spmm_typed(const DevCsr& A, const float* xi, float* y, int64_t ystride, int R,
                const PivotCoef& pc, cudaStream_t s) {
  const int64_t blocks =
      (int64_t)pc.npiv_blocks * pc.nprob + (A.rows + kRowsPerBlock - 1) / kRowsPerBlock;
  const ColIdx ci{A.col, A.off, A.ubase};
  const VT* v = reinterpret_cast<const VT*>(A.val);
  if (A.compressed && A.use_cmp)
    k_spmm_pivots<VT, RS, true><<<(unsigned)blocks, 256, 0, s>>>(A.rows, A.row_ptr, A.row_len,
                                                                 ci, v, xi, y, ystride, R, pc);
  else
    k_spmm_pivots<VT, RS, false><<<(unsigned)blocks, 256, 0, s>>>(A.rows, A.row_ptr, A.row_len,
                                                                  ci, v, xi, y, ystride, R, pc);
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

namespace {
// Reads n 16-byte words through L2 (clean lines, as the elimination leaves
// them before a product) and stores one word so the reads are not dropped.
__global__ void k_l2_flush(const int4* __restrict__ p, int64_t n, int* sink) {
  int acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int4 v = __ldcg(p + i);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x7fffffff) *sink = acc;  // practically never; keeps the loads
}
}  // namespace

void launch_l2_flush(const void* buf, size_t bytes, int* sink, cudaStream_t s, int num_sms) {
  const int64_t n = (int64_t)(bytes / 16);
  k_l2_flush<<<num_sms * 8, 256, 0, s>>>(reinterpret_cast<const int4*>(buf), n, sink);
}

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
