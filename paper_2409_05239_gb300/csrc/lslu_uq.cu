// Low-rank uncertainty quantification of Section 4.2 (lslu_uq).
//
// After k iterations, A^T A ~ L_k G^T G L_k^T with G^T G = W_k (D_k^T D_k)^-1 W_k^T
// (Eq. nhr2).  With lambda = sigma / alpha the posterior covariance
// sigma^2 (lambda^2 I + A^T A)^-1 is approximated by
//
//   Gamma_k = sigma^2 (lambda^2 I + L G^T G L^T)^-1
//           = sigma^2 lambda^-2 (I - L M L^T),  M = (L^T L + lambda^2 (G^T G)^-1)^-1
//
// (Woodbury), and (G^T G)^-1 = X^T (D_k^T D_k) X with X = W_k^-1, so no
// eigendecomposition is needed.  With S = L^T L + lambda^2 X^T D^T D X = R R^T
// (Cholesky), l_i^T M l_i = ||R^-1 l_i||^2, hence
//
//   diag(Gamma_k)_i = sigma^2 / lambda^2 (1 - ||R^-1 l_i||^2),
//   1^T Gamma_k 1   = sigma^2 / lambda^2 (n - ||R^-1 L^T 1||^2).
//
// Kernels: a tiled Gram pass over the bases (L^T L, D_k^T D_k, L^T 1; basis
// type products accumulated per row slice, FP64 across slices, reduced in a
// fixed order), two small FP64 GEMMs, one block for the Cholesky factor R,
// the triangular inverses W^-1 and R^-1 with one warp per column over the GPU,
// and a row pass that forms R^-1 l_i for every row and its squared norm.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "lslu_internal.cuh"

namespace lslu {
std::string& thread_error();  // defined in lslu_api.cu

namespace {

constexpr int kTG = 64;    // Gram output tile (kTG x kTG)
constexpr int kRC = 32;    // rows staged per step
constexpr int kSlicesMax = 64;

// Partial Gram tiles: block (pair, slice) adds B1(r, i) B2(r, j) over its rows
// for the kTG x kTG tile (ti, tj) of the pair list; 256 threads, 4 x 4 outputs
// each.  B1 / B2 column-major with leading dimension ld; cols1 / cols2 columns.
template <typename BT>
__global__ void __launch_bounds__(256)
    k_gram_tiles(const BT* __restrict__ B1, int cols1, const BT* __restrict__ B2, int cols2,
                 int64_t ld, int64_t rows, const int2* __restrict__ pairs, int rows_per_slice,
                 double* __restrict__ part) {
  using CT = BT;  // accumulate in the basis type within a slice
  __shared__ BT s1[kRC][kTG + 1];
  __shared__ BT s2[kRC][kTG + 1];
  const int2 pr = pairs[blockIdx.x];
  const int i0 = pr.x * kTG, j0 = pr.y * kTG;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_slice;
  const int64_t r_end = r_begin + rows_per_slice < rows ? r_begin + rows_per_slice : rows;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads
  CT acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  // stage kRC rows x kTG columns of each operand (zero outside); the next
  // slab's loads are issued into registers before the current one is used
  constexpr int kPer = kRC * kTG / 256;
  BT p1[kPer], p2[kPer];
  auto fetch = [&](int64_t r0) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = (int)threadIdx.x + 256 * u;
      const int rr = e % kRC, cc = e / kRC;
      const int64_t r = r0 + rr;
      const bool in = r < r_end;
      p1[u] = (in && i0 + cc < cols1) ? B1[(int64_t)(i0 + cc) * ld + r] : (BT)0;
      p2[u] = (in && j0 + cc < cols2) ? B2[(int64_t)(j0 + cc) * ld + r] : (BT)0;
    }
  };
  if (r_begin < r_end) fetch(r_begin);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kRC) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = (int)threadIdx.x + 256 * u;
      s1[e % kRC][e / kRC] = p1[u];
      s2[e % kRC][e / kRC] = p2[u];
    }
    __syncthreads();
    if (r0 + kRC < r_end) fetch(r0 + kRC);
#pragma unroll 4
    for (int rr = 0; rr < kRC; ++rr) {
      CT a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = s1[rr][ty + 16 * q];
        b[q] = s2[rr][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  double* out = part + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * (kTG * kTG);
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(ty + 16 * p) * kTG + (tx + 16 * q)] = (double)acc[p][q];
}

// C(i, j) (ld ldc) = sum over slices of the partial tiles, in slice order; for
// symmetric products (B1 == B2) the mirrored entry is written too.
__global__ void k_gram_reduce(const double* __restrict__ part, const int2* __restrict__ pairs,
                              int npairs, int nslices, int cols1, int cols2, int symmetric,
                              double* __restrict__ C, int64_t ldc) {
  const int64_t total = (int64_t)npairs * kTG * kTG;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int pi = (int)(e / (kTG * kTG));
    const int w = (int)(e % (kTG * kTG));
    const int i = pairs[pi].x * kTG + w / kTG, j = pairs[pi].y * kTG + w % kTG;
    if (i >= cols1 || j >= cols2) continue;
    double s = 0.0;
    for (int sl = 0; sl < nslices; ++sl) s += part[((int64_t)sl * npairs + pi) * (kTG * kTG) + w];
    C[(int64_t)j * ldc + i] = s;
    if (symmetric) C[(int64_t)i * ldc + j] = s;
  }
}

// C = alpha op(A) B + beta C0 for k x k FP64 matrices (column-major, ld k);
// op(A) = A or A^T.  16 x 16 tiles.
__global__ void k_gemm_f64(const double* __restrict__ A, int transA, const double* __restrict__ B,
                           const double* __restrict__ C0, double alpha, double beta, int k,
                           double* __restrict__ C) {
  __shared__ double sa[16][17], sb[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int t0 = 0; t0 < k; t0 += 16) {
    const int ar = blockIdx.y * 16 + ty, ac = t0 + tx;
    double av = 0.0;
    if (ar < k && ac < k) av = transA ? A[(int64_t)ar * k + ac] : A[(int64_t)ac * k + ar];
    sa[ty][tx] = av;
    const int br = t0 + ty, bc = blockIdx.x * 16 + tx;
    sb[ty][tx] = (br < k && bc < k) ? B[(int64_t)bc * k + br] : 0.0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) acc = fma(sa[ty][t], sb[t][tx], acc);
    __syncthreads();
  }
  if (row < k && col < k) {
    double v = alpha * acc;
    if (C0) v += beta * C0[(int64_t)col * k + row];
    C[(int64_t)col * k + row] = v;
  }
}

// X = T^-1 for a triangular T (k x k, leading dimension ldt, column-major;
// upper: T(i, l) for i <= l, else lower), one warp per column j of X,
// column-oriented substitution: b = e_j, then for each l from j towards the
// far end, x_l = b_l * (1 / T(l, l)) and b_i -= T(i, l) x_l for the entries
// still ahead, which the warp's lanes update in parallel (b in shared memory).
// Each step is a short chain (a multiply and one FMA per lane entry) instead
// of one thread's dot product, and all columns run at once over the GPU.
constexpr int kTriWarps = 4;
__global__ void __launch_bounds__(kTriWarps * 32)
    k_tri_inverse(const double* __restrict__ T, int64_t ldt, int k, int upper,
                  double* __restrict__ X) {
  extern __shared__ double tsm[];
  double* rd = tsm;                                          // 1 / T(l, l)
  double* b = tsm + k + (int64_t)(threadIdx.x >> 5) * k;     // this warp's b
  const int lane = threadIdx.x & 31;
  for (int l = threadIdx.x; l < k; l += blockDim.x) rd[l] = 1.0 / T[(int64_t)l * ldt + l];
  __syncthreads();
  const int j = blockIdx.x * kTriWarps + (threadIdx.x >> 5);
  if (j >= k) return;
  double* x = X + (int64_t)j * k;
  for (int i = lane; i < k; i += 32) {
    b[i] = (i == j) ? 1.0 : 0.0;
    if (upper ? i > j : i < j) x[i] = 0.0;
  }
  __syncwarp();
  if (upper) {
    for (int l = j; l >= 0; --l) {
      const double xl = b[l] * rd[l];
      if (lane == 0) x[l] = xl;
      const double* tc = T + (int64_t)l * ldt;
      for (int i = lane; i < l; i += 32) b[i] = fma(-tc[i], xl, b[i]);
      __syncwarp();
    }
  } else {
    for (int l = j; l < k; ++l) {
      const double xl = b[l] * rd[l];
      if (lane == 0) x[l] = xl;
      const double* tc = T + (int64_t)l * ldt;
      for (int i = l + 1 + lane; i < k; i += 32) b[i] = fma(-tc[i], xl, b[i]);
      __syncwarp();
    }
  }
}

size_t tri_inverse_smem(int k) { return (size_t)(1 + kTriWarps) * k * sizeof(double); }

// t = R^-1 s (R^-1 lower) and 1^T Gamma 1 = scale (n - ||t||^2); one block.
__global__ void k_uq_tsum(const double* __restrict__ Ri, int k, const double* __restrict__ s,
                          double* __restrict__ t, double n, double scale, double* out_sum) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double v = 0.0;
    for (int l = 0; l <= i; ++l) v = fma(Ri[(int64_t)l * k + i], s[l], v);
    t[i] = v;
    acc = fma(v, v, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    if (out_sum) *out_sum = scale * (n - tot);
  }
}

// S = R R^T in place (lower; err = 1 when S is not positive definite) on one
// thread-block cluster: CTA r of C keeps the
// columns j = r (mod C) of S in shared memory.  Step p: the owner of column p
// takes its square root, scales it and writes it into every CTA's buffer of
// parity p & 1; one cluster barrier; every CTA subtracts its outer product
// from its own columns j > p.  A buffer is rewritten two steps later, after
// the barrier that every reader of it has passed.  The FP64 updates spread
// over C SMs, and a step costs one barrier instead of three.
constexpr int kCholThreads = 512;
__global__ void __launch_bounds__(kCholThreads)
    k_chol_cluster(double* __restrict__ S, int k, double* err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double csm[];
  const int C = (int)cluster.num_blocks(), me = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kCholThreads / 32;
  const int nown = (k - me + C - 1) / C;  // columns me, me + C, ...
  double* own = csm;                       // nown x k, column c/C at (c / C) * k
  double* colp = own + (int64_t)((k + C - 1) / C) * k;  // 2 x k
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int q = 0; q < nown; ++q)
    for (int i = tid; i < k; i += kCholThreads)
      own[(int64_t)q * k + i] = S[(int64_t)(me + q * C) * k + i];
  cluster.sync();
  for (int p = 0; p < k; ++p) {
    double* buf = colp + (p & 1) * k;
    if (p % C == me) {
      double* cp = own + (int64_t)(p / C) * k;
      __shared__ double piv;
      if (tid == 0) {
        const double d = cp[p];
        if (!(d > 0.0) || !isfinite(d)) bad = 1;
        piv = sqrt(d > 0.0 ? d : 1.0);
        cp[p] = piv;
      }
      __syncthreads();
      const double pv = piv;
      for (int i = p + tid; i < k; i += kCholThreads) {
        const double v = i == p ? pv : cp[i] / pv;
        cp[i] = v;
        for (int r = 0; r < C; ++r) *cluster.map_shared_rank(buf + i, r) = v;
      }
    }
    cluster.sync();
    // own columns j > p: S(i, j) -= L(i, p) L(j, p), i >= j
    for (int q = (p + 1 - me + C - 1) / C + warp; q < nown; q += nw) {
      const int j = me + q * C;
      if (j <= p) continue;
      const double lj = buf[j];
      double* col = own + (int64_t)q * k;
      for (int i = j + lane; i < k; i += 32) col[i] -= buf[i] * lj;
    }
    __syncthreads();
  }
  for (int q = 0; q < nown; ++q)
    for (int i = tid; i < k; i += kCholThreads)
      S[(int64_t)(me + q * C) * k + i] = own[(int64_t)q * k + i];
  if (tid == 0 && bad) *err = 1.0;
  cluster.sync();  // no CTA leaves while another may still write its buffer
}

constexpr size_t kCholSmemCap = 200 * 1024;
size_t chol_cluster_smem(int k, int C) {
  return ((size_t)((k + C - 1) / C) * k + 2 * (size_t)k) * sizeof(double);
}

// Row pass: for rows [blockIdx.x * 64, +64) and output columns a-tile
// blockIdx.y (64 of them), t_i(a) = sum_{b <= a} Ri(a, b) l_i(b); the block
// writes sum_a t_i(a)^2 for its tile into part[tile][row].
template <typename BT>
__global__ void __launch_bounds__(256)
    k_uq_rows(const BT* __restrict__ L, int64_t ldl, int64_t n, int k,
              const BT* __restrict__ Ri, double* __restrict__ part) {
  using CT = BT;
  __shared__ BT sl[kRC][kTG + 1];  // L(row, b) for 64 rows x 32 b
  __shared__ BT sr[kRC][kTG + 1];  // Ri(a, b) for 64 a x 32 b
  const int64_t r0 = (int64_t)blockIdx.x * kTG;
  const int a0 = blockIdx.y * kTG;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  CT acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0;
  const int bmax = k < a0 + kTG ? k : a0 + kTG;  // Ri(a, b) = 0 for b > a
  for (int b0 = 0; b0 < bmax; b0 += kRC) {
    for (int e = threadIdx.x; e < kRC * kTG; e += blockDim.x) {
      // consecutive threads on consecutive rows of L (and entries a of Ri):
      // coalesced reads of the column-major operands
      const int cc = e % kTG, bb = e / kTG;
      const int b = b0 + bb;
      const int64_t r = r0 + cc;
      sl[bb][cc] = (b < k && r < n) ? L[(int64_t)b * ldl + r] : (BT)0;
      const int a = a0 + cc;
      sr[bb][cc] = (b < k && a < k) ? Ri[(int64_t)b * k + a] : (BT)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int bb = 0; bb < kRC; ++bb) {
      CT x[4], y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        x[q] = sl[bb][ty + 16 * q];  // rows
        y[q] = sr[bb][tx + 16 * q];  // a
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(x[p], y[q], acc[p][q]);
    }
    __syncthreads();
  }
  // squared norms of this tile's 64 t-entries per row: reduce over tx (16
  // lanes sharing a row) in a fixed butterfly
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) s += (double)acc[p][q] * (double)acc[p][q];
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int64_t r = r0 + ty + 16 * p;
    if (tx == 0 && r < n) part[(int64_t)blockIdx.y * n + r] = s;
  }
}

__global__ void k_uq_diag(const double* __restrict__ part, int ntiles, int64_t n, double scale,
                          double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < ntiles; ++t) s += part[(int64_t)t * n + i];
    out[i] = scale * (1.0 - s);
  }
}

template <typename T>
__global__ void k_to_basis(const double* __restrict__ a, T* __restrict__ b, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}

template <typename T>
__global__ void k_fill(T* __restrict__ p, int64_t count, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

lslu_status fail(Ctx* c, lslu_status st, const std::string& msg) {
  c->err = msg;
  return st;
}

// Gram products B1^T B2 (cols1 x cols2, FP64, ld ldc) on the device.
template <typename BT>
cudaError_t gram(const BT* B1, int cols1, const BT* B2, int cols2, int64_t ld, int64_t rows,
                 bool symmetric, double* C, int64_t ldc, int2* dpairs, double* part,
                 int64_t part_cap, cudaStream_t s) {
  const int t1 = (cols1 + kTG - 1) / kTG, t2 = (cols2 + kTG - 1) / kTG;
  std::vector<int2> pairs;
  for (int i = 0; i < t1; ++i)
    for (int j = symmetric ? i : 0; j < t2; ++j) pairs.push_back(make_int2(i, j));
  const int np = (int)pairs.size();
  int nsl = std::max(1, std::min(kSlicesMax, (960 + np - 1) / np));
  while (nsl > 1 && (int64_t)nsl * np * kTG * kTG > part_cap) --nsl;
  if ((int64_t)nsl * np * kTG * kTG > part_cap) return cudaErrorInvalidValue;
  int64_t rps = (rows + nsl - 1) / nsl;
  rps = (rps + kRC - 1) / kRC * kRC;
  cudaError_t e = cudaMemcpyAsync(dpairs, pairs.data(), np * sizeof(int2), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  k_gram_tiles<BT><<<dim3(np, nsl), 256, 0, s>>>(B1, cols1, B2, cols2, ld, rows, dpairs, (int)rps,
                                                part);
  const int64_t tot = (int64_t)np * kTG * kTG;
  k_gram_reduce<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(
      part, dpairs, np, nsl, cols1, cols2, symmetric ? 1 : 0, C, ldc);
  e = cudaStreamSynchronize(s);  // the host pair list goes out of scope
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename BT>
lslu_status uq_impl(Ctx* c, double sigma2, double lam, double* var_diag, double* var_sum) {
  const int k = c->last_k;
  const int64_t n = c->n, m = c->m;
  cudaStream_t s = c->stream;
  // the k x k Cholesky factor runs on one thread-block cluster whose CTAs hold
  // its columns in shared memory (k up to about 640 with 16 CTAs; beyond that
  // W_k is numerically singular in FP64 for this method anyway)
  const int ccl = projected_cluster_size();
  const size_t smc = ccl > 0 ? chol_cluster_smem(k, ccl) : 0;
  if (ccl <= 0 || smc > kCholSmemCap)
    return fail(c, LSLU_ERR_INVALID_ARG,
                "uq: k = " + std::to_string(k) +
                    " is above what the cluster Cholesky factor holds in shared memory");
  if (cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smc) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LSLU_ERR_CUDA, "uq: cluster Cholesky set-up");
  }
  const BT* L = reinterpret_cast<const BT*>(c->L);
  const BT* D = reinterpret_cast<const BT*>(c->D);
  // work space: 5 k x k FP64, 2 k-vectors, pair list, Gram partials, ones
  // column, row partials
  const int tiles = (k + kTG - 1) / kTG;
  const int64_t part_cap = std::max<int64_t>((int64_t)1024 * kTG * kTG,
                                             (int64_t)tiles * (tiles + 1) / 2 * kTG * kTG);
  const int64_t rows_part = (int64_t)tiles * n;
  const int64_t kk = (int64_t)k * k;
  const size_t bytes = (size_t)(5 * kk + 4 * k + 8) * 8 + (size_t)tiles * tiles * sizeof(int2) +
                       (size_t)std::max(part_cap, rows_part) * 8 + (size_t)c->ldl * sizeof(BT) +
                       (size_t)kk * sizeof(BT) + 16 * 256;
  char* ws = nullptr;
  cudaError_t e = cudaMalloc(&ws, bytes);
  if (e != cudaSuccess) return fail(c, LSLU_ERR_OOM, "uq work space");
  auto take = [&](size_t b) {
    char* p = ws;
    ws += (b + 255) / 256 * 256;
    return p;
  };
  char* base = ws;
  double* GL = (double*)take(kk * 8);
  double* GD = (double*)take(kk * 8);
  double* X = (double*)take(kk * 8);
  double* Y = (double*)take(kk * 8);
  double* Ri = (double*)take(kk * 8);
  double* sL = (double*)take(k * 8);
  double* tv = (double*)take(k * 8);
  double* scal = (double*)take(64);
  int2* pairs = (int2*)take((size_t)tiles * tiles * sizeof(int2) + 16);
  double* part = (double*)take((size_t)std::max(part_cap, rows_part) * 8);
  BT* ones = (BT*)take((size_t)c->ldl * sizeof(BT));
  BT* Rib = (BT*)take((size_t)kk * sizeof(BT));
  const int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
  k_fill<BT><<<g, 256, 0, s>>>(ones, n, (BT)1);
  const double scale = sigma2 / (lam * lam);
  // Gram products
  if ((e = gram<BT>(L, k, L, k, c->ldl, n, true, GL, k, pairs, part, part_cap, s)) != cudaSuccess ||
      (e = gram<BT>(D, k, D, k, c->ldd, m, true, GD, k, pairs, part, part_cap, s)) != cudaSuccess ||
      (e = gram<BT>(L, k, ones, 1, c->ldl, n, false, sL, k, pairs, part, part_cap, s)) !=
          cudaSuccess) {
    cudaFree(base);
    return fail(c, LSLU_ERR_CUDA, std::string("uq gram: ") + cudaGetErrorString(e));
  }
  // X = W^-1, Y = G_D X, S = G_L + lambda^2 X^T Y (into GL)
  const unsigned gt = (unsigned)((k + kTriWarps - 1) / kTriWarps);
  const size_t smt = tri_inverse_smem(k);
  if (smt > 48 * 1024)
    cudaFuncSetAttribute(k_tri_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt);
  k_tri_inverse<<<gt, kTriWarps * 32, smt, s>>>(c->W, c->kmax, k, 1, X);
  const dim3 gg((k + 15) / 16, (k + 15) / 16);
  k_gemm_f64<<<gg, 256, 0, s>>>(GD, 0, X, nullptr, 1.0, 0.0, k, Y);
  k_gemm_f64<<<gg, 256, 0, s>>>(X, 1, Y, GL, lam * lam, 1.0, k, GD);  // GD <- S
  // the Cholesky factor on a thread-block cluster (checked to fit above)
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ccl);
    cfg.blockDim = dim3(kCholThreads);
    cfg.dynamicSmemBytes = smc;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)ccl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaMemsetAsync(scal + 1, 0, sizeof(double), s);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_chol_cluster, GD, k, scal + 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(s);
      cudaFree(base);
      return fail(c, LSLU_ERR_CUDA, std::string("uq: cluster Cholesky: ") + cudaGetErrorString(e));
    }
  }
  k_tri_inverse<<<gt, kTriWarps * 32, smt, s>>>(GD, k, k, 0, Ri);
  k_uq_tsum<<<1, 256, 0, s>>>(Ri, k, sL, tv, (double)n, scale, scal);
  if (var_diag) {
    k_to_basis<BT><<<64, 256, 0, s>>>(Ri, Rib, kk);
    const dim3 gr((unsigned)((n + kTG - 1) / kTG), (unsigned)tiles);
    k_uq_rows<BT><<<gr, 256, 0, s>>>(L, c->ldl, n, k, Rib, part);
    k_uq_diag<<<g, 256, 0, s>>>(part, tiles, n, scale, var_diag);
  }
  double hs[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(hs, scal, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(base);
  if (e != cudaSuccess) return fail(c, LSLU_ERR_CUDA, std::string("uq: ") + cudaGetErrorString(e));
  if (hs[1] != 0.0)
    return fail(c, LSLU_ERR_INVALID_ARG, "uq: L^T L + lambda^2 (G^T G)^-1 is not positive definite");
  if (var_sum) *var_sum = hs[0];
  return LSLU_OK;
}

template <typename BT>
lslu_status gram_products_impl(Ctx* c, int k, const double* v, double* G, double* g) {
  cudaStream_t s = c->stream;
  const int tiles = (k + kTG - 1) / kTG;
  const int64_t part_cap = std::max<int64_t>((int64_t)1024 * kTG * kTG,
                                             (int64_t)tiles * (tiles + 1) / 2 * kTG * kTG);
  int2* pairs = nullptr;
  double* part = nullptr;
  BT* vb = nullptr;
  cudaError_t e = cudaMalloc(&pairs, (size_t)tiles * tiles * sizeof(int2) + 16);
  if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)part_cap * 8);
  if (e == cudaSuccess) e = cudaMalloc(&vb, (size_t)c->ldl * sizeof(BT));
  if (e == cudaSuccess) {
    k_to_basis<BT><<<64, 256, 0, s>>>(v, vb, c->n);
    const BT* L = reinterpret_cast<const BT*>(c->L);
    e = gram<BT>(L, k, L, k, c->ldl, c->n, true, G, k, pairs, part, part_cap, s);
    if (e == cudaSuccess) e = gram<BT>(L, k, vb, 1, c->ldl, c->n, false, g, k, pairs, part, part_cap, s);
  }
  cudaFree(pairs);
  cudaFree(part);
  cudaFree(vb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LSLU_ERR_CUDA, std::string("gram products: ") + cudaGetErrorString(e));
  }
  return LSLU_OK;
}

}  // namespace

lslu_status basis_gram_products(Ctx* c, int k, const double* v, double* G, double* g) {
  return c->value_type == LSLU_F64 ? gram_products_impl<double>(c, k, v, G, g)
                                   : gram_products_impl<float>(c, k, v, G, g);
}

}  // namespace lslu

using namespace lslu;

extern "C" lslu_status lslu_uq(lslu_handle h, double sigma2, double lambda, int32_t ptr_location,
                               double* var_diag, double* var_sum) {
  Ctx* c = h;
  if (!c) {
    thread_error() = "NULL handle";
    return LSLU_ERR_INVALID_ARG;
  }
  if (c->map_m) return fail(c, LSLU_ERR_INVALID_ARG, "lslu_uq takes single-problem handles");
  if (c->last_k < 1) return fail(c, LSLU_ERR_INVALID_ARG, "lslu_uq needs a completed iteration");
  if (!(sigma2 > 0.0) || !(lambda > 0.0) || !std::isfinite(sigma2) || !std::isfinite(lambda))
    return fail(c, LSLU_ERR_INVALID_ARG, "sigma2 and lambda must be finite and > 0");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return fail(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  // host outputs, and the output of a renumbered handle, are staged on the
  // device in the internal numbering
  const bool host = ptr_location == LSLU_HOST;
  const bool stage = var_diag && (host || c->ord_m);
  double* dd = var_diag;
  if (stage) {
    if (cudaMalloc(&dd, c->n * sizeof(double)) != cudaSuccess)
      return fail(c, LSLU_ERR_OOM, "uq output");
  }
  double sum = 0.0;
  lslu_status st = c->value_type == LSLU_F64 ? uq_impl<double>(c, sigma2, lambda, dd, &sum)
                                             : uq_impl<float>(c, sigma2, lambda, dd, &sum);
  if (st == LSLU_OK && stage) {
    cudaError_t e = vec_out(c, false, dd, host, var_diag);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = fail(c, LSLU_ERR_CUDA, cudaGetErrorString(e));
  }
  if (stage) cudaFree(dd);
  if (st == LSLU_OK && var_sum) {
    if (ptr_location == LSLU_HOST) {
      *var_sum = sum;
    } else if (cudaMemcpy(var_sum, &sum, 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      st = fail(c, LSLU_ERR_CUDA, "uq: copying the sum");
    }
  }
  return st;
}
