// Reverse-mode derivative of Hybrid LSLU with the pivots held fixed
// (lslu_adjoint).
//
// With the pivot lists g and t of a completed solve held fixed, x_K is a
// smooth function of b and lambda.  This file runs the exact transpose of the
// forward steps (Algorithms 4 and 5), newest step first.  With 0-based
// indices, iteration k of the forward pass computes
//
//   L side:  q = A^T d_k,  c = T_L^-1 q(g_0..g_{k-1}),  v = q - L_{0:k-1} c,
//            omega = v(g_k) = W(k,k),  l_k = v / omega,  W(0:k-1,k) = c;
//   D side:  u = A l_k,  h = T_D^-1 u(t_0..t_k),  z = u - D_{0:k} h,
//            eta = z(t_{k+1}) = H(k+1,k),  d_{k+1} = z / eta,  H(0:k,k) = h;
//
// with T_L(i,j) = l_j(g_i) and T_D(i,j) = d_j(t_i) unit lower triangular, and
// finally y = (H^T H + lambda^2 I)^-1 H^T (beta e1) (Eq. TSP), x = L y.
// Given xbar = dJ/dx, the reverse pass forms
//
//   ybar = L^T xbar;  with ztil = (H^T H + lambda^2 I)^-1 ybar:
//   Hbar = (beta e1 - H y) ztil^T - (H ztil) y^T,  betabar = (H ztil)_0,
//   lambdabar = -2 lambda ztil^T y;
//
// and then, for k = K-1 .. 0, the D side of iteration k followed by its L
// side.  Each adjoint basis vector is assembled once, when it is complete:
//
//   dbar_{k+1} = A qbar_{k+1} - sum_{k'>k} H(k+1,k') zbar_{k'}
//                + its entries in the T_D terms of later steps;
//   lbar_k     = y_k xbar + A^T ubar_k - sum_{k'>k} W(k,k') vbar_{k'}
//                + its entries in the T_L terms of later steps;
//
// and the step adjoints are
//
//   etabar = Hbar(k+1,k) - dbar_{k+1}.d_{k+1} / eta,
//   zbar = dbar_{k+1} / eta + etabar e_{t_{k+1}},
//   a = T_D^-T (Hbar(0:k,k) - D_{0:k}^T zbar),  ubar = zbar + sum_i a_i e_{t_i},
//   omegabar = -lbar_k.l_k / omega,  vbar = lbar_k / omega + omegabar e_{g_k},
//   a' = T_L^-T (-L_{0:k-1}^T vbar),  qbar = vbar + sum_i a'_i e_{g_i}.
//
// The T terms: T^-1 u(piv) has the adjoint -T^-T cbar c^T with respect to T,
// so basis vector j receives -a_i c_j at pivot row i > j of every later step;
// these are the "pivot-row" corrections, kept in the small matrices A_D, A_L
// (column k' = a of step k').  Finally betabar_total = betabar -
// dbar_0.d_0 / beta and bbar = dbar_0 / beta + betabar_total e_{t_0}.
//
// Per reverse iteration: two sparse products (A^T ubar, A qbar: the forward
// kernels), two assembly passes over the stored adjoints (the shape of the
// forward elimination) and two dot-product passes over the basis.  The
// forward pass keeps every basis vector resident (its elimination needs
// them), so nothing is recomputed.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "lslu_internal.cuh"

namespace lslu {
std::string& thread_error();  // defined in lslu_api.cu

namespace {

constexpr int kT = 256;
constexpr int kNW = kT / 32;
constexpr int kDotRowsMax = 4096;  // rows of one dot-product block (shared-memory bound)

// scalar slots at the start of the FP64 work space
enum { S_ETA_BAR = 0, S_OMEGA_BAR, S_BETA_BAR_PROJ, S_LAMBDA_BAR, S_BETA_BAR, S_ERR, S_COUNT = 8 };

template <typename BT>
struct Vec;
template <>
struct Vec<float> {
  static constexpr int N = 4;
  __device__ static void load(const float* p, float (&o)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct Vec<double> {
  static constexpr int N = 2;
  __device__ static void load(const double* p, double (&o)[2]) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = v.x; o[1] = v.y;
  }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum (result in every thread).
__device__ double block_sum(double v) {
  __shared__ double red[kNW];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kNW; ++i) s += red[i];
  __syncthreads();
  return s;
}

// Sum of the per-block partials 0..nb-1 in a fixed order (every thread gets it).
__device__ double sum_partials(const double* part, int nb) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(part + b);
  return block_sum(s);
}

__device__ bool last_block(DevState* st) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&st->ticket, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) st->ticket = 0;
  }
  return last;
}

// ---- assembly of an adjoint basis vector ---------------------------------
struct AsmArgs {
  int64_t rows;
  const double* xbar;  // out += (*yk) xbar(i) when non-null
  const double* yk;
  const void* part;    // out += part(i) (compute type) when non-null
  const void* V;       // out -= sum_{j<cnt} coef(j) V(:, j)   (basis type)
  int64_t ldv;
  int cnt;
  const double* coef;  // coef(j) = coef[j * cstride]
  int64_t cstride;
  const void* w;       // dot partner (basis type)
  // pivot-row corrections, applied by the last block: for i in [i_lo, i_hi),
  // out(piv[i]) -= sum_{k' = i + kp_off}^{K-1} Am(i, k') crow[k' * crs]
  const double* Am;
  int64_t lda;
  const double* crow;
  int64_t crs;
  const int32_t* piv;
  int i_lo, i_hi, kp_off, K;
  // scalar epilogue: *slot = (ext ? *ext : 0) - dot / *den
  const double* ext;
  const double* den;
  double* slot;
  double* part_dot;
  DevState* st;
};

template <typename BT, typename CT>
__global__ void __launch_bounds__(kT) k_adj_assemble(AsmArgs a, CT* __restrict__ out) {
  constexpr int VEC = Vec<BT>::N;
  constexpr int TILE = 32 * VEC;
  extern __shared__ unsigned char smem_raw[];
  CT* c = reinterpret_cast<CT*>(smem_raw);
  __shared__ CT partw[kNW][TILE];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < a.cnt; j += blockDim.x) c[j] = (CT)a.coef[(int64_t)j * a.cstride];
  __syncthreads();
  const BT* V = reinterpret_cast<const BT*>(a.V);
  const BT* w = reinterpret_cast<const BT*>(a.w);
  const CT* part = reinterpret_cast<const CT*>(a.part);
  const CT yk = a.xbar ? (CT)*a.yk : (CT)0;
  double dot = 0.0;
  const int64_t ntiles = (a.rows + TILE - 1) / TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * TILE;
    CT acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0;
    {
      const BT* bp = V + r0 + lane * VEC;  // V has whole tiles of rows
      int j = warp;
      for (; j + 3 * kNW < a.cnt; j += 4 * kNW) {
        BT b[4][VEC];
#pragma unroll
        for (int u = 0; u < 4; ++u) Vec<BT>::load(bp + (int64_t)(j + u * kNW) * a.ldv, b[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[e] = fma(c[j + u * kNW], (CT)b[u][e], acc[e]);
      }
      for (; j < a.cnt; j += kNW) {
        BT b0[VEC];
        Vec<BT>::load(bp + (int64_t)j * a.ldv, b0);
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = fma(c[j], (CT)b0[e], acc[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) partw[warp][lane * VEC + e] = acc[e];
    __syncthreads();
    if (threadIdx.x < TILE) {
      const int64_t i = r0 + threadIdx.x;
      if (i < a.rows) {
        CT s = 0;
#pragma unroll
        for (int ww = 0; ww < kNW; ++ww) s += partw[ww][threadIdx.x];
        CT val = -s;
        if (part) val += part[i];
        if (a.xbar) val = fma(yk, (CT)a.xbar[i], val);
        out[i] = val;
        dot += (double)val * (double)w[i];
      }
    }
    __syncthreads();
  }
  dot = block_sum(dot);
  if (threadIdx.x == 0) a.part_dot[blockIdx.x] = dot;
  if (!last_block(a.st)) return;
  double tot = sum_partials(a.part_dot, gridDim.x);
  // pivot-row corrections and their share of the dot product
  double extra = 0.0;
  for (int i = a.i_lo + threadIdx.x; i < a.i_hi; i += blockDim.x) {
    double pv = 0.0;
    for (int kp = i + a.kp_off; kp < a.K; ++kp)
      pv -= a.Am[(int64_t)kp * a.lda + i] * a.crow[(int64_t)kp * a.crs];
    const int32_t r = a.piv[i];
    const CT nv = (CT)((double)__ldcg(out + r) + pv);
    __stcg(out + r, nv);
    extra += pv * (double)w[r];
  }
  tot += block_sum(extra);
  if (threadIdx.x == 0) *a.slot = (a.ext ? *a.ext : 0.0) - tot / *a.den;
}

// ---- dot products of a new adjoint vector with the basis ------------------
struct DotArgs {
  int64_t rows;
  int rows_per_block;
  const void* in;         // v(i) = in(i) / den + (i == *prow ? *sval : 0)
  int in_f64;             // in is FP64 (else compute type)
  const double* den;      // null: 1
  const int32_t* prow;    // null: no single-entry term
  const double* sval;
  void* store_b;          // optional copy of v in the basis type
  void* store_c;          // optional copy of v in the compute type
  const void* B;          // sums_j = sum_i B(i, j) v(i), j < cnt
  int64_t ldb;
  int cnt;
  // epilogue: r_j = (ext ? ext[j] : 0) + sgn * sums_j; with Tinv,
  // a_i = sum_{l >= i} Tinv(l, i) r_l is written to out_vec and added to
  // store_c at piv[i]; without, r goes to out_vec
  const double* ext;
  double sgn;
  const void* Tinv;
  int64_t ldt;
  double* out_vec;
  const int32_t* piv;
  double* part;           // gridDim.x x ldp partial sums
  int64_t ldp;
  DevState* st;
};

template <typename BT, typename CT>
__global__ void __launch_bounds__(kT) k_adj_dots(DotArgs a) {
  constexpr int VEC = Vec<BT>::N;
  extern __shared__ unsigned char smem_raw[];
  CT* vs = reinterpret_cast<CT*>(smem_raw);  // this block's v
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t r1 = min(r0 + a.rows_per_block, a.rows);
  const int nr = (int)(r1 - r0);
  const int32_t pr = a.prow ? *a.prow : -1;
  const double den = a.den ? *a.den : 1.0;
  const CT denc = (CT)den;
  for (int i = threadIdx.x; i < a.rows_per_block; i += blockDim.x) {
    CT v = 0;
    if (i < nr) {
      const int64_t gi = r0 + i;
      if (a.in_f64)
        v = (CT)(reinterpret_cast<const double*>(a.in)[gi] / den);
      else
        v = reinterpret_cast<const CT*>(a.in)[gi] / denc;
      if (gi == pr) v += (CT)*a.sval;
      if (a.store_b) reinterpret_cast<BT*>(a.store_b)[gi] = (BT)v;
      if (a.store_c) reinterpret_cast<CT*>(a.store_c)[gi] = v;
    }
    vs[i] = v;  // zero past the end of the rows
  }
  __syncthreads();
  const BT* B = reinterpret_cast<const BT*>(a.B);
  double* part = a.part + (int64_t)blockIdx.x * a.ldp;
  // rows_per_block is a multiple of 32 * VEC; B has whole 128-row tiles
  for (int j = warp; j < a.cnt; j += kNW) {
    const BT* bp = B + (int64_t)j * a.ldb + r0;
    CT acc = 0;
    for (int i = lane * VEC; i < nr; i += 32 * VEC) {
      BT b[VEC];
      Vec<BT>::load(bp + i, b);
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc = fma((CT)b[e], vs[i + e], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) part[j] = (double)acc;
  }
  if (!last_block(a.st)) return;
  extern __shared__ unsigned char smem_raw2[];
  double* r = reinterpret_cast<double*>(smem_raw2);  // reuses the v area (cnt doubles)
  __syncthreads();
  for (int j = threadIdx.x; j < a.cnt; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(a.part + (int64_t)b * a.ldp + j);
    r[j] = (a.ext ? a.ext[j] : 0.0) + a.sgn * s;
  }
  __syncthreads();
  if (!a.Tinv) {
    for (int j = threadIdx.x; j < a.cnt; j += blockDim.x) a.out_vec[j] = r[j];
    return;
  }
  const BT* Ti = reinterpret_cast<const BT*>(a.Tinv);
  CT* sc = reinterpret_cast<CT*>(a.store_c);
  for (int i = threadIdx.x; i < a.cnt; i += blockDim.x) {
    double s = 0.0;
    const BT* col = Ti + (int64_t)i * a.ldt;
    for (int l = i; l < a.cnt; ++l) s += (double)col[l] * r[l];
    a.out_vec[i] = s;
    const int32_t row = a.piv[i];
    __stcg(sc + row, (CT)((double)__ldcg(sc + row) + s));
  }
}

// ---- adjoint of the projected problem (one block, FP64) -------------------
//   M = H^T H + lambda^2 I = R R^T (Cholesky, R lower), ztil = M^-1 ybar,
//   Hbar = (beta e1 - H y) ztil^T - (H ztil) y^T, betabar = (H ztil)_0,
//   lambdabar = -2 lambda ztil^T y.
constexpr int kPT = 1024;

__global__ void __launch_bounds__(kPT)
    k_adj_projected(const double* __restrict__ H, int64_t ldh, int K, const double* y,
                    const DevState* st, const double* lam_ptr, const double* ybar, double* M,
                    double* zt, double* Hbar, double* scal) {
  __shared__ double red[kPT / 32];
  __shared__ int bad;
  const double lam = *lam_ptr;
  const double beta = st->beta;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  // lower triangle of M; H is upper Hessenberg, so column j has rows 0..j+1
  const int64_t npair = (int64_t)K * (K + 1) / 2;
  for (int64_t p = tid; p < npair; p += blockDim.x) {
    // p -> (i, j) with i >= j
    int i = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
    while ((int64_t)i * (i + 1) / 2 > p) --i;
    while ((int64_t)(i + 1) * (i + 2) / 2 <= p) ++i;
    const int j = (int)(p - (int64_t)i * (i + 1) / 2);
    double s = (i == j) ? lam * lam : 0.0;
    const int rmax = min(i, j) + 1;
    for (int r = 0; r <= rmax; ++r) s += H[(int64_t)i * ldh + r] * H[(int64_t)j * ldh + r];
    M[(int64_t)j * K + i] = s;
  }
  __syncthreads();
  // right-looking Cholesky (column-major, lower)
  for (int p = 0; p < K; ++p) {
    if (tid == 0) {
      const double d = M[(int64_t)p * K + p];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      M[(int64_t)p * K + p] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double piv = M[(int64_t)p * K + p];
    for (int i = p + 1 + tid; i < K; i += blockDim.x) M[(int64_t)p * K + i] /= piv;
    __syncthreads();
    const int rem = K - p - 1;
    const int64_t nup = (int64_t)rem * (rem + 1) / 2;
    for (int64_t q = tid; q < nup; q += blockDim.x) {
      int ii = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
      while ((int64_t)ii * (ii + 1) / 2 > q) --ii;
      while ((int64_t)(ii + 1) * (ii + 2) / 2 <= q) ++ii;
      const int jj = (int)(q - (int64_t)ii * (ii + 1) / 2);
      const int i = p + 1 + ii, j = p + 1 + jj;
      M[(int64_t)j * K + i] -= M[(int64_t)p * K + i] * M[(int64_t)p * K + j];
    }
    __syncthreads();
  }
  // R w = ybar, then R^T ztil = w (column oriented)
  for (int i = tid; i < K; i += blockDim.x) zt[i] = ybar[i];
  __syncthreads();
  for (int p = 0; p < K; ++p) {
    if (tid == 0) zt[p] /= M[(int64_t)p * K + p];
    __syncthreads();
    const double zp = zt[p];
    for (int i = p + 1 + tid; i < K; i += blockDim.x) zt[i] -= M[(int64_t)p * K + i] * zp;
    __syncthreads();
  }
  for (int p = K - 1; p >= 0; --p) {
    // zt[p] = (zt[p] - sum_{i>p} R(i,p) zt[i]) / R(p,p)
    double s = 0.0;
    for (int i = p + 1 + tid; i < K; i += blockDim.x) s += M[(int64_t)p * K + i] * zt[i];
    s = warp_sum(s);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kPT / 32; ++w) t += red[w];
      zt[p] = (zt[p] - t) / M[(int64_t)p * K + p];
    }
    __syncthreads();
  }
  // rH = beta e1 - H y and Hz = H ztil (length K+1), kept in M's space
  double* rH = M;
  double* Hz = M + (K + 1);
  for (int r = tid; r <= K; r += blockDim.x) {
    double a1 = (r == 0) ? beta : 0.0, a2 = 0.0;
    for (int j = max(r - 1, 0); j < K; ++j) {
      const double h = H[(int64_t)j * ldh + r];
      a1 -= h * y[j];
      a2 += h * zt[j];
    }
    rH[r] = a1;
    Hz[r] = a2;
  }
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)(K + 1) * K; e += blockDim.x) {
    const int j = (int)(e / (K + 1)), r = (int)(e % (K + 1));
    Hbar[(int64_t)j * ldh + r] = rH[r] * zt[j] - Hz[r] * y[j];
  }
  double s = 0.0;
  for (int j = tid; j < K; j += blockDim.x) s += zt[j] * y[j];
  s = warp_sum(s);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kPT / 32; ++w) t += red[w];
    scal[S_LAMBDA_BAR] = -2.0 * lam * t;
    scal[S_BETA_BAR_PROJ] = Hz[0];
    scal[S_ERR] = bad ? 1.0 : 0.0;
  }
}

// bbar = dbar_0 / beta + betabar e_{t_0}
template <typename CT>
__global__ void k_adj_bbar(const CT* __restrict__ dbar, int64_t m, const DevState* st,
                           const int32_t* tp, const double* scal, double* __restrict__ bbar,
                           double* lam_bar) {
  const double beta = st->beta;
  const int32_t t0 = tp[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)dbar[i] / beta;
    if (i == t0) v += scal[S_BETA_BAR];
    bbar[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && lam_bar) *lam_bar = scal[S_LAMBDA_BAR];
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, (count ? count : 1) * sizeof(T));
}

lslu_status fail(Ctx* c, lslu_status st, const std::string& msg) {
  c->err = msg;
  return st;
}

// FP64 work space layout (doubles)
struct SmallLayout {
  int64_t scal, ybar, zt, Hbar, AD, AL, M, total;
  int64_t ldh, ldAD, ldAL;
};
SmallLayout small_layout(const Ctx* c) {
  SmallLayout L;
  const int64_t K = c->kmax;
  L.ldh = K + 1;
  L.ldAD = K + 1;
  L.ldAL = K + 1;
  L.scal = 0;
  L.ybar = S_COUNT;
  L.zt = L.ybar + K;
  L.Hbar = L.zt + K;
  L.AD = L.Hbar + (K + 1) * K;
  L.AL = L.AD + (K + 1) * K;
  L.M = L.AL + (K + 1) * K;
  L.total = L.M + std::max<int64_t>(K * K, 2 * (K + 1));
  return L;
}

int dot_rows_per_block(int64_t rows, int nblk_target, int vec) {
  const int64_t unit = 32LL * vec;
  int64_t r = (rows + nblk_target - 1) / nblk_target;
  r = (r + unit - 1) / unit * unit;
  if (r > kDotRowsMax) r = kDotRowsMax;
  if (r < unit) r = unit;
  return (int)r;
}

template <typename BT, typename CT>
lslu_status ensure_workspace(Ctx* c) {
  if (c->adj_small) return LSLU_OK;
  const size_t bb = sizeof(BT);
  const int64_t K = c->kmax;
  const int64_t big = std::max(c->ldl, c->ldd);
  const int nt = std::max(c->num_sms * 2, 1);
  const int rpb = dot_rows_per_block(big, nt, Vec<BT>::N);
  const int64_t nblk_max = std::max<int64_t>((big + rpb - 1) / rpb, c->num_sms * 8);
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&c->adj_Vb, (size_t)c->ldl * K * bb)) != cudaSuccess ||
      (e = cudaMalloc(&c->adj_Zb, (size_t)c->ldd * K * bb)) != cudaSuccess ||
      (e = cudaMalloc(&c->adj_vec, (size_t)(3 * c->ldl + 3 * c->ldd + c->ldl) * sizeof(double))) !=
          cudaSuccess ||
      (e = dalloc(&c->adj_small, (size_t)small_layout(c).total)) != cudaSuccess ||
      (e = dalloc(&c->adj_part, (size_t)nblk_max * (K + 2))) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? LSLU_ERR_OOM : LSLU_ERR_CUDA,
                std::string("adjoint work space: ") + cudaGetErrorString(e));
  }
  c->adj_part_rows = (int)nblk_max;
  cudaMemset(c->adj_Vb, 0, (size_t)c->ldl * K * bb);
  cudaMemset(c->adj_Zb, 0, (size_t)c->ldd * K * bb);
  return LSLU_OK;
}

template <typename BT, typename CT>
void launch_assemble(Ctx* c, const AsmArgs& a, CT* out, cudaStream_t s) {
  constexpr int TILE = 32 * Vec<BT>::N;
  const int64_t ntiles = (a.rows + TILE - 1) / TILE;
  int64_t g = std::min<int64_t>(ntiles, (int64_t)c->num_sms * 8);
  if (g < 1) g = 1;
  const size_t smem = (size_t)std::max(a.cnt, 1) * sizeof(CT);
  k_adj_assemble<BT, CT><<<(unsigned)g, kT, smem, s>>>(a, out);
}

template <typename BT, typename CT>
void launch_dots(Ctx* c, DotArgs a, cudaStream_t s) {
  const int nt = std::max(c->num_sms * 2, 1);
  a.rows_per_block = dot_rows_per_block(a.rows, nt, Vec<BT>::N);
  const int64_t g = (a.rows + a.rows_per_block - 1) / a.rows_per_block;
  a.ldp = c->kmax + 2;
  const size_t smem = std::max((size_t)a.rows_per_block * sizeof(CT),
                               (size_t)(c->kmax + 2) * sizeof(double));
  k_adj_dots<BT, CT><<<(unsigned)g, kT, smem, s>>>(a);
}

template <typename BT, typename CT>
lslu_status adjoint_impl(Ctx* c, const double* xbar, double* bbar, double* lam_bar,
                         double* x0bar) {
  lslu_status st = ensure_workspace<BT, CT>(c);
  if (st != LSLU_OK) return st;
  cudaStream_t s = c->stream;
  const int K = c->last_K;
  const int64_t n = c->n, m = c->m;
  const int vt = c->value_type;
  const SmallLayout SL = small_layout(c);
  double* sm = c->adj_small;
  double* scal = sm + SL.scal;
  double* ybar = sm + SL.ybar;
  double* Hbar = sm + SL.Hbar;
  double* AD = sm + SL.AD;
  double* AL = sm + SL.AL;
  const int64_t ldh = c->kmax + 1, ldw = c->kmax;
  const BT* L = reinterpret_cast<const BT*>(c->L);
  const BT* D = reinterpret_cast<const BT*>(c->D);
  BT* Vb = reinterpret_cast<BT*>(c->adj_Vb);
  BT* Zb = reinterpret_cast<BT*>(c->adj_Zb);
  CT* vec = reinterpret_cast<CT*>(c->adj_vec);
  CT* lbar = vec;
  CT* qbar = lbar + c->ldl;
  CT* lpart = qbar + c->ldl;
  CT* dbar = lpart + c->ldl;
  CT* ubar = dbar + c->ldd;
  CT* dpart = ubar + c->ldd;
  // FP64 scratch of length n behind the compute-type vectors
  double* tmp_n = reinterpret_cast<double*>(c->adj_vec) + 3 * c->ldl + 3 * c->ldd;
  const double* lam_ptr = c->proj_out + (K - 1);
  int64_t launches = 0;

  cudaMemsetAsync(scal, 0, S_COUNT * sizeof(double), s);
  // ybar = L^T xbar
  {
    DotArgs a = {};
    a.rows = n;
    a.in = xbar;
    a.in_f64 = 1;
    a.B = L;
    a.ldb = c->ldl;
    a.cnt = K;
    a.sgn = 1.0;
    a.out_vec = ybar;
    a.part = c->adj_part;
    a.st = c->st;
    launch_dots<BT, CT>(c, a, s);
  }
  k_adj_projected<<<1, kPT, 0, s>>>(c->H, ldh, K, c->y, c->st, lam_ptr, ybar, sm + SL.M,
                                    sm + SL.zt, Hbar, scal);
  launches += 3;

  for (int k = K - 1; k >= 0; --k) {
    // ---- D side of iteration k: dbar_{k+1}, zbar_k, a (A_D column k), ubar
    {
      AsmArgs a = {};
      a.rows = m;
      a.part = (k + 1 <= K - 1) ? dpart : nullptr;
      a.V = Zb + (int64_t)(k + 1) * c->ldd;
      a.ldv = c->ldd;
      a.cnt = K - 1 - k;
      a.coef = c->H + (int64_t)(k + 1) * ldh + (k + 1);
      a.cstride = ldh;
      a.w = D + (int64_t)(k + 1) * c->ldd;
      a.Am = AD;
      a.lda = SL.ldAD;
      a.crow = c->H + (k + 1);
      a.crs = ldh;
      a.piv = c->tp;
      a.i_lo = k + 2;
      a.i_hi = K;
      a.kp_off = 0;
      a.K = K;
      a.ext = Hbar + (int64_t)k * ldh + (k + 1);
      a.den = c->H + (int64_t)k * ldh + (k + 1);
      a.slot = scal + S_ETA_BAR;
      a.part_dot = c->adj_part;
      a.st = c->st;
      launch_assemble<BT, CT>(c, a, dbar, s);
    }
    {
      DotArgs a = {};
      a.rows = m;
      a.in = dbar;
      a.den = c->H + (int64_t)k * ldh + (k + 1);
      a.prow = c->tp + (k + 1);
      a.sval = scal + S_ETA_BAR;
      a.store_b = Zb + (int64_t)k * c->ldd;
      a.store_c = ubar;
      a.B = D;
      a.ldb = c->ldd;
      a.cnt = k + 1;
      a.ext = Hbar + (int64_t)k * ldh;
      a.sgn = -1.0;
      a.Tinv = c->TDi;
      a.ldt = c->ldt;
      a.out_vec = AD + (int64_t)k * SL.ldAD;
      a.piv = c->tp;
      a.part = c->adj_part;
      a.st = c->st;
      launch_dots<BT, CT>(c, a, s);
    }
    launch_spmv<CT, CT>(c->AT, vt, ubar, lpart, s, c->num_sms);
    // ---- L side of iteration k: lbar_k, vbar_k, a' (A_L column k), qbar
    {
      AsmArgs a = {};
      a.rows = n;
      a.xbar = xbar;
      a.yk = c->y + k;
      a.part = lpart;
      a.V = Vb + (int64_t)(k + 1) * c->ldl;
      a.ldv = c->ldl;
      a.cnt = K - 1 - k;
      a.coef = c->W + (int64_t)(k + 1) * ldw + k;
      a.cstride = ldw;
      a.w = L + (int64_t)k * c->ldl;
      a.Am = AL;
      a.lda = SL.ldAL;
      a.crow = c->W + k;
      a.crs = ldw;
      a.piv = c->gp;
      a.i_lo = k + 1;
      a.i_hi = K;
      a.kp_off = 1;
      a.K = K;
      a.ext = nullptr;
      a.den = c->W + (int64_t)k * ldw + k;
      a.slot = scal + S_OMEGA_BAR;
      a.part_dot = c->adj_part;
      a.st = c->st;
      launch_assemble<BT, CT>(c, a, lbar, s);
    }
    {
      DotArgs a = {};
      a.rows = n;
      a.in = lbar;
      a.den = c->W + (int64_t)k * ldw + k;
      a.prow = c->gp + k;
      a.sval = scal + S_OMEGA_BAR;
      a.store_b = Vb + (int64_t)k * c->ldl;
      a.store_c = qbar;
      a.B = L;
      a.ldb = c->ldl;
      a.cnt = k;
      a.ext = nullptr;
      a.sgn = -1.0;
      a.Tinv = c->TLi;
      a.ldt = c->ldt;
      a.out_vec = AL + (int64_t)k * SL.ldAL;
      a.piv = c->gp;
      a.part = c->adj_part;
      a.st = c->st;
      launch_dots<BT, CT>(c, a, s);
    }
    launch_spmv<CT, CT>(c->A, vt, qbar, dpart, s, c->num_sms);
    launches += 6;
  }
  // dbar_0 and bbar
  {
    AsmArgs a = {};
    a.rows = m;
    a.part = dpart;
    a.V = Zb;
    a.ldv = c->ldd;
    a.cnt = K;
    a.coef = c->H;
    a.cstride = ldh;
    a.w = D;
    a.Am = AD;
    a.lda = SL.ldAD;
    a.crow = c->H;
    a.crs = ldh;
    a.piv = c->tp;
    a.i_lo = 1;
    a.i_hi = K;
    a.kp_off = 0;
    a.K = K;
    a.ext = scal + S_BETA_BAR_PROJ;
    a.den = &c->st->beta;
    a.slot = scal + S_BETA_BAR;
    a.part_dot = c->adj_part;
    a.st = c->st;
    launch_assemble<BT, CT>(c, a, dbar, s);
  }
  const int g = (int)std::min<int64_t>((m + 255) / 256, (int64_t)c->num_sms * 8);
  k_adj_bbar<CT><<<g, 256, 0, s>>>(dbar, m, c->st, c->tp, scal, bbar, lam_bar);
  launches += 2;
  if (x0bar) {  // r0 = b - A x0: x0bar = xbar - A^T bbar
    launch_spmv<double, double>(c->AT, vt, bbar, tmp_n, s, c->num_sms);
    const int g2 = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
    k_sub<<<g2, 256, 0, s>>>(xbar, tmp_n, x0bar, n);
    launches += 2;
  }
  c->launches = launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, LSLU_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(e));
  double err = 0.0;
  e = cudaMemcpyAsync(&err, scal + S_ERR, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(c, LSLU_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(e));
  if (err != 0.0)
    return fail(c, LSLU_ERR_INVALID_ARG,
                "adjoint: H^T H + lambda^2 I is not positive definite (lambda = 0 and H rank deficient)");
  return LSLU_OK;
}

}  // namespace
}  // namespace lslu

using namespace lslu;

extern "C" lslu_status lslu_adjoint(lslu_handle h, const double* x_bar, int32_t ptr_location,
                                    double* b_bar, double* lambda_bar, double* x0_bar) {
  Ctx* c = h;
  if (!c) {
    thread_error() = "NULL handle";
    return LSLU_ERR_INVALID_ARG;
  }
  if (c->map_m) return fail(c, LSLU_ERR_INVALID_ARG, "lslu_adjoint takes single-problem handles");
  if (!c->adj_valid)
    return fail(c, LSLU_ERR_INVALID_ARG,
                "lslu_adjoint needs a preceding lslu_solve that completed all K iterations");
  if (!x_bar || !b_bar) return fail(c, LSLU_ERR_INVALID_ARG, "x_bar and b_bar are required");
  if (ptr_location != LSLU_HOST && ptr_location != LSLU_DEVICE)
    return fail(c, LSLU_ERR_INVALID_ARG, "unknown ptr_location");
  const bool host = ptr_location == LSLU_HOST;
  const int64_t n = c->n, m = c->m;
  cudaStream_t s = c->stream;
  // device staging: xbar (n), bbar (m), x0bar (n), lambda_bar (1) behind the
  // compute-type vectors of the work space
  lslu_status st = c->value_type == LSLU_F64 ? ensure_workspace<double, double>(c)
                                             : ensure_workspace<float, float>(c);
  if (st != LSLU_OK) return st;
  double* dx = nullptr;
  double* db = nullptr;
  double* dx0 = nullptr;
  double* dl = nullptr;
  cudaError_t e = cudaSuccess;
  // host vectors, and every vector of a renumbered handle, go through a
  // device staging area in the internal numbering
  const bool stage = host || c->ord_m;
  if (stage) {
    if ((e = cudaMalloc(&dx, (size_t)(2 * n + m + 1) * sizeof(double))) != cudaSuccess)
      return fail(c, LSLU_ERR_OOM, "adjoint staging");
    db = dx + n;
    dx0 = x0_bar ? db + m : nullptr;
    dl = db + m + n;
    e = vec_in(c, false, x_bar, host, dx);
  } else {
    dx = const_cast<double*>(x_bar);
    db = b_bar;
    dx0 = x0_bar;
    dl = lambda_bar;
  }
  if (e == cudaSuccess) {
    st = c->value_type == LSLU_F64 ? adjoint_impl<double, double>(c, dx, db, dl, dx0)
                                   : adjoint_impl<float, float>(c, dx, db, dl, dx0);
  } else {
    st = fail(c, LSLU_ERR_CUDA, cudaGetErrorString(e));
  }
  if (stage && st == LSLU_OK) {
    e = vec_out(c, true, db, host, b_bar);
    if (e == cudaSuccess && x0_bar) e = vec_out(c, false, dx0, host, x0_bar);
    if (e == cudaSuccess && lambda_bar)
      e = cudaMemcpyAsync(lambda_bar, dl, 8,
                          host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(c, LSLU_ERR_CUDA, cudaGetErrorString(e));
  }
  if (stage) cudaFree(dx);
  return st;
}
