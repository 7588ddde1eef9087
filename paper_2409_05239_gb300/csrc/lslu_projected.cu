// Projected Tikhonov problem of Hybrid LSLU (Eq. TSP, Section 3.3), FP64.
//
// For the (k+1) x k upper Hessenberg H and beta:
//   1. Householder bidiagonalisation H = P [B; 0] Q^T (B k x k upper
//      bidiagonal), with g = P^T (beta e1);
//   2. singular values of B by Golub-Kahan implicit-shift QR sweeps; the
//      left rotations are applied to g, giving c = beta U^T e1 (Eq. gcv2);
//   3. lambda by the rule: none (0), fixed, GCV (Eq. gcv2) or weighted GCV
//      with omega = (k+1)/m (Eq. wgcv), minimised on a 257-point log grid
//      sigma_1 * 10^[-14, 2] and refined by 64 bisection steps on the sign of
//      dG/d(lambda^2) between the neighbours of the best grid point;
//   4. projected residual ||beta e1 - H y|| = sqrt(sum (f_i c_i)^2 + c_{k+1}^2)
//      with f_i = lambda^2 / (sigma_i^2 + lambda^2);
//   5. y = Q z with z = argmin ||g_{1:k} - B z||^2 + lambda^2 ||z||^2, solved
//      by Givens rotations on the stacked bidiagonal [B; lambda I] (Elden's
//      elimination), or by back substitution when lambda = 0.
// One thread block solves one projected problem; a launch solves the problems
// of sizes k_first..k_last (all of them when histories are requested).
#include <cuda_runtime.h>

#include <cmath>

#include "lslu_internal.cuh"

namespace lslu {

namespace {

constexpr int kT = 256;
constexpr int kGrid = 257;

__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Householder vector of x (length len, stride inc) in place: on return x[0]
// holds the new leading entry beta_h, x[1:] holds v[1:] (v[0] = 1) and tau
// is returned (H = I - tau v v^T maps x to beta_h e1).
__device__ double householder(double* x, int64_t inc, int len, double* red, double* beta_out) {
  double xn2 = 0.0;
  for (int t = 1 + threadIdx.x; t < len; t += blockDim.x) {
    const double a = x[t * inc];
    xn2 = fma(a, a, xn2);
  }
  xn2 = block_sum(xn2, red);
  const double alpha = x[0];
  if (xn2 == 0.0) {
    *beta_out = alpha;
    return 0.0;
  }
  const double nrm = sqrt(fma(alpha, alpha, xn2));
  const double bh = alpha >= 0.0 ? -nrm : nrm;
  const double tau = (bh - alpha) / bh;
  const double sc = 1.0 / (alpha - bh);
  __syncthreads();
  for (int t = 1 + threadIdx.x; t < len; t += blockDim.x) x[t * inc] *= sc;
  __syncthreads();
  *beta_out = bh;
  return tau;
}

__device__ __forceinline__ void givens(double y, double z, double& c, double& s, double& r) {
  if (z == 0.0) {
    c = 1.0;
    s = 0.0;
    r = y;
  } else {
    r = hypot(y, z);
    c = y / r;
    s = z / r;
  }
}

// Golub-Kahan SVD of the upper bidiagonal (d, e) of order n, applying the
// left rotations to g.  Single thread.  Returns 0 on convergence.
__device__ int bidiag_svd(double* d, double* e, double* g, int n) {
  const double eps = 2.220446049250313e-16;
  double bnorm = 0.0;
  for (int i = 0; i < n; ++i) bnorm = fmax(bnorm, fabs(d[i]));
  for (int i = 0; i + 1 < n; ++i) bnorm = fmax(bnorm, fabs(e[i]));
  if (bnorm == 0.0) return 0;
  const int max_steps = 60 * n + 100;
  int steps = 0;
  while (true) {
    for (int i = 0; i + 1 < n; ++i)
      if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;
    int hi = n - 1;
    while (hi > 0 && e[hi - 1] == 0.0) --hi;
    if (hi == 0) return 0;
    int lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;
    if (++steps > max_steps) return 1;
    // a (numerically) zero diagonal entry splits the block after a chase
    int zi = -1;
    for (int i = lo; i <= hi; ++i)
      if (fabs(d[i]) <= eps * bnorm) {
        zi = i;
        break;
      }
    if (zi >= 0) {
      d[zi] = 0.0;
      if (zi < hi) {
        // left rotations of row zi against rows zi+1..hi remove e[zi]
        double f = e[zi];
        e[zi] = 0.0;
        for (int j = zi + 1; j <= hi && f != 0.0; ++j) {
          double c, s, r;
          givens(d[j], f, c, s, r);
          d[j] = r;
          if (j < hi) {
            f = -s * e[j];
            e[j] = c * e[j];
          }
          const double gj = g[j], gz = g[zi];
          g[j] = c * gj + s * gz;
          g[zi] = -s * gj + c * gz;
        }
      } else {
        // right rotations of column hi against columns hi-1..lo remove e[hi-1]
        double f = e[hi - 1];
        e[hi - 1] = 0.0;
        for (int j = hi - 1; j >= lo && f != 0.0; --j) {
          double c, s, r;
          givens(d[j], f, c, s, r);
          d[j] = r;
          if (j > lo) {
            f = -s * e[j - 1];
            e[j - 1] = c * e[j - 1];
          }
        }
      }
      continue;
    }
    // Wilkinson shift from the trailing 2x2 of B^T B on the block
    const double t11 = d[hi - 1] * d[hi - 1] + (hi - 1 > lo ? e[hi - 2] * e[hi - 2] : 0.0);
    const double t12 = d[hi - 1] * e[hi - 1];
    const double t22 = d[hi] * d[hi] + e[hi - 1] * e[hi - 1];
    const double dl = 0.5 * (t11 - t22);
    const double den = dl + (dl >= 0.0 ? 1.0 : -1.0) * hypot(dl, t12);
    const double mu = den != 0.0 ? t22 - t12 * t12 / den : t22;
    double y = d[lo] * d[lo] - mu;
    double z = d[lo] * e[lo];
    for (int p = lo; p < hi; ++p) {
      double c, s, r;
      // right rotation on columns p, p+1 zeroing z in row p-1 (or the
      // implicit first column of B^T B - mu I)
      givens(y, z, c, s, r);
      if (p > lo) e[p - 1] = r;
      const double dp = d[p], ep = e[p];
      d[p] = c * dp + s * ep;
      e[p] = -s * dp + c * ep;
      const double bulge = s * d[p + 1];
      d[p + 1] = c * d[p + 1];
      // left rotation on rows p, p+1 zeroing the bulge at (p+1, p)
      givens(d[p], bulge, c, s, r);
      d[p] = r;
      const double ep2 = e[p], dp1 = d[p + 1];
      e[p] = c * ep2 + s * dp1;
      d[p + 1] = -s * ep2 + c * dp1;
      const double gp = g[p], gq = g[p + 1];
      g[p] = c * gp + s * gq;
      g[p + 1] = -s * gp + c * gq;
      if (p + 1 < hi) {
        z = s * e[p + 1];
        e[p + 1] = c * e[p + 1];
        y = e[p];
      }
    }
  }
}

__device__ double gcv_G(const double* sig, const double* c, int k, double lam, double omega) {
  const double L2 = lam * lam;
  double num = 0.0, den = 1.0;
  for (int i = 0; i < k; ++i) {
    const double s2 = sig[i] * sig[i];
    const double w = s2 + L2;
    const double t = (L2 / w) * c[i];
    num = fma(t, t, num);
    den += ((1.0 - omega) * s2 + L2) / w;
  }
  num = fma(c[k], c[k], num);
  return (double)k * num / (den * den);
}

// sign-carrying derivative of G with respect to mu = lambda^2: N' D - 2 N D'
__device__ double gcv_slope(const double* sig, const double* c, int k, double lam, double omega,
                            double* red) {
  const double L2 = lam * lam;
  double N = 0.0, dN = 0.0, Dn = 0.0, dD = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double s2 = sig[i] * sig[i];
    const double w = s2 + L2;
    const double f = L2 / w;
    const double dfdmu = s2 / (w * w);
    const double c2 = c[i] * c[i];
    N = fma(f * f, c2, N);
    dN = fma(2.0 * f * dfdmu, c2, dN);
    Dn += ((1.0 - omega) * s2 + L2) / w;
    dD += dfdmu;
  }
  N = block_sum(N, red) + c[k] * c[k];
  dN = block_sum(dN, red);
  Dn = 1.0 + block_sum(Dn, red);
  dD = omega * block_sum(dD, red);
  return dN * Dn - 2.0 * N * dD;
}

__global__ void __launch_bounds__(kT) k_projected(ProjArgs a, ProjWork w) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  __shared__ int flag;
  const int kk = a.k_first + (int)blockIdx.x;
  const int kdone = a.st ? a.st->k_done : a.k_last;
  const bool is_final = (kk == a.k_last);
  const int k = is_final ? min(kk, kdone) : kk;
  double* lam_o = a.lam_out ? a.lam_out + (kk - 1) : nullptr;
  double* res_o = a.res_out ? a.res_out + (kk - 1) : nullptr;
  if (k <= 0 || (!is_final && kk > kdone)) {
    if (threadIdx.x == 0) {
      if (lam_o) *lam_o = 0.0;
      if (res_o) *res_o = 0.0;
    }
    return;
  }
  const double beta = a.beta_ptr ? *a.beta_ptr : a.beta_val;
  const int64_t ld = k + 1;
  // workspace: packed by problem size for batched launches
  double* A = w.packed ? w.A + (int64_t)(kk - 1) * kk * (kk + 1) / 3 : w.A;
  double* Qr = w.packed ? w.Q + (int64_t)(kk - 1) * kk * (2 * kk - 1) / 6 : w.Q;  // ld k
  // shared vectors
  double* d = sm;                // k
  double* e = d + (k + 1);       // k
  double* g = e + (k + 1);       // k+1
  double* d0 = g + (k + 1);      // k   (B before the QR sweeps)
  double* e0 = d0 + (k + 1);     // k
  double* g0 = e0 + (k + 1);     // k+1
  double* taur = g0 + (k + 1);   // k
  double* vv = taur + (k + 1);   // k+1 left Householder vector
  double* sig = vv + (k + 1);    // k
  double* cc = sig + (k + 1);    // k+1
  double* z = cc + (k + 1);      // k
  double* Gv = z + (k + 1);      // kGrid

  for (int64_t t = threadIdx.x; t < (int64_t)(k + 1) * k; t += blockDim.x) {
    const int64_t col = t / (k + 1), row = t % (k + 1);
    A[t] = a.H[row + col * a.ldh];
  }
  for (int t = threadIdx.x; t <= k; t += blockDim.x) g[t] = (t == 0) ? beta : 0.0;
  __syncthreads();

  for (int j = 0; j < k; ++j) {
    // left reflector on column j, rows j..k
    const int len = k + 1 - j;
    double bh;
    const double tau = householder(A + j + j * ld, 1, len, red, &bh);
    for (int t = threadIdx.x; t < len; t += blockDim.x) vv[t] = (t == 0) ? 1.0 : A[j + t + j * ld];
    __syncthreads();
    if (threadIdx.x == 0) d[j] = bh;
    if (tau != 0.0) {
      // columns j+1..k-1 and g: one warp per column
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int cidx = j + 1 + warp; cidx <= k; cidx += nw) {
        double* colp = (cidx < k) ? (A + j + cidx * ld) : (g + j);
        double s = 0.0;
        for (int t = lane; t < len; t += 32) s = fma(vv[t], colp[t], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double ts = tau * s;
        for (int t = lane; t < len; t += 32) colp[t] = fma(-ts, vv[t], colp[t]);
      }
    }
    __syncthreads();
    // right reflector on row j, columns j+1..k-1
    if (j < k - 1) {
      const int rl = k - 1 - j;
      double be;
      const double tr = householder(A + j + (j + 1) * ld, ld, rl, red, &be);
      if (threadIdx.x == 0) {
        e[j] = be;
        taur[j] = tr;
      }
      for (int t = threadIdx.x; t < rl; t += blockDim.x)
        Qr[t + j * k] = (t == 0) ? 1.0 : A[j + (j + 1 + t) * ld];
      __syncthreads();
      if (tr != 0.0) {
        // rows j+1..k of columns j+1..k-1: s_r = sum_t A[r, j+1+t] w_t
        for (int r = j + 1 + threadIdx.x; r <= k; r += blockDim.x) {
          double s = 0.0;
          for (int t = 0; t < rl; ++t) s = fma(A[r + (j + 1 + t) * ld], Qr[t + j * k], s);
          const double ts = tr * s;
          for (int t = 0; t < rl; ++t)
            A[r + (j + 1 + t) * ld] = fma(-ts, Qr[t + j * k], A[r + (j + 1 + t) * ld]);
        }
      }
      __syncthreads();
    } else if (threadIdx.x == 0) {
      taur[j] = 0.0;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t <= k; t += blockDim.x) {
    g0[t] = g[t];
    if (t < k) {
      d0[t] = d[t];
      e0[t] = (t + 1 < k) ? e[t] : 0.0;
    }
  }
  __syncthreads();

  // singular values and c = beta U^T e1
  if (threadIdx.x == 0) flag = bidiag_svd(d, e, g, k);
  __syncthreads();
  // sort |d| descending (rank by count of larger, ties by index)
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double si = fabs(d[i]);
    int rank = 0;
    for (int j2 = 0; j2 < k; ++j2) {
      const double sj = fabs(d[j2]);
      rank += (sj > si) || (sj == si && j2 < i);
    }
    sig[rank] = si;
    cc[rank] = g[i];
  }
  if (threadIdx.x == 0) cc[k] = g[k];
  __syncthreads();

  // lambda
  double lam = 0.0;
  if (a.rule == LSLU_LAMBDA_FIXED) {
    lam = a.lambda;
  } else if (a.rule == LSLU_LAMBDA_GCV || a.rule == LSLU_LAMBDA_WGCV) {
    const double omega = a.rule == LSLU_LAMBDA_GCV ? 1.0 : (double)(k + 1) / (double)a.m;
    const double s1 = sig[0];
    if (s1 > 0.0) {
      for (int t = threadIdx.x; t < kGrid; t += blockDim.x) {
        const double lt = s1 * pow(10.0, -14.0 + 0.0625 * t);
        Gv[t] = gcv_G(sig, cc, k, lt, omega);
      }
      __syncthreads();
      __shared__ int ibest;
      if (threadIdx.x == 0) {
        int ib = 0;
        for (int t = 1; t < kGrid; ++t)
          if (Gv[t] < Gv[ib]) ib = t;
        ibest = ib;
      }
      __syncthreads();
      const int ib = ibest;
      lam = s1 * pow(10.0, -14.0 + 0.0625 * ib);
      if (ib > 0 && ib < kGrid - 1) {
        double lo = log(s1 * pow(10.0, -14.0 + 0.0625 * (ib - 1)));
        double hi = log(s1 * pow(10.0, -14.0 + 0.0625 * (ib + 1)));
        const double slo = gcv_slope(sig, cc, k, exp(lo), omega, red);
        const double shi = gcv_slope(sig, cc, k, exp(hi), omega, red);
        if (slo < 0.0 && shi > 0.0) {
          for (int it = 0; it < 64; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (gcv_slope(sig, cc, k, exp(mid), omega, red) < 0.0)
              lo = mid;
            else
              hi = mid;
          }
          const double lb = exp(0.5 * (lo + hi));
          if (!(gcv_G(sig, cc, k, lb, omega) > Gv[ib])) lam = lb;
        }
      }
    }
  }

  // projected residual
  double rs = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double ri;
    if (lam == 0.0) {
      ri = 0.0;
    } else {
      const double L2 = lam * lam;
      ri = L2 / (sig[i] * sig[i] + L2) * cc[i];
    }
    rs = fma(ri, ri, rs);
  }
  rs = block_sum(rs, red);
  if (threadIdx.x == 0) {
    if (lam_o) *lam_o = lam;
    if (res_o) *res_o = sqrt(rs + cc[k] * cc[k]);
    if (flag) {  // the QR sweeps did not converge: report NaN
      if (lam_o) *lam_o = NAN;
      if (res_o) *res_o = NAN;
    }
  }
  if (a.sig)
    for (int i = threadIdx.x; i < k; i += blockDim.x) a.sig[(int64_t)blockIdx.x * a.ldsig + i] = sig[i];
  if (a.cvec)
    for (int i = threadIdx.x; i <= k; i += blockDim.x) a.cvec[(int64_t)blockIdx.x * a.ldc + i] = cc[i];

  if (!(is_final && a.want_y)) return;
  // z = argmin ||g0 - B z||^2 + lam^2 ||z||^2 on the original bidiagonal
  if (threadIdx.x == 0) {
    if (lam == 0.0) {
      for (int i = k - 1; i >= 0; --i) {
        const double ri = g0[i] - (i + 1 < k ? e0[i] * z[i + 1] : 0.0);
        z[i] = ri / d0[i];
      }
    } else {
      // Givens elimination of the lambda rows of [B; lam I] (Elden): the
      // current lambda row holds ell at column i and right-hand side hl; it
      // is rotated into B-row i, and the fill it receives at column i+1 is
      // rotated into lambda row i+1.  d0/e0/g0 become the bidiagonal R and
      // its right-hand side.
      double ell = lam, hl = 0.0;
      for (int i = 0; i < k; ++i) {
        double c, s, r;
        givens(d0[i], ell, c, s, r);
        d0[i] = r;
        const double ei = (i + 1 < k) ? e0[i] : 0.0;
        e0[i] = c * ei;
        const double gi = g0[i];
        g0[i] = c * gi + s * hl;
        const double fill = -s * ei;
        const double hnew = -s * gi + c * hl;
        if (i + 1 < k) {
          double c2, s2, r2;
          givens(lam, fill, c2, s2, r2);
          ell = r2;
          hl = s2 * hnew;
        }
      }
      for (int i = k - 1; i >= 0; --i) {
        const double ri = g0[i] - (i + 1 < k ? e0[i] * z[i + 1] : 0.0);
        z[i] = ri / d0[i];
      }
    }
  }
  __syncthreads();
  // y = Q z = H_0 H_1 ... z : apply the right reflectors in reverse order
  for (int j = k - 2; j >= 0; --j) {
    const double tr = taur[j];
    if (tr == 0.0) continue;
    const int rl = k - 1 - j;
    double s = 0.0;
    for (int t = threadIdx.x; t < rl; t += blockDim.x) s = fma(Qr[t + j * k], z[j + 1 + t], s);
    s = block_sum(s, red);
    for (int t = threadIdx.x; t < rl; t += blockDim.x) z[j + 1 + t] = fma(-tr * s, Qr[t + j * k], z[j + 1 + t]);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) a.y[i] = z[i];
}

}  // namespace

cudaError_t launch_projected(const ProjArgs& a, ProjWork& w, cudaStream_t s) {
  const int nprob = a.k_last - a.k_first + 1;
  if (nprob <= 0) return cudaSuccess;
  if (nprob > 1 && !w.packed) return cudaErrorInvalidValue;
  const int kmax = a.k_last;
  const size_t smem = (size_t)(12 * (kmax + 1) + kGrid) * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_projected, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  k_projected<<<nprob, kT, smem, s>>>(a, w);
  return cudaGetLastError();
}

}  // namespace lslu
