// Projected Tikhonov problem of Hybrid LSLU (Eq. TSP, Section 3.3), FP64.
//
// One thread-block cluster solves the problem for one (k+1) x k upper
// Hessenberg H and beta:
//   1. Householder bidiagonalisation H = P B Q^T with B lower bidiagonal
//      ((k+1) x k: alpha_j on the diagonal, beta_{j+1} below it) and
//      P e1 = e1 (each step first reflects row j from the right, then column
//      j below the diagonal from the left, so no left reflector touches
//      row 0).  Columns of H are dealt round robin to the CTAs of the cluster
//      and stay in shared memory; partial sums travel through global memory
//      between cluster barriers.
//   2. Singular values of B = positive eigenvalues of the Golub-Kahan
//      tridiagonal T (order 2k+1, zero diagonal, off-diagonals alpha_0,
//      beta_1, alpha_1, ..., beta_k): Sturm counts on a geometric grid
//      bracket each one, then Newton's method on det(T - theta I) with
//      bisection safeguards refines it; one thread per singular value.
//   3. c = beta U^T e1 (Eq. gcv2): since P e1 = e1, c_i^2 is 2 beta^2 times the
//      squared first component of T's eigenvector for sigma_i, read off as
//      the residue of e1^T (T - theta)^-1 e1 = det(T_{2:,2:} - theta) /
//      det(T - theta); c_{k+1}^2 = beta^2 / ||u||^2 for the null vector u of B^T.
//   4. lambda by the rule: none (0), fixed, GCV (Eq. gcv2) or weighted GCV
//      with omega = (k+1)/m (Eq. wgcv), minimised on a 257-point log grid
//      sigma_1 * 10^[-14, 2] and refined by 64 bisection steps on the sign of
//      dG/d(lambda^2) between the neighbours of the best grid point.
//   5. Projected residual ||beta e1 - H y|| = sqrt(sum f_i^2 c_i^2 +
//      c_{k+1}^2) with f_i = lambda^2 / (sigma_i^2 + lambda^2).
//   6. y = Q z with z = argmin ||beta e1 - B z||^2 + lambda^2 ||z||^2, by the
//      Givens sweep for damped bidiagonal least squares and back substitution.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>

#include "lslu_internal.cuh"

namespace cg = cooperative_groups;

namespace lslu {

namespace {

constexpr int kT = 256;
constexpr int kGrid = 257;        // lambda grid points
constexpr int kSturmGrid = 2048;  // geometric grid that brackets the singular values
constexpr double kEps = 2.220446049250313e-16;
constexpr size_t kSmemCap = 200 * 1024;

__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Four block-wide sums at once (one pair of barriers).
__device__ void block_sum4(double (&v)[4], double* red4) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red4[q * 32 + w] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double t = lane < nw ? red4[q * 32 + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    v[q] = t;
  }
}

// Reflector I - tau v v^T (v0 = 1, v_rest = rest * scale) mapping
// x = (x0, rest), ||rest||^2 = ss, to bh e1.
__device__ __forceinline__ void house(double x0, double ss, double& tau, double& bh,
                                      double& scale) {
  if (ss == 0.0) {
    tau = 0.0;
    bh = x0;
    scale = 0.0;
    return;
  }
  const double nrm = sqrt(fma(x0, x0, ss));
  bh = x0 >= 0.0 ? -nrm : nrm;
  tau = (bh - x0) / bh;
  scale = 1.0 / (x0 - bh);
}

// Squared off-diagonals t_j^2 of the Golub-Kahan tridiagonal T (1-based j,
// t_j couples rows j and j+1): t_{2i+1} = alpha_i, t_{2i+2} = beta_{i+1}.
// The recurrences below read t2[j]; the FP64 pipe is the scarce resource on
// this GPU, so signs and zero tests use integer operations on the bits and
// the over/underflow check runs once every 8 steps (|p| grows by at most a
// factor (|theta| + 2 max|t|)^8 < 2^160 between checks for the matrices
// solved here, far inside the 2^+-400 rescaling margin).
__device__ __forceinline__ int sign_change(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  // a change, or an exact zero (which counts as a change)
  return (int)(((ia ^ ib) < 0) | ((ia << 1) == 0));
}

__device__ __forceinline__ bool needs_rescale(double p0, double pm1, int& s) {
  const int e0 = (int)((__double_as_longlong(p0) >> 52) & 0x7ff);
  const int e1 = (int)((__double_as_longlong(pm1) >> 52) & 0x7ff);
  const int e = e0 > e1 ? e0 : e1;
  if (e > 1023 + 400) {
    s = -400;
    return true;
  }
  if (e < 1023 - 400 && e0 != 0) {
    s = 400;
    return true;
  }
  return false;
}

// Leading-minor recurrence p_j = -theta p_{j-1} - t_{j-1}^2 p_{j-2} of
// det(T - theta I), optionally with its theta-derivative.  Returns the number
// of sign changes of p_0..p_n (= eigenvalues of T below theta); p, dp receive
// the determinant and derivative scaled by 2^-exp2.
template <bool kDeriv>
__device__ int sturm(const double* t2, int n, double theta, double& p, double& dp, int& exp2) {
  double pm1 = 1.0, p0 = -theta;
  double dm1 = 0.0, d0 = -1.0;
  int cnt = (int)(__double_as_longlong(p0) < 0);
  int e = 0;
  int j = 2;
  while (j <= n) {
    const int jend = min(n, j + 7);
    for (; j <= jend; ++j) {
      const double tt = t2[j - 1];
      const double pj = fma(-theta, p0, -tt * pm1);
      if (kDeriv) {
        const double dj = fma(-theta, d0, fma(-tt, dm1, -p0));
        dm1 = d0;
        d0 = dj;
      }
      cnt += sign_change(pj, p0);
      pm1 = p0;
      p0 = pj;
    }
    int sc;
    if (needs_rescale(p0, pm1, sc)) {
      p0 = ldexp(p0, sc);
      pm1 = ldexp(pm1, sc);
      if (kDeriv) {
        d0 = ldexp(d0, sc);
        dm1 = ldexp(dm1, sc);
      }
      e -= sc;
    }
  }
  p = p0;
  dp = d0;
  exp2 = e;
  return cnt;
}

// det(T_{2:n,2:n} - theta I) by the trailing-minor recurrence, scaled by 2^-exp2.
__device__ double trailing_det(const double* t2, int n, double theta, int& exp2) {
  double r1 = 1.0, r0 = -theta;  // r_{n+1}, r_n
  int e = 0;
  int j = n - 1;
  while (j >= 2) {
    const int jend = max(2, j - 7);
    for (; j >= jend; --j) {
      const double rj = fma(-theta, r0, -t2[j] * r1);
      r1 = r0;
      r0 = rj;
    }
    int sc;
    if (needs_rescale(r0, r1, sc)) {
      r0 = ldexp(r0, sc);
      r1 = ldexp(r1, sc);
      e -= sc;
    }
  }
  exp2 = e;
  return r0;
}

__device__ double gcv_G(const double* sig, const double* c2, int k, double lam, double omega) {
  const double L2 = lam * lam;
  double num = 0.0, den = 1.0;
  for (int i = 0; i < k; ++i) {
    const double s2 = sig[i] * sig[i];
    const double rw = 1.0 / (s2 + L2);
    const double f = L2 * rw;
    num = fma(f * f, c2[i], num);
    den = fma(fma(1.0 - omega, s2, L2), rw, den);
  }
  num += c2[k];
  return (double)k * num / (den * den);
}

// sign-carrying derivative of G with respect to mu = lambda^2: N' D - 2 N D'
__device__ double gcv_slope(const double* sig, const double* c2, int k, double lam, double omega,
                            double* red4) {
  const double L2 = lam * lam;
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // N, N', D - 1, D'/omega
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double s2 = sig[i] * sig[i];
    const double rw = 1.0 / (s2 + L2);
    const double f = L2 * rw;
    const double dfdmu = s2 * rw * rw;
    v[0] = fma(f * f, c2[i], v[0]);
    v[1] = fma(2.0 * f * dfdmu, c2[i], v[1]);
    v[2] = fma(fma(1.0 - omega, s2, L2), rw, v[2]);
    v[3] += dfdmu;
  }
  block_sum4(v, red4);
  const double N = v[0] + c2[k], dN = v[1], Dn = 1.0 + v[2], dD = omega * v[3];
  return dN * Dn - 2.0 * N * dD;
}

// Global work space of one problem of size kk (all cross-CTA traffic).
struct Slots {
  double* part_s;  // CL x (kk+1) partial sums
  double* part_n;  // CL partial norms
  double* x0;      // leading entry of the current row
  double* vl;      // kk+1 left reflector
  double* taul;    // its tau
  double* al;      // kk+1 alpha
  double* be;      // kk+1 beta (be[0] unused)
  double* taur;    // kk+1 right-reflector taus
  double* sig;     // kk+1 singular values
  double* c2;      // kk+1 squared weights
  int* gcnt;       // kSturmGrid Sturm counts
  double* gv;      // kGrid GCV values
  double* Qs;      // kk x kk: right reflector j in row j (entries c >= j)
  double* A;       // (kk+1) x kk slab when shared memory is too small
};

__device__ Slots carve(double* base, int kk, int CL) {
  Slots s;
  double* p = base;
  s.part_s = p; p += (int64_t)CL * (kk + 1);
  s.part_n = p; p += CL;
  s.x0 = p; p += 2;
  s.vl = p; p += kk + 1;
  s.taul = p; p += 2;
  s.al = p; p += kk + 1;
  s.be = p; p += kk + 1;
  s.taur = p; p += kk + 1;
  s.sig = p; p += kk + 1;
  s.c2 = p; p += kk + 1;
  s.gcnt = reinterpret_cast<int*>(p); p += kSturmGrid / 2;
  s.gv = p; p += kGrid + 1;
  s.Qs = p; p += (int64_t)kk * kk;
  s.A = p;
  return s;
}

__device__ __forceinline__ double ldg_cg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kT) k_projected(ProjArgs a, ProjWork w) {
  extern __shared__ double smem[];
  __shared__ double red[33];
  __shared__ double red4[128];
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int prob = blockIdx.x / CL;
  const bool batch = a.nbatch > 1;   // one final problem per batch entry
  const int p = batch ? prob : 0;
  const int kk = batch ? a.k_last : a.k_first + prob;
  const DevState* sp = a.st ? a.st + p : nullptr;
  const int kdone = sp ? sp->k_done : a.k_last;
  const bool is_final = (kk == a.k_last);
  const int k = is_final ? min(kk, kdone) : kk;
  double* lam_o = a.lam_out ? a.lam_out + (batch ? p : kk - 1) : nullptr;
  double* res_o = a.res_out ? a.res_out + (batch ? p : kk - 1) : nullptr;
  double* tr_o = a.tr_out ? a.tr_out + (batch ? p : kk - 1) : nullptr;
  if (k <= 0 || (!is_final && kk > kdone)) {
    if (rank == 0 && threadIdx.x == 0) {
      if (lam_o) *lam_o = 0.0;
      if (res_o) *res_o = 0.0;
      if (tr_o) *tr_o = 0.0;
    }
    return;  // the whole cluster leaves: no barrier is left waiting
  }
  const double beta = sp ? sp->beta : a.beta_val;
  const double* Hp = a.H + (int64_t)p * a.strideH;
  double* yp = a.y ? a.y + (int64_t)p * a.ldy : nullptr;
  Slots S = carve(w.base + (w.packed ? w.offsets[kk] : (int64_t)p * w.slot_stride), kk, CL);
  const int64_t ld = k + 1;
  const int kmax = a.k_last;
  // shared layout: [al, be, sig, c2, vls : 5 x (kmax+1)] [t2 : 2 x (kmax+1)]
  // [slab or scratch]
  double* al = smem;
  double* be = al + (kmax + 1);
  double* sig = be + (kmax + 1);
  double* c2 = sig + (kmax + 1);
  double* vls = c2 + (kmax + 1);
  double* t2 = vls + (kmax + 1);
  double* slab = t2 + 2 * (kmax + 1);
  const bool in_smem = w.slab_in_smem != 0;
  auto col = [&](int c) -> double* {
    return in_smem ? slab + (int64_t)(c / CL) * ld : S.A + (int64_t)c * ld;
  };
  auto first_own = [&](int x) -> int { return x + ((rank - x) % CL + CL) % CL; };
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  unsigned long long* ts = (a.tstamp && is_final && rank == 0 && tid == 0) ? a.tstamp : nullptr;
  if (ts) ts[0] = gtimer();

  for (int c = rank; c < k; c += CL) {
    double* cp = col(c);
    for (int r = tid; r <= k; r += nt) cp[r] = Hp[r + (int64_t)c * a.ldh];
  }
  __syncthreads();

  // ---- 1. bidiagonalisation ------------------------------------------------
  unsigned long long tsec[6] = {0, 0, 0, 0, 0, 0}, tprev = ts ? gtimer() : 0;
  auto lap = [&](int q) {
    if (ts) {
      const unsigned long long now = gtimer();
      tsec[q] += now - tprev;
      tprev = now;
    }
  };
  for (int j = 0; j < k; ++j) {
    // right reflector on row j, columns j..k-1
    if (tid == 0) {
      double ss = 0.0;
      for (int c = first_own(j + 1); c < k; c += CL) {
        const double x = col(c)[j];
        ss = fma(x, x, ss);
      }
      __stcg(S.part_n + rank, ss);
      if (j % CL == rank) __stcg(S.x0, col(j)[j]);
      __threadfence();
    }
    lap(0);
    cluster.sync();
    lap(1);
    double tss = 0.0;
    {
      double pv[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) pv[q] = q < CL ? ldg_cg(S.part_n + q) : 0.0;
      for (int q = 0; q < CL; ++q) tss += pv[q];
    }
    const double x0r = ldg_cg(S.x0);
    double taur, bh, sc;
    house(x0r, tss, taur, bh, sc);
    if (tid == 0) {
      for (int c = first_own(j); c < k; c += CL) {
        const double wc = (c == j) ? 1.0 : col(c)[j] * sc;
        col(c)[j] = wc;
        __stcg(S.Qs + (int64_t)j * k + c, wc);
      }
      if (rank == 0) {
        S.al[j] = bh;
        S.taur[j] = taur;
      }
    }
    __syncthreads();
    // partial s_r = sum_{own c >= j} A[r, c] w_c, r = j+1..k
    const int c0 = first_own(j);
    for (int r = j + 1 + tid; r <= k; r += nt) {
      double s0 = 0.0, s1 = 0.0;
      int c = c0;
      for (; c + CL < k; c += 2 * CL) {
        s0 = fma(col(c)[r], col(c)[j], s0);
        s1 = fma(col(c + CL)[r], col(c + CL)[j], s1);
      }
      if (c < k) s0 = fma(col(c)[r], col(c)[j], s0);
      __stcg(S.part_s + (int64_t)rank * ld + r, s0 + s1);
    }
    __threadfence();
    lap(2);
    cluster.sync();
    lap(1);
    if (taur != 0.0) {
      for (int r = j + 1 + tid; r <= k; r += nt) {
        double pv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) pv[q] = q < CL ? ldg_cg(S.part_s + (int64_t)q * ld + r) : 0.0;
        double s = 0.0;
        for (int q = 0; q < CL; ++q) s += pv[q];
        const double ts = taur * s;
        for (int c = c0; c < k; c += CL) col(c)[r] = fma(-ts, col(c)[j], col(c)[r]);
      }
    }
    __syncthreads();
    // left reflector on column j, rows j+1..k (owner of column j)
    if (j % CL == rank) {
      double* cp = col(j);
      double s2 = 0.0;
      for (int r = j + 2 + tid; r <= k; r += nt) s2 = fma(cp[r], cp[r], s2);
      s2 = block_sum(s2, red);
      double taul, bl, scl;
      house(cp[j + 1], s2, taul, bl, scl);
      for (int r = j + 1 + tid; r <= k; r += nt) __stcg(S.vl + r, (r == j + 1) ? 1.0 : cp[r] * scl);
      if (tid == 0) {
        __stcg(S.taul, taul);
        S.be[j + 1] = bl;
      }
      __threadfence();
    }
    lap(3);
    cluster.sync();
    lap(1);
    const double taul = ldg_cg(S.taul);
    if (taul != 0.0) {
      for (int r = j + 1 + tid; r <= k; r += nt) vls[r] = ldg_cg(S.vl + r);
      __syncthreads();
      // own columns c > j, one warp per column: t = v^T A[j+1:, c]
      for (int c = first_own(j + 1) + warp * CL; c < k; c += CL * nw) {
        double* cp = col(c);
        double t = 0.0;
        for (int r = j + 1 + lane; r <= k; r += 32) t = fma(vls[r], cp[r], t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        const double tt = taul * t;
        for (int r = j + 1 + lane; r <= k; r += 32) cp[r] = fma(-tt, vls[r], cp[r]);
      }
    }
    __syncthreads();
    lap(4);
  }
  if (ts)
    for (int q = 0; q < 5; ++q) ts[8 + q] = tsec[q];
  __threadfence();
  cluster.sync();

  if (ts) ts[1] = gtimer();
  // ---- 2./3. singular values and weights -----------------------------------
  for (int i = tid; i <= k; i += nt) {
    al[i] = i < k ? ldg_cg(S.al + i) : 0.0;
    be[i] = i > 0 ? ldg_cg(S.be + i) : 0.0;
  }
  __syncthreads();
  const int n = 2 * k + 1;
  for (int i = tid; i < k; i += nt) {
    t2[2 * i + 1] = al[i] * al[i];
    t2[2 * i + 2] = be[i + 1] * be[i + 1];
  }
  __syncthreads();
  __shared__ double Gsh;
  if (tid == 0) {  // Gershgorin bound of T
    double gm = 0.0;
    for (int i = 0; i < k; ++i) {
      gm = fmax(gm, fabs(al[i]) + fabs(be[i + 1]));
      if (i + 1 < k) gm = fmax(gm, fabs(be[i + 1]) + fabs(al[i + 1]));
    }
    gm = fmax(gm, fabs(al[0]));
    gm = fmax(gm, fabs(be[k]));
    Gsh = gm;
  }
  __syncthreads();
  const double G = Gsh;
  const int gthreads = CL * nt;
  const int gid = rank * nt + tid;
  // grid theta_g = G 2^(-60 + 60 g / (NG - 1)); gcnt = number of sigma below
  for (int g = gid; g < kSturmGrid; g += gthreads) {
    const double th = G * exp2(-60.0 + 60.0 * g / (kSturmGrid - 1));
    double p, dp;
    int e2;
    __stcg(S.gcnt + g, sturm<false>(t2, n, th, p, dp, e2) - (k + 1));
  }
  __threadfence();
  cluster.sync();
  if (ts) ts[2] = gtimer();
  // sigma_i for i = rank, rank + CL, ... : the FP64 work is spread over the cluster
  for (int i = rank + CL * tid; i < k; i += CL * nt) {
    const int target = k - 1 - i;  // sigma_i (i-th largest) has target sigmas below it
    int glo = 0, ghi = kSturmGrid;  // first grid point with count > target (binary search)
    while (glo < ghi) {
      const int mid = (glo + ghi) >> 1;
      if (__ldcg(S.gcnt + mid) <= target)
        glo = mid + 1;
      else
        ghi = mid;
    }
    const int g = glo;
    double lo = g > 0 ? G * exp2(-60.0 + 60.0 * (g - 1) / (kSturmGrid - 1)) : 0.0;
    double hi = g < kSturmGrid ? G * exp2(-60.0 + 60.0 * g / (kSturmGrid - 1)) : 2.0 * G + 1.0;
    int clo = g > 0 ? __ldcg(S.gcnt + g - 1) : 0;
    int chi = g < kSturmGrid ? __ldcg(S.gcnt + g) : k;
    double th = lo > 0.0 ? sqrt(lo * hi) : 0.5 * hi;
    double p = 0.0, dp = 0.0, pth = -1.0;
    int ep = 0;
    for (int it = 0; it < 200; ++it) {
      if (hi - lo <= 4.0 * kEps * hi) break;
      const int cnt = sturm<true>(t2, n, th, p, dp, ep) - (k + 1);
      pth = th;
      if (cnt <= target) {
        lo = th;
        clo = cnt;
      } else {
        hi = th;
        chi = cnt;
      }
      double nx;
      if (chi - clo == 1 && dp != 0.0) {
        nx = th - p / dp;  // Newton step on det(T - theta I)
        if (fabs(nx - th) <= 4.0 * kEps * th) {  // converged (the step is rounding noise)
          if (nx > lo && nx < hi) th = nx;
          break;
        }
        if (!(nx > lo && nx < hi)) nx = lo > 0.0 ? sqrt(lo * hi) : 0.5 * hi;
      } else {
        nx = (lo > 0.0 && hi / lo > 4.0) ? sqrt(lo * hi) : 0.5 * (lo + hi);
      }
      th = nx;
    }
    // weight: first component^2 of T's eigenvector = -det(T_{2:,2:} - th) / det'(T - th);
    // the derivative of the last Newton evaluation is reused when it was taken
    // at (numerically) the same theta
    if (!(fabs(pth - th) <= 1e-10 * th)) sturm<true>(t2, n, th, p, dp, ep);
    int eq;
    const double q = trailing_det(t2, n, th, eq);
    double wgt = (dp != 0.0) ? ldexp(-q / dp, eq - ep) : 0.0;
    if (!(wgt >= 0.0)) wgt = 0.0;
    __stcg(S.sig + i, th);
    __stcg(S.c2 + i, 2.0 * beta * beta * wgt);
  }
  if (rank == 0 && tid == 0) {
    // null vector of B^T: u_{i+1} = -alpha_i u_i / beta_{i+1}, u_0 = 1
    double u = 1.0, nrm2 = 1.0;
    int e = 0;  // u and nrm2 carry the factors 2^-e/2 and 2^-e
    for (int i = 0; i < k; ++i) {
      if (be[i + 1] == 0.0) break;
      u = -al[i] * u / be[i + 1];
      nrm2 = fma(u, u, nrm2);
      if (nrm2 > 0x1p+600) {
        u = ldexp(u, -300);
        nrm2 = ldexp(nrm2, -600);
        e += 600;
      }
    }
    __stcg(S.c2 + k, ldexp(beta * beta / nrm2, -e));
  }
  __threadfence();
  cluster.sync();
  if (ts) ts[3] = gtimer();
  for (int i = tid; i <= k; i += nt) {
    sig[i] = i < k ? ldg_cg(S.sig + i) : 0.0;
    c2[i] = ldg_cg(S.c2 + i);
  }
  __syncthreads();
  const bool gcv = (a.rule == LSLU_LAMBDA_GCV || a.rule == LSLU_LAMBDA_WGCV) && sig[0] > 0.0;
  const double mrows = a.mvec ? (double)a.mvec[p] : (double)a.m;
  const double omega = a.rule == LSLU_LAMBDA_WGCV ? (double)(k + 1) / mrows : 1.0;
  const double s1 = sig[0];
  // ---- 4. lambda: the grid is shared by the cluster, the refinement by CTA 0
  double* Gv = S.gv;
  if (gcv) {
    for (int t = rank + CL * tid; t < kGrid; t += CL * nt)
      __stcg(Gv + t, gcv_G(sig, c2, k, s1 * pow(10.0, -14.0 + 0.0625 * t), omega));
  }
  __threadfence();
  cluster.sync();
  if (rank != 0) return;
  double lam = 0.0;
  __shared__ int ibest;
  if (a.rule == LSLU_LAMBDA_FIXED) {
    lam = a.lambda;
  } else if (gcv) {
    if (tid == 0) {
      int ib = 0;
      double gb = __ldcg(Gv);
      for (int t = 1; t < kGrid; ++t) {
        const double gt = __ldcg(Gv + t);
        if (gt < gb) {
          gb = gt;
          ib = t;
        }
      }
      ibest = ib;
    }
    __syncthreads();
    const int ib = ibest;
    const double gib = __ldcg(Gv + ib);
    lam = s1 * pow(10.0, -14.0 + 0.0625 * ib);
    if (ib > 0 && ib < kGrid - 1) {
      double lo = log(s1 * pow(10.0, -14.0 + 0.0625 * (ib - 1)));
      double hi = log(s1 * pow(10.0, -14.0 + 0.0625 * (ib + 1)));
      const double slo = gcv_slope(sig, c2, k, exp(lo), omega, red4);
      const double shi = gcv_slope(sig, c2, k, exp(hi), omega, red4);
      if (slo < 0.0 && shi > 0.0) {
        for (int it = 0; it < 64; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (gcv_slope(sig, c2, k, exp(mid), omega, red4) < 0.0)
            lo = mid;
          else
            hi = mid;
        }
        const double lb = exp(0.5 * (lo + hi));
        if (!(gcv_G(sig, c2, k, lb, omega) > gib)) lam = lb;
      }
    }
  }

  // ---- 5. projected residual (and the filter-factor trace of Eq. stop2) ----
  double rs = 0.0, tr = 0.0;
  if (lam != 0.0) {
    const double L2 = lam * lam;
    for (int i = tid; i < k; i += nt) {
      const double f = L2 / (sig[i] * sig[i] + L2);
      rs = fma(f * f, c2[i], rs);
      tr += f;
    }
  }
  rs = block_sum(rs, red);
  if (tr_o) tr = block_sum(tr, red);
  if (tid == 0) {
    if (lam_o) *lam_o = lam;
    if (res_o) *res_o = sqrt(rs + c2[k]);
    if (tr_o) *tr_o = tr;
  }
  if (a.sig)
    for (int i = tid; i < k; i += nt) a.sig[(int64_t)prob * a.ldsig + i] = sig[i];
  if (a.cvec)
    for (int i = tid; i <= k; i += nt) a.cvec[(int64_t)prob * a.ldc + i] = sqrt(c2[i]);
  if (!(is_final && a.want_y && yp)) return;

  if (ts) ts[5] = gtimer();
  // ---- 6. y = Q z ----------------------------------------------------------
  // (the slab is no longer needed: its space holds z and the sweep results)
  double* z = slab;
  double* rho = z + (k + 1);
  double* thv = rho + (k + 1);
  double* ph = thv + (k + 1);
  if (tid == 0) {
    double rbar = al[0], phibar = beta;
    for (int j = 0; j < k; ++j) {
      double rhat = rbar, phib = phibar;
      if (lam != 0.0) {  // rotation that removes lambda-row j
        const double r1 = hypot(rbar, lam);
        phib = (rbar / r1) * phibar;
        rhat = r1;
      }
      const double bj = be[j + 1];  // rotation that removes beta_{j+1}
      const double r = hypot(rhat, bj);
      const double cs = rhat / r, sn = bj / r;
      rho[j] = r;
      ph[j] = cs * phib;
      phibar = sn * phib;
      if (j + 1 < k) {
        thv[j] = sn * al[j + 1];
        rbar = -cs * al[j + 1];
      }
    }
    z[k - 1] = ph[k - 1] / rho[k - 1];
    for (int j = k - 2; j >= 0; --j) z[j] = (ph[j] - thv[j] * z[j + 1]) / rho[j];
  }
  __syncthreads();
  if (ts) ts[6] = gtimer();
  for (int j = k - 1; j >= 0; --j) {  // z <- Q_j z, j = k-1 .. 0
    const double tr = ldg_cg(S.taur + j);
    if (tr == 0.0) continue;
    double s = 0.0;
    for (int c = j + tid; c < k; c += nt) s = fma(ldg_cg(S.Qs + (int64_t)j * k + c), z[c], s);
    s = block_sum(s, red);
    for (int c = j + tid; c < k; c += nt) z[c] = fma(-tr * s, ldg_cg(S.Qs + (int64_t)j * k + c), z[c]);
    __syncthreads();
  }
  for (int i = tid; i < k; i += nt) yp[i] = z[i];
  if (ts) ts[7] = gtimer();
}

// ---- optimal lambda (needs x_true) ----------------------------------------
// y(lam) = Q z(lam) from the factorisation H = P B Q^T that k_projected leaves
// in its work slot (alpha, beta of B, the right reflectors), z(lam) by the
// same Givens sweep as phase 6, and E(lam) - ||x_true||^2 = y^T G y - 2 g^T y
// with G = L^T L (k x k) and g = L^T x_true.  sm holds 4 (k+1) doubles.
__device__ double opt_eval(const Slots& S, int k, double beta, double lam,
                           const double* __restrict__ G, const double* __restrict__ g,
                           double* sm, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double* z = sm;
  double* rho = z + (k + 1);
  double* thv = rho + (k + 1);
  double* ph = thv + (k + 1);
  if (tid == 0) {
    double rbar = ldg_cg(S.al), phibar = beta;
    for (int j = 0; j < k; ++j) {
      double rhat = rbar, phib = phibar;
      if (lam != 0.0) {
        const double r1 = hypot(rbar, lam);
        phib = (rbar / r1) * phibar;
        rhat = r1;
      }
      const double bj = ldg_cg(S.be + j + 1);
      const double r = hypot(rhat, bj);
      const double cs = rhat / r, sn = bj / r;
      rho[j] = r;
      ph[j] = cs * phib;
      phibar = sn * phib;
      if (j + 1 < k) {
        const double an = ldg_cg(S.al + j + 1);
        thv[j] = sn * an;
        rbar = -cs * an;
      }
    }
    z[k - 1] = ph[k - 1] / rho[k - 1];
    for (int j = k - 2; j >= 0; --j) z[j] = (ph[j] - thv[j] * z[j + 1]) / rho[j];
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {  // z <- Q_j z
    const double tr = ldg_cg(S.taur + j);
    if (tr == 0.0) continue;
    double s = 0.0;
    for (int c = j + tid; c < k; c += nt) s = fma(ldg_cg(S.Qs + (int64_t)j * k + c), z[c], s);
    s = block_sum(s, red);
    for (int c = j + tid; c < k; c += nt) z[c] = fma(-tr * s, ldg_cg(S.Qs + (int64_t)j * k + c), z[c]);
    __syncthreads();
  }
  double e = 0.0;
  for (int i = tid; i < k; i += nt) {
    double t = 0.0;
    for (int jj = 0; jj < k; ++jj) t = fma(G[(int64_t)jj * k + i], z[jj], t);
    e = fma(z[i], t - 2.0 * g[i], e);
  }
  return block_sum(e, red);
}

// One block per point of the lambda grid (the grid of the GCV search).
__global__ void __launch_bounds__(kT) k_opt_grid(ProjWork w, int K, const DevState* st,
                                                 const double* G, const double* g, double* Eg) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  const Slots S = carve(w.base, K, w.cluster);
  const int k = min(K, st->k_done);
  const double s1 = ldg_cg(S.sig);
  if (k <= 0 || !(s1 > 0.0)) {
    if (threadIdx.x == 0) Eg[blockIdx.x] = 0.0;
    return;
  }
  const double lam = s1 * pow(10.0, -14.0 + 0.0625 * (int)blockIdx.x);
  const double e = opt_eval(S, k, st->beta, lam, G, g, sm, red);
  if (threadIdx.x == 0) Eg[blockIdx.x] = e;
}

// The best grid point (ties: the smaller lambda), then 64 golden-section
// steps in log(lambda) between its neighbours; one block.
__global__ void __launch_bounds__(kT) k_opt_refine(ProjWork w, int K, const DevState* st,
                                                   const double* G, const double* g,
                                                   const double* Eg, double* lam_out) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  __shared__ int ib;
  const Slots S = carve(w.base, K, w.cluster);
  const int k = min(K, st->k_done);
  const double s1 = ldg_cg(S.sig);
  if (k <= 0 || !(s1 > 0.0)) {
    if (threadIdx.x == 0) *lam_out = 0.0;
    return;
  }
  if (threadIdx.x == 0) {
    int b = 0;
    for (int i = 1; i < kGrid; ++i)
      if (Eg[i] < Eg[b]) b = i;
    ib = b;
  }
  __syncthreads();
  const int b = ib;
  double lam = s1 * pow(10.0, -14.0 + 0.0625 * b);
  if (b > 0 && b < kGrid - 1) {
    const double phi = 0.5 * (sqrt(5.0) - 1.0);
    double lo = log(s1 * pow(10.0, -14.0 + 0.0625 * (b - 1)));
    double hi = log(s1 * pow(10.0, -14.0 + 0.0625 * (b + 1)));
    const double beta = st->beta;
    double c = hi - phi * (hi - lo), d = lo + phi * (hi - lo);
    double ec = opt_eval(S, k, beta, exp(c), G, g, sm, red);
    double ed = opt_eval(S, k, beta, exp(d), G, g, sm, red);
    for (int it = 0; it < 64; ++it) {
      if (ec < ed) {
        hi = d;
        d = c;
        ed = ec;
        c = hi - phi * (hi - lo);
        ec = opt_eval(S, k, beta, exp(c), G, g, sm, red);
      } else {
        lo = c;
        c = d;
        ec = ed;
        d = lo + phi * (hi - lo);
        ed = opt_eval(S, k, beta, exp(d), G, g, sm, red);
      }
    }
    const double lm = exp(0.5 * (lo + hi));
    if (opt_eval(S, k, beta, lm, G, g, sm, red) <= Eg[b]) lam = lm;
  }
  if (threadIdx.x == 0) *lam_out = lam;
}

}  // namespace

int64_t projected_slot_doubles(int kk, int CL) {
  return (int64_t)CL * (kk + 1) + CL + 2 + (kk + 1) + 2 + 6 * (kk + 1) + kSturmGrid / 2 + kGrid + 1 +
         (int64_t)kk * kk + (int64_t)(kk + 1) * kk + 64;
}

int projected_cluster_size() {
  static int cs = 0;
  if (cs) return cs;
  cudaFuncSetAttribute(k_projected, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_projected, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  int best = 1;
  for (int cand : {16, 8, 4, 2}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cand, 1, 1);
    cfg.blockDim = dim3(kT, 1, 1);
    cfg.dynamicSmemBytes = kSmemCap;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cand;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_projected, &cfg) == cudaSuccess &&
        nclusters > 0) {
      best = cand;
      break;
    }
    cudaGetLastError();
  }
  cs = best;
  return cs;
}

cudaError_t launch_projected(const ProjArgs& a, ProjWork& w, cudaStream_t s) {
  // one cluster per projected problem: every k of k_first..k_last (histories),
  // or one final problem per batch entry
  const bool batch = a.nbatch > 1;
  if (batch && (a.k_first != a.k_last || w.packed)) return cudaErrorInvalidValue;
  const int nprob = batch ? a.nbatch : a.k_last - a.k_first + 1;
  if (nprob <= 0) return cudaSuccess;
  if (!batch && nprob > 1 && !w.packed) return cudaErrorInvalidValue;
  const int CL = w.cluster;
  const int kmax = a.k_last;
  const int ncl = (kmax + CL - 1) / CL;
  const size_t vecs = (size_t)7 * (kmax + 1) * sizeof(double);
  const size_t slab = (size_t)ncl * (kmax + 1) * sizeof(double);
  const size_t scratch = (size_t)4 * (kmax + 1) * sizeof(double);
  w.slab_in_smem = (vecs + slab <= kSmemCap) ? 1 : 0;
  size_t dyn = vecs + (w.slab_in_smem ? (slab > scratch ? slab : scratch) : scratch);
  if (dyn > kSmemCap) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nprob * CL), 1, 1);
  cfg.blockDim = dim3(kT, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_projected, a, w);
}

}  // namespace lslu

namespace lslu {

cudaError_t launch_optimal_lambda(const ProjWork& w, int K, const DevState* st, const double* G,
                                  const double* g, double* Eg, double* lam_out, cudaStream_t s) {
  const size_t smem = (size_t)4 * (K + 1) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_opt_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_opt_refine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_opt_grid<<<kGrid, kT, smem, s>>>(w, K, st, G, g, Eg);
  k_opt_refine<<<1, kT, smem, s>>>(w, K, st, G, g, Eg, lam_out);
  return cudaGetLastError();
}

}  // namespace lslu
