// Projected Tikhonov problem of Hybrid LSLU (Eq. TSP, Section 3.2.1), FP64.
//
// For one (k+1) x k upper Hessenberg H and beta (or one per batch entry, or
// one per k of a history) these kernels run in sequence:
//   1. k_bidiag, one thread-block cluster per problem (16 CTAs; 8 for the
//      many problems of a history, largest k first): Householder
//      bidiagonalisation H = P B Q^T with B lower bidiagonal ((k+1) x k:
//      alpha_j on the diagonal, beta_{j+1} below it) and P e1 = e1 (each step
//      first reflects row j from the right, then column j below the diagonal
//      from the left, so no left reflector touches row 0).  Columns of H are
//      dealt round robin to the CTAs and stay in shared memory.  The right
//      reflector's product s = A w is formed before the reflector is known,
//      s = A(:, j) + scale * A(:, j+1:) A(j, j+1:)^T, so one exchange per step
//      carries both the row norm and s: every CTA publishes its partial
//      products (and the owner of column j that column) in its own shared
//      memory, and after one cluster barrier every CTA reads them all through
//      distributed shared memory, sums them in a fixed order and computes both
//      reflectors of the step itself.  The partial sums run over 16 virtual
//      ranks in one fixed order whatever the cluster size.
//   2. k_sigma, one warp per singular value over the whole GPU: the singular
//      values of B are the positive eigenvalues of the Golub-Kahan tridiagonal
//      T (order 2k+1, zero diagonal, off-diagonals alpha_0, beta_1, alpha_1,
//      ..., beta_k).  Sturm counts at 32 points per round (one per lane,
//      geometric spacing while the bracket spans more than an octave) shrink
//      the bracket of sigma_i 33-fold per round.  c = beta U^T e1 (Eq. gcv2):
//      since P e1 = e1, c_i^2 is 2 beta^2 times the squared first component of
//      T's eigenvector for sigma_i, the residue of e1^T (T - theta)^-1 e1 =
//      det(T_{2:,2:} - theta) / det(T - theta), with the leading and trailing
//      minors evaluated by two lanes of the warp together; one more warp
//      forms c_{k+1}^2 = beta^2 / ||u||^2 for the null vector u of B^T.
//      k_sigma_lanes does the same for the non-final problems of a history,
//      one lane per singular value, where that finishes first.  k_weights
//      then keeps sum c_i^2 + c_{k+1}^2 = beta^2 where a numerically zero
//      singular value breaks the residue formula.
//   3. k_gcv_grid (GCV rules only), one warp per point of the 257-point log
//      grid sigma_1 * 10^[-14, 2] of lambda: the GCV function (Eq. gcv2), or
//      weighted GCV with omega = (k+1)/m (Eq. wgcv).
//   4. k_finish, one block per problem: lambda by the rule (none: 0, fixed, or
//      the best grid point refined between its neighbours to the root of
//      dG/d(lambda^2) by safeguarded Newton steps), the projected residual
//      ||beta e1 - H y|| = sqrt(sum f_i^2 c_i^2 + c_{k+1}^2) with
//      f_i = lambda^2 / (sigma_i^2 + lambda^2), and y = Q z with
//      z = argmin ||beta e1 - B z||^2 + lambda^2 ||z||^2 by the Givens sweep
//      for damped bidiagonal least squares and back substitution.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <mutex>

#include <cmath>

#include "lslu_internal.cuh"

namespace cg = cooperative_groups;

namespace lslu {

namespace {

constexpr int kT = 256;   // threads of the one-block-per-problem kernels
constexpr int kTB = 128;  // threads of a bidiagonalisation CTA: one warp per SM sub-partition,
                          // whose FP64 pipe is the scarce resource
constexpr int kWB = 4;    // warps per block of the warp-per-item kernels
constexpr int kWS = 2;    // warps per block of the singular-value kernel
constexpr int kMaxCluster = 16;
constexpr int kHistoryCluster = 8;  // CTAs per problem of a history's bidiagonalisation
constexpr int kGrid = 257;  // lambda grid points
constexpr double kEps = 2.220446049250313e-16;
constexpr size_t kSmemCap = 200 * 1024;
constexpr size_t kSmemOnePerSm = 120 * 1024;  // more than half of an SM's shared memory

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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

// Four block-wide sums at once.  Within a warp the four values are first
// reduce-scattered (lanes 0-15 keep the first two, then lanes with bit 3
// clear keep one of those, ...), so a warp spends 6 FP64 adds instead of 20;
// the warps' results meet in red4 (2 x 32 entries, alternating between
// calls so that one barrier per call suffices).
__device__ void block_sum4(double (&v)[4], double* red4, int& parity) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool up = lane & 16, up8 = lane & 8;
  double a0 = up ? v[2] : v[0], a1 = up ? v[3] : v[1];
  const double b0 = up ? v[0] : v[2], b1 = up ? v[1] : v[3];
  a0 += __shfl_xor_sync(0xffffffffu, b0, 16);
  a1 += __shfl_xor_sync(0xffffffffu, b1, 16);
  double c = up8 ? a1 : a0;
  c += __shfl_xor_sync(0xffffffffu, up8 ? a0 : a1, 8);
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  // lane 8 q holds quantity q of this warp
  double* r = red4 + parity * 32;
  parity ^= 1;
  if ((lane & 7) == 0) r[(lane >> 3) * 8 + warp] = c;
  __syncthreads();
  // lane 8 q + w (w < nw) reads quantity q of warp w; sum over the warps
  double t = ((lane & 7) < nw) ? r[(lane >> 3) * 8 + (lane & 7)] : 0.0;
  t += __shfl_xor_sync(0xffffffffu, t, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = __shfl_sync(0xffffffffu, t, 8 * q);
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
  // with q = x0^2 + ss and nrm = sqrt(q): bh = -sign(x0) nrm,
  // tau = (bh - x0) / bh = (|x0| + nrm) / nrm and 1 / (x0 - bh) =
  // sign(x0) / (|x0| + nrm); one rsqrt and one division (each costs about as
  // much as seven dependent FP64 FMAs here, a sqrt ten)
  const double q = fma(x0, x0, ss);
  const double rn = rsqrt(q);
  const double nrm = q * rn;
  const double d = fabs(x0) + nrm;
  const bool neg = x0 < 0.0;
  bh = neg ? nrm : -nrm;
  tau = d * rn;
  const double id = 1.0 / d;
  scale = neg ? -id : id;
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
// Number of eigenvalues of T below theta: sign changes along the leading
// minors p_0 = 1, p_1 = -theta, p_j = -theta p_{j-1} - t_{j-1}^2 p_{j-2}.
// The product -t_j^2 p_{j-1} of the next step does not depend on p_j; it is
// issued right after p_j's FMA so that in-order issue does not stall on it
// (t2[n] must be readable; its value is not used).
__device__ int sturm_count(const double* t2, int n, double theta) {
  double pm1 = 1.0, p0 = -theta;
  int cnt = (int)(__double_as_longlong(p0) < 0);
  double x = -t2[1] * pm1;
  int j = 2;
  while (j <= n) {
    const int jend = min(n, j + 7);
#pragma unroll 4
    for (; j <= jend; ++j) {
      const double pj = fma(-theta, p0, x);
      x = -t2[j] * p0;
      cnt += sign_change(pj, p0);
      pm1 = p0;
      p0 = pj;
    }
    int sc;
    if (needs_rescale(p0, pm1, sc)) {  // x is proportional to pm1
      p0 = ldexp(p0, sc);
      pm1 = ldexp(pm1, sc);
      x = ldexp(x, sc);
    }
  }
  return cnt;
}

// Leading minors p_j = -theta p_{j-1} - t_{j-1}^2 p_{j-2} of det(T - theta I)
// with their theta-derivative (trailing = false), or the trailing minors
// r_j = -theta r_{j+1} - t_j^2 r_{j+2}, j = n-1 .. 2, of det(T_{2:n,2:n} -
// theta I) (trailing = true; the derivative is then unused).  Both run the
// same steps on different entries of t2, so two lanes of one warp evaluate
// them together.  v and dv are scaled by 2^-e.
__device__ void minors(const double* t2, int n, double theta, bool trailing, double& v,
                       double& dv, int& e) {
  // step m (m = 0 ..) uses tt_m = t2[m + 1] (leading) or t2[n - 1 - m]
  // (trailing); the next step's products x = -tt p_{j-1} and
  // z = -tt d_{j-1} - p_j are formed as soon as their inputs exist
  double pm1 = 1.0, p0 = -theta, dm1 = 0.0, d0 = -1.0;
  int ex = 0;
  const int stride = trailing ? -1 : 1;
  const double* tp = t2 + (trailing ? n - 1 : 1);
  double x = -tp[0] * pm1;
  double z = fma(-tp[0], dm1, -p0);
  const int common = n - 2;  // steps both recurrences take
  int m = 0;
  while (m < common) {
    const int mend = min(common, m + 8);
#pragma unroll 2
    for (; m < mend; ++m) {
      const double pj = fma(-theta, p0, x);
      const double dj = fma(-theta, d0, z);
      const double tn = tp[(m + 1) * stride];
      x = -tn * p0;
      z = fma(-tn, d0, -pj);
      pm1 = p0;
      p0 = pj;
      dm1 = d0;
      d0 = dj;
    }
    int sc;
    if (needs_rescale(p0, pm1, sc)) {  // x and z scale with the minors
      p0 = ldexp(p0, sc);
      pm1 = ldexp(pm1, sc);
      d0 = ldexp(d0, sc);
      dm1 = ldexp(dm1, sc);
      x = ldexp(x, sc);
      z = ldexp(z, sc);
      ex -= sc;
    }
  }
  if (!trailing) {  // the leading recurrence has one step more
    const double pj = fma(-theta, p0, x);
    d0 = fma(-theta, d0, z);
    p0 = pj;
  }
  v = p0;
  dv = d0;
  e = ex;
}

// The GCV function (Eqs. gcv2/wgcv) N / D^2 scaled by k and its sign-carrying
// derivative with respect to mu = lambda^2, N' D - 2 N D', evaluated by the
// whole block (sig2 = sigma_i^2).
struct GcvSums {
  double N, dN, D, dD;
};
__device__ GcvSums gcv_sums(const double* sig2, const double* c2, int k, double mu, double omega,
                            double* red4, int& parity) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // N, N', D - 1, D'/omega
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double s2 = sig2[i];
    const double rw = 1.0 / (s2 + mu);
    const double f = mu * rw;
    const double dfdmu = s2 * rw * rw;
    v[0] = fma(f * f, c2[i], v[0]);
    v[1] = fma(2.0 * f * dfdmu, c2[i], v[1]);
    v[2] = fma(fma(1.0 - omega, s2, mu), rw, v[2]);
    v[3] += dfdmu;
  }
  block_sum4(v, red4, parity);
  return {v[0] + c2[k], v[1], 1.0 + v[2], omega * v[3]};
}

// The slope s(mu) = N' D - 2 N D' of G = N / D^2 (same sign as dG/dlambda)
// and its derivative s'(mu) = N'' D - N' D' - 2 N D'' for the safeguarded
// Newton refinement of lambda; f = mu / (s2 + mu), f' = s2 / (s2 + mu)^2,
// f'' = -2 s2 / (s2 + mu)^3, N = sum f^2 c2 + c2_{k+1}, D = 1 + sum
// ((1 - omega) s2 + mu) / (s2 + mu), D' = omega sum f', D'' = omega sum f''.
struct SlopeAndDerivative {
  double s, ds, N, D;
};
__device__ SlopeAndDerivative gcv_slope2(const double* sig2, const double* c2, int k, double mu,
                                         double omega, double* red4, int& parity) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // N, N', N'', D - 1
  double w[4] = {0.0, 0.0, 0.0, 0.0};  // sum f', sum f'', unused
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double s2 = sig2[i];
    const double rw = 1.0 / (s2 + mu);
    const double f = mu * rw;
    const double fp = s2 * rw * rw;
    const double fpp = -2.0 * fp * rw;
    const double c = c2[i];
    v[0] = fma(f * f, c, v[0]);
    v[1] = fma(2.0 * f * fp, c, v[1]);
    v[2] = fma(2.0 * fma(fp, fp, f * fpp), c, v[2]);
    v[3] = fma(fma(1.0 - omega, s2, mu), rw, v[3]);
    w[0] += fp;
    w[1] += fpp;
  }
  block_sum4(v, red4, parity);
  block_sum4(w, red4, parity);
  const double N = v[0] + c2[k], dN = v[1], ddN = v[2], D = 1.0 + v[3];
  const double dD = omega * w[0], ddD = omega * w[1];
  return {dN * D - 2.0 * N * dD, ddN * D - dN * dD - 2.0 * N * ddD, N, D};
}

// Global work space of one problem of size kk.
struct Slots {
  double* al;    // kk+1: alpha_j, the diagonal of B
  double* be;    // kk+1: beta_j below it (be[0] unused)
  double* taur;  // kk+1: right-reflector taus
  double* sig;   // kk+1: singular values, largest first
  double* c2;    // kk+1: c_i^2, then c_{k+1}^2
  double* gv;    // kGrid+1: GCV function on the lambda grid
  double* Qs;    // kk x kk: right reflector j in row j (entries c >= j)
  double* A;     // (kk+1) x kk column slab when shared memory is too small
};

__device__ Slots carve(double* base, int kk, int /*CL*/) {
  Slots s;
  double* p = base;
  s.al = p; p += kk + 1;
  s.be = p; p += kk + 1;
  s.taur = p; p += kk + 1;
  s.sig = p; p += kk + 1;
  s.c2 = p; p += kk + 1;
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

// Which problem a block works on, and its size (k = 0: nothing to solve).
struct ProbInfo {
  int p;          // batch entry (0 without a batch)
  int kk;         // problem size before clamping to the iterations done
  int k;          // columns of H solved
  bool is_final;  // the problem of size k_last (the one that yields y)
  double beta;
};

__device__ ProbInfo prob_info(const ProjArgs& a, int prob) {
  ProbInfo r;
  const bool batch = a.nbatch > 1;
  r.p = batch ? prob : 0;
  r.kk = batch ? a.k_last : a.k_first + prob;
  const DevState* sp = a.st ? a.st + r.p : nullptr;
  const int kdone = sp ? sp->k_done : a.k_last;
  r.is_final = (r.kk == a.k_last);
  r.k = r.is_final ? min(r.kk, kdone) : r.kk;
  if (r.k <= 0 || (!r.is_final && r.kk > kdone)) r.k = 0;
  r.beta = sp ? sp->beta : a.beta_val;
  return r;
}

__device__ Slots slot_of(const ProjWork& w, const ProbInfo& pi) {
  return carve(w.base + (w.packed ? w.offsets[pi.kk] : (int64_t)pi.p * w.slot_stride), pi.kk,
               w.cluster);
}

// ---- 1. bidiagonalisation ---------------------------------------------------
__global__ void __launch_bounds__(kTB) k_bidiag(ProjArgs a, ProjWork w) {
  extern __shared__ double smem[];
  __shared__ double red[kTB / 32];
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int local = blockIdx.x / CL, nlocal = gridDim.x / CL;
  const int prob = w.prob0 + (w.desc ? nlocal - 1 - local : local);
  const ProbInfo pi = prob_info(a, prob);
  const int k = pi.k;
  if (k == 0) return;  // every CTA of the cluster sees the same k: no barrier is left waiting
  const Slots S = slot_of(w, pi);
  const double* Hp = a.H + (int64_t)pi.p * a.strideH;
  const int K1 = (w.kcap > 0 ? w.kcap : a.k_last) + 1;
  const int64_t ld = k + 1;
  // The partial products are summed over kMaxCluster virtual ranks (columns
  // c = v mod kMaxCluster) in one fixed order whatever the cluster size; a
  // CTA holds the V = kMaxCluster / CL virtual ranks rank + t CL, so results
  // do not depend on CL.
  const int V = kMaxCluster / CL;
  // shared layout: [Ps, cj, sv : K1 each] [xP : 2 V x K1] [xC : 2 x K1] [slab]
  double* Ps = smem;             // summed partial products, rows j..k
  double* cj = Ps + K1;          // column j (from its owner), then the left reflector
  double* sv = cj + K1;          // s = A w, rows j+1..k
  double* xP = sv + K1;          // this CTA's partial products, by step parity and virtual rank
  double* xC = xP + 2 * V * K1;  // the owner's copy of the next column, by step parity
  double* slab = xC + 2 * K1;
  const bool in_smem = w.slab_in_smem != 0;
  auto col = [&](int c) -> double* {
    return in_smem ? slab + (int64_t)(c / CL) * ld : S.A + (int64_t)c * ld;
  };
  auto first_own = [&](int x) -> int { return x + ((rank - x) % CL + CL) % CL; };
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  unsigned long long* ts = (a.tstamp && pi.is_final && rank == 0 && tid == 0) ? a.tstamp : nullptr;
  if (ts) ts[0] = gtimer();

  for (int c = rank; c < k; c += CL) {
    double* cp = col(c);
    for (int r = tid; r <= k; r += nt) cp[r] = Hp[r + (int64_t)c * a.ldh];
  }
  __syncthreads();

  // What step jn needs from this CTA: P_r = sum over own columns c > jn of
  // A[r, c] A[jn, c] for r = jn..k (r = jn: the partial squared norm of row
  // jn), and from the owner of column jn a copy of it.
  auto publish = [&](int jn) {
    for (int t = 0; t < V; ++t) {
      double* P = xP + ((jn & 1) * V + t) * K1;
      const int v = rank + t * CL;
      const int c0 = jn + 1 + ((v - jn - 1) % kMaxCluster + kMaxCluster) % kMaxCluster;
      for (int r = jn + tid; r <= k; r += nt) {
        double s0 = 0.0, s1 = 0.0;
        int c = c0;
        for (; c + kMaxCluster < k; c += 2 * kMaxCluster) {
          s0 = fma(col(c)[r], col(c)[jn], s0);
          s1 = fma(col(c + kMaxCluster)[r], col(c + kMaxCluster)[jn], s1);
        }
        if (c < k) s0 = fma(col(c)[r], col(c)[jn], s0);
        P[r] = s0 + s1;
      }
    }
    if (jn % CL == rank) {
      double* C = xC + (jn & 1) * K1;
      const double* cp = col(jn);
      for (int r = jn + tid; r <= k; r += nt) C[r] = cp[r];
    }
  };

  unsigned long long tsec[4] = {0, 0, 0, 0}, tprev = ts ? gtimer() : 0;
  auto lap = [&](int q) {
    if (ts) {
      const unsigned long long now = gtimer();
      tsec[q] += now - tprev;
      tprev = now;
    }
  };
  publish(0);
  for (int j = 0; j < k; ++j) {
    const int par = j & 1;
    lap(0);
    // Step j's partials are complete in every CTA.  The buffers of parity
    // par are rewritten only in step j+2, after the next barrier, which no
    // CTA passes before all have finished reading them below.
    cluster.sync();
    lap(1);
    {
      const double* oc = cluster.map_shared_rank(xC + par * K1, j % CL);
      for (int r = j + tid; r <= k; r += nt) {
        double pv[kMaxCluster];
#pragma unroll
        for (int q = 0; q < kMaxCluster; ++q)
          pv[q] = *cluster.map_shared_rank(xP + (par * V + q / CL) * K1 + r, q % CL);
#pragma unroll
        for (int h = kMaxCluster / 2; h >= 1; h >>= 1)  // fixed pairwise order
#pragma unroll
          for (int q = 0; q < h; ++q) pv[q] += pv[q + h];
        Ps[r] = pv[0];
        cj[r] = oc[r];
      }
    }
    __syncthreads();
    // right reflector on row j (w_j = 1, w_c = sc A[j, c] for c > j), computed
    // by every thread from the same values
    double taur, bh, sc;
    house(cj[j], Ps[j], taur, bh, sc);
    // s_r = sum_c A[r, c] w_c and column j after the right reflector, rows j+1..k
    double s2 = 0.0;
    for (int r = j + 1 + tid; r <= k; r += nt) {
      const double s = fma(sc, Ps[r], cj[r]);
      sv[r] = s;
      const double v = fma(-taur, s, cj[r]);
      cj[r] = v;
      if (r >= j + 2) s2 = fma(v, v, s2);
    }
    s2 = warp_sum_d(s2);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    s2 = 0.0;
    for (int q = 0; q < nw; ++q) s2 += red[q];
    // left reflector on column j, rows j+1..k
    double taul, bl, scl;
    house(cj[j + 1], s2, taul, bl, scl);
    __syncthreads();  // cj[j+1] and red are read by all before they change
    for (int r = j + 1 + tid; r <= k; r += nt) cj[r] = (r == j + 1) ? 1.0 : cj[r] * scl;
    if (rank == 0 && tid == 0) {
      S.al[j] = bh;
      S.be[j + 1] = bl;
      S.taur[j] = taur;
      S.Qs[(int64_t)j * k + j] = 1.0;
    }
    __syncthreads();
    lap(2);
    // own columns c > j, two per warp at a time: the right reflector, then the
    // left one (t = v^T A[j+1:, c]); the two dots are reduced together
    for (int c = first_own(j + 1) + warp * CL; c < k; c += 2 * CL * nw) {
      const int c2 = c + CL * nw;
      const bool two = c2 < k;
      double* cp = col(c);
      double* cq = col(two ? c2 : c);
      const double wc = cp[j] * sc, wq = two ? cq[j] * sc : 0.0;
      if (lane == 0) {
        __stcg(S.Qs + (int64_t)j * k + c, wc);
        if (two) __stcg(S.Qs + (int64_t)j * k + c2, wq);
      }
      const double g = taur * wc, gq = taur * wq;
      double t = 0.0, tq = 0.0;
      for (int r = j + 1 + lane; r <= k; r += 32) {
        const double sr = sv[r], vr = cj[r];
        const double v = fma(-g, sr, cp[r]);
        cp[r] = v;
        t = fma(vr, v, t);
        if (two) {
          const double vq = fma(-gq, sr, cq[r]);
          cq[r] = vq;
          tq = fma(vr, vq, tq);
        }
      }
      // lanes 0-15 finish t, lanes 16-31 tq
      const bool hiL = lane & 16;
      double u = hiL ? tq : t;
      u += __shfl_xor_sync(0xffffffffu, hiL ? t : tq, 16);
      u += __shfl_xor_sync(0xffffffffu, u, 8);
      u += __shfl_xor_sync(0xffffffffu, u, 4);
      u += __shfl_xor_sync(0xffffffffu, u, 2);
      u += __shfl_xor_sync(0xffffffffu, u, 1);
      t = __shfl_sync(0xffffffffu, u, 0);
      tq = __shfl_sync(0xffffffffu, u, 16);
      const double h = taul * t, hq = taul * tq;
      if (h != 0.0 || hq != 0.0)
        for (int r = j + 1 + lane; r <= k; r += 32) {
          const double vr = cj[r];
          cp[r] = fma(-h, vr, cp[r]);
          if (two) cq[r] = fma(-hq, vr, cq[r]);
        }
    }
    __syncthreads();
    lap(3);
    if (j + 1 < k) publish(j + 1);
  }
  // no CTA leaves while another may still read its shared memory
  cluster.sync();
  if (ts) {
    ts[1] = gtimer();
    for (int q = 0; q < 4; ++q) ts[8 + q] = tsec[q];
  }
}

// ---- 2. singular values and weights ----------------------------------------
// Block (x, prob) serves sigma_i for i = x kWS + warp; warp i = k forms
// c_{k+1}^2.  Shared: t2 (2 (kmax+1)), alpha and beta (kmax+1 each).  Each
// warp is a chain of dependent FP64 operations: when the grid fits on the GPU
// at once, the launcher asks for enough shared memory that every SM holds one
// block, so no two warps share an FP64 pipe.
__global__ void __launch_bounds__(kWS * 32) k_sigma(ProjArgs a, ProjWork w) {
  extern __shared__ double sh[];
  __shared__ unsigned long long gmax[kWS];
  const ProbInfo pi = prob_info(a, w.prob0 + blockIdx.y);
  const int k = pi.k;
  const int i0 = blockIdx.x * kWS;
  if (k == 0 || i0 > k) return;
  const Slots S = slot_of(w, pi);
  const int K1 = a.k_last + 1;
  double* t2 = sh;            // t2[j] = t_j^2, j = 1..2k
  double* alv = t2 + 2 * K1;  // alpha_0..alpha_{k-1}
  double* bev = alv + K1;     // beta_1..beta_k at 1..k
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = 2 * k + 1;
  // spectral bound of T: 2 max |t_j| (no eigenvalue of a zero-diagonal
  // tridiagonal reaches it), the maximum taken on the bit patterns
  unsigned long long mx = 0;
  for (int i = tid; i < k; i += blockDim.x) {
    const double al = ldg_cg(S.al + i), be = ldg_cg(S.be + i + 1);
    alv[i] = al;
    bev[i + 1] = be;
    t2[2 * i + 1] = al * al;
    t2[2 * i + 2] = be * be;
    const unsigned long long ba = (unsigned long long)__double_as_longlong(al) & 0x7fffffffffffffffull;
    const unsigned long long bb = (unsigned long long)__double_as_longlong(be) & 0x7fffffffffffffffull;
    mx = max(mx, max(ba, bb));
  }
  if (tid == 0) t2[2 * k + 1] = 0.0;  // read (not used) by the last Sturm step
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) gmax[warp] = mx;
  __syncthreads();
  for (int q = 0; q < kWS; ++q) mx = max(mx, gmax[q]);
  const double G = 2.0 * __longlong_as_double((long long)mx);
  const int i = i0 + warp;
  if (i > k) return;
  if (i == k) {  // null vector of B^T: u_{i+1} = -alpha_i u_i / beta_{i+1}, u_0 = 1
    if (lane == 0) {
      double u = 1.0, nrm2 = 1.0;
      int e = 0;  // u and nrm2 carry the factors 2^-e/2 and 2^-e
      for (int q = 0; q < k; ++q) {
        if (bev[q + 1] == 0.0) break;
        u = -alv[q] * u / bev[q + 1];
        nrm2 = fma(u, u, nrm2);
        if (nrm2 > 0x1p+600) {
          u = ldexp(u, -300);
          nrm2 = ldexp(nrm2, -600);
          e += 600;
        }
      }
      __stcg(S.c2 + k, ldexp(pi.beta * pi.beta / nrm2, -e));
    }
    return;
  }
  // sigma_i, the i-th largest, has target = k-1-i singular values below it;
  // the bracket keeps count(lo) <= target < count(hi), both counts evaluated
  const int target = k - 1 - i;
  double lo = 0.0, hi = G;
  int rounds = 0;
  if (G > 0.0) {
    const double tiny = G * 0x1p-200;  // below this a singular value is zero
    const double f = (double)(lane + 1) * (1.0 / 33.0);
    for (; rounds < 64; ++rounds) {
      if (hi - lo <= 4.0 * kEps * hi || hi <= tiny) break;
      double th;
      if (lo == 0.0)
        th = hi * exp2(-60.0 * (1.0 - f));  // geometric points down to hi 2^-60
      else if (hi > 2.0 * lo)
        th = lo * exp2(log2(hi / lo) * f);
      else
        th = fma(hi - lo, f, lo);
      const int cnt = sturm_count(t2, n, th) - (k + 1);
      const unsigned above = __ballot_sync(0xffffffffu, cnt > target);
      const int fl = above ? __ffs(above) - 1 : 32;  // first point above the target
      const double nhi = __shfl_sync(0xffffffffu, th, fl < 32 ? fl : 0);
      const double nlo = __shfl_sync(0xffffffffu, th, fl > 0 ? fl - 1 : 0);
      const double hi2 = fl < 32 ? nhi : hi, lo2 = fl > 0 ? nlo : lo;
      if (hi2 == hi && lo2 == lo) break;  // the points no longer split the bracket
      lo = lo2;
      hi = hi2;
    }
  }
  if (a.tstamp && pi.is_final && lane == 0) {  // multisection rounds (timing mode)
    atomicMax(a.tstamp + 13, (unsigned long long)rounds);
    atomicAdd(a.tstamp + 14, (unsigned long long)rounds);
  }
  const double th = lo > 0.0 ? 0.5 * (lo + hi) : 0.5 * hi;
  // weight: first component^2 of T's eigenvector = -det(T_{2:,2:} - th) / det'(T - th)
  double v, dv;
  int ev;
  minors(t2, n, th, lane == 1, v, dv, ev);
  const double q = __shfl_sync(0xffffffffu, v, 1);
  const int eq = __shfl_sync(0xffffffffu, ev, 1);
  if (lane == 0) {
    double wgt = (dv != 0.0) ? ldexp(-q / dv, eq - ev) : 0.0;
    if (!(wgt >= 0.0)) wgt = 0.0;
    __stcg(S.sig + i, th);
    __stcg(S.c2 + i, 2.0 * pi.beta * pi.beta * wgt);
  }
}

// ---- 2'. the same, one lane per singular value ------------------------------
// For the many problems of a history (every k of 1..K).  An FP64 warp
// instruction holds its sub-partition's FP64 pipe for the same time whatever
// its lanes do, so 32 lanes spent on one singular value (33-fold bracket
// shrink per round) buy about 5 bits per round where 32 lanes bisecting 32
// singular values buy 32.  Each lane bisects
// its own sigma_i: through the exponent (halving the number of octaves) while
// the bracket spans at least two, then linearly; once the bracket holds
// sigma_i alone and is 2^-16 narrow, Newton steps on det(T - theta) finish
// it (about 24 rounds and 3 steps of two rounds' cost instead of ~60
// rounds), else bisection goes on to the same final width as k_sigma
// (k = 1..300: 8.4 ms; 15.3 with bisection alone; multisection 46.8).  A
// warp serves 32 consecutive i of one problem, so its lanes read the same t2
// entries; blocks take the problems largest k first.  Shared: as k_sigma.
constexpr int kWL = 4;           // warps per block
constexpr int kMaxBisect = 160;  // rounds (the bracket needs ~13 + 52 at most)
constexpr int kNewtonSteps = 4;

__device__ __forceinline__ int biased_exponent(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// One bisection round of a lane (work = false: evaluate, keep the bracket,
// so that the warp stays converged).  Trial point: 2^-16 hi while lo = 0;
// lo 2^(d/2) while hi spans d >= 2 octaves above lo (exact scalings); else
// the midpoint.
__device__ __forceinline__ void bisect_round(const double* t2, int n, int k, int target, bool work,
                                             double& lo, double& hi, int& clo, int& chi) {
  const int d = biased_exponent(hi) - biased_exponent(lo);
  double th;
  if (lo == 0.0)
    th = hi * 0x1p-16;
  else if (d >= 2 && biased_exponent(lo) > 0)
    th = lo * __longlong_as_double((long long)(1023 + d / 2) << 52);
  else
    th = fma(0.5, hi - lo, lo);
  const int cnt = sturm_count(t2, n, th) - (k + 1);
  if (work) {
    if (cnt > target) {
      hi = th;
      chi = cnt;
    } else {
      lo = th;
      clo = cnt;
    }
  }
}

__global__ void __launch_bounds__(kWL * 32) k_sigma_lanes(ProjArgs a, ProjWork w) {
  extern __shared__ double sh[];
  __shared__ unsigned long long gmax[kWL];
  const ProbInfo pi = prob_info(a, w.prob0 + (int)(gridDim.y - 1 - blockIdx.y));
  const int k = pi.k;
  const int i0 = blockIdx.x * kWL * 32;
  if (k == 0 || i0 > k) return;
  const Slots S = slot_of(w, pi);
  const int K1 = a.k_last + 1;
  double* t2 = sh;            // t2[j] = t_j^2, j = 1..2k
  double* alv = t2 + 2 * K1;  // alpha_0..alpha_{k-1}
  double* bev = alv + K1;     // beta_1..beta_k at 1..k
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = 2 * k + 1;
  unsigned long long mx = 0;
  for (int q = tid; q < k; q += blockDim.x) {
    const double al = ldg_cg(S.al + q), be = ldg_cg(S.be + q + 1);
    alv[q] = al;
    bev[q + 1] = be;
    t2[2 * q + 1] = al * al;
    t2[2 * q + 2] = be * be;
    const unsigned long long ba = (unsigned long long)__double_as_longlong(al) & 0x7fffffffffffffffull;
    const unsigned long long bb = (unsigned long long)__double_as_longlong(be) & 0x7fffffffffffffffull;
    mx = max(mx, max(ba, bb));
  }
  if (tid == 0) t2[2 * k + 1] = 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) gmax[warp] = mx;
  __syncthreads();
  for (int q = 0; q < kWL; ++q) mx = max(mx, gmax[q]);
  const double G = 2.0 * __longlong_as_double((long long)mx);
  const int wbase = i0 + warp * 32;
  if (wbase > k) return;  // whole warp past the problem (warp-uniform)
  const int i = wbase + lane;
  // lanes with i >= k run the rounds on a settled bracket and store nothing
  const bool mine = i < k;
  const int target = k - 1 - i;
  // bracket with its counts (eigenvalues of T below it, minus k + 1):
  // clo <= target < chi; clo = -1 while lo = 0 has not been evaluated
  double lo = 0.0, hi = G, x = 0.0;
  int clo = -1, chi = k;
  bool by_newton = false;
  if (G > 0.0) {
    const double tiny = G * 0x1p-200;  // below this a singular value is zero
    auto settled = [&]() { return !mine || hi - lo <= 4.0 * kEps * hi || hi <= tiny; };
    // A. bisection until settled, or until the bracket holds sigma_i alone
    // and is 2^-16 narrow
    int r = 0;
    for (; r < kMaxBisect; ++r) {
      const bool isolated = clo == target && chi == target + 1 && hi - lo <= 0x1p-16 * hi;
      const bool stop = settled() || isolated;
      if (__all_sync(0xffffffffu, stop)) break;
      bisect_round(t2, n, k, target, !stop, lo, hi, clo, chi);
    }
    // B. safeguarded Newton steps on det(T - theta) from the midpoint of the
    // isolating bracket (quadratic from there unless another singular value
    // lies just outside it); a step that leaves the bracket, or no step below
    // 2^-40 x within kNewtonSteps, hands the lane back to bisection
    bool nt = !settled() && clo == target && chi == target + 1;
    x = 0.5 * (lo + hi);
    for (int it = 0; it < kNewtonSteps; ++it) {
      if (!__any_sync(0xffffffffu, nt && !by_newton)) break;
      double v, dv;
      int e;
      minors(t2, n, x, false, v, dv, e);
      if (nt && !by_newton) {
        const double xn = x - v / dv;
        if (!(xn > lo && xn < hi)) {
          nt = false;
        } else {
          by_newton = fabs(xn - x) <= 0x1p-40 * xn;
          x = xn;
        }
      }
    }
    // C. the lanes left bisect to the final width
    for (; r < kMaxBisect; ++r) {
      const bool stop = settled() || by_newton;
      if (__all_sync(0xffffffffu, stop)) break;
      bisect_round(t2, n, k, target, !stop, lo, hi, clo, chi);
    }
  }
  if (mine) {
    const double th = by_newton ? x : lo > 0.0 ? 0.5 * (lo + hi) : 0.5 * hi;
    // weight as in k_sigma, both minors on this lane
    double v, dv, q, dq;
    int ev, eq;
    minors(t2, n, th, false, v, dv, ev);
    minors(t2, n, th, true, q, dq, eq);
    double wgt = (dv != 0.0) ? ldexp(-q / dv, eq - ev) : 0.0;
    if (!(wgt >= 0.0)) wgt = 0.0;
    __stcg(S.sig + i, th);
    __stcg(S.c2 + i, 2.0 * pi.beta * pi.beta * wgt);
  }
  if (i == k) {  // null vector of B^T, as in k_sigma
    double u = 1.0, nrm2 = 1.0;
    int e = 0;
    for (int q = 0; q < k; ++q) {
      if (bev[q + 1] == 0.0) break;
      u = -alv[q] * u / bev[q + 1];
      nrm2 = fma(u, u, nrm2);
      if (nrm2 > 0x1p+600) {
        u = ldexp(u, -300);
        nrm2 = ldexp(nrm2, -600);
        e += 600;
      }
    }
    __stcg(S.c2 + k, ldexp(pi.beta * pi.beta / nrm2, -e));
  }
}

// ---- 2''. weights of numerically zero singular values ----------------------
// U is orthogonal, so sum_i c_i^2 + c_{k+1}^2 = beta^2.  The residue formula
// keeps that to rounding for every separated singular value, tiny ones
// included, but at an exactly or numerically zero one (a rank-deficient H;
// never an unreduced Hessenberg H of the basis loop) it degenerates at the
// near-triple eigenvalue 0 of T and the sum is off.  Such a sigma_i (<= (k+1)
// eps sigma_1) has its left singular vector, and c_i, fixed only up to the
// null space of H^T; only the sum of those c_i^2 and c_{k+1}^2 enters G, the
// residual and y (f_i = 1 for them, sigma_i c_i / (sigma_i^2 + lambda^2)
// vanishes with sigma_i, and lambda = 0 drops them).  So where the sum misses
// beta^2 by more than rounding (64 k eps beta^2), those c_i^2 share equally
// what is left of beta^2.  One block per problem.
__global__ void __launch_bounds__(kT) k_weights(ProjArgs a, ProjWork w) {
  __shared__ double red[33];  // block_sum's scratch
  const ProbInfo pi = prob_info(a, blockIdx.x);
  const int k = pi.k;
  if (k == 0) return;  // block-uniform
  const Slots S = slot_of(w, pi);
  const double thr = (double)(k + 1) * kEps * ldg_cg(S.sig);
  double rest = 0.0, zero = 0.0, nzero = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double c2 = ldg_cg(S.c2 + i);
    if (ldg_cg(S.sig + i) <= thr) {
      nzero += 1.0;
      zero += c2;
    } else {
      rest += c2;
    }
  }
  nzero = block_sum(nzero, red);  // exact: a count below 2^53
  if (nzero == 0.0) return;       // block-uniform
  rest = block_sum(rest, red) + ldg_cg(S.c2 + k);
  zero = block_sum(zero, red);
  const double b2 = pi.beta * pi.beta;
  if (fabs(b2 - rest - zero) <= 64.0 * k * kEps * b2) return;  // consistent
  const double each = fmax(0.0, b2 - rest) / nzero;
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (ldg_cg(S.sig + i) <= thr) __stcg(S.c2 + i, each);
}

// Which of the two singular-value kernels finishes first: per warp, rounds
// times the Sturm length 2k+1, either along the longest warp's chain or
// spread over the GPU's sub-partitions (rounds: ~11 for k_sigma, measured at
// k = 300; ~30 round equivalents for k_sigma_lanes, ~60 where Newton steps
// do not take over).
bool sigma_by_lanes(const ProjArgs& a, int nprob, int num_sms) {
  if (num_sms <= 0) return false;
  double multi = 0.0, lanes = 0.0;
  int kmax = 0;
  for (int p = 0; p < nprob; ++p) {  // problems k_first .. k_first + nprob - 1
    const int k = a.k_first + p;
    kmax = k > kmax ? k : kmax;
    multi += (double)(k + 1) * (2 * k + 1);
    lanes += (double)((k + 32) / 32) * (2 * k + 1);
  }
  const double spread = 4.0 * num_sms;
  const double c_multi = 11.0 * fmax(2 * kmax + 1, multi / spread);
  const double c_lanes = 30.0 * fmax(2 * kmax + 1, lanes / spread);
  return c_lanes < c_multi;
}

// ---- 3. GCV function on the lambda grid: one warp per grid point ------------
__global__ void __launch_bounds__(kWB * 32) k_gcv_grid(ProjArgs a, ProjWork w) {
  const ProbInfo pi = prob_info(a, blockIdx.y);
  const int k = pi.k;
  const int t = blockIdx.x * kWB + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k == 0 || t >= kGrid) return;
  const Slots S = slot_of(w, pi);
  const double s1 = ldg_cg(S.sig);
  if (!(s1 > 0.0)) return;
  const double mrows = a.mvec ? (double)a.mvec[pi.p] : (double)a.m;
  const double omega = a.rule == LSLU_LAMBDA_WGCV ? (double)(k + 1) / mrows : 1.0;
  const double lam = s1 * pow(10.0, -14.0 + 0.0625 * t);
  const double L2 = lam * lam;
  double num = 0.0, den = 0.0;
  for (int i = lane; i < k; i += 32) {
    const double s = ldg_cg(S.sig + i), s2 = s * s;
    const double rw = 1.0 / (s2 + L2);
    const double f = L2 * rw;
    num = fma(f * f, ldg_cg(S.c2 + i), num);
    den = fma(fma(1.0 - omega, s2, L2), rw, den);
  }
  num = warp_sum_d(num);
  den = warp_sum_d(den);
  if (lane == 0) {
    num += ldg_cg(S.c2 + k);
    den += 1.0;
    __stcg(S.gv + t, (double)k * num / (den * den));
  }
}

// ---- 4. lambda, residual and y: one block per problem -----------------------
constexpr int kTF = 128;
constexpr int kQPer = (kMaxIter + kTF - 1) / kTF;


// Shared: sigma^2, c2, alpha, beta and three vectors of the sweep (kmax+1 each).
// y = Q z with Q = H_0 ... H_{k-1}: z <- (I - tau_j w_j w_j^T) z for
// j = k-1 .. 0 (w_j in row j of Qs, entries c >= j).  Thread t owns entries
// c = t + kTF e, e < NP, in registers; the row of step j-1 is loaded during
// step j.
template <int NP>
__device__ void apply_q(const Slots& S, int k, const double* z, double* yp,
                        double (*qred)[kTF / 32]) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double zr[NP], qc[NP], qn[NP];
#pragma unroll
  for (int e = 0; e < NP; ++e) {
    const int c = tid + kTF * e;
    zr[e] = c < k ? z[c] : 0.0;
    qn[e] = (c < k && c >= k - 1) ? ldg_cg(S.Qs + (int64_t)(k - 1) * k + c) : 0.0;
  }
  double taun = ldg_cg(S.taur + (k - 1));
  for (int j = k - 1; j >= 0; --j) {
    const double tj = taun;
#pragma unroll
    for (int e = 0; e < NP; ++e) qc[e] = qn[e];
    if (j > 0) {
      taun = ldg_cg(S.taur + (j - 1));
#pragma unroll
      for (int e = 0; e < NP; ++e) {
        const int c = tid + kTF * e;
        qn[e] = (c < k && c >= j - 1) ? ldg_cg(S.Qs + (int64_t)(j - 1) * k + c) : 0.0;
      }
    }
    if (tj == 0.0) continue;  // the same for every thread
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < NP; ++e) s = fma(qc[e], zr[e], s);
    s = warp_sum_d(s);
    if (lane == 0) qred[j & 1][warp] = s;
    __syncthreads();
    s = 0.0;
#pragma unroll
    for (int q = 0; q < kTF / 32; ++q) s += qred[j & 1][q];
    const double h = tj * s;
#pragma unroll
    for (int e = 0; e < NP; ++e) zr[e] = fma(-h, qc[e], zr[e]);
  }
#pragma unroll
  for (int e = 0; e < NP; ++e) {
    const int c = tid + kTF * e;
    if (c < k) yp[c] = zr[e];
  }
}

__global__ void __launch_bounds__(kTF) k_finish(ProjArgs a, ProjWork w) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  __shared__ double red4[64];
  __shared__ double qred[2][kTF / 32];
  __shared__ int ibest;
  const int prob = blockIdx.x;
  const ProbInfo pi = prob_info(a, prob);
  const int k = pi.k;
  const bool batch = a.nbatch > 1;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  double* lam_o = a.lam_out ? a.lam_out + (batch ? pi.p : pi.kk - 1) : nullptr;
  double* res_o = a.res_out ? a.res_out + (batch ? pi.p : pi.kk - 1) : nullptr;
  double* tr_o = a.tr_out ? a.tr_out + (batch ? pi.p : pi.kk - 1) : nullptr;
  if (k == 0) {
    if (tid == 0) {
      if (lam_o) *lam_o = 0.0;
      if (res_o) *res_o = 0.0;
      if (tr_o) *tr_o = 0.0;
    }
    return;
  }
  const Slots S = slot_of(w, pi);
  const int K1 = a.k_last + 1;
  double* sig2 = sm;
  double* c2 = sig2 + K1;
  double* al = c2 + K1;
  double* be = al + K1;
  double* rinv = be + K1;
  double* thv = rinv + K1;
  double* ph = thv + K1;
  unsigned long long* ts = (a.tstamp && pi.is_final && tid == 0) ? a.tstamp : nullptr;
  if (ts) ts[3] = gtimer();
  const double s1 = ldg_cg(S.sig);
  for (int i = tid; i <= k; i += nt) {
    if (i < k) {
      const double sg = ldg_cg(S.sig + i);
      sig2[i] = sg * sg;
      if (a.sig) a.sig[(int64_t)prob * a.ldsig + i] = sg;
    }
    c2[i] = ldg_cg(S.c2 + i);
    al[i] = i < k ? ldg_cg(S.al + i) : 0.0;
    be[i] = i > 0 ? ldg_cg(S.be + i) : 0.0;
  }
  __syncthreads();
  const bool gcv = (a.rule == LSLU_LAMBDA_GCV || a.rule == LSLU_LAMBDA_WGCV) && s1 > 0.0;
  const double mrows = a.mvec ? (double)a.mvec[pi.p] : (double)a.m;
  const double omega = a.rule == LSLU_LAMBDA_WGCV ? (double)(k + 1) / mrows : 1.0;
  const double beta = pi.beta;
  int par = 0;
  double lam = 0.0;
  if (a.rule == LSLU_LAMBDA_FIXED) {
    lam = a.lambda;
  } else if (gcv) {
    if (warp == 0) {  // best grid point, ties to the smaller lambda (G >= 0: bit order)
      unsigned long long bk = ~0ull;
      int bi = 0;
      for (int t = lane; t < kGrid; t += 32) {
        const double g = ldg_cg(S.gv + t);
        const unsigned long long key =
            (g == g) ? (unsigned long long)__double_as_longlong(g) : ~0ull;
        if (key < bk) {
          bk = key;
          bi = t;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ok < bk || (ok == bk && oi < bi)) {
          bk = ok;
          bi = oi;
        }
      }
      if (lane == 0) ibest = bi;
    }
    __syncthreads();
    const int ib = ibest;
    const double gib = ldg_cg(S.gv + ib);
    lam = s1 * pow(10.0, -14.0 + 0.0625 * ib);
    if (ib > 0 && ib < kGrid - 1) {
      // bisection in log(lambda) between the neighbours: the midpoint of
      // log(lo) and log(hi) is log(sqrt(lo hi)), and mu = lambda^2 = lo hi
      double lo = s1 * pow(10.0, -14.0 + 0.0625 * (ib - 1));
      double hi = s1 * pow(10.0, -14.0 + 0.0625 * (ib + 1));
      auto slope = [&](double mu) {
        const GcvSums g = gcv_sums(sig2, c2, k, mu, omega, red4, par);
        return g.dN * g.D - 2.0 * g.N * g.dD;
      };
      if (slope(lo * lo) < 0.0 && slope(hi * hi) > 0.0) {
        // the root of the slope inside the bracket [a, b] (in mu = lambda^2):
        // Newton steps, kept only while they stay inside the bracket (else
        // the geometric midpoint), the bracket narrowed by the slope's sign;
        // it ends when a step moves mu by less than 1e-13 relative (near the
        // root the slope is rounding noise, and steps below that only wander
        // inside it) or cannot move it at all
        double a2 = lo * lo, b2 = hi * hi, mu = lo * hi;
        for (int it = 0; it < 60; ++it) {
          const SlopeAndDerivative sd = gcv_slope2(sig2, c2, k, mu, omega, red4, par);
          if (sd.s == 0.0) break;
          if (sd.s < 0.0)
            a2 = mu;
          else
            b2 = mu;
          double nx = (sd.ds > 0.0) ? mu - sd.s / sd.ds : -1.0;
          if (!(nx > a2 && nx < b2)) nx = sqrt(a2) * sqrt(b2);
          if (!(nx > a2 && nx < b2) || nx == mu) break;
          const bool done = fabs(nx - mu) <= 1e-13 * mu;
          mu = nx;
          if (done) break;
        }
        const GcvSums g = gcv_sums(sig2, c2, k, mu, omega, red4, par);
        if (!((double)k * g.N / (g.D * g.D) > gib)) lam = sqrt(mu);
      }
    }
  }
  if (ts) ts[4] = gtimer();

  // ---- projected residual (and the filter-factor trace of Eq. stop2) --------
  double rs = 0.0, tr = 0.0;
  if (lam != 0.0) {
    const double L2 = lam * lam;
    for (int i = tid; i < k; i += nt) {
      const double f = L2 / (sig2[i] + L2);
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
  if (a.cvec)
    for (int i = tid; i <= k; i += nt) a.cvec[(int64_t)prob * a.ldc + i] = sqrt(c2[i]);
  double* yp = a.y ? a.y + (int64_t)pi.p * a.ldy : nullptr;
  if (!(pi.is_final && a.want_y && yp)) return;

  if (ts) ts[5] = gtimer();
  // ---- z = argmin ||beta e1 - B z||^2 + lambda^2 ||z||^2 ---------------------
  // Givens sweep on B / sigma_1 (rotations do not depend on the scale; the
  // scaled entries cannot overflow when squared), one thread.
  if (tid == 0) {
    const double sc = s1 > 0.0 ? 1.0 / s1 : 1.0;
    const double lm = lam * sc;
    const double L2 = lm * lm;
    double rbar = al[0] * sc, phibar = beta * sc;
    for (int j = 0; j < k; ++j) {
      const double bj = be[j + 1] * sc;
      const double q = fma(rbar, rbar, L2);  // r1^2 after removing lambda-row j
      const double ir = rsqrt(fma(bj, bj, q));  // 1 / r after removing beta_{j+1}
      double c1 = 1.0, r1 = rbar;  // lambda = 0: no first rotation
      if (lm != 0.0) {
        const double iq = rsqrt(q);
        c1 = rbar * iq;
        r1 = q * iq;
      }
      const double cs = r1 * ir, sn = bj * ir;
      const double phib = c1 * phibar;
      rinv[j] = ir;
      ph[j] = cs * phib;
      phibar = sn * phib;
      if (j + 1 < k) {
        const double an = al[j + 1] * sc;
        thv[j] = sn * an;
        rbar = -cs * an;
      }
    }
    // back substitution; z overwrites ph
    ph[k - 1] *= rinv[k - 1];
    for (int j = k - 2; j >= 0; --j) ph[j] = (ph[j] - thv[j] * ph[j + 1]) * rinv[j];
  }
  __syncthreads();
  if (ts) ts[6] = gtimer();
  // ---- y = Q z ----------------------------------------------------------------
  const int np = (k + kTF - 1) / kTF;
  if (np <= 1)
    apply_q<1>(S, k, ph, yp, qred);
  else if (np <= 2)
    apply_q<2>(S, k, ph, yp, qred);
  else if (np <= 3)
    apply_q<3>(S, k, ph, yp, qred);
  else if (np <= 4)
    apply_q<4>(S, k, ph, yp, qred);
  else if (np <= 8)
    apply_q<8>(S, k, ph, yp, qred);
  else
    apply_q<kQPer>(S, k, ph, yp, qred);
  if (ts) ts[7] = gtimer();
}

// ---- optimal lambda (needs x_true) ----------------------------------------
// y(lam) = Q z(lam) from the factorisation H = P B Q^T that k_bidiag leaves
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

// Refinement of the best grid point (ties: the smaller lambda) by
// multisection in log(lambda): round r evaluates kOptPts points spaced evenly
// inside its bracket, one block each, all at once (each evaluation is a chain
// of dependent FP64 operations, so rounds of parallel points take far less
// time than one point after another); the next bracket is the best point
// (ties: the smaller) and its two neighbours.  The bracket holds its centre
// as a point (kOptPts is odd), so the best value never increases; it shrinks
// by (kOptPts + 1) / 2 per round, to about 1e-8 of the grid's log spacing
// after kOptRounds rounds, below the resolution to which the minimiser of an
// error that is quadratic at its minimum is defined (~sqrt(eps)).
constexpr int kOptPts = 63;
constexpr int kOptRounds = 5;

// The bracket [lo, hi] (log lambda) that round r samples; false when the
// grid's best point is at an end of the grid (no refinement), with lo the
// log of that grid point.  One thread.
__device__ bool opt_bracket(int r, double s1, const double* Eg, const double* Er, double& lo,
                            double& hi) {
  int b = 0;
  for (int i = 1; i < kGrid; ++i)
    if (Eg[i] < Eg[b]) b = i;
  if (b == 0 || b == kGrid - 1) {
    lo = hi = log(s1 * pow(10.0, -14.0 + 0.0625 * b));
    return false;
  }
  lo = log(s1 * pow(10.0, -14.0 + 0.0625 * (b - 1)));
  hi = log(s1 * pow(10.0, -14.0 + 0.0625 * (b + 1)));
  for (int q = 0; q < r; ++q) {
    const double h = (hi - lo) / (kOptPts + 1);
    int j = 0;
    for (int i = 1; i < kOptPts; ++i)
      if (Er[q * kOptPts + i] < Er[q * kOptPts + j]) j = i;
    const double t = lo + (j + 1) * h;
    lo = t - h;
    hi = t + h;
  }
  return true;
}

// Round r of the refinement: block i evaluates point i of the round's bracket.
__global__ void __launch_bounds__(kT) k_opt_round(ProjWork w, int K, const DevState* st,
                                                  const double* G, const double* g,
                                                  const double* Eg, double* Er, int r) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  __shared__ double br[2];
  __shared__ bool go;
  const Slots S = carve(w.base, K, w.cluster);
  const int k = min(K, st->k_done);
  const double s1 = ldg_cg(S.sig);
  if (k <= 0 || !(s1 > 0.0)) return;
  if (threadIdx.x == 0) {
    double lo, hi;
    go = opt_bracket(r, s1, Eg, Er, lo, hi);
    br[0] = lo;
    br[1] = hi;
  }
  __syncthreads();
  if (!go) return;
  const double lam = exp(br[0] + (blockIdx.x + 1) * ((br[1] - br[0]) / (kOptPts + 1)));
  const double e = opt_eval(S, k, st->beta, lam, G, g, sm, red);
  if (threadIdx.x == 0) Er[r * kOptPts + blockIdx.x] = e;
}

// The refined lambda: the best point of the last round (or the grid point
// when it lies at an end of the grid).  One thread.
__global__ void k_opt_pick(ProjWork w, int K, const DevState* st, const double* Eg,
                           const double* Er, double* lam_out) {
  const Slots S = carve(w.base, K, w.cluster);
  const int k = min(K, st->k_done);
  const double s1 = ldg_cg(S.sig);
  if (k <= 0 || !(s1 > 0.0)) {
    *lam_out = 0.0;
    return;
  }
  double lo, hi;
  if (!opt_bracket(kOptRounds, s1, Eg, Er, lo, hi)) {
    *lam_out = exp(lo);
    return;
  }
  *lam_out = exp(0.5 * (lo + hi));  // the last round's best point
}

}  // namespace

int64_t projected_slot_doubles(int kk, int /*CL*/) {
  return 5 * (int64_t)(kk + 1) + kGrid + 1 + (int64_t)kk * kk + (int64_t)(kk + 1) * kk + 64;
}

// Per-device set-up of the projected kernels: their attributes (cluster size
// above 8, dynamic shared memory above 48 KB) are properties of the device
// they are set on, so they are set once for every device the process uses,
// with the cluster size found there and the device's SM count.  A mutex
// guards the first call on each device.
namespace {
constexpr int kProjMaxDevices = 64;
struct ProjDeviceSetup {
  int cluster = 0;  // 0: not set up yet
  int num_sms = 0;
};
ProjDeviceSetup g_proj_setup[kProjMaxDevices];
std::mutex g_proj_setup_mutex;

ProjDeviceSetup setup_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kProjMaxDevices) {
    cudaGetLastError();
    return ProjDeviceSetup{1, 0};
  }
  std::lock_guard<std::mutex> lock(g_proj_setup_mutex);
  ProjDeviceSetup& d = g_proj_setup[dev];
  if (d.cluster) return d;
  if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    d.num_sms = 0;
  cudaFuncSetAttribute(k_bidiag, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_bidiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  cudaFuncSetAttribute(k_sigma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  cudaFuncSetAttribute(k_sigma_lanes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  cudaFuncSetAttribute(k_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  int best = 1;
  for (int cand : {kMaxCluster, 8, 4, 2}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cand, 1, 1);
    cfg.blockDim = dim3(kTB, 1, 1);
    cfg.dynamicSmemBytes = kSmemCap;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cand;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_bidiag, &cfg) == cudaSuccess &&
        nclusters > 0) {
      best = cand;
      break;
    }
    cudaGetLastError();
  }
  d.cluster = best;
  return d;
}
}  // namespace

int projected_cluster_size() { return setup_current_device().cluster; }

cudaError_t launch_projected(const ProjArgs& a, ProjWork& w, cudaStream_t s, int* nlaunch) {
  if (nlaunch) *nlaunch = 0;
  // one problem per k of k_first..k_last (histories), or one final problem
  // per batch entry
  const bool batch = a.nbatch > 1;
  if (batch && (a.k_first != a.k_last || w.packed)) return cudaErrorInvalidValue;
  const int nprob = batch ? a.nbatch : a.k_last - a.k_first + 1;
  if (nprob <= 0) return cudaSuccess;
  if (!batch && nprob > 1 && !w.packed) return cudaErrorInvalidValue;
  if (w.cluster < 1 || w.cluster > kMaxCluster) return cudaErrorInvalidValue;
  const ProjDeviceSetup dev_setup = setup_current_device();
  const int kmax = a.k_last;
  const size_t K1 = (size_t)kmax + 1;
  // shared memory of k_bidiag: 5 + 2 kMaxCluster / cl vectors, and the slab
  // of the CTA's columns when it fits beside them
  auto vec_bytes = [&](int cl) { return (size_t)(5 + 2 * (kMaxCluster / cl)) * K1 * sizeof(double); };
  auto slab_bytes = [&](int cl) { return (size_t)((kmax + cl - 1) / cl) * K1 * sizeof(double); };
  // A history (problems of every size up to kmax) with more CTAs than two
  // per SM keeps the GPU busy with many clusters at once: there 8 CTAs per
  // problem, largest k first, do the whole batch in about 0.56 of the time 16
  // take (k = 1..300), although one problem alone is fastest on 16.
  int CL = w.cluster;
  w.desc = 0;
  if (!batch && nprob * CL > 2 * dev_setup.num_sms && CL > kHistoryCluster &&
      vec_bytes(kHistoryCluster) + slab_bytes(kHistoryCluster) <= kSmemCap) {
    CL = kHistoryCluster;
    w.desc = 1;
  }
  w.prob0 = 0;
  w.kcap = 0;
  const size_t vecs = vec_bytes(CL), slab = slab_bytes(CL);
  w.slab_in_smem = (vecs + slab <= kSmemCap) ? 1 : 0;
  const size_t dyn1 = vecs + (w.slab_in_smem ? slab : 0);
  const size_t dyn2 = 4 * K1 * sizeof(double);
  const size_t dyn4 = 7 * K1 * sizeof(double);
  if (dyn1 > kSmemCap || dyn2 > kSmemCap || dyn4 > kSmemCap) return cudaErrorInvalidValue;
  // 1. bidiagonalisation, one cluster per problem
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nprob * CL), 1, 1);
  cfg.blockDim = dim3(kTB, 1, 1);
  cfg.dynamicSmemBytes = dyn1;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_bidiag, a, w);
  if (e != cudaSuccess) return e;
  // 2. singular values and weights.  Final problems (the one of size k_last,
  // every batch entry) always take k_sigma, so that x does not depend on
  // whether histories were asked for or on the batch a problem was solved
  // in; the other problems of a history take k_sigma_lanes where that
  // finishes first.
  const int nlanes =
      (!batch && nprob > 1 && sigma_by_lanes(a, nprob - 1, dev_setup.num_sms)) ? nprob - 1 : 0;
  if (nlanes > 0) {
    w.prob0 = 0;
    const dim3 gl((unsigned)((K1 + kWL * 32 - 1) / (kWL * 32)), (unsigned)nlanes);
    k_sigma_lanes<<<gl, kWL * 32, dyn2, s>>>(a, w);
  }
  {
    w.prob0 = nlanes;
    const dim3 g2((unsigned)((K1 + kWS - 1) / kWS), (unsigned)(nprob - nlanes));
    size_t sm2 = dyn2;
    if ((int64_t)g2.x * g2.y <= dev_setup.num_sms && sm2 < kSmemOnePerSm) sm2 = kSmemOnePerSm;
    k_sigma<<<g2, kWS * 32, sm2, s>>>(a, w);
    w.prob0 = 0;
  }
  k_weights<<<(unsigned)nprob, kT, 0, s>>>(a, w);
  // 3. the GCV function on the lambda grid
  const bool grid = a.rule == LSLU_LAMBDA_GCV || a.rule == LSLU_LAMBDA_WGCV;
  if (grid) {
    const dim3 g3((unsigned)((kGrid + kWB - 1) / kWB), (unsigned)nprob);
    k_gcv_grid<<<g3, kWB * 32, 0, s>>>(a, w);
  }
  // 4. lambda, residual, y
  k_finish<<<(unsigned)nprob, kTF, dyn4, s>>>(a, w);
  if (nlaunch) *nlaunch = 4 + (nlanes > 0 ? 1 : 0) + (grid ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace lslu

namespace lslu {

int optimal_lambda_work_doubles() { return kOptRounds * kOptPts; }

cudaError_t launch_optimal_lambda(const ProjWork& w, int K, const DevState* st, const double* G,
                                  const double* g, double* Eg, double* Er, double* lam_out,
                                  cudaStream_t s) {
  const size_t smem = (size_t)4 * (K + 1) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_opt_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_opt_round, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_opt_grid<<<kGrid, kT, smem, s>>>(w, K, st, G, g, Eg);
  for (int r = 0; r < kOptRounds; ++r)
    k_opt_round<<<kOptPts, kT, smem, s>>>(w, K, st, G, g, Eg, Er, r);
  k_opt_pick<<<1, 1, 0, s>>>(w, K, st, Eg, Er, lam_out);
  return cudaGetLastError();
}

}  // namespace lslu
