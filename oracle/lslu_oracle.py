"""Plain FP64 oracle of LSLU and Hybrid LSLU (arXiv 2409.05239).

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  It is deliberately slow and plain,
FP64 numpy / scipy with library primitives (sparse mat-vec, dense SVD) as
single steps, and computes what the method defines:
  - the two bases of Section 2.2 (Eqs. nhr, nhr2): each new vector is A^T d_k
    or A l_k with the earlier basis vectors of its side removed, one at a
    time, by its own entries at their pivot rows, then divided by its largest
    unpivoted entry, whose row becomes the next pivot;
  - the projected Tikhonov problem of Section 3 (Eq. TSP) through the SVD of
    H_{k+1,k} (Eqs. 3-4), with lambda_k from Eqs. (gcv2) / (wgcv_projected1);
  - x_k = x_0 + L_k y_k.
Indices are 0-based (the paper is 1-based).

Parity pins (tests/test_oracle_pins.py) tie each function to something other
than itself; every function below is pinned.

Readings of the paper where it is silent or ambiguous (all also listed in the
design notes):
  R1  argmax ties go to the lowest index.
  R2  the basis step continues while some unpivoted entry is non-zero; with no
      unpivoted candidate, or all of them exactly zero, it breaks down.
  R3  on a breakdown the iterate of the last completed iteration is returned.
  R4  elimination runs sequentially in j (Algorithm 4 order).
  R6  beta is the signed entry of largest magnitude of r0.
  R7  with x0 != 0 the regulariser is lambda^2 ||y||^2 (Eq. TSP).
  R8  the GCV numerator keeps the factor k.
  R9  the weighted-GCV numerator is the GCV numerator (Eq. gcv2); the '+'
      between its two terms is missing in the printed formula.
  R11 lambda = argmin G: G is evaluated on 257 log-spaced points
      sigma_1 * 10^[-14, 2]; the best grid point (ties -> smaller lambda) is
      refined by 64 bisection steps in log(lambda) on the sign of dG/d(lambda^2)
      inside its two neighbours, kept only if it does not increase G.
  R12 stopping function (Eq. stop2): its numerator is read as n times the
      projected residual ||beta e1 - H y_k||^2 (the printed formula has a '+'
      where the filter factor multiplies [U^T e1]_i; its derivation gives the
      product), its denominator as ((m - k) + sum_i lam_k^2/(sigma_i^2+lam_k^2))^2
      with lam_k the parameter chosen at iteration k; the iteration stops at the
      first k with |G^(k+1) - G^(k)| / G^(1) < tol (Eq. tol) and returns x_k.
  R15 sampled pivots (Section 2.2): pick t (t = 0 for r0, 2k+1 for q and 2k+2
      for u at iteration k) takes the largest |entry| among the unpivoted
      indices of row t of a given sample table (ties -> lowest index); when no
      sampled unpivoted entry is non-zero it falls back to the full search.
      The random indices are inputs, drawn by the caller.
  R16 uncertainty quantification (Section 4.2): with lambda = sigma / alpha the
      posterior covariance is sigma^2 (lambda^2 I + A^T A)^-1, so the low-rank
      Gamma_k uses lambda^2 where the printed formulas show lambda; D_k, W_k
      are the first k columns / the k x k block (A^T D_k = L_k W_k, Eq. nhr2).
      The Woodbury step keeps the factor lambda^-2 on the low-rank term:
      Gamma_k = sigma^2 lambda^-2 (I - Z Delta Z^T) (the last line of the
      printed derivation drops the factor its previous line carries).
  R17 optimal lambda (Section 3.2.1, Eq. lambda; needs x_true): lam_k minimises
      E(lam) = ||L_k y_k(lam) - x_true||^2; searched on the grid of R11, then 64
      golden-section steps in log(lam) between the best point's neighbours
      (kept only if E does not increase).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# status codes (shared meaning with the C library, defined independently)
OK = 0
BREAKDOWN_BETA = 5
BREAKDOWN_W = 6
BREAKDOWN_H = 7

RULES = ("none", "fixed", "gcv", "wgcv")


@dataclasses.dataclass
class OracleResult:
    x: np.ndarray
    gp: np.ndarray          # column pivots g (k_done)
    tp: np.ndarray          # row pivots t (k_done + 1)
    beta: float
    H: np.ndarray           # (k_done+1) x k_done
    W: np.ndarray           # k_done x k_done
    L: np.ndarray           # n x k_done
    D: np.ndarray           # m x (k_done+1)
    lam_hist: np.ndarray    # lambda_k for k = 1..k_done
    res_hist: np.ndarray    # ||beta e1 - H_{k+1,k} y_k|| for k = 1..k_done
    status: int
    k_done: int


def _argmax_abs_unpivoted(v: np.ndarray, pivoted: np.ndarray):
    """Index of the largest |v| outside the pivoted set, lowest index on ties
    (Algorithm 4, pivot search; reading R1).  None when no candidate exists."""
    a = np.abs(v)
    a = np.where(pivoted, -1.0, a)
    if not np.any(~pivoted):
        return None
    return int(np.argmax(a))  # numpy argmax returns the first maximum


def _sampled_pivot(v, pivoted, sample):
    """Pivot of Section 2.2's sampled variant (reading R15), or None when no
    sampled unpivoted entry is non-zero."""
    best, bi = 0.0, None
    for i in sorted(set(int(j) for j in sample)):
        if pivoted[i]:
            continue
        a = abs(v[i])
        if a > best:
            best, bi = a, i
    return bi


def _pick(v, pivoted, samples, t):
    if samples is not None:
        i = _sampled_pivot(v, pivoted, samples[t])
        if i is not None:
            return i
    return _argmax_abs_unpivoted(v, pivoted)


def hessenberg_rect_pivoted(A, b, x0, K, samples=None):
    """Hessenberg process with pivoting for rectangular A (Algorithm 4).

    A is an m x n scipy sparse matrix (or dense array), b length m, x0 length n
    or None.  Runs up to K iterations.  Returns a dict with L (n x k),
    D (m x (k+1)), H ((k+1) x k), W (k x k), pivots gp (k), tp (k+1), beta,
    status and k (completed iterations).  Relations (Eqs. nhr / nhr2):
    A L_k = D_{k+1} H_{k+1,k} and A^T D_k = L_k W_k.  samples (optional, one
    row of indices per pivot pick, 2K+1 rows) selects the sampled pivoting of
    Section 2.2 (reading R15).
    """
    m, n = A.shape
    r0 = np.array(b, dtype=np.float64, copy=True)
    if x0 is not None:
        r0 = r0 - A @ np.asarray(x0, dtype=np.float64)
    L = np.zeros((n, K))
    D = np.zeros((m, K + 1))
    H = np.zeros((K + 1, K))
    W = np.zeros((K, K))
    gp = np.zeros(K, dtype=np.int64)
    tp = np.zeros(K + 1, dtype=np.int64)
    g_used = np.zeros(n, dtype=bool)
    t_used = np.zeros(m, dtype=bool)

    # initialisation: beta = signed max-abs entry of r0 (R6), d_1 = r0 / beta
    i = _pick(r0, t_used, samples, 0)
    if i is None or r0[i] == 0.0 or not np.isfinite(r0[i]):
        return dict(L=L[:, :0], D=D[:, :0], H=H[:0, :0], W=W[:0, :0], gp=gp[:0],
                    tp=tp[:0], beta=0.0, status=BREAKDOWN_BETA, k=0)
    beta = float(r0[i])
    D[:, 0] = r0 / beta
    tp[0] = i
    t_used[i] = True

    status = OK
    k_done = 0
    for k in range(K):
        # q = A^T d_k, then eliminate against l_0 .. l_{k-1} in order (R4)
        q = np.asarray(A.T @ D[:, k], dtype=np.float64).reshape(-1)
        for j in range(k):
            W[j, k] = q[gp[j]]
            q = q - W[j, k] * L[:, j]
        i = _pick(q, g_used, samples, 2 * k + 1)
        if i is None or q[i] == 0.0:
            status = BREAKDOWN_W
            break
        W[k, k] = q[i]
        L[:, k] = q / W[k, k]
        gp[k] = i
        g_used[i] = True

        # u = A l_k, then eliminate against d_0 .. d_k in order
        u = np.asarray(A @ L[:, k], dtype=np.float64).reshape(-1)
        for j in range(k + 1):
            H[j, k] = u[tp[j]]
            u = u - H[j, k] * D[:, j]
        i = _pick(u, t_used, samples, 2 * k + 2)
        if i is None or u[i] == 0.0:
            status = BREAKDOWN_H
            break
        H[k + 1, k] = u[i]
        D[:, k + 1] = u / H[k + 1, k]
        tp[k + 1] = i
        t_used[i] = True
        k_done = k + 1

    k = k_done
    return dict(L=L[:, :k], D=D[:, :k + 1], H=H[:k + 1, :k], W=W[:k, :k],
                gp=gp[:k], tp=tp[:k + 1], beta=beta, status=status, k=k)


def projected_svd(H: np.ndarray, beta: float):
    """SVD quantities of the projected problem (Section 3.2.1, Eqs. 3-4, gcv2).

    H = U Sigma V^T with U (k+1) x (k+1).  Returns sigma (k), c = beta U^T e1
    (length k+1) and V (k x k).
    """
    U, s, Vt = np.linalg.svd(H, full_matrices=True)
    c = beta * U[0, :]
    return s, c, Vt.T


def tikhonov_y(sigma, c, V, lam):
    """y = argmin ||beta e1 - H y||^2 + lam^2 ||y||^2 (Eq. TSP) via the SVD:
    y = V diag(sigma_i / (sigma_i^2 + lam^2)) c_{1:k} (Eq. 4).  For lam = 0
    (plain LSLU) singular values below (k+1) * eps * sigma_1 are dropped."""
    k = sigma.shape[0]
    if k == 0:
        return np.zeros(0)
    if lam == 0.0:
        keep = sigma > (k + 1) * np.finfo(np.float64).eps * sigma[0]
        f = np.where(keep, 1.0 / np.where(keep, sigma, 1.0), 0.0)
    else:
        f = sigma / (sigma ** 2 + lam ** 2)
    return V @ (f * c[:k])


def projected_residual(sigma, c, lam):
    """||beta e1 - H y_lam|| from the SVD: the components are
    lam^2/(sigma_i^2+lam^2) c_i (i <= k) and c_{k+1}."""
    k = sigma.shape[0]
    if lam == 0.0:
        keep = sigma > (k + 1) * np.finfo(np.float64).eps * sigma[0] if k else sigma > 0
        r = np.where(keep, 0.0, c[:k])
    else:
        r = lam ** 2 / (sigma ** 2 + lam ** 2) * c[:k]
    return math.sqrt(float(np.sum(r ** 2) + c[k] ** 2))


def gcv_value(sigma, c, lam, omega=1.0):
    """(Weighted) GCV function of the projected problem, Eqs. (gcv2)/(wgcv):
    G = k (sum_i (f_i c_i)^2 + c_{k+1}^2) / (1 + sum_i (1 - omega (1 - f_i)))^2
    with f_i = lam^2/(sigma_i^2+lam^2); omega = 1 is plain GCV (R8, R9)."""
    k = sigma.shape[0]
    L2 = lam * lam
    s2 = sigma * sigma
    f = L2 / (s2 + L2)
    num = k * (np.sum((f * c[:k]) ** 2) + c[k] ** 2)
    den = 1.0 + np.sum(((1.0 - omega) * s2 + L2) / (s2 + L2))
    return float(num / den ** 2)


def gcv_slope(sigma, c, lam, omega=1.0):
    """Sign-carrying derivative N' D - 2 N D' of G = N / D^2 with respect to
    mu = lam^2 (same sign as dG/dlam for lam > 0)."""
    L2 = lam * lam
    s2 = sigma * sigma
    k = sigma.shape[0]
    w = s2 + L2
    f = L2 / w
    dfdmu = s2 / (w * w)
    N = np.sum((f * c[:k]) ** 2) + c[k] ** 2
    dN = np.sum(2.0 * f * dfdmu * c[:k] ** 2)
    Dn = 1.0 + np.sum(((1.0 - omega) * s2 + L2) / w)
    dD = omega * np.sum(dfdmu)
    return float(dN * Dn - 2.0 * N * dD)


def lambda_grid(sigma1):
    return sigma1 * 10.0 ** np.linspace(-14.0, 2.0, 257)


def select_lambda(sigma, c, omega=1.0):
    """lambda_k = argmin_lambda G(lambda) (reading R11)."""
    if sigma.shape[0] == 0 or sigma[0] == 0.0:
        return 0.0
    grid = lambda_grid(sigma[0])
    G = np.array([gcv_value(sigma, c, l, omega) for l in grid])
    i = int(np.argmin(G))  # first minimum: ties go to the smaller lambda
    if i == 0 or i == grid.shape[0] - 1:
        return float(grid[i])
    a, bnd = math.log(grid[i - 1]), math.log(grid[i + 1])
    if not (gcv_slope(sigma, c, math.exp(a), omega) < 0.0
            and gcv_slope(sigma, c, math.exp(bnd), omega) > 0.0):
        return float(grid[i])
    for _ in range(64):
        mid = 0.5 * (a + bnd)
        if gcv_slope(sigma, c, math.exp(mid), omega) < 0.0:
            a = mid
        else:
            bnd = mid
    lam = math.exp(0.5 * (a + bnd))
    if gcv_value(sigma, c, lam, omega) > G[i]:
        return float(grid[i])
    return lam


def _lambda_for(rule, lam_fixed, sigma, c, k, m):
    if rule == "none":
        return 0.0
    if rule == "fixed":
        return float(lam_fixed)
    if rule == "gcv":
        return select_lambda(sigma, c, 1.0)
    if rule == "wgcv":
        return select_lambda(sigma, c, (k + 1) / m)  # omega = (k+1)/m
    raise ValueError(rule)


def hybrid_lslu(A, b, x0=None, K=10, rule="gcv", lam=0.0, histories=True, samples=None):
    """Hybrid LSLU (Algorithm 5); rule 'none' is plain LSLU (lambda = 0).

    Returns an OracleResult with x_k for the last completed iteration k,
    the pivots, H, W, the bases and (if histories) lambda_k and the projected
    residual for every k.
    """
    if rule not in RULES:
        raise ValueError(rule)
    m, n = A.shape
    hp = hessenberg_rect_pivoted(A, b, x0, K, samples)
    k = hp["k"]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    lam_hist = np.zeros(k)
    res_hist = np.zeros(k)
    kk_list = range(1, k + 1) if histories else ([k] if k > 0 else [])
    y = None
    for kk in kk_list:
        Hk = hp["H"][:kk + 1, :kk]
        s, c, V = projected_svd(Hk, hp["beta"])
        lk = _lambda_for(rule, lam, s, c, kk, m)
        lam_hist[kk - 1] = lk
        res_hist[kk - 1] = projected_residual(s, c, lk)
        if kk == k:
            y = tikhonov_y(s, c, V, lk)
    if k > 0:
        x = x + hp["L"] @ y
    return OracleResult(x=x, gp=hp["gp"], tp=hp["tp"], beta=hp["beta"], H=hp["H"],
                        W=hp["W"], L=hp["L"], D=hp["D"], lam_hist=lam_hist,
                        res_hist=res_hist, status=hp["status"], k_done=k)


def stopping_gcv_value(sigma, c, lam, n, m):
    """G^(k) of Eq. (stop2) for one k (reading R12): sigma (k), c = beta U^T e1
    (k+1), lam = lam_k, n and m the dimensions of A."""
    k = sigma.shape[0]
    L2 = lam * lam
    f = L2 / (sigma * sigma + L2)
    num = n * (float(np.sum((f * c[:k]) ** 2)) + float(c[k] ** 2))
    den = (m - k) + float(np.sum(f))
    return num / (den * den)


def stopping_iteration(G, tol):
    """First k (1-based) with |G(k+1) - G(k)| / G(1) < tol (Eq. tol), or the
    last k when the test never passes.  G[i] holds G^(i+1)."""
    for k in range(1, len(G)):
        if abs((G[k] - G[k - 1]) / G[0]) < tol:
            return k
    return len(G)


def hybrid_lslu_stopping(A, b, K_max, rule="wgcv", lam=0.0, tol=1e-6):
    """Hybrid LSLU with the stopping criterion of Section 3.2.2: runs up to K_max
    iterations, evaluates G^(k) for every k with the lambda_k of the rule and
    returns (x_k at the stopping iteration, k, G history)."""
    m, n = A.shape
    hp = hessenberg_rect_pivoted(A, b, None, K_max)
    kd = hp["k"]
    G = np.zeros(kd)
    lams = np.zeros(kd)
    for kk in range(1, kd + 1):
        Hk = hp["H"][:kk + 1, :kk]
        s_, c_, _ = projected_svd(Hk, hp["beta"])
        lk = _lambda_for(rule, lam, s_, c_, kk, m)
        lams[kk - 1] = lk
        G[kk - 1] = stopping_gcv_value(s_, c_, lk, n, m)
    k = stopping_iteration(G, tol) if kd > 0 else 0
    x = np.zeros(n)
    if k > 0:
        Hk = hp["H"][:k + 1, :k]
        s_, c_, V = projected_svd(Hk, hp["beta"])
        x = hp["L"][:, :k] @ tikhonov_y(s_, c_, V, lams[k - 1])
    return x, k, G


def uq_lowrank(L, D, W, lam, sigma2):
    """Low-rank posterior covariance of Section 4.2 (reading R16).

    A^T A ~ L_k W_k (D_k^T D_k)^-1 W_k^T L_k^T = L_k G^T G L_k^T; with the
    eigendecomposition G^T G = V diag(s2) V^T and Z = L_k V,
    Gamma_k = sigma^2 lam^-2 (I - Z Delta Z^T), Delta = (Z^T Z + lam^2 diag(s2)^-1)^-1
    (Woodbury).  Returns (diag(Gamma_k), 1^T Gamma_k 1)."""
    n, k = L.shape
    Dk = D[:, :k]
    GtG = W @ np.linalg.solve(Dk.T @ Dk, W.T)
    GtG = 0.5 * (GtG + GtG.T)
    s2, V = np.linalg.eigh(GtG)
    Z = L @ V
    Delta = np.linalg.inv(Z.T @ Z + lam * lam * np.diag(1.0 / s2))
    diag = sigma2 / (lam * lam) * (1.0 - np.einsum("ij,jk,ik->i", Z, Delta, Z))
    zs = Z.T @ np.ones(n)
    total = sigma2 / (lam * lam) * (n - zs @ Delta @ zs)
    return diag, float(total)


GOLDEN = (math.sqrt(5.0) - 1.0) / 2.0


def optimal_lambda(L, sigma, c, V, x_true):
    """Optimal Tikhonov parameter of the projected problem (reading R17):
    argmin_lam ||L y(lam) - x_true||^2 with y from Eq. (4)."""
    def E(lam):
        r = L @ tikhonov_y(sigma, c, V, lam) - x_true
        return float(r @ r)

    if sigma.shape[0] == 0 or sigma[0] == 0.0:
        return 0.0
    grid = lambda_grid(sigma[0])
    Eg = np.array([E(l) for l in grid])
    i = int(np.argmin(Eg))
    if i == 0 or i == grid.shape[0] - 1:
        return float(grid[i])
    a, b = math.log(grid[i - 1]), math.log(grid[i + 1])
    cpt = b - GOLDEN * (b - a)
    dpt = a + GOLDEN * (b - a)
    ec, ed = E(math.exp(cpt)), E(math.exp(dpt))
    for _ in range(64):
        if ec < ed:
            b, dpt, ed = dpt, cpt, ec
            cpt = b - GOLDEN * (b - a)
            ec = E(math.exp(cpt))
        else:
            a, cpt, ec = cpt, dpt, ed
            dpt = a + GOLDEN * (b - a)
            ed = E(math.exp(dpt))
    lam = math.exp(0.5 * (a + b))
    return lam if E(lam) <= Eg[i] else float(grid[i])


def hybrid_lslu_optimal(A, b, K, x_true):
    """Hybrid LSLU at iteration K with the optimal lambda (R17): returns
    (x_K, lam_K, E)."""
    hp = hessenberg_rect_pivoted(A, b, None, K)
    k = hp["k"]
    s_, c_, V = projected_svd(hp["H"][:k + 1, :k], hp["beta"])
    lam = optimal_lambda(hp["L"], s_, c_, V, x_true)
    x = hp["L"] @ tikhonov_y(s_, c_, V, lam)
    return x, lam, float(np.sum((x - x_true) ** 2))
