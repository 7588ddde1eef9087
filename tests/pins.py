"""Checks that tie the FP64 oracle to facts fixed by the paper and by
mathematics, independent of the oracle's own code.

Each check takes the oracle module as an argument so that the mutation tests
can run the same checks against a deliberately broken copy of the oracle.
Every check raises AssertionError when the pin does not hold.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# small dense problems
# ----------------------------------------------------------------------------


def random_problem(m, n, seed, decay=0.85):
    """Dense ill-posed test matrix A = U diag(decay^i) V^T, x_true, b."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    r = min(m, n)
    s = decay ** np.arange(r)
    A = U[:, :r] @ np.diag(s) @ V[:, :r].T
    x = rng.standard_normal(n)
    b = A @ x + 1e-3 * rng.standard_normal(m)
    return A, x, b


def square_hessenberg_pivoted(M, r0, K):
    """Algorithm 2 (Hessenberg process with pivoting, square M), written
    independently of the rectangular oracle.  Returns L (n x K+1), pivots p,
    Hessenberg Hs ((K+1) x K)."""
    n = M.shape[0]
    L = np.zeros((n, K + 1))
    Hs = np.zeros((K + 1, K))
    perm = np.arange(n)
    i = int(np.argmax(np.abs(r0)))
    beta = r0[i]
    L[:, 0] = r0 / beta
    perm[[0, i]] = perm[[i, 0]]
    for k in range(K):
        u = M @ L[:, k]
        for j in range(k + 1):
            Hs[j, k] = u[perm[j]]
            u = u - Hs[j, k] * L[:, j]
        rest = perm[k + 1:]
        ii = int(np.argmax(np.abs(u[rest]))) + k + 1
        Hs[k + 1, k] = u[perm[ii]]
        L[:, k + 1] = u / Hs[k + 1, k]
        perm[[k + 1, ii]] = perm[[ii, k + 1]]
    return L, perm[:K + 1], Hs


# ----------------------------------------------------------------------------
# basis pins (Algorithm 4, Eqs. nhr, nhr2, h1, h2)
# ----------------------------------------------------------------------------


def check_unit_pivot_structure(hp, max_abs_one=True):
    """Each basis vector has a 1 at its own pivot, exact zeros at all earlier
    pivots and max-abs 1 (Algorithm 4: elimination then max-abs scaling; the
    last property only with the full pivot search)."""
    for Bmat, piv in ((hp["L"], hp["gp"]), (hp["D"], hp["tp"])):
        k = Bmat.shape[1]
        assert len(set(piv.tolist())) == len(piv), "pivot list repeats an index"
        for j in range(k):
            col = Bmat[:, j]
            assert col[piv[j]] == 1.0, f"basis vector {j} not 1 at its pivot"
            assert np.all(col[piv[:j]] == 0.0), f"basis vector {j} not 0 at earlier pivots"
            if max_abs_one:
                assert np.max(np.abs(col)) == 1.0, f"basis vector {j} has max-abs != 1"


def check_hessenberg_relations(A, hp, tol=1e-12):
    """A L_k = D_{k+1} H_{k+1,k} (Eq. nhr) and A^T D_k = L_k W_k (Eq. nhr2)."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    L, D, H, W = hp["L"], hp["D"], hp["H"], hp["W"]
    k = L.shape[1]
    scale = np.linalg.norm(Ad) * max(np.linalg.norm(L), np.linalg.norm(D))
    r1 = np.linalg.norm(Ad @ L - D @ H)
    r2 = np.linalg.norm(Ad.T @ D[:, :k] - L @ W)
    assert r1 <= tol * scale, f"A L != D H: {r1 / scale:.3e}"
    assert r2 <= tol * scale, f"A^T D != L W: {r2 / scale:.3e}"
    assert np.all(np.tril(H, -2) == 0.0), "H is not upper Hessenberg"
    assert np.all(np.tril(W, -1) == 0.0), "W is not upper triangular"


def check_normal_equation_equivalence(O, A, b, K, tol=1e-9):
    """Algorithm 4 equals Algorithm 2 applied to A^T A (start A^T r0) and to
    A A^T (start r0): same bases and pivots, with Hessenberg matrices
    W_{k+1} H_{k+1,k} and H_{k+2,k+1} W_{k+1} (Eqs. h1, h2)."""
    hp = O.hessenberg_rect_pivoted(A, b, None, K)
    assert hp["k"] == K
    L2, p2, Hs = square_hessenberg_pivoted(A.T @ A, A.T @ b, K - 1)
    assert np.array_equal(hp["gp"], p2), f"column pivots differ: {hp['gp']} vs {p2}"
    assert np.allclose(hp["L"], L2, rtol=0, atol=tol), "L differs from Algorithm 2 on A^T A"
    WH = hp["W"] @ hp["H"][:K, :K - 1]
    assert np.allclose(WH, Hs, rtol=0, atol=tol * np.abs(Hs).max()), "W H differs"
    D2, t2, Hd = square_hessenberg_pivoted(A @ A.T, b, K)
    assert np.array_equal(hp["tp"], t2), f"row pivots differ: {hp['tp']} vs {t2}"
    assert np.allclose(hp["D"], D2, rtol=0, atol=tol), "D differs from Algorithm 2 on A A^T"
    HW = hp["H"] @ hp["W"]
    assert np.allclose(HW, Hd, rtol=0, atol=tol * np.abs(Hd).max()), "H W differs"


def _principal_sines(X, Y):
    Qx, _ = np.linalg.qr(X)
    Qy, _ = np.linalg.qr(Y)
    s = np.linalg.svd(Qx.T @ Qy, compute_uv=False)
    return np.sqrt(np.maximum(0.0, 1.0 - np.min(s) ** 2))


def check_krylov_spans(O, A, b, K, tol=1e-7):
    """R(L_k) = K_k(A^T A, A^T r0) and R(D_{k+1}) = K_{k+1}(A A^T, r0)
    (Eqs. K1, K2, Pk, Ck), compared by principal angles."""
    hp = O.hessenberg_rect_pivoted(A, b, None, K)
    v = A.T @ b
    P = np.column_stack([np.linalg.matrix_power(A.T @ A, j) @ v for j in range(K)])
    C = np.column_stack([np.linalg.matrix_power(A @ A.T, j) @ b for j in range(K + 1)])
    assert _principal_sines(hp["L"], P) < tol, "R(L_k) != K_k(A^T A, A^T r0)"
    assert _principal_sines(hp["D"], C) < tol, "R(D_k+1) != K_k+1(A A^T, r0)"


# ----------------------------------------------------------------------------
# projected problem pins (Eqs. TSP, 3, 4, gcv1, gcv2, wgcv)
# ----------------------------------------------------------------------------


def check_tikhonov_vs_stacked_lstsq(O, H, beta, lams, tol=1e-10):
    """y from the SVD formula equals the least-squares solution of the
    stacked system [H; lam I] y = [beta e1; 0] (Eq. TSP), and the SVD
    residual equals ||beta e1 - H y||."""
    kp1, k = H.shape
    e1 = np.zeros(kp1)
    e1[0] = beta
    s, c, V = O.projected_svd(H, beta)
    for lam in lams:
        y = O.tikhonov_y(s, c, V, lam)
        if lam == 0.0:
            y_ref = np.linalg.lstsq(H, e1, rcond=None)[0]
        else:
            Ms = np.vstack([H, lam * np.eye(k)])
            y_ref = np.linalg.lstsq(Ms, np.concatenate([e1, np.zeros(k)]), rcond=None)[0]
        assert np.linalg.norm(y - y_ref) <= tol * np.linalg.norm(y_ref), f"y mismatch at lam={lam}"
        res = O.projected_residual(s, c, lam)
        res_ref = np.linalg.norm(e1 - H @ y_ref)
        assert abs(res - res_ref) <= 1e-9 * max(res_ref, 1e-300) + 1e-14 * abs(beta), \
            f"residual mismatch at lam={lam}: {res} vs {res_ref}"


def gcv_explicit(H, beta, lam, omega=1.0):
    """Eq. (gcv1) / (wgcv_projected1) with the explicit regularised inverse."""
    kp1, k = H.shape
    e1 = np.zeros(kp1)
    e1[0] = beta
    Hl = np.linalg.solve(H.T @ H + lam ** 2 * np.eye(k), H.T)
    P = H @ Hl
    num = k * np.linalg.norm((np.eye(kp1) - P) @ e1) ** 2
    den = np.trace(np.eye(kp1) - omega * P) ** 2
    return num / den


def check_gcv_forms(O, H, beta, lams, omegas=(1.0, 0.3), tol=1e-9):
    s, c, _ = O.projected_svd(H, beta)
    for om in omegas:
        for lam in lams:
            g = O.gcv_value(s, c, lam, om)
            ge = gcv_explicit(H, beta, lam, om)
            assert abs(g - ge) <= tol * abs(ge), f"G mismatch lam={lam} omega={om}: {g} vs {ge}"


def check_lambda_is_minimiser(O, H, beta, omega=1.0):
    """lambda_k from select_lambda minimises G: no point of a 20001-point
    log grid over the search range is lower, and a bounded scalar minimiser
    (scipy) started around it agrees."""
    from scipy.optimize import minimize_scalar

    s, c, _ = O.projected_svd(H, beta)
    lam = O.select_lambda(s, c, omega)
    Gs = O.gcv_value(s, c, lam, omega)
    grid = s[0] * 10.0 ** np.linspace(-14.0, 2.0, 20001)
    Gg = np.array([O.gcv_value(s, c, l, omega) for l in grid])
    j = int(np.argmin(Gg))
    assert Gs <= Gg[j] * (1 + 1e-9), f"G(lambda*)={Gs} above grid min {Gg[j]}"
    if 0 < j < grid.shape[0] - 1:
        res = minimize_scalar(lambda t: O.gcv_value(s, c, np.exp(t), omega),
                              bounds=(np.log(grid[j - 1]), np.log(grid[j + 1])),
                              method="bounded", options={"xatol": 1e-10})
        assert abs(np.log(lam) - res.x) < 1e-3, f"lambda {lam} vs scipy {np.exp(res.x)}"


def wgcv_from_definition(H, beta, lam, omega):
    """G(omega, lambda) of Eq. (wgcv_projected1) from its definition, without
    an SVD: y_lambda from a QR of the stacked matrix [H; lambda I], the
    residual (I - H H_lambda^+) beta e1 = beta e1 - H y_lambda, and
    trace(H H_lambda^+) = ||Q_1||_F^2 with Q_1 the first k+1 rows of Q
    (H = Q_1 R and H_lambda^+ = R^-1 Q_1^T), so the denominator is
    ((k+1) - omega ||Q_1||_F^2)^2."""
    kp1, k = H.shape
    Q, R = np.linalg.qr(np.vstack([H, lam * np.eye(k)]))
    rhs = np.zeros(kp1 + k)
    rhs[0] = beta
    y = np.linalg.solve(R, Q.T @ rhs)
    r = rhs[:kp1] - H @ y
    tr = float(np.sum(Q[:kp1] ** 2))
    return k * float(r @ r) / (kp1 - omega * tr) ** 2


def check_wgcv_rule(O, A, b, K, npts=801):
    """The weighted-GCV rule (Section 3.2.1): at every iteration k, lambda_k
    minimises G(omega, lambda) with omega = (k+1)/m, m the row count of A.
    G comes from wgcv_from_definition and omega is computed here from k and
    m, so neither the oracle's SVD form nor its omega is reused.  lambda_k
    must reach the minimum of an npts-point log grid over
    sigma_1 10^[-14, 2] and, when that minimum is interior, agree with a
    bounded scalar minimiser (scipy) between its neighbours to 1e-3 in
    log(lambda)."""
    from scipy.optimize import minimize_scalar

    m = A.shape[0]
    res = O.hybrid_lslu(A, b, None, K, "wgcv")
    assert res.k_done == K, f"wgcv run stopped at {res.k_done}"
    for k in range(1, K + 1):
        H = res.H[:k + 1, :k]
        omega = (k + 1) / m
        lam = float(res.lam_hist[k - 1])

        def G(t):
            return wgcv_from_definition(H, res.beta, t, omega)

        s1 = np.linalg.norm(H, 2)
        grid = s1 * 10.0 ** np.linspace(-14.0, 2.0, npts)
        Gg = np.array([G(t) for t in grid])
        j = int(np.argmin(Gg))
        assert lam > 0.0 and G(lam) <= Gg[j] * (1 + 1e-9), \
            f"k={k}: G(lambda_k)={G(lam)} above the grid minimum {Gg[j]}"
        if 0 < j < npts - 1:
            r = minimize_scalar(lambda t: G(np.exp(t)), method="bounded",
                                bounds=(np.log(grid[j - 1]), np.log(grid[j + 1])),
                                options={"xatol": 1e-10})
            assert abs(np.log(lam) - r.x) < 1e-3, \
                f"k={k}: lambda_k={lam} but the minimiser is {np.exp(r.x)}"


# ----------------------------------------------------------------------------
# whole-iterate pins (Eq. quasi, Eq. TP, Theorems 1 and 2)
# ----------------------------------------------------------------------------


def check_oblique_bruteforce(O, A, b, K, lam, rule, tol=1e-9):
    """x_k = argmin over x in R(L_k) of ||D^+_{k+1}(b - A x)||^2 +
    lam^2 ||L_k^+ x||^2 (Eqs. quasi and TP with x0 = 0), solved densely."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    res = O.hybrid_lslu(A, b, None, K, rule, lam)
    L, D = res.L, res.D
    Dp = np.linalg.pinv(D)
    M = Dp @ Ad @ L
    rhs = Dp @ b
    lam_used = res.lam_hist[-1]
    k = L.shape[1]
    if lam_used == 0.0:
        y = np.linalg.lstsq(M, rhs, rcond=None)[0]
    else:
        y = np.linalg.lstsq(np.vstack([M, lam_used * np.eye(k)]),
                            np.concatenate([rhs, np.zeros(k)]), rcond=None)[0]
    x_ref = L @ y
    err = np.linalg.norm(res.x - x_ref) / np.linalg.norm(x_ref)
    assert err <= tol, f"x_k differs from brute-force oblique LS: {err:.3e}"


def check_theorem_bounds(O, A, b, K, lam):
    """Theorem 1 (lam = 0) and Theorem 2 (fixed lam): the LSQR residual
    bounds the LSLU residual from below, kappa times it from above."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    m, n = Ad.shape
    rule = "none" if lam == 0.0 else "fixed"
    res = O.hybrid_lslu(A, b, None, K, rule, lam)
    k = res.k_done
    Q, _ = np.linalg.qr(res.L)  # orthonormal basis of K_k(A^T A, A^T b)
    AQ = Ad @ Q
    if lam == 0.0:
        z = np.linalg.lstsq(AQ, b, rcond=None)[0]
        r_qr = np.linalg.norm(b - AQ @ z)
        r_lu = np.linalg.norm(b - Ad @ res.x)
        kappa = np.linalg.cond(res.D)
    else:
        Ms = np.vstack([AQ, lam * Q])
        z = np.linalg.lstsq(Ms, np.concatenate([b, np.zeros(n)]), rcond=None)[0]
        x_qr = Q @ z
        r_qr = np.sqrt(np.linalg.norm(b - Ad @ x_qr) ** 2 + lam ** 2 * np.linalg.norm(x_qr) ** 2)
        r_lu = np.sqrt(np.linalg.norm(b - Ad @ res.x) ** 2 + lam ** 2 * np.linalg.norm(res.x) ** 2)
        Dbar = np.zeros((m + n, 2 * k + 1))
        Dbar[:m, :k + 1] = res.D
        Dbar[m:, k + 1:] = res.L
        sv = np.linalg.svd(Dbar, compute_uv=False)
        kappa = sv[0] / sv[-1]
    assert r_qr <= r_lu * (1 + 1e-10), f"lower bound violated: {r_qr} > {r_lu}"
    assert r_lu <= kappa * r_qr * (1 + 1e-10), f"upper bound violated: {r_lu} > {kappa} * {r_qr}"
    return r_qr, r_lu, kappa
