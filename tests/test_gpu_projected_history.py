"""The projected problems of a whole history (lslu_projected_history: Eq. TSP
for every leading block H_{k+1,k} of one H, Eqs. gcv2 / wgcv for lambda_k)
against the oracle's rule on the same blocks.

With K = 160 the launcher runs the blocks as one throughput batch: 8-CTA
bidiagonalisations, one lane per singular value (bisection, then Newton steps
on det(T - theta)) for k < K, 32-point multisection for k = K.  The spectra:
a Hessenberg H of the 32x32 CT problem, a graded dense H, the same with a zero
column (zero singular values from there on), and a lower bidiagonal H whose
blocks have near-multiple singular values (where the Newton steps hand lanes
back to bisection)."""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import lslu, tomo

pytestmark = pytest.mark.gpu

K = 160


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_05239_gb300 import build

    build.build()


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


@pytest.fixture(scope="module")
def handle(ct32):
    with lslu.from_problem(ct32, "f64", K) as s:
        yield s


def ct_hessenberg(P):
    hp = O.hessenberg_rect_pivoted(P.scipy(), P.b, None, K)
    return hp["H"][:K + 1, :K], float(hp["beta"])


def graded(seed=3):
    rng = np.random.default_rng(seed)
    H = rng.standard_normal((K + 1, K)) * 10.0 ** (-10.0 * np.arange(K) / K)
    return H, 2.5


def zero_column(seed=3):
    H, beta = graded(seed)
    H[:, 57] = 0.0
    return H, beta


def near_multiple(seed=5):
    """alpha_j in four groups of equal values up to 1e-9 relative, beta_{j+1}
    = 1e-6 alpha_j: every block's singular values come in groups a few 1e-6
    wide (well inside the 2^-16 bracket at which Newton steps would start)."""
    rng = np.random.default_rng(seed)
    base = np.repeat([1.0, 1e-2, 1e-4, 1e-6], K // 4)
    alpha = base * (1.0 + 1e-9 * rng.standard_normal(K))
    H = np.zeros((K + 1, K))
    H[np.arange(K), np.arange(K)] = alpha
    H[np.arange(1, K + 1), np.arange(K)] = 1e-6 * alpha
    return H, 1.0


def gcv_min_spread(sig, c, omega, lam_ref, trials=6):
    """How far the minimum of G moves (relative) when sigma and c take
    perturbations within the backward error of any stable SVD of the block
    (a few units of roundoff of sigma_1 and |c|; and numerically zero
    singular values, <= (k+1) eps sigma_1, set to zero, as they are exactly
    for a rank-deficient block): the resolution to which the rule fixes G's
    minimum here.  On a flat weighted-GCV curve the noise value LAPACK gives a
    zero singular value decides where the smallest lambda lands."""
    eps = np.finfo(float).eps
    rng = np.random.default_rng(11)
    G0 = O.gcv_value(sig, c, lam_ref, omega)
    k = sig.shape[0]
    zeroed = np.where(sig <= (k + 1) * eps * sig[0], 0.0, sig)
    d = abs(O.gcv_value(sig, c, O.select_lambda(zeroed, c, omega), omega) - G0) / G0
    for _ in range(trials):
        sp = np.sort(np.abs(sig + 4 * eps * sig[0] * rng.standard_normal(sig.shape)))[::-1]
        cp = c + 4 * eps * np.linalg.norm(c) * rng.standard_normal(c.shape)
        lp = O.select_lambda(sp, cp, omega)
        d = max(d, abs(O.gcv_value(sig, c, lp, omega) - G0) / G0)
    return d


def residual_range(sig, c, lam):
    """The oracle's residual at lam with every numerically zero singular value
    (<= (k+1) eps sigma_1, a value within the SVD's backward error) anywhere
    between that bound and 0: the residual falls as such a sigma_i grows."""
    k = sig.shape[0]
    thr = (k + 1) * np.finfo(float).eps * sig[0]
    z = sig <= thr
    return (O.projected_residual(np.where(z, thr, sig), c, lam),
            O.projected_residual(np.where(z, 0.0, sig), c, lam))


CASES = {"ct32": None, "graded": graded, "zero-column": zero_column,
         "near-multiple": near_multiple}


def make(name, ct32):
    return ct_hessenberg(ct32) if name == "ct32" else CASES[name]()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("rule", ["gcv", "wgcv"])
def test_history_against_the_oracle_rule(handle, ct32, name, rule):
    H, beta = make(name, ct32)
    m = ct32.m
    out = handle.projected_history(H, beta, rule, m=m)
    for k in range(1, K + 1):
        sig, c, _ = O.projected_svd(H[:k + 1, :k], beta)
        omega = 1.0 if rule == "gcv" else (k + 1) / m
        lam_ref = O.select_lambda(sig, c, omega)
        lam = out["lam_hist"][k - 1]
        G_ref = O.gcv_value(sig, c, lam_ref, omega)
        G = O.gcv_value(sig, c, lam, omega)
        if G > G_ref * (1 + 1e-9):
            tol = 10 * gcv_min_spread(sig, c, omega, lam_ref)
            assert G <= G_ref * (1 + max(1e-9, tol)), (k, lam, lam_ref)
        lo, hi = residual_range(sig, c, lam)
        r = out["res_hist"][k - 1]
        assert lo * (1 - 1e-8) - 1e-14 * abs(beta) <= r <= hi * (1 + 1e-8) + 1e-14 * abs(beta), k
    # the final block runs as a single problem does
    assert out["lam_hist"][K - 1] == handle.projected(H, beta, rule, m=m)["lam"]


@pytest.mark.parametrize("name", ["ct32", "zero-column"])
def test_history_fixed_lambda(handle, ct32, name):
    H, beta = make(name, ct32)
    lam = 3e-3
    out = handle.projected_history(H, beta, "fixed", lam)
    assert np.all(out["lam_hist"] == lam)
    for k in range(1, K + 1):
        sig, c, _ = O.projected_svd(H[:k + 1, :k], beta)
        res = O.projected_residual(sig, c, lam)
        assert abs(out["res_hist"][k - 1] - res) <= 1e-9 * res + 1e-14 * abs(beta), k


@pytest.mark.parametrize("k", [58, 120])
def test_single_problem_with_a_zero_singular_value(handle, k):
    """One block with a zero column: its zero singular value takes the weight
    that U's orthogonality leaves (beta^2 minus the others), so G, the
    residual and y are the oracle's."""
    H, beta = zero_column()
    Hk = H[:k + 1, :k]
    sig, c, V = O.projected_svd(Hk, beta)
    lam_ref = O.select_lambda(sig, c, 1.0)
    out = handle.projected(Hk, beta, "gcv")
    assert out["sigma"][-1] <= (k + 1) * np.finfo(float).eps * out["sigma"][0]
    G_ref = O.gcv_value(sig, c, lam_ref)
    assert O.gcv_value(sig, c, out["lam"]) <= G_ref * (1 + 1e-9)
    res = O.projected_residual(sig, c, out["lam"])
    assert abs(out["resid"] - res) <= 1e-9 * res
    y_ref = O.tikhonov_y(sig, c, V, out["lam"])
    assert np.linalg.norm(out["y"] - y_ref) <= 1e-9 * np.linalg.norm(y_ref)
    assert abs(np.sum(out["c"] ** 2) - beta ** 2) <= 1e-12 * beta ** 2


def test_history_equals_the_solve_histories(ct32):
    """A solve's histories are this entry point on the solve's own H."""
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve(ct32.b, K, "wgcv", histories=True)
        st = s.state(r["k_done"])
        out = s.projected_history(st["H"], st["beta"], "wgcv")
    assert np.array_equal(out["lam_hist"], r["lam_hist"])
    assert np.array_equal(out["res_hist"], r["res_hist"])


def test_history_argument_checks(handle):
    H, beta = graded()
    with pytest.raises(lslu.LsluError):  # K above the handle's max_iter
        handle.projected_history(np.zeros((K + 2, K + 1)), beta)
    with pytest.raises(lslu.LsluError):
        handle.projected_history(H, beta, "fixed", -1.0)
    with pytest.raises(lslu.LsluError):
        handle.projected_history(H, beta, "wgcv", m=-1)
