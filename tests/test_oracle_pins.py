"""Pins of the FP64 oracle against what the paper and mathematics fix."""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import tomo
from tests import pins


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


@pytest.fixture(scope="module")
def ct32_run(ct32):
    return O.hessenberg_rect_pivoted(ct32.scipy(), ct32.b, None, 50)


@pytest.mark.parametrize("shape", [(30, 20), (20, 30), (25, 25)])
def test_normal_equation_equivalence_dense(shape):
    A, _, b = pins.random_problem(*shape, seed=sum(shape), decay=0.8)
    pins.check_normal_equation_equivalence(O, A, b, K=7)


def test_normal_equation_equivalence_tomo(ct32):
    A = ct32.scipy()
    pins.check_normal_equation_equivalence(O, A.toarray(), ct32.b, K=6, tol=1e-8)


def test_unit_pivot_structure_ct32(ct32_run):
    assert ct32_run["status"] == O.OK and ct32_run["k"] == 50
    pins.check_unit_pivot_structure(ct32_run)


def test_hessenberg_relations_ct32(ct32, ct32_run):
    pins.check_hessenberg_relations(ct32.scipy(), ct32_run)


@pytest.mark.parametrize("shape", [(40, 25), (25, 40)])
def test_krylov_spans(shape):
    A, _, b = pins.random_problem(*shape, seed=7, decay=0.7)
    pins.check_krylov_spans(O, A, b, K=5)


def test_x0_shift(ct32):
    """With x0 != 0 the process starts from r0 = b - A x0: running from x0
    equals running on b - A x0 from zero and adding x0."""
    A = ct32.scipy()
    x0 = np.linspace(0.0, 1.0, ct32.n)
    r1 = O.hybrid_lslu(A, ct32.b, x0, 12, "fixed", 1e-2)
    r2 = O.hybrid_lslu(A, ct32.b - A @ x0, None, 12, "fixed", 1e-2)
    assert np.array_equal(r1.gp, r2.gp)
    assert np.allclose(r1.x, r2.x + x0, rtol=0, atol=1e-12 * np.linalg.norm(r1.x))


@pytest.mark.parametrize("k", [1, 2, 5, 17, 40])
def test_tikhonov_vs_stacked_lstsq(ct32_run, k):
    H = ct32_run["H"][:k + 1, :k]
    pins.check_tikhonov_vs_stacked_lstsq(O, H, ct32_run["beta"], [0.0, 1e-4, 1e-2, 0.5, 30.0])


@pytest.mark.parametrize("k", [1, 3, 10, 30])
def test_gcv_forms(ct32_run, k):
    H = ct32_run["H"][:k + 1, :k]
    pins.check_gcv_forms(O, H, ct32_run["beta"], [1e-4, 1e-2, 0.3, 4.0])


def test_wgcv_omega_one_is_gcv(ct32_run):
    H = ct32_run["H"][:21, :20]
    s, c, _ = O.projected_svd(H, ct32_run["beta"])
    for lam in (1e-3, 0.1, 2.0):
        assert O.gcv_value(s, c, lam, 1.0) == O.gcv_value(s, c, lam)


@pytest.mark.parametrize("k", [1, 4, 12, 35, 50])
@pytest.mark.parametrize("omega", [1.0, 0.02])
def test_lambda_is_minimiser(ct32_run, k, omega):
    H = ct32_run["H"][:k + 1, :k]
    pins.check_lambda_is_minimiser(O, H, ct32_run["beta"], omega)


@pytest.mark.parametrize("m,n,seed,decay", [(40, 25, 5, 0.8), (40, 25, 7, 0.7), (60, 30, 3, 0.85),
                                             (25, 40, 9, 0.8)])
def test_wgcv_rule_minimises_definition(m, n, seed, decay):
    """Weighted GCV with omega = (k+1)/m (Section 3.2.1): the oracle's
    lambda_k minimises Eq. (wgcv_projected1) built from its definition, at
    every k, on problems where m != n and m is small enough that omega moves
    the minimiser."""
    A, _, b = pins.random_problem(m, n, seed=seed, decay=decay)
    pins.check_wgcv_rule(O, A, b, 14)


def test_wgcv_rule_ct32(ct32):
    """The same on the 32x32 tomography workload (m = 2070 rows, n = 1024)."""
    pins.check_wgcv_rule(O, ct32.scipy(), ct32.b, 20, npts=401)


def test_gcv_k1_closed_form():
    """For k = 1 the GCV minimiser has the closed form f* = c2^2 / c1^2 with
    f = lam^2 / (sigma^2 + lam^2) (set dG/df = 0 in Eq. gcv2)."""
    sigma = np.array([2.0])
    c = np.array([1.0, 0.5])
    lam = O.select_lambda(sigma, c, 1.0)
    f = 0.25
    lam_ref = np.sqrt(f * sigma[0] ** 2 / (1 - f))
    assert abs(lam - lam_ref) <= 1e-12 * lam_ref


@pytest.mark.parametrize("rule,lam", [("none", 0.0), ("fixed", 1e-2), ("fixed", 0.5), ("gcv", 0.0),
                                      ("wgcv", 0.0)])
def test_oblique_bruteforce_ct32(ct32, rule, lam):
    pins.check_oblique_bruteforce(O, ct32.scipy(), ct32.b, 15, lam, rule)


@pytest.mark.parametrize("shape", [(40, 25), (25, 40)])
def test_oblique_bruteforce_dense(shape):
    A, _, b = pins.random_problem(*shape, seed=11, decay=0.8)
    pins.check_oblique_bruteforce(O, A, b, 8, 1e-2, "fixed")
    pins.check_oblique_bruteforce(O, A, b, 8, 0.0, "none")


def test_lambda_zero_is_lslu(ct32):
    """Hybrid LSLU with lambda = 0 reproduces LSLU, whose y_k solves
    min ||beta e1 - H_{k+1,k} y|| (Section 2.2)."""
    A = ct32.scipy()
    r = O.hybrid_lslu(A, ct32.b, None, 30, "fixed", 0.0)
    e1 = np.zeros(31)
    e1[0] = r.beta
    y = np.linalg.lstsq(r.H, e1, rcond=None)[0]
    assert np.linalg.norm(r.x - r.L @ y) <= 1e-10 * np.linalg.norm(r.x)
    r2 = O.hybrid_lslu(A, ct32.b, None, 30, "none", 0.0)
    assert np.array_equal(r.x, r2.x)


@pytest.mark.parametrize("K", [3, 10, 25])
@pytest.mark.parametrize("lam", [0.0, 1e-2])
def test_theorem_bounds_ct32(ct32, K, lam):
    pins.check_theorem_bounds(O, ct32.scipy(), ct32.b, K, lam)


def test_breakdown_beta():
    A, _, _ = pins.random_problem(10, 8, seed=3)
    r = O.hybrid_lslu(A, np.zeros(10), None, 5, "gcv")
    assert r.status == O.BREAKDOWN_BETA and r.k_done == 0 and np.all(r.x == 0)


def test_breakdown_w_exact():
    """Hand-worked case: A = diag(1, 2) padded to 4 x 3, b = ones.  Exact
    arithmetic gives d1 = b, l1 = (1/2, 1, 0), l2 = e0, d3 = (0, 0, 1, 1) and
    then A^T d3 = 0, so the third q vanishes: breakdown in the W step after two
    completed iterations (Algorithm 4, first break)."""
    A = np.zeros((4, 3))
    A[0, 0], A[1, 1] = 1.0, 2.0
    hp = O.hessenberg_rect_pivoted(A, np.ones(4), None, 5)
    assert hp["status"] == O.BREAKDOWN_W and hp["k"] == 2
    assert hp["gp"].tolist() == [1, 0] and hp["tp"].tolist() == [0, 1, 2]
    assert np.array_equal(hp["L"][:, 0], [0.5, 1.0, 0.0])
    assert np.array_equal(hp["L"][:, 1], [1.0, 0.0, 0.0])
    assert np.array_equal(hp["D"][:, 2], [0.0, 0.0, 1.0, 1.0])
    assert hp["beta"] == 1.0 and hp["W"][0, 0] == 2.0 and hp["H"][0, 0] == 0.5


def test_breakdown_h_exact():
    """A = I, b = (1, 1/2): u = A l1 equals d1, so eliminating d1 leaves u = 0
    and the H step breaks down in the first iteration; no iterate is formed and
    x = x0 is returned (Algorithm 5, second break; reading R3)."""
    r = O.hybrid_lslu(np.eye(2), np.array([1.0, 0.5]), None, 3, "gcv")
    assert r.status == O.BREAKDOWN_H and r.k_done == 0
    assert np.all(r.x == 0.0)


def test_histories_shape_and_final(ct32):
    A = ct32.scipy()
    r = O.hybrid_lslu(A, ct32.b, None, 20, "gcv")
    r_last = O.hybrid_lslu(A, ct32.b, None, 20, "gcv", histories=False)
    assert r.lam_hist.shape == (20,) and r.res_hist.shape == (20,)
    assert np.array_equal(r.x, r_last.x)
    # projected residual of LSLU (lambda = 0) is non-increasing in k: the
    # search spaces are nested and H_{k+1,k} is a leading block of H_{k+2,k+1}
    r0 = O.hybrid_lslu(A, ct32.b, None, 20, "none")
    assert np.all(np.diff(r0.res_hist) <= 1e-12 * r0.res_hist[0])


def test_reconstruction_quality(ct32):
    """Semi-convergence sanity on the 32x32 workload: the GCV iterate is a
    usable reconstruction (relative error well below 1)."""
    r = O.hybrid_lslu(ct32.scipy(), ct32.b, None, 50, "gcv")
    err = np.linalg.norm(r.x - ct32.x_true) / np.linalg.norm(ct32.x_true)
    assert err < 0.3


def test_method_commutes_with_a_renumbering():
    """Max-abs pivoting picks the same entries whatever the numbering of rows
    and columns (Algorithm 4), so Hybrid LSLU on P_r A P_c^T with P_r b gives
    the pivots mapped through the renumbering and x = P_c^T x_hat, up to
    rounding (the renumbered handle of the CUDA path relies on this)."""
    from paper_2409_05239_gb300 import tomo

    P = tomo.make_config("ct32")
    rng = np.random.default_rng(21)
    for ro, co in (tomo.locality_order(P), (rng.permutation(P.m), rng.permutation(P.n))):
        ir, ic = np.argsort(ro), np.argsort(co)
        Ah = P.scipy()[ir][:, ic].tocsr()
        for rule, lam in (("gcv", 0.0), ("fixed", 1e-2)):
            ref = O.hybrid_lslu(P.scipy(), P.b, None, 40, rule, lam)
            alt = O.hybrid_lslu(Ah, P.b[ir], None, 40, rule, lam)
            assert np.array_equal(ic[alt.gp], ref.gp) and np.array_equal(ir[alt.tp], ref.tp)
            assert np.linalg.norm(alt.x[co] - ref.x) <= 1e-12 * np.linalg.norm(ref.x)
            assert np.allclose(alt.H, ref.H, rtol=0, atol=1e-12 * np.abs(ref.H).max())


def test_zero_singular_value_weight_enters_only_as_a_sum():
    """For a rank-deficient block (a zero column) the weight c_i of its zero
    singular value is fixed only up to the null space of H^T: G (Eqs. gcv2,
    wgcv) and the projected residual see it only through c_i^2 + c_{k+1}^2,
    y (Eq. 4) only through sigma_i c_i / (sigma_i^2 + lambda^2), which
    vanishes with sigma_i, and sum c^2 = beta^2 since U is orthogonal.  This
    is why the GPU may place that weight differently (a reading of the
    paper's formulas at a singular H, which the paper does not discuss)."""
    rng = np.random.default_rng(8)
    k = 12
    H = rng.standard_normal((k + 1, k))
    H[:, 5] = 0.0
    beta = 1.7
    sig, c, V = O.projected_svd(H, beta)
    assert abs(np.sum(c ** 2) - beta ** 2) <= 1e-13 * beta ** 2
    z = sig <= (k + 1) * np.finfo(float).eps * sig[0]
    assert z.sum() == 1 and z[-1]
    assert np.linalg.norm(H @ V[:, -1]) <= 1e-13 * sig[0]
    moved = c.copy()
    moved[k] = np.hypot(c[k], c[k - 1])
    moved[k - 1] = 0.0
    for lam in [0.0] + [f * sig[0] for f in (1e-6, 1e-3, 0.3, 5.0)]:
        if lam > 0.0:
            for omega in (1.0, 0.2):
                assert np.isclose(O.gcv_value(sig, moved, lam, omega),
                                  O.gcv_value(sig, c, lam, omega), rtol=1e-12, atol=0)
        assert np.isclose(O.projected_residual(sig, moved, lam),
                          O.projected_residual(sig, c, lam), rtol=1e-12, atol=0)
        y0 = O.tikhonov_y(sig, c, V, lam)
        term = 0.0 if lam == 0.0 else sig[-1] * abs(c[k - 1]) / (sig[-1] ** 2 + lam ** 2)
        dy = np.linalg.norm(O.tikhonov_y(sig, moved, V, lam) - y0)
        assert dy <= term * (1 + 1e-9) + 1e-12 * np.linalg.norm(y0)
