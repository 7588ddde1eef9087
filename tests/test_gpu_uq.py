"""Low-rank uncertainty quantification (Section 4.2) on the GPU (lslu_uq)
against the oracle's eigendecomposition/Woodbury form on the same basis."""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import lslu, tomo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_05239_gb300 import build

    build.build()


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


def noise_var(P):
    return (P.eta * np.linalg.norm(P.b_clean)) ** 2 / P.m


@pytest.mark.parametrize("K,lam", [(10, 0.05), (25, 0.3)])
def test_uq_f64_vs_oracle(ct32, K, lam):
    s2 = noise_var(ct32)
    hp = O.hessenberg_rect_pivoted(ct32.scipy(), ct32.b, None, K)
    d_ref, t_ref = O.uq_lowrank(hp["L"], hp["D"], hp["W"], lam, s2)
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve(ct32.b, K, "gcv")
        assert np.array_equal(r["gp"], hp["gp"])
        u = s.uq(s2, lam)
    assert np.allclose(u["var_diag"], d_ref, rtol=1e-8, atol=0)
    assert abs(u["var_sum"] - t_ref) <= 1e-8 * abs(t_ref)


def test_uq_f32_vs_oracle(ct32):
    K, lam = 15, 0.05
    s2 = noise_var(ct32)
    A = ct32.scipy(tomo.round_values(ct32.vals, "f32"))
    hp = O.hessenberg_rect_pivoted(A, ct32.b, None, K)
    d_ref, t_ref = O.uq_lowrank(hp["L"], hp["D"], hp["W"], lam, s2)
    with lslu.from_problem(ct32, "f32", K) as s:
        r = s.solve(ct32.b, K, "gcv")
        assert np.array_equal(r["gp"], hp["gp"])
        u = s.uq(s2, lam)
    assert np.max(np.abs(u["var_diag"] - d_ref)) <= 1e-4 * np.max(d_ref)
    assert abs(u["var_sum"] - t_ref) <= 1e-4 * abs(t_ref)


def test_uq_large_properties():
    P = tomo.make_config("ct256")
    K, lam = 50, 1.0
    s2 = noise_var(P)
    with lslu.from_problem(P, "f32", K) as s:
        s.solve(P.b, K, "gcv")
        u = s.uq(s2, lam)
    d = u["var_diag"]
    prior = s2 / lam ** 2
    assert np.all(d > 0) and np.all(d <= prior * (1 + 1e-5))
    assert np.min(d) < 0.999 * prior  # the data reduce some variances
    assert u["var_sum"] > 0


def test_uq_argument_checks(ct32):
    with lslu.from_problem(ct32, "f64", 5) as s:
        with pytest.raises(lslu.LsluError):  # no solve yet
            s.uq(1.0, 0.1)
        s.solve(ct32.b, 5, "gcv")
        with pytest.raises(lslu.LsluError):
            s.uq(1.0, 0.0)


def test_uq_refuses_k_beyond_the_cluster_factor(ct32):
    """The k x k Cholesky factor runs on one cluster that holds its columns in
    shared memory; at k = 660 it does not fit, and (as the oracle shows on
    this problem: cond(W) ~ 1e18) W_k is numerically singular there anyway.
    lslu_uq refuses instead of computing a meaningless covariance."""
    K = 660
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve(ct32.b, K, "gcv")
        assert r["k_done"] == K
        with pytest.raises(lslu.LsluError, match="cluster Cholesky"):
            s.uq(noise_var(ct32), 0.05)
