"""Stopping criterion G^(k) on the GPU (lslu_solve_stopping) against the
oracle (Eqs. stop2, tol).  The graph loop mode stops online: the basis runs
in chunks of 8 iterations and G^(k) is returned for the iterations evaluated
(at least through k_stop + 1), zero past them."""
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


CHUNK = 8


def evaluated(G):
    """Number of leading entries of a returned G history that were evaluated."""
    nz = np.flatnonzero(G)
    return 0 if nz.size == 0 else int(nz[-1]) + 1


def check_online_history(G, G_ref, k_stop, K):
    """The evaluated prefix equals the oracle's; it covers k_stop + 1 (or K)
    and ends on a chunk boundary or at K; zeros after it."""
    ne = evaluated(G)
    assert ne >= min(k_stop + 1, K)
    assert ne == K or ne % CHUNK == 0
    assert np.allclose(G[:ne], G_ref[:ne], rtol=1e-8, atol=0)
    assert np.all(G[ne:] == 0.0)


def margin_ok(G, k, tol, rel=1e-6):
    """True when no step before k (nor at k) sits within rel of the threshold,
    so two correct FP64 implementations must stop at the same k."""
    d = np.abs(np.diff(G)) / abs(G[0])
    return all(abs(v - tol) > rel * tol for v in d[:k])


@pytest.mark.parametrize("rule,lam", [("wgcv", 0.0), ("gcv", 0.0), ("fixed", 1e-2)])
@pytest.mark.parametrize("tol", [1e-6, 1e-4])
def test_stopping_f64_vs_oracle(ct32, rule, lam, tol):
    K = 50
    x_ref, k_ref, G_ref = O.hybrid_lslu_stopping(ct32.scipy(), ct32.b, K, rule, lam, tol)
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve_stopping(ct32.b, K, rule, lam, tol)
        if margin_ok(G_ref, k_ref, tol):
            assert r["k_stop"] == k_ref
        check_online_history(r["G"], G_ref, r["k_stop"], K)
        ref_k = s.solve(ct32.b, r["k_stop"], rule, lam)
    # x at the stopping iteration equals the plain solve with K = k_stop
    assert np.array_equal(r["x"], ref_k["x"])
    if r["k_stop"] == k_ref:
        assert np.linalg.norm(r["x"] - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_stopping_mixed_and_large():
    P = tomo.make_config("ct256")
    with lslu.from_problem(P, "f32", 150) as s:
        r = s.solve_stopping(P.b, 150, "wgcv", 0.0, 1e-6)
        k = r["k_stop"]
        assert 1 <= k <= 150
        assert np.all(r["G"][:k] > 0)
        ref = s.solve(P.b, k, "wgcv")
    assert np.array_equal(r["x"], ref["x"])


def test_stopping_argument_checks(ct32):
    with lslu.from_problem(ct32, "f64", 10) as s:
        with pytest.raises(lslu.LsluError):
            s.solve_stopping(ct32.b, 1, "gcv")
        with pytest.raises(lslu.LsluError):
            s.solve_stopping(ct32.b, 10, "gcv", tol=0.0)


@pytest.mark.parametrize("tol", [1e-6, 1e-3])
def test_online_stop_equals_the_full_run(ct32, tol):
    """The online stop (graph loop mode) against the run to K_max (a persistent
    loop handle takes that path: every projected problem, then the
    selection): the same stopping k, G^(k) on the evaluated prefix and x."""
    K = 50
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve_stopping(ct32.b, K, "gcv", 0.0, tol)
    with lslu.from_problem(ct32, "f64", K) as s:
        s.set_loop("persistent")
        full = s.solve_stopping(ct32.b, K, "gcv", 0.0, tol)
    assert evaluated(full["G"]) == K
    if margin_ok(full["G"], full["k_stop"], tol):
        assert r["k_stop"] == full["k_stop"]
    ne = evaluated(r["G"])
    assert np.allclose(r["G"][:ne], full["G"][:ne], rtol=1e-10, atol=0)
    if r["k_stop"] == full["k_stop"]:
        assert np.linalg.norm(r["x"] - full["x"]) <= 1e-10 * np.linalg.norm(full["x"])


def test_online_stop_runs_to_k_max_when_the_criterion_never_holds(ct32):
    K = 20
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve_stopping(ct32.b, K, "gcv", 0.0, 1e-300)
        ref = s.solve(ct32.b, K, "gcv")
    assert r["k_stop"] == K and evaluated(r["G"]) == K
    assert np.array_equal(r["x"], ref["x"])


def test_online_stop_at_a_breakdown_in_a_later_chunk():
    """A = diag(1..12), b generic: the process breaks down at k_done = 11, in
    the second chunk; with a criterion that never holds the run stops there,
    G^(k) for k <= 11 against the oracle and zero after."""
    n, K = 12, 16
    A = np.diag(np.arange(1.0, n + 1))
    b = np.linspace(1.0, 2.0, n)
    x_ref, k_ref, G_ref = O.hybrid_lslu_stopping(A, b, K, "gcv", 0.0, 1e-300)
    assert k_ref == 11
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    with lslu.Solver(n, n, rp, ci, np.arange(1.0, n + 1), "f64", K) as s:
        r = s.solve_stopping(b, K, "gcv", 0.0, 1e-300)
    assert r["k_stop"] == k_ref
    assert np.allclose(r["G"][:k_ref], G_ref[:k_ref], rtol=1e-8, atol=0)
    assert np.all(r["G"][k_ref:] == 0.0)
    assert np.linalg.norm(r["x"] - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_online_stop_with_x0(ct32):
    K = 30
    x0 = 0.1 * np.sin(np.arange(ct32.n))
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve_stopping(ct32.b, K, "gcv", 0.0, 1e-4, x0=x0)
        ref = s.solve(ct32.b, r["k_stop"], "gcv", x0=x0)
    assert 1 <= r["k_stop"] <= K
    assert np.array_equal(r["x"], ref["x"])
