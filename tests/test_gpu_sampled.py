"""Sampled pivoting (Section 2.2) on the GPU against the oracle with the same
sample table."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("s", [25, 50, 100])
@pytest.mark.parametrize("rule,lam", [("gcv", 0.0), ("fixed", 1e-2)])
def test_sampled_f64_parity(ct32, s, rule, lam):
    K = 40
    S = lslu.sample_table(K, s, ct32.m, ct32.n, seed=s)
    ref = O.hybrid_lslu(ct32.scipy(), ct32.b, None, K, rule, lam, histories=False,
                        samples=list(S))
    with lslu.from_problem(ct32, "f64", K) as h:
        r = h.solve_sampled(ct32.b, K, S, rule, lam)
    assert r["status"] == ref.status and r["k_done"] == ref.k_done
    assert np.array_equal(r["gp"], ref.gp) and np.array_equal(r["tp"], ref.tp)
    assert rel(r["x"], ref.x) <= 1e-10


def test_sampled_mixed(ct32):
    K = 30
    S = lslu.sample_table(K, 50, ct32.m, ct32.n, seed=9)
    A = ct32.scipy(tomo.round_values(ct32.vals, "f32"))
    ref = O.hybrid_lslu(A, ct32.b, None, K, "gcv", histories=False, samples=list(S))
    with lslu.from_problem(ct32, "f32", K) as h:
        r = h.solve_sampled(ct32.b, K, S, "gcv")
        r2 = h.solve_sampled(ct32.b, K, S, "gcv")  # graph replay
    assert np.array_equal(r["gp"][:5], ref.gp[:5]) and np.array_equal(r["tp"][:5], ref.tp[:5])
    assert rel(r["x"], ref.x) <= 2e-4
    assert np.array_equal(r["x"], r2["x"])


def test_full_table_equals_standard_pivoting(ct32):
    """Every row covering its whole index space (the n-space rows repeat
    their indices to the common length m) reduces to the standard search."""
    K = 20
    full_m = np.arange(ct32.m, dtype=np.int32)
    S = np.stack([full_m if t % 2 == 0 else np.resize(np.arange(ct32.n, dtype=np.int32), ct32.m)
                  for t in range(2 * K + 1)])
    with lslu.from_problem(ct32, "f64", K) as h:
        a = h.solve(ct32.b, K, "gcv")
        b = h.solve_sampled(ct32.b, K, S, "gcv")
    assert np.array_equal(a["gp"], b["gp"]) and np.array_equal(a["tp"], b["tp"])
    assert np.array_equal(a["x"], b["x"])


def test_sampled_table_validation(ct32):
    K = 5
    S = lslu.sample_table(K, 10, ct32.m, ct32.n, seed=1)
    S[1, 0] = ct32.n  # odd row indexes [0, n)
    with lslu.from_problem(ct32, "f64", K) as h:
        with pytest.raises(lslu.LsluError):
            h.solve_sampled(ct32.b, K, S, "gcv")
