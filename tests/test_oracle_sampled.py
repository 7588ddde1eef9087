"""Pins of the sampled-pivot variant (Section 2.2) in the oracle.

* every index sampled reduces it to the standard max-abs pivoting;
* with random samples the basis keeps the invariants of Algorithm 4 (unit
  pivot, zeros at earlier pivots) and the relations (nhr), (nhr2), and every
  new vector is bounded by 1 in magnitude on its own sample with the bound
  attained at its pivot (the pivot is the sample's largest entry);
* the reconstruction error stays comparable to full pivoting.
"""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import tomo
from tests import pins


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


def table(K, s, m, n, seed):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, m if t % 2 == 0 else n, size=s) for t in range(2 * K + 1)]


def test_full_sample_is_standard_pivoting(ct32):
    K = 20
    full = [np.arange(ct32.m if t % 2 == 0 else ct32.n) for t in range(2 * K + 1)]
    a = O.hessenberg_rect_pivoted(ct32.scipy(), ct32.b, None, K)
    b = O.hessenberg_rect_pivoted(ct32.scipy(), ct32.b, None, K, full)
    assert np.array_equal(a["gp"], b["gp"]) and np.array_equal(a["tp"], b["tp"])
    assert np.array_equal(a["L"], b["L"])


@pytest.mark.parametrize("s", [25, 100])
def test_sampled_basis_invariants(ct32, s):
    K = 20
    S = table(K, s, ct32.m, ct32.n, seed=s)
    A = ct32.scipy()
    hp = O.hessenberg_rect_pivoted(A, ct32.b, None, K, S)
    assert hp["status"] == O.OK
    pins.check_unit_pivot_structure(hp, max_abs_one=False)
    pins.check_hessenberg_relations(A, hp)
    for k in range(K):
        lk = hp["L"][:, k]
        smp = [j for j in S[2 * k + 1] if j not in set(hp["gp"][:k].tolist())]
        assert np.max(np.abs(lk[smp])) == 1.0 and hp["gp"][k] in smp
        dk = hp["D"][:, k + 1]
        smp = [j for j in S[2 * k + 2] if j not in set(hp["tp"][:k + 1].tolist())]
        assert np.max(np.abs(dk[smp])) == 1.0 and hp["tp"][k + 1] in smp
    # the full max-abs exceeds 1 somewhere: the sample really restricts the search
    assert np.max(np.abs(hp["L"])) > 1.0


def test_sampled_reconstruction_comparable(ct32):
    K = 40
    A = ct32.scipy()
    full = O.hybrid_lslu(A, ct32.b, None, K, "wgcv", histories=False)
    smp = O.hybrid_lslu(A, ct32.b, None, K, "wgcv", histories=False,
                        samples=table(K, 50, ct32.m, ct32.n, seed=3))
    e_full = np.linalg.norm(full.x - ct32.x_true) / np.linalg.norm(ct32.x_true)
    e_smp = np.linalg.norm(smp.x - ct32.x_true) / np.linalg.norm(ct32.x_true)
    assert e_smp < 2.0 * e_full
