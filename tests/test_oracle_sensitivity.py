"""How far two correct FP64 evaluations of Algorithm 4 drift apart: the oracle
against itself with a permuted (equally valid) summation order.  This fixes
what parity against the oracle can demand of any other implementation."""
import numpy as np

import oracle.lslu_oracle as O
from oracle.perturb import PermutedOperator, first_difference
from paper_2409_05239_gb300 import tomo


def test_ct32_insensitive_to_summation_order():
    P = tomo.make_config("ct32")
    A = P.scipy()
    r1 = O.hybrid_lslu(A, P.b, None, 50, "gcv")
    r2 = O.hybrid_lslu(PermutedOperator(A), P.b, None, 50, "gcv")
    assert np.array_equal(r1.gp, r2.gp) and np.array_equal(r1.tp, r2.tp)
    assert np.linalg.norm(r1.x - r2.x) <= 1e-12 * np.linalg.norm(r1.x)


def test_permuted_operator_is_the_same_matrix():
    P = tomo.make_config("ct32")
    A = P.scipy()
    Ap = PermutedOperator(A)
    v = np.random.default_rng(0).standard_normal(P.n)
    u = np.random.default_rng(1).standard_normal(P.m)
    assert np.allclose(Ap @ v, A @ v, rtol=1e-13, atol=1e-12)
    assert np.allclose(Ap.T @ u, A.T @ u, rtol=1e-13, atol=1e-12)
    assert first_difference([1, 2, 3], [1, 2, 4]) == 2
