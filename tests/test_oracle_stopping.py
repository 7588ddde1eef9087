"""Pins of the stopping criterion G^(k) (Eq. stop2) and its rule (Eq. tol).

* numerator: n ||D_{k+1}^+ (b - A x_k)||^2 with a dense pseudo-inverse of the
  D basis (the quantity the paper approximates the GCV numerator by);
* denominator: (trace(I_m - A A_k^+))^2 with A_k^+ = L_k H_lambda^+ D_{k+1}^+
  formed densely;
* the rule on hand-made sequences, and the returned iterate equals the
  oracle's x_k at the stopping iteration.
"""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from tests import pins


def dense_G(A, b, K, lam):
    m, n = A.shape
    hp = O.hessenberg_rect_pivoted(A, b, None, K)
    L, D, H = hp["L"], hp["D"], hp["H"]
    Dp = np.linalg.pinv(D)
    Hl = np.linalg.solve(H.T @ H + lam * lam * np.eye(K), H.T)  # H_lambda^+
    Ak = L @ Hl @ Dp                                              # A_k^+
    xk = Ak @ b
    num = n * np.sum((Dp @ (b - A @ xk)) ** 2)
    den = np.trace(np.eye(m) - A @ Ak)
    return num / den ** 2, hp


@pytest.mark.parametrize("K,lam", [(3, 0.05), (6, 0.2), (10, 0.01)])
def test_stopping_value_against_dense_definition(K, lam):
    A, _, b = pins.random_problem(40, 25, seed=21, decay=0.8)
    G_dense, hp = dense_G(A, b, K, lam)
    s, c, _ = O.projected_svd(hp["H"], hp["beta"])
    G = O.stopping_gcv_value(s, c, lam, A.shape[1], A.shape[0])
    assert abs(G - G_dense) <= 1e-9 * abs(G_dense)


def test_stopping_rule_on_sequences():
    assert O.stopping_iteration(np.array([1.0, 0.5, 0.4, 0.3999995, 0.3]), 1e-5) == 3
    assert O.stopping_iteration(np.array([2.0, 1.0, 0.5]), 1e-6) == 3  # never passes
    assert O.stopping_iteration(np.array([1.0, 1.0]), 1e-6) == 1
    # relative to G(1): the same step passes or fails with the scale of G(1)
    assert O.stopping_iteration(np.array([100.0, 99.99999, 50.0]), 1e-6) == 1
    assert O.stopping_iteration(np.array([1.0, 0.9999, 0.5]), 1e-6) == 3


def test_stopping_solve_returns_x_at_k():
    A, _, b = pins.random_problem(60, 40, seed=22, decay=0.75)
    x, k, G = O.hybrid_lslu_stopping(A, b, 20, "gcv", tol=1e-3)
    assert 1 <= k <= 20 and G.shape == (20,)
    ref = O.hybrid_lslu(A, b, None, k, "gcv", histories=False)
    assert np.allclose(x, ref.x, rtol=1e-12, atol=0)
