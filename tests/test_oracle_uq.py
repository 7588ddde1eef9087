"""Pins of the low-rank uncertainty quantification (Section 4.2) in the oracle.

The oracle follows the paper's steps (G^T G, its eigendecomposition, Z, the
Woodbury form).  The pins form the same covariance densely from its
definition: Gamma_k = sigma^2 (lam^2 I + A^T D_k D_k^+ A)^-1 with a dense
pseudo-inverse of D_k, its diagonal and the sum of all its entries."""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import tomo
from tests import pins


def dense_gamma(A, D, k, lam, sigma2):
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    Dk = D[:, :k]
    M = Ad.T @ Dk @ np.linalg.pinv(Dk) @ Ad
    return sigma2 * np.linalg.inv(lam * lam * np.eye(Ad.shape[1]) + M)


@pytest.mark.parametrize("K,lam", [(4, 0.05), (8, 0.3), (12, 0.02)])
def test_uq_against_dense_definition(K, lam):
    A, _, b = pins.random_problem(30, 18, seed=31, decay=0.8)
    hp = O.hessenberg_rect_pivoted(A, b, None, K)
    diag, total = O.uq_lowrank(hp["L"], hp["D"], hp["W"], lam, 0.7)
    G = dense_gamma(A, hp["D"], K, lam, 0.7)
    assert np.allclose(diag, np.diag(G), rtol=1e-8, atol=0)
    assert abs(total - G.sum()) <= 1e-8 * abs(G.sum())


def test_uq_on_tomography():
    P = tomo.make_config("ct32")
    A = P.scipy()
    hp = O.hessenberg_rect_pivoted(A, P.b, None, 15)
    lam, s2 = 0.05, (0.01 * np.linalg.norm(P.b_clean)) ** 2 / P.m
    diag, total = O.uq_lowrank(hp["L"], hp["D"], hp["W"], lam, s2)
    G = dense_gamma(A, hp["D"], 15, lam, s2)
    assert np.allclose(diag, np.diag(G), rtol=1e-7, atol=0)
    assert abs(total - G.sum()) <= 1e-7 * abs(G.sum())
    # a variance never exceeds the prior's sigma^2 / lam^2
    assert np.all(diag <= s2 / lam ** 2 * (1 + 1e-12)) and np.all(diag > 0)
