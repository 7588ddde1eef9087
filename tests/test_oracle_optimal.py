"""Pins of the optimal-lambda rule (needs x_true): the chosen lambda
minimises ||L_k y(lambda) - x_true|| against a dense 20001-point log grid
and scipy's bounded scalar minimiser, on a dense problem and on the 32x32
tomography workload."""
import math

import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import tomo
from tests import pins


def err(L, s, c, V, x, lam):
    r = L @ O.tikhonov_y(s, c, V, lam) - x
    return float(r @ r)


def check(A, b, x_true, K):
    hp = O.hessenberg_rect_pivoted(A, b, None, K)
    s, c, V = O.projected_svd(hp["H"], hp["beta"])
    lam = O.optimal_lambda(hp["L"], s, c, V, x_true)
    e = err(hp["L"], s, c, V, x_true, lam)
    fine = s[0] * 10.0 ** np.linspace(-14.0, 2.0, 20001)
    e_fine = min(err(hp["L"], s, c, V, x_true, l) for l in fine)
    assert e <= e_fine * (1 + 1e-10)
    from scipy.optimize import minimize_scalar
    r = minimize_scalar(lambda t: err(hp["L"], s, c, V, x_true, math.exp(t)),
                        bounds=(math.log(lam) - 1.0, math.log(lam) + 1.0), method="bounded",
                        options={"xatol": 1e-10})
    assert e <= r.fun * (1 + 1e-9)
    return lam, e


def test_optimal_lambda_dense():
    A, x, b = pins.random_problem(40, 30, seed=41, decay=0.8)
    check(A, b, x, 12)


def test_optimal_lambda_tomography():
    P = tomo.make_config("ct32")
    lam, e = check(P.scipy(), P.b, P.x_true, 20)
    x, lam2, e2 = O.hybrid_lslu_optimal(P.scipy(), P.b, 20, P.x_true)
    assert lam2 == lam and abs(e2 - e) <= 1e-12 * e
    # no worse than the GCV choice at the same iteration
    g = O.hybrid_lslu(P.scipy(), P.b, None, 20, "gcv", histories=False)
    assert e2 <= float(np.sum((g.x - P.x_true) ** 2))
