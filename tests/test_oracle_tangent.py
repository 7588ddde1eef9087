"""Pins of the tangent oracle (forward-mode derivative of Hybrid LSLU with
fixed pivots) against what the mathematics fixes:

* its primal part equals the pinned oracle (same pivots, same x_K);
* central finite differences of x_K(b, lambda) with the pivots held fixed;
* Euler's identity: x_K is 1-homogeneous in b (d_1 = b / beta does not depend
  on the scale of b, y scales with beta), so dx along db = b is x itself;
* a consistent full-basis problem, A (n+1) x n of full rank, b = A x*, K = n,
  lambda = 0: x_K = x* and dx = dx* along db = A dx*;
* planted mistakes in a copy of the module fail at least one pin.
"""
import inspect
import sys
import types

import numpy as np
import pytest

import oracle.lslu_oracle as O
import oracle.lslu_tangent as T
from paper_2409_05239_gb300 import tomo
from tests import pins


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


def primal_pivots(A, b, K):
    hp = O.hessenberg_rect_pivoted(A, b, None, K)
    assert hp["status"] == O.OK
    return hp["gp"], hp["tp"]


def check_primal(Tm, A, b, K, lam):
    ref = O.hybrid_lslu(A, b, None, K, "fixed", lam, histories=False)
    x, _, _ = Tm.hybrid_lslu_tangent(A, b, np.zeros_like(b), lam, 0.0, K, ref.gp, ref.tp)
    assert rel(x, ref.x) <= 1e-9


def check_fd(Tm, A, b, K, lam, seed):
    gp, tp = primal_pivots(A, b, K)
    rng = np.random.default_rng(seed)
    db = rng.standard_normal(b.shape[0]) * np.linalg.norm(b) / np.sqrt(b.shape[0])
    dlam = 0.7 * lam
    _, dx, _ = Tm.hybrid_lslu_tangent(A, b, db, lam, dlam, K, gp, tp)
    h = 1e-6
    xp, _, _ = Tm.hybrid_lslu_tangent(A, b + h * db, db, lam + h * dlam, 0.0, K, gp, tp)
    xm, _, _ = Tm.hybrid_lslu_tangent(A, b - h * db, db, lam - h * dlam, 0.0, K, gp, tp)
    fd = (xp - xm) / (2 * h)
    assert rel(dx, fd) <= 1e-6, rel(dx, fd)


def check_euler(Tm, A, b, K, lam):
    gp, tp = primal_pivots(A, b, K)
    x, dx, _ = Tm.hybrid_lslu_tangent(A, b, b, lam, 0.0, K, gp, tp)
    assert rel(dx, x) <= 1e-10


def check_consistent_full_basis(Tm, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n + 1, n))
    xs = rng.standard_normal(n)
    dxs = rng.standard_normal(n)
    b = A @ xs
    gp, tp = primal_pivots(A, b, n)
    x, dx, _ = Tm.hybrid_lslu_tangent(A, b, A @ dxs, 0.0, 0.0, n, gp, tp)
    assert rel(x, xs) <= 1e-8
    assert rel(dx, dxs) <= 1e-7


def test_primal_matches_oracle(ct32):
    check_primal(T, ct32.scipy(), ct32.b, 20, 1e-2)


@pytest.mark.parametrize("lam", [1e-2, 0.3])
def test_tangent_vs_central_differences(ct32, lam):
    check_fd(T, ct32.scipy(), ct32.b, 15, lam, seed=3)


def test_tangent_dense_problem_fd():
    A, _, b = pins.random_problem(40, 25, seed=9, decay=0.8)
    check_fd(T, A, b, 12, 0.05, seed=4)


def test_euler_homogeneity(ct32):
    check_euler(T, ct32.scipy(), ct32.b, 20, 1e-2)


@pytest.mark.parametrize("n,seed", [(6, 1), (12, 2)])
def test_consistent_full_basis(n, seed):
    check_consistent_full_basis(T, n, seed)


def test_loss_directional_derivative(ct32):
    A = ct32.scipy()
    gp, tp = primal_pivots(A, ct32.b, 15)
    rng = np.random.default_rng(11)
    db = rng.standard_normal(ct32.m)
    lam = 1e-2
    J, dJ = T.loss_and_directional(A, ct32.b, lam, 15, gp, tp, ct32.x_true, db, 0.4)
    h = 1e-6
    Jp, _ = T.loss_and_directional(A, ct32.b + h * db, lam * np.exp(0.4 * h), 15, gp, tp,
                                   ct32.x_true, db, 0.0)
    Jm, _ = T.loss_and_directional(A, ct32.b - h * db, lam * np.exp(-0.4 * h), 15, gp, tp,
                                   ct32.x_true, db, 0.0)
    assert abs(dJ - (Jp - Jm) / (2 * h)) <= 1e-6 * abs(dJ)


MUTATIONS = {
    "dropped_basis_tangent": ("dq = dq - dW[j, k] * L[:, j] - W[j, k] * dL[:, j]",
                              "dq = dq - dW[j, k] * L[:, j]"),
    "wrong_quotient_sign": ("dL[:, k] = (dq - L[:, k] * dW[k, k]) / W[k, k]",
                            "dL[:, k] = (dq + L[:, k] * dW[k, k]) / W[k, k]"),
    "h_tangent_row": ("dH[j, k] = du[tp[j]]", "dH[j, k] = du[tp[0]]"),
    "beta_tangent_dropped": ("dD[:, 0] = (dr0 - D[:, 0] * dbeta) / beta", "dD[:, 0] = dr0 / beta"),
    "lambda_term_sign": ("- 2.0 * lam * dlam * y", "+ 2.0 * lam * dlam * y"),
    "transposed_dH": ("rhs = dH.T @ (beta * e1 - H @ y)", "rhs = dH[:K, :].T @ (beta * e1[:K] - H[:K, :] @ y)"),
    "dy_dropped": ("dx = dL @ y + L @ dy", "dx = dL @ y"),
}


def mutated(name):
    src = inspect.getsource(T)
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mod = types.ModuleType(f"tangent_mutant_{name}")
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(src.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_tangent_mistake_is_caught(ct32, name):
    Tm = mutated(name)
    A = ct32.scipy()
    failed = []
    for label, fn in (("primal", lambda: check_primal(Tm, A, ct32.b, 12, 1e-2)),
                      ("fd", lambda: check_fd(Tm, A, ct32.b, 12, 1e-2, seed=3)),
                      ("euler", lambda: check_euler(Tm, A, ct32.b, 12, 1e-2)),
                      ("full_basis", lambda: check_consistent_full_basis(Tm, 6, 1))):
        try:
            fn()
        except (AssertionError, np.linalg.LinAlgError, ValueError, IndexError):
            failed.append(label)
    assert failed, f"mutation {name} passed every pin"
