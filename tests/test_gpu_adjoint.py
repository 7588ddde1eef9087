"""Reverse-mode derivative of Hybrid LSLU (lslu_adjoint), pivots held fixed.

Checked through the C ABI against:
* the FP64 tangent oracle (forward mode, an independent derivation): the
  directional derivative of J = ||x_K - x_true||^2 along random directions,
  along unit vectors at pivot rows (where the pivot-row terms act) and along
  x0 and log(lambda);
* Euler's identity bbar . b = xbar . x (x_K is 1-homogeneous in b);
* central differences of the GPU's own solve with the pivots replayed
  (lslu_solve_fixed_pivots);
* the torch.autograd wrapper against the direct call.
"""
import numpy as np
import pytest

import oracle.lslu_oracle as O
import oracle.lslu_tangent as T
from paper_2409_05239_gb300 import lslu, tomo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_05239_gb300 import build

    build.build()


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


def directions(P, gp, tp, seed):
    rng = np.random.default_rng(seed)
    out = [rng.standard_normal(P.m) for _ in range(2)]
    for i in (0, 1, len(tp) // 2, len(tp) - 1):  # pivot rows of the D side
        e = np.zeros(P.m)
        e[tp[i]] = 1.0
        out.append(e)
    e = np.zeros(P.m)
    e[int(rng.integers(P.m))] = 1.0
    out.append(e)
    return out


def gpu_run(P, vt, K, lam, rule="fixed"):
    with lslu.from_problem(P, vt, K) as s:
        r = s.solve(P.b, K, rule, lam)
        assert r["status"] == lslu.OK
        xbar = 2.0 * (r["x"] - P.x_true)
        adj = s.adjoint(xbar, want_x0=True)
    return r, xbar, adj


@pytest.mark.parametrize("K,lam", [(15, 1e-2), (30, 0.3)])
def test_f64_adjoint_vs_tangent_oracle(ct32, K, lam):
    r, xbar, adj = gpu_run(ct32, "f64", K, lam)
    A = ct32.scipy()
    ref = O.hybrid_lslu(A, ct32.b, None, K, "fixed", lam, histories=False)
    assert np.array_equal(r["gp"], ref.gp) and np.array_equal(r["tp"], ref.tp)
    bb, lb = adj["b_bar"], adj["lambda_bar"]
    for j, db in enumerate(directions(ct32, r["gp"], r["tp"], seed=K)):
        dl = 0.3 if j == 0 else 0.0
        _, dJ = T.loss_and_directional(A, ct32.b, lam, K, r["gp"], r["tp"], ct32.x_true, db, dl)
        g = bb @ db + lb * lam * dl
        scale = np.linalg.norm(bb) * np.linalg.norm(db) + abs(lb * lam * dl)
        assert abs(g - dJ) <= 1e-9 * scale, (j, g, dJ)
    # x0 direction: x = x0 + L y, r0 = b - A x0
    rng = np.random.default_rng(5)
    dx0 = rng.standard_normal(ct32.n)
    x, dx, _ = T.hybrid_lslu_tangent(A, ct32.b, np.zeros(ct32.m), lam, 0.0, K, r["gp"], r["tp"],
                                     x0=np.zeros(ct32.n), dx0=dx0)
    dJ = 2.0 * (x - ct32.x_true) @ dx
    g = adj["x0_bar"] @ dx0
    assert abs(g - dJ) <= 1e-9 * np.linalg.norm(adj["x0_bar"]) * np.linalg.norm(dx0)


def test_euler_identity(ct32):
    r, xbar, adj = gpu_run(ct32, "f64", 20, 1e-2)
    lhs = adj["b_bar"] @ ct32.b
    rhs = xbar @ r["x"]
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_f64_central_differences_fixed_pivots(ct32):
    K, lam = 20, 1e-2
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve(ct32.b, K, "fixed", lam)
        xbar = 2.0 * (r["x"] - ct32.x_true)
        adj = s.adjoint(xbar)
        rng = np.random.default_rng(7)
        db = rng.standard_normal(ct32.m)
        h = 1e-6 * np.linalg.norm(ct32.b) / np.linalg.norm(db)

        def J(b, lm):
            o = s.solve_fixed_pivots(b, K, r["gp"], r["tp"], "fixed", lm)
            assert o["status"] == lslu.OK
            return float(np.sum((o["x"] - ct32.x_true) ** 2))

        fd_b = (J(ct32.b + h * db, lam) - J(ct32.b - h * db, lam)) / (2 * h)
        e = 1e-4  # smaller steps lose more to cancellation in J than they gain
        fd_l = (J(ct32.b, lam * np.exp(e)) - J(ct32.b, lam * np.exp(-e))) / (2 * e)
    assert abs(adj["b_bar"] @ db - fd_b) <= 1e-6 * abs(fd_b)
    assert abs(adj["lambda_bar"] * lam - fd_l) <= 1e-6 * abs(fd_l)


def test_fixed_pivot_replay_reproduces_solve(ct32):
    with lslu.from_problem(ct32, "f32", 25) as s:
        r = s.solve(ct32.b, 25, "fixed", 1e-2)
        o = s.solve_fixed_pivots(ct32.b, 25, r["gp"], r["tp"], "fixed", 1e-2)
        assert np.array_equal(o["x"], r["x"])
        with pytest.raises(lslu.LsluError):  # repeated pivot row
            g = r["gp"].copy()
            g[3] = g[2]
            s.solve_fixed_pivots(ct32.b, 25, g, r["tp"], "fixed", 1e-2)


@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_mixed_adjoint_vs_f64_oracle(ct32, vt):
    """FP32 basis and adjoint vectors against the FP64 tangent oracle on the
    same rounded matrix values and pivots."""
    K, lam = 15, 1e-2
    r, xbar, adj = gpu_run(ct32, vt, K, lam)
    A = ct32.scipy(tomo.round_values(ct32.vals, vt))
    bb, lb = adj["b_bar"], adj["lambda_bar"]
    for j, db in enumerate(directions(ct32, r["gp"], r["tp"], seed=3)):
        dl = 0.3 if j == 0 else 0.0
        _, dJ = T.loss_and_directional(A, ct32.b, lam, K, r["gp"], r["tp"], ct32.x_true, db, dl)
        g = bb @ db + lb * lam * dl
        scale = np.linalg.norm(bb) * np.linalg.norm(db) + abs(lb * lam * dl)
        assert abs(g - dJ) <= 2e-4 * scale, (j, g, dJ)


def test_torch_autograd_matches_adjoint(ct32):
    import torch

    dev = torch.device("cuda", 0)
    K, lam = 15, 2e-2
    with lslu.from_problem(ct32, "f32", K) as s:
        b = torch.tensor(ct32.b, device=dev, requires_grad=True)
        ll = torch.tensor(np.log(lam), dtype=torch.float64, device=dev, requires_grad=True)
        xt = torch.tensor(ct32.x_true, device=dev)
        x = lslu.hybrid_lslu(s, b, ll, K)
        loss = ((x - xt) ** 2).sum()
        loss.backward()
        ref = s.solve(ct32.b, K, "fixed", lam)
        adj = s.adjoint(2.0 * (ref["x"] - ct32.x_true))
    assert np.array_equal(x.detach().cpu().numpy(), ref["x"])
    assert np.allclose(b.grad.cpu().numpy(), adj["b_bar"], rtol=0, atol=1e-12 * np.abs(adj["b_bar"]).max())
    assert abs(ll.grad.item() - adj["lambda_bar"] * lam) <= 1e-12 * abs(adj["lambda_bar"] * lam)


def test_backward_after_another_solve_is_refused(ct32):
    import torch

    dev = torch.device("cuda", 0)
    with lslu.from_problem(ct32, "f32", 10) as s:
        b = torch.tensor(ct32.b, device=dev, requires_grad=True)
        ll = torch.tensor(-3.0, dtype=torch.float64, device=dev, requires_grad=True)
        x = lslu.hybrid_lslu(s, b, ll, 10)
        s.solve(ct32.b, 10, "gcv")
        with pytest.raises(RuntimeError):
            x.sum().backward()


def test_adjoint_state_checks(ct32):
    with lslu.from_problem(ct32, "f64", 10) as s:
        with pytest.raises(lslu.LsluError):  # no solve yet
            s.adjoint(np.ones(ct32.n))
        r = s.solve(ct32.b, 10, "fixed", 1e-2)
        s.projected(np.triu(np.ones((6, 5)), -1), 1.0)  # reuses the projected work space
        with pytest.raises(lslu.LsluError):
            s.adjoint(np.ones(ct32.n))
        s.solve(np.zeros(ct32.m), 10, "fixed", 1e-2)  # breakdown
        with pytest.raises(lslu.LsluError):
            s.adjoint(np.ones(ct32.n))
        assert r["status"] == lslu.OK


@pytest.fixture(scope="module")
def ct256():
    return tomo.make_config("ct256")


@pytest.mark.parametrize("vt,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_ct256_adjoint_vs_tangent_oracle(ct256, vt, tol):
    """256x256 workload at K = 10, where x_K(b) with fixed pivots is still
    well conditioned (beyond K ~ 20 the rounding noise of the recurrence
    dominates its b-derivative, in the FP64 oracle as much as on the GPU)."""
    K, lam = 10, 1.8
    r, xbar, adj = gpu_run(ct256, vt, K, lam)
    A = ct256.scipy(tomo.round_values(ct256.vals, vt)) if vt != "f64" else ct256.scipy()
    rng = np.random.default_rng(1)
    db = rng.standard_normal(ct256.m)
    _, dJ = T.loss_and_directional(A, ct256.b, lam, K, r["gp"], r["tp"], ct256.x_true, db, 0.5)
    g = adj["b_bar"] @ db + adj["lambda_bar"] * lam * 0.5
    assert abs(g - dJ) <= tol * abs(dJ), (g, dJ)


def test_ct256_k100_lambda_gradient(ct256):
    """The differentiable-solve workload (256x256, FP32, K = 100): d J / d log
    lambda from the adjoint against central differences of the GPU solve with
    the pivots replayed (step 1e-3 in log lambda).  lambda enters only the
    projected problem, so this derivative stays well conditioned at K = 100."""
    K = 100
    with lslu.from_problem(ct256, "f32", K) as s:
        lam = float(s.solve(ct256.b, K, "gcv", histories=True)["lam_hist"][-1])
        r = s.solve(ct256.b, K, "fixed", lam)
        assert r["status"] == lslu.OK
        adj = s.adjoint(2.0 * (r["x"] - ct256.x_true))

        def J(lm):
            o = s.solve_fixed_pivots(ct256.b, K, r["gp"], r["tp"], "fixed", lm)
            return float(np.sum((o["x"] - ct256.x_true) ** 2))

        e = 1e-3
        fd = (J(lam * np.exp(e)) - J(lam * np.exp(-e))) / (2 * e)
    assert abs(adj["lambda_bar"] * lam - fd) <= 1e-4 * abs(fd)


def test_ct256_b_gradient_conditioning(ct256):
    """With the pivots fixed, dJ/db at the differentiable-solve workload's
    K = 100 is not determined in floating point: two FP64 evaluations of the
    oracle's own tangent that differ only in summation order
    (oracle.perturb.PermutedOperator) disagree by several per cent, because
    the recurrence amplifies rounding by ~100x every few iterations.  At
    K = 10 they agree to 1e-13 and the FP64 adjoint must match to 1e-10; at
    K = 100 the spread itself is asserted (> 1%), and the FP64 adjoint is held
    to ten times it.  Along b itself the map is exactly 1-homogeneous
    (x_K(a b) = a x_K(b) with fixed pivots and lambda), so Euler's identity
    b_bar . b = x_bar . x stays a sharp check at K = 100."""
    from oracle.perturb import PermutedOperator

    lam = 1.8
    A = ct256.scipy()
    db = np.random.default_rng(1).standard_normal(ct256.m)
    spread, err = {}, {}
    for K in (10, 100):
        r, xbar, adj = gpu_run(ct256, "f64", K, lam)
        g = float(adj["b_bar"] @ db)
        _, t_nat = T.loss_and_directional(A, ct256.b, lam, K, r["gp"], r["tp"], ct256.x_true,
                                          db, 0.0)
        _, t_perm = T.loss_and_directional(PermutedOperator(A), ct256.b, lam, K, r["gp"],
                                           r["tp"], ct256.x_true, db, 0.0)
        spread[K] = abs(t_perm - t_nat) / abs(t_nat)
        err[K] = abs(g - t_nat) / abs(t_nat)
        if K == 100:
            euler = float(adj["b_bar"] @ ct256.b)
            assert abs(euler - xbar @ r["x"]) <= 1e-8 * abs(xbar @ r["x"]), (euler, xbar @ r["x"])
    assert spread[10] < 1e-12 and err[10] <= 1e-10, (spread, err)
    assert spread[100] > 1e-2, spread
    assert err[100] <= 10 * spread[100], (spread, err)
