"""Parity of the CUDA path (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import lslu, tomo

pytestmark = pytest.mark.gpu

# FP64 tolerance on x_k: the oracle and the GPU differ only in summation order
# (warp-tree sums, forward substitution versus sequential elimination, FMA
# contraction); perturbing the oracle's own summation order moves x_50 by
# ~6e-15 on the 32x32 workload, so 1e-10 leaves ample room.
TOL_F64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_05239_gb300 import build

    build.build()
    import torch

    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("rule,lam", [("none", 0.0), ("fixed", 1e-2), ("gcv", 0.0), ("wgcv", 0.0)])
def test_ct32_f64_parity(ct32, rule, lam):
    K = 50
    ref = O.hybrid_lslu(ct32.scipy(), ct32.b, None, K, rule, lam)
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve(ct32.b, K, rule, lam, histories=True)
        st = s.state(r["k_done"])
    assert r["status"] == lslu.OK and r["k_done"] == K
    assert np.array_equal(r["gp"], ref.gp), "column pivots differ"
    assert np.array_equal(r["tp"], ref.tp), "row pivots differ"
    assert rel(r["x"], ref.x) <= TOL_F64
    assert np.allclose(r["res_hist"], ref.res_hist, rtol=1e-9, atol=0)
    assert np.allclose(r["lam_hist"], ref.lam_hist, rtol=1e-8, atol=0)
    assert st["beta"] == ref.beta
    assert rel(st["H"], ref.H) <= 1e-12 and rel(st["W"], ref.W) <= 1e-12
    assert rel(st["L"], ref.L) <= 1e-12 and rel(st["D"], ref.D) <= 1e-12


def test_ct32_f64_exact_structure(ct32):
    """Pivot entries are exactly 1 and earlier pivots exactly 0 on the GPU too
    (Algorithm 4); every |entry| <= 1."""
    K = 50
    with lslu.from_problem(ct32, "f64", K) as s:
        r = s.solve(ct32.b, K, "gcv")
        st = s.state(r["k_done"])
    for Bm, piv in ((st["L"], r["gp"]), (st["D"], r["tp"])):
        for j in range(Bm.shape[1]):
            assert Bm[piv[j], j] == 1.0
            assert np.all(Bm[piv[:j], j] == 0.0)
            assert np.max(np.abs(Bm[:, j])) == 1.0


def test_ct32_final_only_equals_histories(ct32):
    with lslu.from_problem(ct32, "f64", 30) as s:
        a = s.solve(ct32.b, 30, "gcv", histories=True)
        b = s.solve(ct32.b, 30, "gcv", histories=False)
        c = s.solve(ct32.b, 30, "gcv", histories=False)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(b["x"], c["x"])


@pytest.mark.parametrize("rule", ["gcv", "wgcv"])
def test_long_history_against_the_oracle_rule(ct32, rule):
    """A history of K = 200 projected problems is solved as a throughput batch
    (8-CTA bidiagonalisations, largest k first; one lane per singular value
    for every problem but the last), the final one as in a final-only solve.
    Each lambda_k must minimise the oracle's (w)GCV function of the GPU's own
    H_{k+1,k} as well as the oracle's choice does, each residual must be the
    oracle's at that lambda_k, and x must be bit for bit the final-only x."""
    K = 200
    with lslu.from_problem(ct32, "f64", K) as s:
        a = s.solve(ct32.b, K, rule, histories=True)
        st = s.state(a["k_done"])
        b = s.solve(ct32.b, K, rule, histories=False)
    assert a["status"] == lslu.OK and a["k_done"] == K
    assert np.array_equal(a["x"], b["x"])
    H, beta = st["H"], st["beta"]
    for k in list(range(1, K + 1, 9)) + [K - 1, K]:
        sig, c, _ = O.projected_svd(H[:k + 1, :k], beta)
        omega = 1.0 if rule == "gcv" else (k + 1) / ct32.m
        lam_ref = O.select_lambda(sig, c, omega)
        lam = a["lam_hist"][k - 1]
        G_ref = O.gcv_value(sig, c, lam_ref, omega)
        assert O.gcv_value(sig, c, lam, omega) <= G_ref * (1 + 1e-9), k
        res = O.projected_residual(sig, c, lam)
        assert abs(a["res_hist"][k - 1] - res) <= 1e-9 * res, k


@pytest.mark.parametrize("k", [1, 2, 5, 20, 50])
@pytest.mark.parametrize("rule,lam", [("none", 0.0), ("fixed", 0.05), ("gcv", 0.0), ("wgcv", 0.0)])
def test_projected_solve_parity(ct32, k, rule, lam):
    hp = O.hessenberg_rect_pivoted(ct32.scipy(), ct32.b, None, 50)
    H = hp["H"][:k + 1, :k]
    s_ref, c_ref, V = O.projected_svd(H, hp["beta"])
    lam_ref = O._lambda_for(rule, lam, s_ref, c_ref, k, ct32.m)
    y_ref = O.tikhonov_y(s_ref, c_ref, V, lam_ref)
    with lslu.from_problem(ct32, "f64", 50) as s:
        out = s.projected(H, hp["beta"], rule, lam)
    assert np.allclose(out["sigma"], s_ref, rtol=1e-12, atol=1e-14 * s_ref[0])
    assert np.allclose(np.abs(out["c"]), np.abs(c_ref), rtol=1e-10, atol=1e-13 * abs(hp["beta"]))
    if lam_ref == 0.0:
        assert out["lam"] == 0.0
    else:
        assert abs(out["lam"] - lam_ref) <= 1e-8 * lam_ref
    assert rel(out["y"], y_ref) <= 1e-10
    assert abs(out["resid"] - O.projected_residual(s_ref, c_ref, lam_ref)) <= 1e-10 * abs(hp["beta"])


@pytest.mark.parametrize("vt,tol", [("f32", 2e-4), ("bf16", 2e-4)])
def test_ct32_mixed_precision(ct32, vt, tol):
    """FP32 basis and accumulation with A stored in FP32 / BF16, against the
    FP64 oracle run on the same rounded matrix values."""
    K = 50
    A = ct32.scipy(tomo.round_values(ct32.vals, vt))
    ref = O.hybrid_lslu(A, ct32.b, None, K, "gcv")
    with lslu.from_problem(ct32, vt, K) as s:
        r = s.solve(ct32.b, K, "gcv")
    assert r["status"] == lslu.OK and r["k_done"] == K
    assert rel(r["x"], ref.x) <= tol
    # the first pivots are identical (later near-ties may resolve differently)
    assert np.array_equal(r["gp"][:5], ref.gp[:5]) and np.array_equal(r["tp"][:5], ref.tp[:5])


def test_x0_nonzero(ct32):
    x0 = np.linspace(0.0, 0.5, ct32.n)
    ref = O.hybrid_lslu(ct32.scipy(), ct32.b, x0, 12, "fixed", 1e-2)
    with lslu.from_problem(ct32, "f64", 12) as s:
        r = s.solve(ct32.b, 12, "fixed", 1e-2, x0=x0)
    assert np.array_equal(r["gp"], ref.gp)
    assert rel(r["x"], ref.x) <= TOL_F64


def test_breakdown_beta_on_gpu(ct32):
    with lslu.from_problem(ct32, "f64", 5) as s:
        r = s.solve(np.zeros(ct32.m), 5, "gcv")
    assert r["status"] == lslu.BREAKDOWN_BETA and r["k_done"] == 0
    assert np.all(r["x"] == 0.0) and np.all(r["gp"] == -1) and np.all(r["tp"] == -1)


def test_breakdown_w_exact_case():
    """The hand-worked case of the oracle pins: A = diag(1, 2) padded to 4 x 3,
    b = ones breaks down in the W step after two iterations."""
    rp = np.array([0, 1, 2, 2, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    v = np.array([1.0, 2.0])
    Ad = np.zeros((4, 3))
    Ad[0, 0], Ad[1, 1] = 1.0, 2.0
    ref = O.hybrid_lslu(Ad, np.ones(4), None, 5, "none")
    with lslu.Solver(4, 3, rp, ci, v, "f64", 5) as s:
        r = s.solve(np.ones(4), 5, "none")
    assert r["status"] == lslu.BREAKDOWN_W and r["k_done"] == 2
    assert r["gp"].tolist() == [1, 0, -1, -1, -1]
    assert r["tp"].tolist() == [0, 1, 2, -1, -1, -1]
    assert rel(r["x"], ref.x) <= TOL_F64


def test_breakdown_h_exact_case():
    rp = np.array([0, 1, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    with lslu.Solver(2, 2, rp, ci, np.ones(2), "f64", 3) as s:
        r = s.solve(np.array([1.0, 0.5]), 3, "gcv")
    assert r["status"] == lslu.BREAKDOWN_H and r["k_done"] == 0
    assert np.all(r["x"] == 0.0)


def test_nonfinite_b_rejected(ct32):
    b = ct32.b.copy()
    b[3] = np.nan
    with lslu.from_problem(ct32, "f64", 5) as s:
        with pytest.raises(lslu.LsluError):
            s.solve(b, 5, "gcv")


def test_graph_replay_matches_direct_launches(ct32, monkeypatch):
    """Solves replayed from the captured CUDA graph (with and without timing
    events) equal kernel-by-kernel launches bit for bit."""
    with lslu.from_problem(ct32, "f32", 40) as s:
        a = s.solve(ct32.b, 40, "gcv")
        b = s.solve(ct32.b, 40, "gcv")  # graph replay
        s.profile(True)
        c = s.solve(ct32.b, 40, "gcv")
        s.profile(False)
        n, ms = s.timing()
    monkeypatch.setenv("LSLU_NO_GRAPHS", "1")
    with lslu.from_problem(ct32, "f32", 40) as s2:
        d = s2.solve(ct32.b, 40, "gcv")
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["x"], c["x"])
    assert np.array_equal(a["x"], d["x"]) and np.array_equal(a["gp"], d["gp"])
    assert n == 80 and ms > 0


@pytest.mark.parametrize("shape", range(16))
def test_every_spmv_shape_keeps_f64_parity(ct32, shape):
    """All row shapes of the sparse products (the autotuner's choices) give the
    oracle's pivots and x within the FP64 tolerance."""
    K = 30
    ref = O.hybrid_lslu(ct32.scipy(), ct32.b, None, K, "gcv", histories=False)
    with lslu.from_problem(ct32, "f64", K) as s:
        s.set_spmv_shape(shape, (shape + 1) % 16)
        r = s.solve(ct32.b, K, "gcv")
        r2 = s.solve(ct32.b, K, "gcv")
    assert np.array_equal(r["gp"], ref.gp) and np.array_equal(r["tp"], ref.tp)
    assert rel(r["x"], ref.x) <= TOL_F64
    assert np.array_equal(r["x"], r2["x"])


def test_autotuner_picks_a_shape(ct32):
    K = 20
    A32 = ct32.scipy(tomo.round_values(ct32.vals, "f32"))
    ref = O.hybrid_lslu(A32, ct32.b, None, K, "gcv", histories=False)
    with lslu.from_problem(ct32, "f32", K) as s:
        t = s.tune_spmv(reps=3)
        assert 0 <= t["shape_A"] < 16 and 0 <= t["shape_AT"] < 16
        for key, shp in (("us_A", t["shape_A"]), ("us_AT", t["shape_AT"])):
            best = min(t[key].values())
            chosen = t[key][s.SHAPES[shp]]
            # the fastest shape, or the default (16x2 for FP32) within 3% of it
            assert chosen == best or (shp == 0 and best > 0.97 * chosen)
        r = s.solve(ct32.b, K, "gcv")
    assert rel(r["x"], ref.x) <= 2e-4
