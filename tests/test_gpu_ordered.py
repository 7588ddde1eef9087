"""Renumbered handles (lslu_create_ordered) through the C ABI.

A handle made with a row order and a column order stores A_hat = P_r A P_c^T,
solves with b_hat = P_r b, and maps vectors, bases and pivot indices back to
the caller's numbering; a pivot search still breaks ties by the caller's
index, so the pivots are those of a handle without a renumbering.  Checked
against the FP64 oracle run on A_hat (inputs with no tied search, where the
two definitions agree), against a handle without a renumbering at every entry
point that takes or returns a vector (equal up to rounding), and on a
hand-worked case whose first pivot is a four-way tie.
"""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import lslu, tomo

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_05239_gb300 import build

    build.build()


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def renumbered(P, ro, co, vals=None):
    """A_hat = P_r A P_c^T (internal row ro[i] = caller row i) and the maps
    internal -> caller."""
    ir = np.argsort(ro)
    ic = np.argsort(co)
    Ah = P.scipy(vals)[ir][:, ic].tocsr()
    Ah.sort_indices()
    return Ah, ir, ic


def orders(P, kind, seed=0):
    if kind == "tiles":
        return tomo.locality_order(P)
    rng = np.random.default_rng(seed)
    return (rng.permutation(P.m).astype(np.int32), rng.permutation(P.n).astype(np.int32))


@pytest.mark.parametrize("kind", ["tiles", "random"])
@pytest.mark.parametrize("rule,lam", [("gcv", 0.0), ("fixed", 1e-2)])
def test_ct32_f64_against_oracle_on_renumbered_problem(ct32, kind, rule, lam):
    K = 50
    ro, co = orders(ct32, kind)
    Ah, ir, ic = renumbered(ct32, ro, co)
    ref = O.hybrid_lslu(Ah, ct32.b[ir], None, K, rule, lam)
    with lslu.from_problem(ct32, "f64", K, order=(ro, co)) as s:
        r = s.solve(ct32.b, K, rule, lam, histories=True)
        st = s.state(r["k_done"])
    assert r["status"] == lslu.OK and r["k_done"] == K
    # pivots come back in the caller's numbering
    assert np.array_equal(r["gp"], ic[ref.gp]) and np.array_equal(r["tp"], ir[ref.tp])
    assert rel(r["x"], ref.x[co]) <= TOL_F64
    assert np.allclose(r["res_hist"], ref.res_hist, rtol=1e-9, atol=0)
    assert np.allclose(r["lam_hist"], ref.lam_hist, rtol=1e-8, atol=0)
    assert st["beta"] == ref.beta
    assert rel(st["H"], ref.H) <= 1e-12 and rel(st["W"], ref.W) <= 1e-12
    # bases in the caller's numbering: caller row j is internal row co[j]
    assert rel(st["L"], ref.L[co]) <= 1e-12 and rel(st["D"], ref.D[ro]) <= 1e-12
    # and the same solve as a handle without a renumbering
    ref0 = O.hybrid_lslu(ct32.scipy(), ct32.b, None, K, rule, lam, histories=False)
    assert np.array_equal(r["gp"], ref0.gp) and np.array_equal(r["tp"], ref0.tp)
    assert rel(r["x"], ref0.x) <= TOL_F64


@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_ct32_mixed_precision_renumbered(ct32, vt):
    K = 50
    ro, co = orders(ct32, "random", seed=3)
    Ah, ir, ic = renumbered(ct32, ro, co, tomo.round_values(ct32.vals, vt))
    ref = O.hybrid_lslu(Ah, ct32.b[ir], None, K, "gcv", histories=False)
    with lslu.from_problem(ct32, vt, K, order=(ro, co)) as s:
        r = s.solve(ct32.b, K, "gcv")
    assert r["status"] == lslu.OK and r["k_done"] == K
    assert rel(r["x"], ref.x[co]) <= 2e-4
    assert np.array_equal(r["gp"][:5], ic[ref.gp[:5]])
    assert np.array_equal(r["tp"][:5], ir[ref.tp[:5]])


def test_only_one_order_given(ct32):
    """A NULL order is the identity."""
    K = 20
    ro, co = orders(ct32, "random", seed=5)
    with lslu.from_problem(ct32, "f64", K) as s0:
        r0 = s0.solve(ct32.b, K, "gcv")
    for order in ((ro, None), (None, co)):
        with lslu.from_problem(ct32, "f64", K, order=order) as s:
            r = s.solve(ct32.b, K, "gcv")
        assert np.array_equal(r["gp"], r0["gp"]) and np.array_equal(r["tp"], r0["tp"])
        assert rel(r["x"], r0["x"]) <= TOL_F64


def test_every_entry_point_matches_the_natural_handle(ct32):
    K = 30
    ro, co = orders(ct32, "tiles")
    x0 = np.linspace(0.0, 0.3, ct32.n)
    rng = np.random.default_rng(11)
    x_bar = rng.standard_normal(ct32.n)
    S = lslu.sample_table(K, 64, ct32.m, ct32.n, seed=12)
    out = []
    for order in (None, (ro, co)):
        with lslu.from_problem(ct32, "f64", K, order=order) as s:
            o = {}
            r = s.solve(ct32.b, K, "fixed", 1e-2, x0=x0, histories=True)
            o["solve"] = r
            o["fixed"] = s.solve_fixed_pivots(ct32.b, K, r["gp"], r["tp"], "fixed", 1e-2, x0=x0)
            o["sampled"] = s.solve_sampled(ct32.b, K, S, "gcv")
            o["stop"] = s.solve_stopping(ct32.b, K, "wgcv", tol=1e-4)
            o["opt"] = s.solve_optimal(ct32.b, K, ct32.x_true)
            r = s.solve(ct32.b, K, "gcv")
            o["adj"] = s.adjoint(x_bar, want_x0=True)
            o["uq"] = s.uq(1e-4, 1e-1)
            out.append(o)
    a, b = out
    assert np.array_equal(a["solve"]["gp"], b["solve"]["gp"])
    assert np.array_equal(a["solve"]["tp"], b["solve"]["tp"])
    assert rel(b["solve"]["x"], a["solve"]["x"]) <= TOL_F64
    assert np.allclose(b["solve"]["res_hist"], a["solve"]["res_hist"], rtol=1e-9, atol=0)
    # replaying the caller-numbered pivots reproduces the solve
    assert rel(b["fixed"]["x"], b["solve"]["x"]) <= 1e-12
    assert np.array_equal(a["sampled"]["gp"], b["sampled"]["gp"])
    assert np.array_equal(a["sampled"]["tp"], b["sampled"]["tp"])
    assert rel(b["sampled"]["x"], a["sampled"]["x"]) <= TOL_F64
    assert a["stop"]["k_stop"] == b["stop"]["k_stop"]
    assert rel(b["stop"]["x"], a["stop"]["x"]) <= TOL_F64
    assert rel(b["stop"]["G"], a["stop"]["G"]) <= 1e-9
    # the optimal lambda minimises an error that is quadratic at its minimum,
    # so rounding moves the minimiser by ~sqrt(eps) relative, and x with it
    assert abs(b["opt"]["lam"] - a["opt"]["lam"]) <= 1e-6 * a["opt"]["lam"]
    assert rel(b["opt"]["x"], a["opt"]["x"]) <= 1e-6
    assert rel(b["adj"]["b_bar"], a["adj"]["b_bar"]) <= 1e-9
    assert rel(b["adj"]["x0_bar"], a["adj"]["x0_bar"]) <= 1e-9
    assert abs(b["adj"]["lambda_bar"] - a["adj"]["lambda_bar"]) <= 1e-9 * abs(
        a["adj"]["lambda_bar"])
    assert rel(b["uq"]["var_diag"], a["uq"]["var_diag"]) <= 1e-9
    assert abs(b["uq"]["var_sum"] - a["uq"]["var_sum"]) <= 1e-9 * abs(a["uq"]["var_sum"])


def test_device_pointers(ct32):
    import torch

    K = 25
    ro, co = orders(ct32, "random", seed=7)
    dev = torch.device("cuda", 0)
    with lslu.from_problem(ct32, "f32", K, order=(ro, co)) as s:
        r = s.solve(ct32.b, K, "gcv")
        b = torch.from_numpy(ct32.b).to(dev)
        x = torch.zeros(ct32.n, dtype=torch.float64, device=dev)
        gp = torch.zeros(K, dtype=torch.int32, device=dev)
        tp = torch.zeros(K + 1, dtype=torch.int32, device=dev)
        s.solve_device(b, x, K, "gcv", gp=gp, tp=tp)
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy(), r["x"])
        assert np.array_equal(gp.cpu().numpy(), r["gp"])
        assert np.array_equal(tp.cpu().numpy(), r["tp"])
        xb = torch.from_numpy(np.ones(ct32.n)).to(dev)
        bb = torch.zeros(ct32.m, dtype=torch.float64, device=dev)
        s.adjoint_device(xb, bb)
        torch.cuda.synchronize()
        assert np.array_equal(bb.cpu().numpy(), s.adjoint(np.ones(ct32.n))["b_bar"])


def test_invalid_orders_refused(ct32):
    P = ct32
    good_r, good_c = tomo.locality_order(P)
    bad = good_c.copy()
    bad[3] = bad[4]  # a repeated entry
    for ro, co in ((good_r, bad), (np.full(P.m, P.m, np.int32), good_c),
                   (good_r, -np.ones(P.n, np.int32))):
        with pytest.raises(lslu.LsluError, match="permutation"):
            lslu.from_problem(P, "f64", 5, order=(ro, co))
    with lslu.from_problem(P, "f32", 5, order=(good_r, good_c)) as s:
        import torch

        x = torch.zeros(P.n, dtype=torch.float32, device="cuda")
        y = torch.zeros(P.m, dtype=torch.float32, device="cuda")
        with pytest.raises(lslu.LsluError, match="renumbering"):
            s.spmv(0, x, y)


def test_ct256_f64_renumbered_matches_natural():
    """At 65536 unknowns: the same pivots and x_12 as the natural handle (the
    FP64 oracle run in both numberings agrees to 4e-15 at k = 12; rounding
    noise grows ~100x every few iterations after that)."""
    P = tomo.make_config("ct256")
    ro, co = tomo.locality_order(P)
    K = 12
    with lslu.from_problem(P, "f64", K) as s0, \
            lslu.from_problem(P, "f64", K, order=(ro, co)) as s1:
        r0 = s0.solve(P.b, K, "gcv")
        r1 = s1.solve(P.b, K, "gcv")
    assert np.array_equal(r0["gp"], r1["gp"]) and np.array_equal(r0["tp"], r1["tp"])
    assert rel(r1["x"], r0["x"]) <= 1e-10


def test_breakdowns_renumbered(ct32):
    """b = 0 breaks down before the first iteration; and the hand-worked W-step
    breakdown of the oracle pins (A = diag(1, 2) padded to 4 x 3, b = ones)
    with both numberings reversed: the first row pivot is a four-way tie,
    which goes to the lowest caller index (row 0, not internal row 0 = caller
    row 3), so the solve is the natural one."""
    ro, co = orders(ct32, "random", seed=9)
    with lslu.from_problem(ct32, "f64", 5, order=(ro, co)) as s:
        r = s.solve(np.zeros(ct32.m), 5, "gcv")
    assert r["status"] == lslu.BREAKDOWN_BETA and r["k_done"] == 0
    assert np.all(r["x"] == 0.0) and np.all(r["gp"] == -1) and np.all(r["tp"] == -1)
    rp = np.array([0, 1, 2, 2, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    Ad = np.zeros((4, 3))
    Ad[0, 0], Ad[1, 1] = 1.0, 2.0
    ref = O.hybrid_lslu(Ad, np.ones(4), None, 5, "none")
    ro = np.array([3, 2, 1, 0], np.int32)
    co = np.array([2, 1, 0], np.int32)
    with lslu.Solver(4, 3, rp, ci, np.array([1.0, 2.0]), "f64", 5, row_order=ro,
                     col_order=co) as s:
        r = s.solve(np.ones(4), 5, "none")
    assert r["status"] == ref.status == lslu.BREAKDOWN_W and r["k_done"] == ref.k_done == 2
    assert r["gp"].tolist() == [1, 0, -1, -1, -1]
    assert r["tp"].tolist() == [0, 1, 2, -1, -1, -1]
    assert rel(r["x"], ref.x) <= TOL_F64
    # the sampled search breaks ties the same way: a sample of all four rows
    S = np.tile(np.array([3, 2, 1, 0], np.int32), (11, 1))
    S[1::2] = np.array([2, 1, 0, 2], np.int32)
    with lslu.Solver(4, 3, rp, ci, np.array([1.0, 2.0]), "f64", 5, row_order=ro,
                     col_order=co) as s, lslu.Solver(4, 3, rp, ci, np.array([1.0, 2.0]), "f64",
                                                     5) as s0:
        a = s.solve_sampled(np.ones(4), 5, S, "none")
        b = s0.solve_sampled(np.ones(4), 5, S, "none")
    assert a["status"] == b["status"] and a["k_done"] == b["k_done"]
    assert np.array_equal(a["gp"], b["gp"]) and np.array_equal(a["tp"], b["tp"])
    assert a["tp"][0] == 0


def test_device_csr_and_orders(ct32):
    """CSR arrays and both orders in device memory (ptr_location = device)."""
    import torch

    dev = torch.device("cuda", 0)
    ro, co = orders(ct32, "random", seed=13)

    def t(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)

    with lslu.Solver(ct32.m, ct32.n, t(ct32.row_ptr, np.int64), t(ct32.col_idx, np.int32),
                     t(ct32.vals, np.float64), "f64", 20, row_order=t(ro, np.int32),
                     col_order=t(co, np.int32)) as s_dev, \
            lslu.from_problem(ct32, "f64", 20, order=(ro, co)) as s_host:
        a = s_dev.solve(ct32.b, 20, "gcv")
        b = s_host.solve(ct32.b, 20, "gcv")
    assert np.array_equal(a["x"], b["x"])
    assert np.array_equal(a["gp"], b["gp"]) and np.array_equal(a["tp"], b["tp"])
