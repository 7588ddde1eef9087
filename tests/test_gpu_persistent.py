"""The persistent basis loops of lslu_set_loop against the FP64 oracle and
the launched kernels:

* LSLU_LOOP_PERSISTENT (one cooperative launch with bounded grid barriers
  runs the r0 pivot and all K iterations of Algorithm 4): across block
  counts, on breakdowns and batches, and with a barrier wait that runs out;
* LSLU_LOOP_CLUSTER (one thread-block cluster with hardware cluster
  barriers, for one small problem): the same parity, breakdowns and the
  refusal of problems that do not fit."""
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


@pytest.mark.parametrize("rule,lam", [("none", 0.0), ("fixed", 1e-2), ("gcv", 0.0), ("wgcv", 0.0)])
def test_ct32_f64_parity(ct32, rule, lam):
    """The 32x32 workload in FP64 (K = 50): identical pivots, x within 1e-10 of
    the oracle, bases and Hessenberg matrices within 1e-12, exact unit-pivot
    structure."""
    K = 50
    ref = O.hybrid_lslu(ct32.scipy(), ct32.b, None, K, rule, lam)
    with lslu.from_problem(ct32, "f64", K) as s:
        s.set_loop("persistent")
        r = s.solve(ct32.b, K, rule, lam, histories=True)
        st = s.state(r["k_done"])
    assert r["status"] == lslu.OK and r["k_done"] == K
    assert np.array_equal(r["gp"], ref.gp) and np.array_equal(r["tp"], ref.tp)
    assert rel(r["x"], ref.x) <= TOL_F64
    assert np.allclose(r["lam_hist"], ref.lam_hist, rtol=1e-8, atol=0)
    assert st["beta"] == ref.beta
    assert rel(st["H"], ref.H) <= 1e-12 and rel(st["W"], ref.W) <= 1e-12
    assert rel(st["L"], ref.L) <= 1e-12 and rel(st["D"], ref.D) <= 1e-12
    for Bm, piv in ((st["L"], r["gp"]), (st["D"], r["tp"])):
        for j in range(Bm.shape[1]):
            assert Bm[piv[j], j] == 1.0 and np.all(Bm[piv[:j], j] == 0.0)
            assert np.max(np.abs(Bm[:, j])) == 1.0


@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_ct32_mixed_precision(ct32, vt):
    K = 50
    A = ct32.scipy(tomo.round_values(ct32.vals, vt))
    ref = O.hybrid_lslu(A, ct32.b, None, K, "gcv")
    with lslu.from_problem(ct32, vt, K) as s:
        s.set_loop("persistent")
        r = s.solve(ct32.b, K, "gcv")
    assert r["status"] == lslu.OK and r["k_done"] == K
    assert rel(r["x"], ref.x) <= 2e-4
    assert np.array_equal(r["gp"][:5], ref.gp[:5]) and np.array_equal(r["tp"][:5], ref.tp[:5])


def test_block_counts_give_the_same_bits(ct32):
    """Every row is summed by one lane group in a fixed order and every pivot
    search is reduced in block order, so the block count changes nothing."""
    K = 40
    with lslu.from_problem(ct32, "f64", K) as s:
        s.set_loop("persistent")
        cfg = s.loop_config()
        assert cfg["mode"] == "persistent" and 1 <= cfg["blocks"] <= cfg["max_blocks"]
        base = s.solve(ct32.b, K, "gcv")
        for blocks in (1, 2, 7, cfg["max_blocks"]):
            s.set_loop("persistent", blocks=blocks)
            r = s.solve(ct32.b, K, "gcv")
            assert np.array_equal(r["gp"], base["gp"]) and np.array_equal(r["tp"], base["tp"])
            assert np.array_equal(r["x"], base["x"]), blocks
        with pytest.raises(lslu.LsluError):
            s.set_loop("persistent", blocks=cfg["max_blocks"] + 1)


def test_matches_launched_kernels(ct32):
    K = 50
    with lslu.from_problem(ct32, "f64", K) as s:
        g = s.solve(ct32.b, K, "gcv")
        s.set_loop("persistent")
        p = s.solve(ct32.b, K, "gcv")
        p2 = s.solve(ct32.b, K, "gcv")  # replayed graph of the persistent launch
        s.set_loop("graph")
        g2 = s.solve(ct32.b, K, "gcv")
    assert np.array_equal(p["gp"], g["gp"]) and np.array_equal(p["tp"], g["tp"])
    assert rel(p["x"], g["x"]) <= 1e-12
    assert np.array_equal(p["x"], p2["x"]) and np.array_equal(g["x"], g2["x"])


def test_renumbered_handle_picks_the_natural_pivots(ct32):
    K = 40
    with lslu.from_problem(ct32, "f64", K) as s:
        s.set_loop("persistent")
        a = s.solve(ct32.b, K, "gcv")
    with lslu.from_problem(ct32, "f64", K, order=tomo.locality_order(ct32)) as s:
        s.set_loop("persistent")
        b = s.solve(ct32.b, K, "gcv")
    assert np.array_equal(a["gp"], b["gp"]) and np.array_equal(a["tp"], b["tp"])
    assert rel(b["x"], a["x"]) <= 1e-10


def test_breakdowns(ct32):
    with lslu.from_problem(ct32, "f64", 5) as s:
        s.set_loop("persistent")
        r = s.solve(np.zeros(ct32.m), 5, "gcv")
    assert r["status"] == lslu.BREAKDOWN_BETA and r["k_done"] == 0 and np.all(r["x"] == 0.0)
    # hand-worked W-step breakdown after two iterations (oracle pins)
    rp = np.array([0, 1, 2, 2, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    Ad = np.zeros((4, 3))
    Ad[0, 0], Ad[1, 1] = 1.0, 2.0
    ref = O.hybrid_lslu(Ad, np.ones(4), None, 5, "none")
    with lslu.Solver(4, 3, rp, ci, np.array([1.0, 2.0]), "f64", 5) as s:
        s.set_loop("persistent")
        r = s.solve(np.ones(4), 5, "none")
    assert r["status"] == lslu.BREAKDOWN_W and r["k_done"] == 2
    assert r["gp"].tolist() == [1, 0, -1, -1, -1] and r["tp"].tolist() == [0, 1, 2, -1, -1, -1]
    assert rel(r["x"], ref.x) <= TOL_F64
    # H-step breakdown in the first iteration
    rp = np.array([0, 1, 2], dtype=np.int64)
    with lslu.Solver(2, 2, rp, np.array([0, 1], dtype=np.int32), np.ones(2), "f64", 3) as s:
        s.set_loop("persistent")
        r = s.solve(np.array([1.0, 0.5]), 3, "gcv")
    assert r["status"] == lslu.BREAKDOWN_H and r["k_done"] == 0 and np.all(r["x"] == 0.0)


def test_unsupported_requests_are_refused(ct32):
    with lslu.from_problem(ct32, "f64", 10) as s:
        s.set_loop("persistent")
        with pytest.raises(lslu.LsluError, match="persistent"):
            s.solve(ct32.b, 10, "gcv", x0=np.ones(ct32.n))
        r = s.solve(ct32.b, 10, "gcv")
        with pytest.raises(lslu.LsluError, match="persistent"):
            s.solve_fixed_pivots(ct32.b, 10, r["gp"], r["tp"])


def test_barrier_wait_runs_out_and_the_handle_recovers(ct32):
    """A test-only flag makes the first grid barrier wait on a word that
    nothing writes: every block gives up after the 2 ms limit, the solve
    returns LSLU_ERR_TIMEOUT, and the same handle then solves normally."""
    K = 20
    with lslu.from_problem(ct32, "f64", K) as s:
        s.set_loop("persistent", wait_limit_ns=2_000_000, stall_first_barrier=True)
        with pytest.raises(lslu.LsluError) as ei:
            s.solve(ct32.b, K, "gcv")
        assert ei.value.status == lslu.ERR_TIMEOUT
        s.set_loop("persistent")
        r = s.solve(ct32.b, K, "gcv")
    ref = O.hybrid_lslu(ct32.scipy(), ct32.b, None, K, "gcv", histories=False)
    assert r["status"] == lslu.OK and np.array_equal(r["gp"], ref.gp)
    assert rel(r["x"], ref.x) <= TOL_F64


@pytest.fixture(scope="module")
def small_batch():
    return tomo.make_uneven_batch(count=6, seed=4100, N_range=(12, 40), ang_range=(8, 40))


@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_batch_vs_oracle_and_launched_kernels(small_batch, vt):
    K = 30
    b = np.concatenate([P.b for P in small_batch])
    with lslu.from_problems(small_batch, vt, K) as bs:
        g = bs.solve(b, K, "gcv")
        bs.set_loop("persistent")
        r = bs.solve(b, K, "gcv")
    for p, P in enumerate(small_batch):
        A = P.scipy(tomo.round_values(P.vals, vt))
        ref = O.hybrid_lslu(A, P.b, None, K, "gcv", histories=False)
        assert r["status"][p] == lslu.OK and r["k_done"][p] == K
        assert np.array_equal(r["gp"][p][:5], ref.gp[:5])
        assert np.array_equal(r["tp"][p][:5], ref.tp[:5])
        assert rel(r["x"][p], ref.x) <= 2e-4, p
        assert rel(r["x"][p], g["x"][p]) <= 2e-4, p


def test_batch_breakdowns_stay_local(small_batch):
    tiny = tomo.make_problem(4, 6, 6, 3, 0.01, seed=77)  # 16 pixels: runs out of pivots
    probs = [small_batch[0], tiny, small_batch[1], small_batch[2]]
    bs_ = [P.b for P in probs]
    bs_[2] = np.zeros(probs[2].m)
    K = 20
    with lslu.from_problems(probs, "f32", K) as bs:
        g = bs.solve(np.concatenate(bs_), K, "gcv")
        bs.set_loop("persistent")
        r = bs.solve(np.concatenate(bs_), K, "gcv")
    for p in range(len(probs)):
        assert r["status"][p] == g["status"][p] and r["k_done"][p] == g["k_done"][p], p
        if g["status"][p] == lslu.OK:
            assert rel(r["x"][p], g["x"][p]) <= 2e-4, p
    # the 16-pixel problem ends with a full basis, whose projected problem is
    # ill conditioned: the two rounding orders (FP32) differ by ~0.7% there
    assert rel(r["x"][1], g["x"][1]) <= 2e-2
    # the 16-pixel problem runs out of pivots before K, the zero data breaks
    # down at once, the others complete
    assert g["status"][1] in (lslu.BREAKDOWN_W, lslu.BREAKDOWN_H) and g["k_done"][1] < K
    assert g["status"][2] == lslu.BREAKDOWN_BETA and g["k_done"][2] == 0
    assert g["status"][0] == lslu.OK and g["status"][3] == lslu.OK


def test_batch_barrier_timeout(small_batch):
    K = 10
    b = np.concatenate([P.b for P in small_batch])
    with lslu.from_problems(small_batch, "f32", K) as bs:
        bs.set_loop("persistent", wait_limit_ns=2_000_000, stall_first_barrier=True)
        with pytest.raises(lslu.LsluError) as ei:
            bs.solve(b, K, "gcv")
        assert ei.value.status == lslu.ERR_TIMEOUT
        bs.set_loop("persistent")
        r = bs.solve(b, K, "gcv")
    assert np.all(r["status"] == lslu.OK)


# ---------------------------------------------------------------------------
# the cluster loop
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("rule,lam", [("none", 0.0), ("fixed", 1e-2), ("gcv", 0.0), ("wgcv", 0.0)])
def test_cluster_ct32_f64_parity(ct32, rule, lam):
    K = 50
    ref = O.hybrid_lslu(ct32.scipy(), ct32.b, None, K, rule, lam)
    with lslu.from_problem(ct32, "f64", K) as s:
        s.set_loop("cluster")
        cfg = s.loop_config()
        assert cfg["mode"] == "cluster" and cfg["blocks"] in (8, 16)
        r = s.solve(ct32.b, K, rule, lam, histories=True)
        st = s.state(r["k_done"])
    assert r["status"] == lslu.OK and r["k_done"] == K
    assert np.array_equal(r["gp"], ref.gp) and np.array_equal(r["tp"], ref.tp)
    assert rel(r["x"], ref.x) <= TOL_F64
    assert np.allclose(r["lam_hist"], ref.lam_hist, rtol=1e-8, atol=0)
    assert st["beta"] == ref.beta
    assert rel(st["H"], ref.H) <= 1e-12 and rel(st["W"], ref.W) <= 1e-12
    assert rel(st["L"], ref.L) <= 1e-12 and rel(st["D"], ref.D) <= 1e-12
    for Bm, piv in ((st["L"], r["gp"]), (st["D"], r["tp"])):
        for j in range(Bm.shape[1]):
            assert Bm[piv[j], j] == 1.0 and np.all(Bm[piv[:j], j] == 0.0)
            assert np.max(np.abs(Bm[:, j])) == 1.0


@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_cluster_ct32_mixed_precision(ct32, vt):
    K = 50
    A = ct32.scipy(tomo.round_values(ct32.vals, vt))
    ref = O.hybrid_lslu(A, ct32.b, None, K, "gcv")
    with lslu.from_problem(ct32, vt, K) as s:
        s.set_loop("cluster")
        r = s.solve(ct32.b, K, "gcv")
        r2 = s.solve(ct32.b, K, "gcv")
    assert r["status"] == lslu.OK and r["k_done"] == K
    assert rel(r["x"], ref.x) <= 2e-4
    assert np.array_equal(r["gp"][:5], ref.gp[:5]) and np.array_equal(r["tp"][:5], ref.tp[:5])
    assert np.array_equal(r["x"], r2["x"])


def test_cluster_matches_launched_kernels_and_renumbering(ct32):
    K = 50
    with lslu.from_problem(ct32, "f64", K) as s:
        g = s.solve(ct32.b, K, "gcv")
        s.set_loop("cluster")
        c = s.solve(ct32.b, K, "gcv")
    with lslu.from_problem(ct32, "f64", K, order=tomo.locality_order(ct32)) as s:
        s.set_loop("cluster")
        o = s.solve(ct32.b, K, "gcv")
    assert np.array_equal(c["gp"], g["gp"]) and np.array_equal(c["tp"], g["tp"])
    assert rel(c["x"], g["x"]) <= 1e-12
    assert np.array_equal(o["gp"], g["gp"]) and np.array_equal(o["tp"], g["tp"])
    assert rel(o["x"], g["x"]) <= 1e-10


def test_cluster_breakdowns(ct32):
    with lslu.from_problem(ct32, "f64", 5) as s:
        s.set_loop("cluster")
        r = s.solve(np.zeros(ct32.m), 5, "gcv")
    assert r["status"] == lslu.BREAKDOWN_BETA and r["k_done"] == 0 and np.all(r["x"] == 0.0)
    rp = np.array([0, 1, 2, 2, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    Ad = np.zeros((4, 3))
    Ad[0, 0], Ad[1, 1] = 1.0, 2.0
    ref = O.hybrid_lslu(Ad, np.ones(4), None, 5, "none")
    with lslu.Solver(4, 3, rp, ci, np.array([1.0, 2.0]), "f64", 5) as s:
        s.set_loop("cluster")
        r = s.solve(np.ones(4), 5, "none")
    assert r["status"] == lslu.BREAKDOWN_W and r["k_done"] == 2
    assert r["gp"].tolist() == [1, 0, -1, -1, -1] and r["tp"].tolist() == [0, 1, 2, -1, -1, -1]
    assert rel(r["x"], ref.x) <= TOL_F64
    rp = np.array([0, 1, 2], dtype=np.int64)
    with lslu.Solver(2, 2, rp, np.array([0, 1], dtype=np.int32), np.ones(2), "f64", 3) as s:
        s.set_loop("cluster")
        r = s.solve(np.array([1.0, 0.5]), 3, "gcv")
    assert r["status"] == lslu.BREAKDOWN_H and r["k_done"] == 0 and np.all(r["x"] == 0.0)


def test_cluster_refusals(ct32, small_batch):
    with lslu.from_problems(small_batch, "f32", 10) as bs:
        with pytest.raises(lslu.LsluError, match="single problems"):
            bs.set_loop("cluster")
    P = tomo.make_config("ct256")
    with lslu.from_problem(P, "f32", 200) as s:
        with pytest.raises(lslu.LsluError, match="does not fit"):
            s.set_loop("cluster")
    with lslu.from_problem(ct32, "f64", 10) as s:
        s.set_loop("cluster")
        with pytest.raises(lslu.LsluError, match="x0 = 0"):
            s.solve(ct32.b, 10, "gcv", x0=np.ones(ct32.n))
