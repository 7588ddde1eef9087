"""Batched Hybrid LSLU (lslu_create_batched / lslu_solve_batched).

Every problem of a batch runs Algorithm 5 on its own: its pivots, lambda
choice, breakdowns and x must equal those of a single-problem solve of the
same problem with the same value type, bit for bit (the batched kernels do
the same arithmetic in the same order per problem), and so must match the
FP64 oracle to the mixed-precision tolerance of the single-problem path.
"""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import lslu, tomo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_05239_gb300 import build

    build.build()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def small_batch():
    # uneven, ragged sizes (none a multiple of the 128-row tile)
    return tomo.make_uneven_batch(count=6, seed=4100, N_range=(12, 40), ang_range=(8, 40))


def single(P, vt, K, rule, lam=0.0, b=None):
    with lslu.from_problem(P, vt, K) as s:
        return s.solve(P.b if b is None else b, K, rule, lam)


@pytest.mark.parametrize("vt", ["f32", "bf16"])
@pytest.mark.parametrize("rule,lam", [("gcv", 0.0), ("wgcv", 0.0), ("fixed", 1e-2), ("none", 0.0)])
def test_batched_equals_single(small_batch, vt, rule, lam):
    K = 30
    with lslu.from_problems(small_batch, vt, K) as bs:
        r = bs.solve(np.concatenate([P.b for P in small_batch]), K, rule, lam)
    for p, P in enumerate(small_batch):
        s = single(P, vt, K, rule, lam)
        assert r["status"][p] == s["status"] and r["k_done"][p] == s["k_done"]
        assert np.array_equal(r["gp"][p], s["gp"]) and np.array_equal(r["tp"][p], s["tp"])
        assert np.array_equal(r["x"][p], s["x"]), p


def test_batched_vs_oracle(small_batch):
    K = 30
    with lslu.from_problems(small_batch, "f32", K) as bs:
        r = bs.solve(np.concatenate([P.b for P in small_batch]), K, "gcv")
    for p, P in enumerate(small_batch):
        A = P.scipy(tomo.round_values(P.vals, "f32"))
        ref = O.hybrid_lslu(A, P.b, None, K, "gcv", histories=False)
        assert r["k_done"][p] == K
        assert np.array_equal(r["gp"][p][:5], ref.gp[:5])
        assert np.array_equal(r["tp"][p][:5], ref.tp[:5])
        assert rel(r["x"][p], ref.x) <= 2e-4, p


def test_breakdowns_stay_local(small_batch):
    """A zero right-hand side (beta breakdown) and a problem with fewer
    columns than K (runs out of pivots) stop only themselves."""
    tiny = tomo.make_problem(4, 6, 6, 3, 0.01, seed=77)  # 16 pixels, 36 rays
    probs = [small_batch[0], tiny, small_batch[1], small_batch[2]]
    bs_ = [P.b for P in probs]
    bs_[2] = np.zeros(probs[2].m)
    K = 20
    with lslu.from_problems(probs, "f32", K) as bs:
        r = bs.solve(np.concatenate(bs_), K, "gcv")
    for p, P in enumerate(probs):
        s = single(P, "f32", K, "gcv", b=bs_[p])
        assert r["status"][p] == s["status"] and r["k_done"][p] == s["k_done"], p
        assert np.array_equal(r["gp"][p], s["gp"]) and np.array_equal(r["tp"][p], s["tp"])
        assert np.array_equal(r["x"][p], s["x"]), p
    assert r["status"][2] == lslu.BREAKDOWN_BETA and r["k_done"][2] == 0
    assert np.all(r["x"][2] == 0.0) and np.all(r["gp"][2] == -1)
    assert r["status"][1] in (lslu.BREAKDOWN_W, lslu.BREAKDOWN_H) and r["k_done"][1] <= 16
    assert r["status"][0] == lslu.OK and r["k_done"][0] == K


def test_single_problem_batch(small_batch):
    P = small_batch[3]
    with lslu.from_problems([P], "f32", 25) as bs:
        r = bs.solve(P.b, 25, "gcv")
    s = single(P, "f32", 25, "gcv")
    assert np.array_equal(r["x"][0], s["x"]) and np.array_equal(r["gp"][0], s["gp"])


def test_replay_and_device_pointers(small_batch):
    import torch

    K = 25
    b = np.concatenate([P.b for P in small_batch])
    with lslu.from_problems(small_batch, "f32", K) as bs:
        a = bs.solve(b, K, "gcv")
        c = bs.solve(b, K, "gcv")  # replays the captured graph
        dev = torch.device("cuda", 0)
        nP = len(small_batch)
        bd = torch.tensor(b, dtype=torch.float64, device=dev)
        xd = torch.zeros(sum(P.n for P in small_batch), dtype=torch.float64, device=dev)
        gd = torch.zeros((nP, K), dtype=torch.int32, device=dev)
        kd = torch.zeros(nP, dtype=torch.int32, device=dev)
        bs.solve_device(bd, xd, K, "gcv", gp=gd, k_done=kd)
        torch.cuda.synchronize()
    xa = np.concatenate(a["x"])
    assert np.array_equal(xa, np.concatenate(c["x"]))
    assert np.array_equal(xa, xd.cpu().numpy())
    assert np.array_equal(a["gp"], gd.cpu().numpy()) and np.array_equal(a["k_done"], kd.cpu().numpy())


def test_fixed_lambda_validation(small_batch):
    with lslu.from_problems(small_batch[:2], "f32", 5) as bs:
        with pytest.raises(lslu.LsluError):
            bs.solve(np.concatenate([P.b for P in small_batch[:2]]), 5, "fixed", -1.0)
        with pytest.raises(lslu.LsluError):
            bs.solve(np.concatenate([P.b for P in small_batch[:2]]), 6, "gcv")


@pytest.mark.parametrize("vt", ["f32", "bf16"])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 16])
def test_shared_matrix_rhs_equal_single_solves(vt, nrhs):
    """Right-hand sides sharing one matrix (one pass over A per product for
    all of them) give each the single-problem result bit for bit."""
    Ps = tomo.make_shared_rhs("ct32", nrhs, seed=5100)
    K = 30
    b = np.concatenate([P.b for P in Ps])
    with lslu.shared_rhs(Ps[0], nrhs, vt, K) as bs:
        r = bs.solve(b, K, "gcv")
        r2 = bs.solve(b, K, "gcv")  # graph replay
    for p, P in enumerate(Ps):
        s = single(P, vt, K, "gcv")
        assert r["status"][p] == s["status"] and r["k_done"][p] == s["k_done"]
        assert np.array_equal(r["gp"][p], s["gp"]) and np.array_equal(r["tp"][p], s["tp"])
        assert np.array_equal(r["x"][p], s["x"]), p
        assert np.array_equal(r2["x"][p], s["x"])


def test_shared_matrix_breakdown_is_local():
    Ps = tomo.make_shared_rhs("ct32", 4, seed=5200)
    bs_ = [P.b for P in Ps]
    bs_[1] = np.zeros(Ps[1].m)
    with lslu.shared_rhs(Ps[0], 4, "f32", 12) as bs:
        r = bs.solve(np.concatenate(bs_), 12, "wgcv")
    assert r["status"][1] == lslu.BREAKDOWN_BETA and np.all(r["x"][1] == 0.0)
    for p in (0, 2, 3):
        s = single(Ps[p], "f32", 12, "wgcv")
        assert np.array_equal(r["x"][p], s["x"])


@pytest.mark.parametrize("kind", ["tiles", "random"])
def test_batched_renumbered_equals_single_renumbered(small_batch, kind):
    """lslu_create_batched_ordered: every problem renumbered inside its own
    range gives, bit for bit, the single-problem renumbered handle's solve
    (same stored rows, same kernels), with x and pivots in the caller's
    numbering."""
    K = 30
    rng = np.random.default_rng(31)
    orders = [tomo.locality_order(P) if kind == "tiles" else
              (rng.permutation(P.m), rng.permutation(P.n)) for P in small_batch]
    b = np.concatenate([P.b for P in small_batch])
    with lslu.from_problems(small_batch, "f32", K, orders=orders) as bs:
        r = bs.solve(b, K, "gcv")
    with lslu.from_problems(small_batch, "f32", K) as bn:
        r0 = bn.solve(b, K, "gcv")
    for p, P in enumerate(small_batch):
        with lslu.from_problem(P, "f32", K, order=orders[p]) as s:
            q = s.solve(P.b, K, "gcv")
        assert r["status"][p] == q["status"] and r["k_done"][p] == q["k_done"]
        assert np.array_equal(r["gp"][p], q["gp"]) and np.array_equal(r["tp"][p], q["tp"])
        assert np.array_equal(r["x"][p], q["x"]), p
        # and, with no tied pivot search, the natural batch up to FP32 rounding
        # (each is within 2e-4 of the FP64 oracle, test_batched_vs_oracle)
        assert np.array_equal(r["gp"][p][:5], r0["gp"][p][:5])
        assert rel(r["x"][p], r0["x"][p]) <= 4e-4


def test_batched_order_must_stay_in_its_problem(small_batch):
    """A permutation that swaps row 0 of problem 0 with row 0 of problem 1 is
    refused; so is a shared-matrix order that is not a permutation."""
    P0, P1 = small_batch[0], small_batch[1]
    ro0 = np.arange(P0.m)
    ro0[0] = P0.m  # stacked with offset 0: global row P0.m (problem 1)
    ro1 = np.arange(P1.m)
    ro1[0] = -P0.m  # stacked with offset P0.m: global row 0 (problem 0)
    with pytest.raises(lslu.LsluError, match="onto themselves"):
        lslu.from_problems([P0, P1], "f32", 5, orders=[(ro0, None), (ro1, None)])
    bad = np.zeros(P0.m, np.int32)
    with pytest.raises(lslu.LsluError, match="permutation"):
        lslu.shared_rhs(P0, 2, "f32", 5, order=(bad, None))


def test_batched_renumbered_ties_follow_the_caller_numbering():
    """Two copies of the hand-worked W-step breakdown (A = diag(1, 2) padded to
    4 x 3, b = ones: the first row pivot is a four-way tie), renumbered in
    reverse: every pivot, tie included, is the natural batch's."""
    rp = np.array([0, 1, 2, 2, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    v = np.array([1.0, 2.0])
    csr = [(4, 3, rp, ci, v), (4, 3, rp, ci, 2.0 * v)]
    rev = (np.array([3, 2, 1, 0]), np.array([2, 1, 0]))
    b = np.ones(8)
    with lslu.BatchedSolver(csr, "f32", 5) as bn, \
            lslu.BatchedSolver(csr, "f32", 5, orders=[rev, rev]) as bo:
        r0 = bn.solve(b, 5, "none")
        r1 = bo.solve(b, 5, "none")
    assert np.array_equal(r0["status"], r1["status"]) and np.array_equal(r0["k_done"],
                                                                          r1["k_done"])
    assert np.array_equal(r0["gp"], r1["gp"]) and np.array_equal(r0["tp"], r1["tp"])
    assert r1["tp"][0][0] == 0 and r1["tp"][1][0] == 0
    for p in range(2):
        assert np.allclose(r0["x"][p], r1["x"][p], rtol=1e-6, atol=0)


@pytest.mark.parametrize("nrhs", [3, 16])
def test_shared_matrix_renumbered_equals_single_renumbered(nrhs):
    """lslu_create_shared_ordered: the one matrix renumbered for every
    right-hand side gives each the renumbered single-problem result bit for
    bit, x and pivots in the caller's numbering."""
    Ps = tomo.make_shared_rhs("ct32", nrhs, seed=5300)
    K = 30
    order = tomo.locality_order(Ps[0])
    b = np.concatenate([P.b for P in Ps])
    with lslu.shared_rhs(Ps[0], nrhs, "f32", K, order=order) as bs:
        r = bs.solve(b, K, "gcv")
    for p, P in enumerate(Ps):
        with lslu.from_problem(P, "f32", K, order=order) as s:
            q = s.solve(P.b, K, "gcv")
        assert r["status"][p] == q["status"] and r["k_done"][p] == q["k_done"]
        assert np.array_equal(r["gp"][p], q["gp"]) and np.array_equal(r["tp"][p], q["tp"])
        assert np.array_equal(r["x"][p], q["x"]), p
