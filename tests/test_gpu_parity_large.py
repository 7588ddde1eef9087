"""Parity at the benchmark's sizes.

* 256x256 workload (m = 65160, n = 65536, ~15M non-zeros) in FP64 against the
  FP64 oracle: identical pivots, x_K within 1e-10.
* 512x512 workload (m = 260640, n = 262144, ~120M non-zeros, K = 300, FP32
  values and basis, GCV) in the launch configuration the benchmark times
  (autotuned shapes; natural numbering and the renumbered handle),
  checked through properties that hold at any size and on sampled outputs the
  oracle computes one by one:
    - exact pivot structure of every basis vector (Algorithm 4);
    - the recurrences A l_j = D_{j+1} H(:, j) and A^T d_j = L_j W(:, j)
      (Eqs. nhr, nhr2) on sampled columns, recomputed in FP64 on the host;
    - the projected solve on the GPU's own H against the oracle's SVD-based
      solve of that H (FP64 on both sides);
    - x = L y recomputed in FP64 from the exported basis.
"""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import lslu, tomo

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_05239_gb300 import build

    build.build()


def test_ct256_f64_parity():
    """Algorithm 4 amplifies rounding differences on this workload: two FP64
    runs of the oracle that differ only in summation order drift apart by
    ~100x every 2-3 iterations past k ~ 10 and pick different pivots at
    k = 26.  So the GPU must (a) keep the oracle's pivots about as long as the
    oracle keeps its own, (b) match x to within 10x of the oracle's
    self-difference while the pivots agree, and (c) give the same
    reconstruction quality at K = 80."""
    from oracle.perturb import PermutedOperator, first_difference

    P = tomo.make_config("ct256")
    A = P.scipy()
    Ap = PermutedOperator(A)
    K = 40
    ref = O.hessenberg_rect_pivoted(A, P.b, None, K)
    alt = O.hessenberg_rect_pivoted(Ap, P.b, None, K)
    with lslu.from_problem(P, "f64", 80) as s:
        r = s.solve(P.b, K, "gcv")
        self_div = first_difference(ref["gp"], alt["gp"])
        gpu_div = first_difference(ref["gp"], r["gp"])
        # the divergence point is set by rounding noise growth: within a few
        # iterations of the oracle's own (26 for three different permutations)
        assert gpu_div >= min(self_div, K) - 3, (gpu_div, self_div)
        Ks = 12
        x_ref = O.hybrid_lslu(A, P.b, None, Ks, "gcv", histories=False).x
        x_alt = O.hybrid_lslu(Ap, P.b, None, Ks, "gcv", histories=False).x
        rs = s.solve(P.b, Ks, "gcv")
        tol = max(1e-10, 10 * rel(x_alt, x_ref))
        assert rel(rs["x"], x_ref) <= tol
        r80 = s.solve(P.b, 80, "gcv")
    e_ref = np.linalg.norm(O.hybrid_lslu(A, P.b, None, 80, "gcv", histories=False).x - P.x_true)
    e_gpu = np.linalg.norm(r80["x"] - P.x_true)
    # permuted-oracle runs land within 3% of the oracle's error
    assert abs(e_gpu - e_ref) <= 0.08 * e_ref


def test_ct256_f32_k200_against_oracle():
    """The 256x256 workload in its named configuration (FP32 values and
    basis, K = 200, GCV) against the FP64 oracle on the same FP32-rounded
    matrix, through the whole run.  The FP64 oracle itself is stable here
    (a permuted summation order, or b perturbed by 2^-24 per entry, keeps all
    200 pivot pairs and moves x by < 1e-5), but FP32 rounding in every step of
    the recurrence grows ~100x every few iterations: the GPU's pivots leave
    the oracle's at k = 18-19 (measured, both numberings) and x_200 differs
    by 3.9-4.0%, with the reconstruction error within 3.5% of the oracle's
    (12.95% / 13.36% against 12.91%).  The bars: the first 12 pivot pairs
    identical, x within 8%, reconstruction error within 8% of the oracle's."""
    from oracle.perturb import first_difference

    P = tomo.make_config("ct256")
    K = 200
    A = P.scipy(tomo.round_values(P.vals, "f32"))
    ref = O.hybrid_lslu(A, P.b, None, K, "gcv", histories=False)
    e_ref = np.linalg.norm(ref.x - P.x_true) / np.linalg.norm(P.x_true)
    for order in (None, tomo.locality_order(P)):
        with lslu.from_problem(P, "f32", K, order=order) as s:
            r = s.solve(P.b, K, "gcv")
        assert r["status"] == lslu.OK and r["k_done"] == K
        assert first_difference(r["gp"], ref.gp) >= 12 and first_difference(r["tp"], ref.tp) >= 12
        assert rel(r["x"], ref.x) <= 0.08
        e = np.linalg.norm(r["x"] - P.x_true) / np.linalg.norm(P.x_true)
        assert abs(e - e_ref) <= 0.08 * e_ref, (e, e_ref)


@pytest.fixture(scope="module", params=["natural", "tiles"])
def ct512_run(request):
    """The benchmark's solve: autotuned product shapes, the matrix as numbered
    or renumbered by tomo.locality_order (lslu_create_ordered; vectors, bases
    and pivots come back in the natural numbering, so every check below reads
    the same)."""
    P = tomo.make_config("ct512")
    K = 300
    order = tomo.locality_order(P) if request.param == "tiles" else None
    with lslu.from_problem(P, "f32", K, order=order) as s:
        s.tune_spmv(reps=2)
        r = s.solve(P.b, K, "gcv")
        st = s.state(r["k_done"])
    return P, K, r, st


def test_ct512_exact_structure(ct512_run):
    P, K, r, st = ct512_run
    assert r["status"] == lslu.OK and r["k_done"] == K
    for Bm, piv in ((st["L"], r["gp"]), (st["D"], r["tp"])):
        assert len(set(piv.tolist())) == len(piv)
        for j in range(Bm.shape[1]):
            col = Bm[:, j]
            assert col[piv[j]] == 1.0
            assert np.all(col[piv[:j]] == 0.0)
            assert np.max(np.abs(col)) == 1.0


def test_ct512_recurrences_sampled(ct512_run):
    """A l_j = D_{j+1} H(:, j) and A^T d_j = L_j W(:, j) hold to FP32 rounding
    (basis stored in FP32, accumulation in FP32)."""
    P, K, r, st = ct512_run
    A = P.scipy(tomo.round_values(P.vals, "f32"))
    L = st["L"].astype(np.float64)
    D = st["D"].astype(np.float64)
    nA = np.sqrt(np.sum(A.data ** 2))
    for j in (0, 1, 57, 150, 299):
        lhs = A @ L[:, j]
        rhs = D[:, :j + 2] @ st["H"][:j + 2, j]
        assert np.linalg.norm(lhs - rhs) <= 1e-4 * nA * np.linalg.norm(L[:, j]), j
        lhs2 = A.T @ D[:, j]
        rhs2 = L[:, :j + 1] @ st["W"][:j + 1, j]
        assert np.linalg.norm(lhs2 - rhs2) <= 1e-4 * nA * np.linalg.norm(D[:, j]), j


def test_ct512_projected_and_recombination(ct512_run):
    P, K, r, st = ct512_run
    s_ref, c_ref, V = O.projected_svd(st["H"], st["beta"])
    lam = O.select_lambda(s_ref, c_ref, 1.0)
    y = O.tikhonov_y(s_ref, c_ref, V, lam)
    x_ref = st["L"].astype(np.float64) @ y
    assert rel(r["x"], x_ref) <= 1e-8
    err = np.linalg.norm(r["x"] - P.x_true) / np.linalg.norm(P.x_true)
    assert err < 0.2


@pytest.fixture(scope="module")
def ct512_prefix_ref():
    P = tomo.make_config("ct512")
    K = 12
    A = P.scipy(tomo.round_values(P.vals, "f32"))
    return P, K, O.hybrid_lslu(A, P.b, None, K, "gcv", histories=False)


@pytest.mark.parametrize("order", ["natural", "tiles"])
def test_ct512_mixed_vs_oracle_prefix(ct512_prefix_ref, order):
    """The first 12 iterations of the 512x512 FP32 solve against the FP64 oracle
    on the same FP32-rounded matrix: identical pivots, x within FP32 tolerance
    (the renumbered handle too: its pivots, mapped back, can differ only
    where a search ties)."""
    P, K, ref = ct512_prefix_ref
    o = tomo.locality_order(P) if order == "tiles" else None
    with lslu.from_problem(P, "f32", K, order=o) as s:
        r = s.solve(P.b, K, "gcv")
    assert np.array_equal(r["gp"], ref.gp) and np.array_equal(r["tp"], ref.tp)
    assert rel(r["x"], ref.x) <= 1e-4
