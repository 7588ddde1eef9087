"""Pins of the seeded tomography inputs (Siddon projector, phantom, noise)."""
import math

import numpy as np
import pytest

from paper_2409_05239_gb300 import tomo


def _dense(N, n_ang, p):
    rp, ci, v = tomo.siddon_csr(N, n_ang, p)
    A = np.zeros((n_ang * p, N * N))
    for r in range(n_ang * p):
        A[r, ci[rp[r]:rp[r + 1]]] = v[rp[r]:rp[r + 1]]
    return rp, ci, v, A


def test_csr_well_formed():
    rp, ci, v = tomo.siddon_csr(16, 9, 24)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == ci.shape[0]
    assert ci.dtype == np.int32 and ci.min() >= 0 and ci.max() < 256
    assert np.all(v > 0) and np.all(v <= math.sqrt(2) + 1e-12)
    for r in range(rp.shape[0] - 1):
        seg = ci[rp[r]:rp[r + 1]]
        assert np.all(np.diff(seg) > 0), "columns not strictly increasing in a row"


def test_angle_zero_covers_each_pixel_once():
    """At theta = 0 with an even ray count the rays run along pixel-row centres,
    so every pixel is crossed by exactly one ray with length 1."""
    N, p = 12, 16
    _, _, _, A = _dense(N, 4, p)
    assert np.allclose(A[:p].sum(axis=0), 1.0, atol=1e-12)
    assert np.allclose(A[2 * p:3 * p].sum(axis=0), 1.0, atol=1e-12)  # theta = 90 deg


@pytest.mark.parametrize("N,p", [(8, 12), (10, 15)])
def test_chord_lengths_45_degrees(N, p):
    """At 45 degrees the ray with offset s crosses the square [-h, h]^2 over a
    chord of length 2 sqrt(2) h - 2|s| (|s| < sqrt(2) h)."""
    _, _, _, A = _dense(N, 4, p)
    h = N / 2
    s = np.arange(p) - (p - 1) / 2
    chord = np.maximum(0.0, 2 * math.sqrt(2) * h - 2 * np.abs(s))
    assert np.allclose(A[p:2 * p].sum(axis=1), chord, atol=1e-10)


def test_siddon_against_sampling():
    """Brute force: walk each ray in tiny steps and bin the steps by pixel."""
    N, n_ang, p = 6, 7, 9
    _, _, _, A = _dense(N, n_ang, p)
    h = N / 2
    step = 2e-4
    t = np.arange(-2 * N, 2 * N, step) + step / 2
    for a in range(n_ang):
        th = a * math.pi / n_ang
        for r in range(p):
            s = r - (p - 1) / 2
            x = -s * math.sin(th) + t * math.cos(th)
            y = s * math.cos(th) + t * math.sin(th)
            ok = (x > -h) & (x < h) & (y > -h) & (y < h)
            ix = np.floor(x[ok] + h).astype(int)
            iy = np.floor(y[ok] + h).astype(int)
            est = np.bincount(iy * N + ix, minlength=N * N) * step
            assert np.allclose(A[a * p + r], est, atol=4 * step)


def test_phantom_and_noise_level():
    P = tomo.make_problem(16, 10, 24, 5, 0.02, seed=42)
    assert P.x_true.shape == (256,) and P.x_true.min() >= 0.0 and P.x_true.max() > 0.0
    assert P.x_true.max() <= 5.0
    rel = np.linalg.norm(P.b - P.b_clean) / np.linalg.norm(P.b_clean)
    assert abs(rel - 0.02) < 1e-12
    A = P.scipy()
    assert np.allclose(A @ P.x_true, P.b_clean, rtol=1e-13, atol=1e-13)


def test_seeded_reproducible():
    a = tomo.make_problem(16, 10, 24, 5, 0.01, seed=7)
    b = tomo.make_problem(16, 10, 24, 5, 0.01, seed=7)
    c = tomo.make_problem(16, 10, 24, 5, 0.01, seed=8)
    assert np.array_equal(a.b, b.b) and np.array_equal(a.x_true, b.x_true)
    assert not np.array_equal(a.x_true, c.x_true)


def test_config_shapes():
    P = tomo.make_config("ct32")
    assert (P.m, P.n) == (2070, 1024)
    assert 55000 < P.nnz < 62000


def test_round_values_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.uniform(0, 1.5, 10000), rng.standard_normal(1000) * 1e3,
                        [0.0, 1.0, 1.00390625, 1.005859375, 2.0 ** -20]])
    mine = tomo.round_values(v, "bf16")
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mine, ref)
    assert np.array_equal(tomo.round_values(v, "f32"), v.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("N,n_ang,p", [(32, 45, 46), (13, 7, 19)])
def test_locality_order_tiles(N, n_ang, p):
    """Both orders are permutations; away from the edges the 2x4 pixels of a
    tile, and the 4 angles x 2 rays of a sinogram tile, take consecutive
    internal indices (partial tiles at ragged edges stay whole)."""
    P = tomo.make_problem(N, n_ang, p, 3, 0.01, seed=1)
    ro, co = tomo.locality_order(P)
    assert ro.dtype == np.int32 and co.dtype == np.int32
    assert np.array_equal(np.sort(ro), np.arange(P.m))
    assert np.array_equal(np.sort(co), np.arange(P.n))
    # pixel j = iy*N + ix; tile (tx, ty) covers ix in [2tx, 2tx+2), iy in [4ty, 4ty+4)
    for ty in range(N // 4):
        for tx in range(N // 2):
            idx = [co[(4 * ty + dy) * N + 2 * tx + dx] for dy in range(4) for dx in range(2)]
            assert idx == list(range(idx[0], idx[0] + 8))
    for ta in range(n_ang // 4):
        for tr in range(p // 2):
            idx = [ro[(4 * ta + da) * p + 2 * tr + dr] for da in range(4) for dr in range(2)]
            assert idx == list(range(idx[0], idx[0] + 8))
    # every partial tile is contiguous too
    cells = {}
    for j in range(P.n):
        cells.setdefault(((j // N) // 4, (j % N) // 2), []).append(co[j])
    for v in cells.values():
        assert sorted(v) == list(range(min(v), min(v) + len(v)))


def test_same_matrix_equals_make_problem():
    """Another instance on the same projector draws phantom and noise exactly
    as make_problem does with that seed and noise level."""
    P = tomo.make_problem(20, 12, 28, 3, 0.01, seed=9)
    Q = tomo.same_matrix(P, seed=17, eta=0.02, n_ellipses=4)
    R = tomo.make_problem(20, 12, 28, 4, 0.02, seed=17)
    assert np.array_equal(Q.x_true, R.x_true) and np.array_equal(Q.b, R.b)
    assert Q.row_ptr is P.row_ptr and Q.eta == 0.02 and Q.seed == 17
