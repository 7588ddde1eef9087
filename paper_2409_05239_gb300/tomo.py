"""Seeded synthetic 2-D parallel-beam tomography inputs.

This module produces the workloads that both the CUDA path and the CPU oracle
consume: a sparse system matrix A (CSR, ray-pixel intersection lengths), a
seeded ellipse phantom x_true and noisy data b = A x_true + e.  It holds none
of the solver's arithmetic and imports nothing but numpy.

The workload stands in for the IR Tools PRtomo test problem that the paper
uses in Section 4 (a 256x256 image, A of size 65160 x 65536, noise level
||e|| / ||A x_true|| = 1e-2); that package and its data are not used here.

Geometry (all sizes in pixel units):
  * the image is N x N unit pixels covering [-N/2, N/2]^2; pixel j = iy*N + ix
    covers x in [-N/2+ix, -N/2+ix+1], y in [-N/2+iy, -N/2+iy+1];
  * projection angle a = 0..n_ang-1 has theta_a = a*pi/n_ang and ray
    direction (cos theta, sin theta);
  * ray r = 0..p-1 passes through s_r * (-sin theta, cos theta) with
    s_r = r - (p-1)/2 (unit detector spacing, centred);
  * row index of A is a*p + r; A[row, j] is the length of the ray inside
    pixel j (Siddon's method: the ray is cut at every grid line it crosses).
Phantom: a sum of E ellipses in normalised coordinates [-1,1]^2 with centres
U[-0.6,0.6]^2, semi-axes U[0.05,0.4], orientation U[0,pi) and intensity U[0,1];
a pixel whose centre lies inside an ellipse receives its intensity.
Noise: e = eta * ||A x_true|| * z / ||z|| with z ~ N(0, I).
Seeds: numpy PCG64; phantom seed = 1000*config + instance, noise seed = phantom
seed + 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "TomoProblem",
    "siddon_csr",
    "ellipse_phantom",
    "make_problem",
    "same_matrix",
    "CONFIGS",
    "round_values",
    "csr_matvec_f64",
    "locality_order",
]


@dataclasses.dataclass
class TomoProblem:
    """A CSR system matrix with its phantom and data (all FP64 on the host)."""

    N: int
    n_ang: int
    p: int
    m: int
    n: int
    row_ptr: np.ndarray  # int64, m+1
    col_idx: np.ndarray  # int32, nnz (sorted within each row)
    vals: np.ndarray     # float64, nnz
    x_true: np.ndarray   # float64, n
    b_clean: np.ndarray  # float64, m
    b: np.ndarray        # float64, m
    eta: float
    seed: int

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def scipy(self, vals=None):
        import scipy.sparse as sp

        v = self.vals if vals is None else vals
        return sp.csr_matrix((v, self.col_idx, self.row_ptr), shape=(self.m, self.n))


def _siddon_angle(N: int, theta: float, s: np.ndarray):
    """Intersections of the parallel rays s at angle theta with the pixel grid.

    Returns (ray, pixel, length) triples with ray local to this angle.
    """
    half = 0.5 * N
    c, sn = math.cos(theta), math.sin(theta)
    px = -s * sn
    py = s * c
    p = s.shape[0]
    grid = np.arange(N + 1, dtype=np.float64) - half
    eps = 1e-12
    t_parts = []
    t_lo = np.full(p, -np.inf)
    t_hi = np.full(p, np.inf)
    inside = np.ones(p, dtype=bool)
    for (dcomp, pcomp) in ((c, px), (sn, py)):
        if abs(dcomp) > eps:
            t = (grid[None, :] - pcomp[:, None]) / dcomp
            t_parts.append(t)
            lo = np.minimum(t[:, 0], t[:, -1])
            hi = np.maximum(t[:, 0], t[:, -1])
            t_lo = np.maximum(t_lo, lo)
            t_hi = np.minimum(t_hi, hi)
        else:
            # the ray is parallel to these grid lines: it is inside the
            # slab only when its fixed coordinate lies strictly inside
            inside &= np.abs(pcomp) < half
    inside &= t_hi > t_lo
    T = np.concatenate(t_parts, axis=1)
    T = np.clip(T, t_lo[:, None], t_hi[:, None])
    T = np.concatenate([t_lo[:, None], T, t_hi[:, None]], axis=1)
    T.sort(axis=1)
    seg = np.diff(T, axis=1)
    tm = 0.5 * (T[:, 1:] + T[:, :-1])
    ix = np.floor(px[:, None] + tm * c + half).astype(np.int64)
    iy = np.floor(py[:, None] + tm * sn + half).astype(np.int64)
    keep = (seg > 1e-10) & inside[:, None] & (ix >= 0) & (ix < N) & (iy >= 0) & (iy < N)
    ray = np.broadcast_to(np.arange(p)[:, None], seg.shape)[keep]
    pix = (iy * N + ix)[keep]
    return ray, pix, seg[keep]


def siddon_csr(N: int, n_ang: int, p: int):
    """CSR (row_ptr int64, col_idx int32, vals float64) of the projector.

    Within each row the column indices are sorted ascending; pieces of one
    chord that fall in the same pixel are merged into one entry.
    """
    s = np.arange(p, dtype=np.float64) - 0.5 * (p - 1)
    cols_all, vals_all = [], []
    counts = np.zeros(n_ang * p, dtype=np.int64)
    for a in range(n_ang):
        theta = a * math.pi / n_ang
        ray, pix, seg = _siddon_angle(N, theta, s)
        key = ray * (N * N) + pix
        order = np.argsort(key, kind="stable")
        key = key[order]
        seg = seg[order]
        first = np.ones(key.shape[0], dtype=bool)
        first[1:] = key[1:] != key[:-1]
        starts = np.flatnonzero(first)
        if starts.size:
            seg = np.add.reduceat(seg, starts)
        key = key[starts]
        counts[a * p:(a + 1) * p] = np.bincount(key // (N * N), minlength=p)
        cols_all.append((key % (N * N)).astype(np.int32))
        vals_all.append(seg.astype(np.float64))
    row_ptr = np.zeros(n_ang * p + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, np.concatenate(cols_all), np.concatenate(vals_all)


def locality_order(P: "TomoProblem", pixel_tile=(2, 4), ray_tile=(4, 2)):
    """A renumbering of the unknowns and the rays that keeps neighbours close in
    memory (for lslu_create_ordered): pixels in tiles of pixel_tile = (w, h)
    pixels (w along x, h along y), the tiles row by row; rays in tiles of
    ray_tile = (a, r) = a consecutive angles x r neighbouring rays, the tiles
    of a block of a angles ray by ray.  A ray then meets a few pixels of each
    tile it crosses, and a pixel a few rays of each tile of the sinogram.
    Returns (row_order, col_order), int32: caller row i -> internal row
    row_order[i], caller column j -> internal column col_order[j].  Partial
    tiles at the edges are kept whole."""
    tw, th = pixel_tile
    wa, wr = ray_tile
    j = np.arange(P.N * P.N)
    ix, iy = j % P.N, j // P.N
    cols = np.lexsort((ix % tw, iy % th, ix // tw, iy // th))
    i = np.arange(P.n_ang * P.p)
    a, r = i // P.p, i % P.p
    rows = np.lexsort((r % wr, a % wa, r // wr, a // wa))
    col_order = np.empty(P.n, dtype=np.int32)
    col_order[cols] = np.arange(P.n, dtype=np.int32)
    row_order = np.empty(P.m, dtype=np.int32)
    row_order[rows] = np.arange(P.m, dtype=np.int32)
    return row_order, col_order


def ellipse_phantom(N: int, n_ellipses: int, rng: np.random.Generator) -> np.ndarray:
    """Sum of random ellipses sampled at pixel centres, length N*N (row-major)."""
    coords = (np.arange(N, dtype=np.float64) + 0.5 - 0.5 * N) / (0.5 * N)
    X, Y = np.meshgrid(coords, coords, indexing="xy")  # Y varies along rows (iy)
    img = np.zeros((N, N), dtype=np.float64)
    for _ in range(n_ellipses):
        cx, cy = rng.uniform(-0.6, 0.6, size=2)
        ax, ay = rng.uniform(0.05, 0.4, size=2)
        phi = rng.uniform(0.0, math.pi)
        inten = rng.uniform(0.0, 1.0)
        dx, dy = X - cx, Y - cy
        u = dx * math.cos(phi) + dy * math.sin(phi)
        v = -dx * math.sin(phi) + dy * math.cos(phi)
        img[(u / ax) ** 2 + (v / ay) ** 2 <= 1.0] += inten
    return img.reshape(-1)


def csr_matvec_f64(row_ptr, col_idx, vals, x):
    """y = A x for a CSR matrix in FP64 (numpy, used to synthesise data)."""
    m = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    return np.bincount(rows, weights=vals * x[col_idx], minlength=m)


def make_problem(N: int, n_ang: int, p: int, n_ellipses: int, eta: float,
                 seed: int) -> TomoProblem:
    """Projector, phantom and noisy data for one seeded instance."""
    row_ptr, col_idx, vals = siddon_csr(N, n_ang, p)
    rng = np.random.Generator(np.random.PCG64(seed))
    x_true = ellipse_phantom(N, n_ellipses, rng)
    b_clean = csr_matvec_f64(row_ptr, col_idx, vals, x_true)
    nrng = np.random.Generator(np.random.PCG64(seed + 1))
    z = nrng.standard_normal(b_clean.shape[0])
    e = eta * np.linalg.norm(b_clean) * z / np.linalg.norm(z)
    return TomoProblem(N=N, n_ang=n_ang, p=p, m=n_ang * p, n=N * N,
                       row_ptr=row_ptr, col_idx=col_idx, vals=vals,
                       x_true=x_true, b_clean=b_clean, b=b_clean + e,
                       eta=eta, seed=seed)


# Workloads: image size N, angles, rays per angle, ellipses, noise levels.
CONFIGS = {
    # 32x32 image, 45 angles x 46 rays, 5 ellipses, 1% noise, FP64, 50 iterations
    "ct32": dict(N=32, n_ang=45, p=46, n_ellipses=5, etas=(0.01,), seed_base=1000, K=50),
    # 256x256 image, 180 angles x 362 rays, 5 ellipses, 1% noise, FP32, 200 iterations
    "ct256": dict(N=256, n_ang=180, p=362, n_ellipses=5, etas=(0.01,), seed_base=2000, K=200),
    # 512x512 image, 360 angles x 724 rays, 20 ellipses, 0.5% and 2% noise, 300 iterations
    "ct512": dict(N=512, n_ang=360, p=724, n_ellipses=20, etas=(0.005, 0.02), seed_base=3000, K=300),
}


def make_config(name: str, instance: int = 0, eta: float | None = None) -> TomoProblem:
    c = CONFIGS[name]
    e = c["etas"][0] if eta is None else eta
    return make_problem(c["N"], c["n_ang"], c["p"], c["n_ellipses"], e,
                        seed=c["seed_base"] + instance)


def same_matrix(P: TomoProblem, seed: int, eta: float, n_ellipses: int) -> TomoProblem:
    """Another seeded instance on P's projector: a phantom of n_ellipses drawn
    from PCG64(seed) and noise at level eta from PCG64(seed + 1), as
    make_problem draws them (so same_matrix(P, s, eta, E) equals
    make_problem(P.N, P.n_ang, P.p, E, eta, s) without rebuilding A)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x_true = ellipse_phantom(P.N, n_ellipses, rng)
    b_clean = csr_matvec_f64(P.row_ptr, P.col_idx, P.vals, x_true)
    nrng = np.random.Generator(np.random.PCG64(seed + 1))
    z = nrng.standard_normal(b_clean.shape[0])
    e = eta * np.linalg.norm(b_clean) * z / np.linalg.norm(z)
    return TomoProblem(N=P.N, n_ang=P.n_ang, p=P.p, m=P.m, n=P.n, row_ptr=P.row_ptr,
                       col_idx=P.col_idx, vals=P.vals, x_true=x_true, b_clean=b_clean,
                       b=b_clean + e, eta=eta, seed=seed)


def round_values(vals: np.ndarray, value_type: str) -> np.ndarray:
    """FP64 copy of vals rounded to the storage type (round to nearest even).

    'f64' returns vals unchanged, 'f32' rounds to binary32, 'bf16' rounds to
    binary32 first and then to bfloat16 (the upper 16 bits of binary32, round
    to nearest, ties to even).  Finite inputs only.
    """
    if value_type == "f64":
        return np.asarray(vals, dtype=np.float64)
    f = np.asarray(vals, dtype=np.float32)
    if value_type == "f32":
        return f.astype(np.float64)
    if value_type == "bf16":
        u = f.view(np.uint32).astype(np.uint64)
        lsb = (u >> 16) & 1
        r = ((u + 0x7FFF + lsb) >> 16) << 16
        return r.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(f"unknown value type {value_type!r}")


def bf16_bits(vals: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of round_values(vals, 'bf16')."""
    r = round_values(vals, "bf16").astype(np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


def make_uneven_batch(count: int = 64, seed: int = 4000, N_range=(64, 256),
                      ang_range=(30, 180), eta_range=(0.005, 0.03),
                      n_ellipses: int = 5) -> list[TomoProblem]:
    """Independent problems of uneven size for a batched solve: image side N
    and angle count drawn uniformly from the inclusive ranges, round(1.41 N)
    rays per angle, and each problem's own seeded phantom and noise level
    (uniform in eta_range)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        n_ang = int(rng.integers(ang_range[0], ang_range[1] + 1))
        eta = float(rng.uniform(eta_range[0], eta_range[1]))
        out.append(make_problem(N, n_ang, int(round(1.41 * N)), n_ellipses, eta,
                                seed=seed + 10 * (i + 1)))
    return out


def make_shared_rhs(name: str = "ct256", nrhs: int = 16, seed: int = 5000) -> list[TomoProblem]:
    """nrhs right-hand sides for one projector: the workload's A with a
    different seeded phantom and noise draw per right-hand side."""
    c = CONFIGS[name]
    base = make_problem(c["N"], c["n_ang"], c["p"], c["n_ellipses"], c["etas"][0], seed)
    out = [base]
    for r in range(1, nrhs):
        rng = np.random.Generator(np.random.PCG64(seed + 10 * r))
        x_true = ellipse_phantom(c["N"], c["n_ellipses"], rng)
        b_clean = csr_matvec_f64(base.row_ptr, base.col_idx, base.vals, x_true)
        nrng = np.random.Generator(np.random.PCG64(seed + 10 * r + 1))
        z = nrng.standard_normal(b_clean.shape[0])
        e = c["etas"][0] * np.linalg.norm(b_clean) * z / np.linalg.norm(z)
        out.append(TomoProblem(N=base.N, n_ang=base.n_ang, p=base.p, m=base.m, n=base.n,
                               row_ptr=base.row_ptr, col_idx=base.col_idx, vals=base.vals,
                               x_true=x_true, b_clean=b_clean, b=b_clean + e,
                               eta=base.eta, seed=seed + 10 * r))
    return out
