"""Every row shape of the sparse products (lanes per row x chunks in flight,
32-bit columns or 16-bit offsets) through the C ABI (lslu_set_spmv_shape,
lslu_spmv) against the FP64 product of scipy within the rounding bound of the
accumulation type, on matrices with empty rows, rows of mixed length (ragged
ends of the 8-entry units and of the 64-entry transposed blocks), one long
row and many one-entry rows; and the refusal of an out-of-range shape."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2409_05239_gb300 import lslu

pytestmark = pytest.mark.gpu

NSHAPES = len(lslu.Solver.SHAPES)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_05239_gb300 import build

    build.build()


def random_csr(m, n, lens, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for r, L in enumerate(lens):
        c = rng.choice(n, size=L, replace=False)
        rows.append(np.full(L, r))
        cols.append(np.sort(c))
    r = np.concatenate(rows) if rows else np.zeros(0, int)
    c = np.concatenate(cols) if cols else np.zeros(0, int)
    v = rng.uniform(-1.0, 1.0, size=r.shape[0])
    return sp.csr_matrix((v, (r, c)), shape=(m, n))


def product(A, vt, shape, x, transpose=False):
    import torch

    A = A.tocsr()
    dev = torch.device("cuda", 0)
    dt = torch.float64 if vt == "f64" else torch.float32
    s = lslu.Solver(A.shape[0], A.shape[1], A.indptr.astype(np.int64), A.indices.astype(np.int32),
                    A.data, vt, 8)
    try:
        s.set_spmv_shape(shape, shape)
        xin = torch.tensor(x, dtype=dt, device=dev)
        y = torch.zeros(A.shape[1] if transpose else A.shape[0], dtype=dt, device=dev)
        s.spmv(1 if transpose else 0, xin, y)
        y2 = torch.zeros_like(y)
        s.spmv(1 if transpose else 0, xin, y2)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.float64), y2.cpu().numpy().astype(np.float64)
    finally:
        s.close()


def stored(A, vt):
    """A with the values the library stores for this value type."""
    B = A.copy().astype(np.float64)
    if vt == "f32":
        B.data = B.data.astype(np.float32).astype(np.float64)
    elif vt == "bf16":
        import torch

        B.data = torch.tensor(B.data, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    return B


def check(A, vt, shape, seed=0, transpose=False):
    rng = np.random.default_rng(seed)
    n_in = A.shape[0] if transpose else A.shape[1]
    x = rng.standard_normal(n_in)
    xs = x if vt == "f64" else x.astype(np.float32).astype(np.float64)
    y, y2 = product(A, vt, shape, x, transpose)
    M = stored(A, vt)
    M = M.T.tocsr() if transpose else M
    ref = M @ xs
    scale = abs(M) @ np.abs(xs)
    # rounding bound of a recursive FMA sum of len terms in the accumulation
    # type (the values and x are stored exactly): (len + 2) u sum |a_i x_i|
    u = 2.0 ** -53 if vt == "f64" else 2.0 ** -24
    lens = np.diff(M.indptr)
    bound = (lens + 2) * u * scale
    assert np.all(np.abs(y - ref) <= bound), np.max(np.abs(y - ref) - bound)
    assert np.array_equal(y, y2)  # bitwise reproducible


@pytest.mark.parametrize("vt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape", range(NSHAPES))
def test_rows_of_mixed_length_and_empty_rows(vt, shape):
    rng = np.random.default_rng(1)
    lens = rng.integers(0, 300, size=3000)
    lens[rng.random(3000) < 0.1] = 0
    lens[:5] = 0
    lens[-7:] = 0
    A = random_csr(3000, 2000, lens, seed=2)
    check(A, vt, shape, seed=3)
    check(A, vt, shape, seed=4, transpose=True)


@pytest.mark.parametrize("shape", range(NSHAPES))
def test_many_one_entry_rows(shape):
    n = 20000
    A = sp.diags(np.linspace(1.0, 2.0, n)).tocsr() + sp.eye(n, k=7, format="csr")
    check(A.tocsr(), "f32", shape, seed=5)


@pytest.mark.parametrize("shape", [0, 6, 12, 13])
def test_one_long_row(shape):
    """One row of 4099 entries (many 64-entry blocks and a ragged tail) among
    short rows."""
    lens = np.full(600, 5)
    lens[300] = 4099
    A = random_csr(600, 8192, lens, seed=6)
    check(A, "f32", shape, seed=7)
    check(A, "f64", shape, seed=8, transpose=True)


def test_shape_out_of_range_refused():
    lens = np.full(100, 3)
    A = random_csr(100, 400, lens, seed=8)
    s = lslu.Solver(100, 400, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data,
                    "f32", 8)
    try:
        with pytest.raises(lslu.LsluError, match=r"\[0, 16\)"):
            s.set_spmv_shape(NSHAPES, 0)
        t = s.tune_spmv(reps=1)
        assert set(t["us_A"]) <= set(lslu.Solver.SHAPES) and 0 <= t["shape_A"] < NSHAPES
    finally:
        s.close()
