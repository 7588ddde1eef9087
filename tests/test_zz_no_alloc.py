"""The allocation-free projected solve (lslu_projected_noalloc) matches the
handle-based lslu_projected.

Some callers cannot allocate device memory (a framework's memory pool owns
every allocation, or a hot loop cannot take an allocation's synchronisation);
they call lslu_projected_noalloc, whose work space is a fixed device array in
the library.  This file sorts last so that, if it fails, a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import lslu, tomo
from tests import pins

pytestmark = pytest.mark.gpu


def _colmajor(torch, H, dev):
    """H as a column-major FP64 device tensor with leading dimension rows."""
    out = torch.empty_strided(H.shape, (1, H.shape[0]), dtype=torch.float64, device=dev)
    out.copy_(torch.from_numpy(np.ascontiguousarray(H)))
    return out


def _outputs(torch, k, dev):
    return dict(y=torch.zeros(k, dtype=torch.float64, device=dev),
                sigma=torch.zeros(k, dtype=torch.float64, device=dev),
                c=torch.zeros(k + 1, dtype=torch.float64, device=dev),
                lam_out=torch.zeros(1, dtype=torch.float64, device=dev),
                resid_out=torch.zeros(1, dtype=torch.float64, device=dev))


@pytest.mark.parametrize("rule,lam", [("gcv", 0.0), ("fixed", 0.05), ("none", 0.0)])
def test_noalloc_matches_projected(rule, lam):
    import torch

    from paper_2409_05239_gb300 import build

    build.build()
    dev = torch.device("cuda", 0)
    P = tomo.make_config("ct32")
    hp = O.hessenberg_rect_pivoted(P.scipy(), P.b, None, 60)
    with lslu.from_problem(P, "f64", 60) as s:
        for k in (37, 60):  # two calls in a row on the shared work space
            H = hp["H"][:k + 1, :k]
            ref = s.projected(H, hp["beta"], rule, lam)
            Hd = _colmajor(torch, H, dev)
            out = _outputs(torch, k, dev)
            lslu.projected_noalloc(Hd, hp["beta"], rule, lam, P.m, **out)
            torch.cuda.synchronize()
            tol = 1e-10
            assert np.allclose(out["y"].cpu().numpy(), ref["y"], rtol=tol, atol=tol * np.abs(ref["y"]).max())
            assert np.allclose(out["sigma"].cpu().numpy(), ref["sigma"], rtol=tol, atol=0)
            assert np.allclose(out["c"].cpu().numpy(), ref["c"], rtol=tol, atol=tol * abs(hp["beta"]))
            assert abs(out["lam_out"].item() - ref["lam"]) <= tol * max(ref["lam"], 1e-300)
            assert abs(out["resid_out"].item() - ref["resid"]) <= tol * abs(hp["beta"])


def _hessenberg(k, seed):
    """A well-conditioned random (k+1) x k upper Hessenberg matrix."""
    rng = np.random.default_rng(seed)
    H = np.triu(rng.uniform(-1.0, 1.0, size=(k + 1, k)), -1)
    H[np.arange(k), np.arange(k)] += 3.0 * np.sign(H[np.arange(k), np.arange(k)] + 0.5)
    return H


@pytest.mark.parametrize("k", [1, 2, 256])
@pytest.mark.parametrize("rule,lam", [("gcv", 0.0), ("wgcv", 0.0), ("fixed", 0.3), ("none", 0.0)])
def test_noalloc_at_the_edges(k, rule, lam):
    """k = 1, 2 and 256 (the largest problem the fixed array serves; its slot
    then fills most of the array), each called twice in a row after a call of
    another size: bit for bit the handle-based lslu_projected (the same
    kernels on a handle's work space), and the oracle's SVD solve (Eqs. TSP,
    3-4, gcv2, wgcv) within tolerances set by the conditioning of H."""
    import torch

    from paper_2409_05239_gb300 import build

    build.build()
    dev = torch.device("cuda", 0)
    # H and beta of the Hessenberg process on a dense ill-posed problem
    # (decaying singular values give an interior GCV minimum)
    A, _, b = pins.random_problem(600, 300, seed=40 + k, decay=0.97)
    hp = O.hessenberg_rect_pivoted(A, b, None, k)
    assert hp["k"] == k
    m = A.shape[0]
    beta = hp["beta"]
    H = hp["H"]
    s_ref, c_ref, V = O.projected_svd(H, beta)
    lam_ref = O._lambda_for(rule, lam, s_ref, c_ref, k, m)
    y_ref = O.tikhonov_y(s_ref, c_ref, V, lam_ref)
    res_ref = O.projected_residual(s_ref, c_ref, lam_ref)
    P = tomo.make_config("ct32")
    with lslu.from_problem(P, "f64", 256) as s:
        ref_h = s.projected(H, beta, rule, lam, m=m)
    Hd = _colmajor(torch, H, dev)
    other = _colmajor(torch, O.hessenberg_rect_pivoted(A, b, None, 40)["H"], dev)
    lslu.projected_noalloc(other, 1.0, "gcv", 0.0, 500, **_outputs(torch, 40, dev))
    # effective condition of the regularised projected problem: a backward
    # stable solve gets y to about eps * sigma_1 / max(lambda, sigma_k)
    kappa = s_ref[0] / max(lam_ref, s_ref[-1])
    tol_y = max(1e-10, 10.0 * np.finfo(float).eps * kappa)
    for _ in range(2):
        out = _outputs(torch, k, dev)
        lslu.projected_noalloc(Hd, beta, rule, lam, m, **out)
        torch.cuda.synchronize()
        got = {key: v.cpu().numpy() for key, v in out.items()}
        for key, hkey in (("y", "y"), ("sigma", "sigma"), ("c", "c")):
            assert np.array_equal(got[key], np.abs(ref_h[hkey]) if key == "c" else ref_h[hkey])
        assert got["lam_out"][0] == ref_h["lam"] and got["resid_out"][0] == ref_h["resid"]
        assert np.allclose(got["sigma"], s_ref, rtol=1e-12, atol=1e-14 * s_ref[0])
        # two LAPACK SVD drivers differ by 2.2e-14 |beta| in c at k = 256
        assert np.allclose(got["c"], np.abs(c_ref), rtol=1e-10, atol=1e-12 * abs(beta))
        if lam_ref == 0.0:
            assert got["lam_out"][0] == 0.0
        else:
            assert abs(got["lam_out"][0] - lam_ref) <= 1e-8 * lam_ref
        assert np.linalg.norm(got["y"] - y_ref) <= tol_y * np.linalg.norm(y_ref)
        assert abs(got["resid_out"][0] - res_ref) <= 1e-10 * abs(beta)


def test_noalloc_checks_tensor_layouts():
    """The binding refuses layouts the C entry point cannot see through raw
    pointers (a row-major H, a short output), before any launch."""
    import torch

    dev = torch.device("cuda", 0)
    k = 5
    H = torch.from_numpy(_hessenberg(k, 3)).to(dev)  # row-major
    with pytest.raises(ValueError, match="column-major"):
        lslu.projected_noalloc(H, 1.0, "gcv", 0.0, 100)
    Hc = _colmajor(torch, _hessenberg(k, 3), dev)
    with pytest.raises(ValueError, match="at least 6"):
        lslu.projected_noalloc(Hc, 1.0, "gcv", 0.0, 100,
                               c=torch.zeros(k, dtype=torch.float64, device=dev))


def test_noalloc_rejects_k_beyond_limit():
    import torch

    dev = torch.device("cuda", 0)
    k = 257
    H = _colmajor(torch, np.zeros((k + 1, k)), dev)
    with pytest.raises(lslu.LsluError, match=r"k must be in \[1, 256\]"):
        lslu.projected_noalloc(H, 1.0, "gcv", 0.0, 1000)
