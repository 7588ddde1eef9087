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

pytestmark = pytest.mark.gpu


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
            Hd = torch.from_numpy(np.asfortranarray(H)).to(dev).t().contiguous().t()
            out = _outputs(torch, k, dev)
            lslu.projected_noalloc(Hd, hp["beta"], rule, lam, P.m, **out)
            torch.cuda.synchronize()
            tol = 1e-10
            assert np.allclose(out["y"].cpu().numpy(), ref["y"], rtol=tol, atol=tol * np.abs(ref["y"]).max())
            assert np.allclose(out["sigma"].cpu().numpy(), ref["sigma"], rtol=tol, atol=0)
            assert np.allclose(out["c"].cpu().numpy(), ref["c"], rtol=tol, atol=tol * abs(hp["beta"]))
            assert abs(out["lam_out"].item() - ref["lam"]) <= tol * max(ref["lam"], 1e-300)
            assert abs(out["resid_out"].item() - ref["resid"]) <= tol * abs(hp["beta"])


def test_noalloc_rejects_k_beyond_limit():
    import torch

    dev = torch.device("cuda", 0)
    k = 257
    H = torch.zeros((k + 1, k), dtype=torch.float64, device=dev).t().contiguous().t()
    with pytest.raises(lslu.LsluError, match=r"k must be in \[1, 256\]"):
        lslu.projected_noalloc(H, 1.0, "gcv", 0.0, 1000)
