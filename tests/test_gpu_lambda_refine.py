"""The regularization parameter of the projected problem (Section 3.2.1, Eqs.
(gcv2) and (wgcv)) on synthetic projected problems whose singular values and
data coefficients are prescribed, against the oracle's rule.

H = Q[:, :k] diag(sigma) V^T with Q the reflector whose first row is c / beta,
so that U^T (beta e1) = c exactly: the spectra can be chosen to make the GCV
curve steep, flat, or its minimum sit near a grid point.  The GPU refines the
best grid point by safeguarded Newton steps on the slope, the oracle by
bisection; both must reach the same minimum of G (to rounding), and where the
minimum is well curved, the same lambda."""
import numpy as np
import pytest

from oracle import lslu_oracle as O
from paper_2409_05239_gb300 import lslu, tomo

pytestmark = pytest.mark.gpu


def synthetic_H(sigma, c, seed):
    """(k+1) x k H with singular values sigma and U^T (beta e1) = c (length
    k+1); returns (H, beta)."""
    k = sigma.shape[0]
    beta = float(np.linalg.norm(c))
    q = c / beta
    e1 = np.zeros(k + 1)
    e1[0] = 1.0
    w = e1 - q
    nw = np.linalg.norm(w)
    Q = np.eye(k + 1) - (2.0 / (nw * nw)) * np.outer(w, w) if nw > 0 else np.eye(k + 1)
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    H = (Q[:, :k] * sigma) @ V.T
    return H, beta


def cases():
    out = []
    rng = np.random.default_rng(7)
    for k, decades, picard, noise in [(20, 8, 1.2, 1e-4), (50, 12, 1.0, 1e-3), (120, 14, 1.5, 1e-6),
                                      (200, 10, 1.1, 1e-2)]:
        s = 10.0 ** (-decades * np.arange(k) / max(k - 1, 1))
        c = np.empty(k + 1)
        c[:k] = s ** picard * rng.choice([-1.0, 1.0], k) + noise * rng.standard_normal(k)
        c[k] = noise * 3.0
        out.append((f"picard-k{k}", s, c))
    k = 40  # white coefficients: a flat curve
    s = 10.0 ** (-6 * np.arange(k) / (k - 1))
    out.append(("white-k40", s, np.full(k + 1, 0.3)))
    k = 30  # clustered singular values
    s = np.concatenate([np.full(10, 1.0), np.full(10, 1e-3), np.full(10, 1e-6)]) * (
        1 + 1e-3 * np.arange(30))
    c = np.concatenate([np.full(10, 1.0), np.full(10, 1e-2), np.full(10, 1e-2), [1e-3]])
    out.append(("clusters-k30", s, c))
    return out


CASES = cases()


@pytest.fixture(scope="module")
def handle():
    P = tomo.make_config("ct32")
    with lslu.from_problem(P, "f64", 200) as s:
        yield s


def spread_under_backward_error(s_ref, c_ref, V, omega, lam_ref, trials=6):
    """How far the oracle's lambda, G(lambda) and y move when sigma and c take
    perturbations of a few units of roundoff of sigma_1 and |c| (the backward
    error of any stable SVD of H): the resolution to which the rule itself
    fixes them for this spectrum."""
    eps = np.finfo(float).eps
    rng = np.random.default_rng(11)
    G0 = O.gcv_value(s_ref, c_ref, lam_ref, omega)
    y0 = O.tikhonov_y(s_ref, c_ref, V, lam_ref)
    dl = dg = dy = 0.0
    for _ in range(trials):
        sp = np.abs(s_ref + 4 * eps * s_ref[0] * rng.standard_normal(s_ref.shape))
        order = np.argsort(-sp)
        sp = sp[order]
        cp = c_ref.copy()
        cp[:-1] = cp[:-1][order]
        cp = cp + 4 * eps * np.linalg.norm(c_ref) * rng.standard_normal(cp.shape)
        lp = O.select_lambda(sp, cp, omega)
        dl = max(dl, abs(lp - lam_ref) / lam_ref)
        dg = max(dg, abs(O.gcv_value(s_ref, c_ref, lp, omega) - G0) / G0)
        yp = O.tikhonov_y(sp, cp, V[:, order], lp)
        dy = max(dy, np.linalg.norm(yp - y0) / np.linalg.norm(y0))
    return dl, dg, dy


@pytest.mark.parametrize("name,sigma,c", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("rule", ["gcv", "wgcv"])
def test_lambda_matches_oracle(handle, name, sigma, c, rule):
    k = sigma.shape[0]
    m = 4 * k + 3  # row count of A for the weight omega = (k+1)/m
    H, beta = synthetic_H(sigma, c, seed=k)
    s_ref, c_ref, V = O.projected_svd(H, beta)
    omega = 1.0 if rule == "gcv" else (k + 1) / m
    lam_ref = O.select_lambda(s_ref, c_ref, omega)
    dl, dg, dy = spread_under_backward_error(s_ref, c_ref, V, omega, lam_ref)
    out = handle.projected(H, beta, rule, 0.0, m=m)
    lam = out["lam"]
    G = lambda x: O.gcv_value(s_ref, c_ref, x, omega)  # noqa: E731
    # lambda and the minimum of G to the resolution the rule has for this
    # spectrum (1e-8 relative where the slope resolves it better)
    assert abs(lam - lam_ref) <= max(1e-8, 10 * dl) * lam_ref
    assert abs(G(lam) - G(lam_ref)) <= max(1e-12, 10 * dg) * G(lam_ref)
    # the projected solution
    y_ref = O.tikhonov_y(s_ref, c_ref, V, lam_ref)
    assert np.linalg.norm(out["y"] - y_ref) <= max(1e-9, 10 * dy) * np.linalg.norm(y_ref)
