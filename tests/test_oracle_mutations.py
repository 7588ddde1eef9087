"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them.  The mistakes live only in the in-memory copy."""
import inspect
import sys
import types

import numpy as np
import pytest

import oracle.lslu_oracle as O
from paper_2409_05239_gb300 import tomo
from tests import pins

MUTATIONS = {
    "elimination_sign": ("q = q - W[j, k] * L[:, j]", "q = q + W[j, k] * L[:, j]"),
    "pivot_without_abs": ("a = np.abs(v)", "a = np.array(v, dtype=np.float64)"),
    "h_coefficient_row": ("H[j, k] = u[tp[j]]", "H[j, k] = u[tp[0]]"),
    "h_elimination_short": ("for j in range(k + 1):", "for j in range(k):"),
    "w_scaling": ("L[:, k] = q / W[k, k]", "L[:, k] = q / abs(W[k, k])"),
    "beta_unsigned": ("beta = float(r0[i])", "beta = float(abs(r0[i]))"),
    "svd_transposed": ("c = beta * U[0, :]", "c = beta * U[:, 0]"),
    "tikhonov_filter": ("f = sigma / (sigma ** 2 + lam ** 2)", "f = sigma / (sigma ** 2 + lam)"),
    "gcv_dropped_term": ("num = k * (np.sum((f * c[:k]) ** 2) + c[k] ** 2)",
                         "num = k * (np.sum((f * c[:k]) ** 2))"),
    "wgcv_weight": ("den = 1.0 + np.sum(((1.0 - omega) * s2 + L2) / (s2 + L2))",
                    "den = 1.0 + np.sum(((1.0 - omega) * L2 + s2) / (s2 + L2))"),
    "slope_sign": ("return float(dN * Dn - 2.0 * N * dD)", "return float(dN * Dn + 2.0 * N * dD)"),
    "recombination_basis": ("x = x + hp[\"L\"] @ y", "x = x + hp[\"L\"][:, ::-1] @ y"),
    "wgcv_omega_k_over_m": ("return select_lambda(sigma, c, (k + 1) / m)",
                            "return select_lambda(sigma, c, k / m)"),
    "wgcv_omega_columns": ("lk = _lambda_for(rule, lam, s, c, kk, m)",
                           "lk = _lambda_for(rule, lam, s, c, kk, n)"),
}


def mutated(name):
    src = inspect.getsource(O)
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mod = types.ModuleType(f"oracle_mutant_{name}")
    sys.modules[mod.__name__] = mod  # dataclasses look their module up
    try:
        exec(compile(src.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


@pytest.fixture(scope="module")
def ct32():
    return tomo.make_config("ct32")


def run_all_pins(M, P):
    """Runs the pin suite on module M; returns the list of pins that failed."""
    A = P.scipy()
    failures = []

    def attempt(label, fn):
        try:
            fn()
        except (AssertionError, FloatingPointError, np.linalg.LinAlgError, ValueError,
                IndexError, ZeroDivisionError) as e:
            failures.append((label, str(e)[:80]))

    def basis():
        hp = M.hessenberg_rect_pivoted(A, P.b, None, 12)
        pins.check_unit_pivot_structure(hp)
        pins.check_hessenberg_relations(A, hp)

    Ad, _, bd = pins.random_problem(30, 20, seed=50, decay=0.8)
    attempt("basis", basis)
    attempt("normal_eq", lambda: pins.check_normal_equation_equivalence(M, Ad, bd, 6))
    hp = O.hessenberg_rect_pivoted(A, P.b, None, 12)
    H = hp["H"]
    attempt("stacked", lambda: pins.check_tikhonov_vs_stacked_lstsq(M, H, hp["beta"], [0.0, 1e-2, 0.5]))
    attempt("gcv_forms", lambda: pins.check_gcv_forms(M, H, hp["beta"], [1e-3, 0.1, 2.0]))
    attempt("lambda_min", lambda: pins.check_lambda_is_minimiser(M, H, hp["beta"], 1.0))
    attempt("oblique", lambda: pins.check_oblique_bruteforce(M, A, P.b, 10, 1e-2, "fixed"))
    attempt("oblique_gcv", lambda: pins.check_oblique_bruteforce(M, A, P.b, 10, 0.0, "gcv"))
    Aw, _, bw = pins.random_problem(40, 25, seed=5, decay=0.8)
    attempt("wgcv_rule", lambda: pins.check_wgcv_rule(M, Aw, bw, 14, npts=401))
    return failures


def test_unmutated_oracle_passes_all(ct32):
    assert run_all_pins(O, ct32) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(ct32, name):
    with np.errstate(all="ignore"):
        failures = run_all_pins(mutated(name), ct32)
    assert failures, f"mutation {name} passed every pin"
