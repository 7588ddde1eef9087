"""ctypes binding of the LSLU C ABI (include/lslu.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Importing this module never compiles anything; it raises if the library has
not been built (paper_2409_05239_gb300.build.build()).  Host arrays are numpy
arrays; device buffers are torch CUDA tensors (only their data pointers are
passed to the library).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblslu.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT = 0, 1, 2, 3, 4
BREAKDOWN_BETA, BREAKDOWN_W, BREAKDOWN_H, ERR_NONFINITE = 5, 6, 7, 8
BREAKDOWNS = (BREAKDOWN_BETA, BREAKDOWN_W, BREAKDOWN_H)
VALUE_TYPES = {"f64": 0, "f32": 1, "bf16": 2}
RULES = {"none": 0, "fixed": 1, "gcv": 2, "wgcv": 3}
HOST, DEVICE = 0, 1

EXPORTS = ("lslu_create", "lslu_solve", "lslu_get_state", "lslu_spmv", "lslu_projected",
           "lslu_projected_noalloc", "lslu_profile", "lslu_timing", "lslu_last_launch_count",
           "lslu_error_string", "lslu_destroy", "lslu_create_batched", "lslu_solve_batched",
           "lslu_adjoint", "lslu_solve_fixed_pivots", "lslu_create_shared",
           "lslu_solve_stopping", "lslu_solve_sampled", "lslu_set_spmv_shape",
           "lslu_tune_spmv", "lslu_uq", "lslu_solve_optimal", "lslu_spmv_config",
           "lslu_create_ordered", "lslu_create_batched_ordered", "lslu_create_shared_ordered",
           "lslu_set_loop", "lslu_loop_config", "lslu_projected_history")

_lib = None


class LsluError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lslu status {status}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load the shared library (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing "
                           "(run paper_2409_05239_gb300.build.build())")
    lib = ctypes.CDLL(p)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.lslu_create.argtypes = [i64, i64, i64, vp, vp, vp, i32, i32, i32, vp, ctypes.POINTER(vp)]
    lib.lslu_create.restype = i32
    lib.lslu_create_ordered.argtypes = [i64, i64, i64, vp, vp, vp, i32, i32, vp, vp, i32, vp,
                                        ctypes.POINTER(vp)]
    lib.lslu_create_ordered.restype = i32
    lib.lslu_create_batched_ordered.argtypes = [i32, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp,
                                                ctypes.POINTER(vp)]
    lib.lslu_create_batched_ordered.restype = i32
    lib.lslu_create_shared_ordered.argtypes = [i64, i64, vp, vp, vp, i32, i32, i32, vp, vp, vp,
                                               ctypes.POINTER(vp)]
    lib.lslu_create_shared_ordered.restype = i32
    lib.lslu_solve.argtypes = [vp, vp, vp, i32, i32, f64, i32, vp, vp, vp, vp, vp, vp]
    lib.lslu_solve.restype = i32
    lib.lslu_get_state.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    lib.lslu_get_state.restype = i32
    lib.lslu_spmv.argtypes = [vp, i32, vp, vp]
    lib.lslu_spmv.restype = i32
    lib.lslu_projected.argtypes = [vp, i32, vp, i32, f64, i32, f64, i64, i32, vp, vp, vp, vp, vp]
    lib.lslu_projected.restype = i32
    lib.lslu_projected_history.argtypes = [vp, i32, vp, i32, f64, i32, f64, i64, i32, vp, vp]
    lib.lslu_projected_history.restype = i32
    lib.lslu_projected_noalloc.argtypes = [i32, vp, i32, f64, i32, f64, i64, vp, vp, vp, vp,
                                           vp, vp]
    lib.lslu_projected_noalloc.restype = i32
    lib.lslu_profile.argtypes = [vp, i32]
    lib.lslu_profile.restype = i32
    lib.lslu_timing.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(f64)]
    lib.lslu_timing.restype = i32
    lib.lslu_last_launch_count.argtypes = [vp]
    lib.lslu_last_launch_count.restype = i64
    lib.lslu_error_string.argtypes = [vp]
    lib.lslu_error_string.restype = ctypes.c_char_p
    lib.lslu_create_batched.argtypes = [i32, vp, vp, vp, vp, vp, i32, i32, vp,
                                        ctypes.POINTER(vp)]
    lib.lslu_create_batched.restype = i32
    lib.lslu_create_shared.argtypes = [i64, i64, vp, vp, vp, i32, i32, i32, vp,
                                       ctypes.POINTER(vp)]
    lib.lslu_create_shared.restype = i32
    lib.lslu_solve_batched.argtypes = [vp, vp, i32, i32, f64, i32, vp, vp, vp, vp, vp]
    lib.lslu_solve_batched.restype = i32
    lib.lslu_solve_fixed_pivots.argtypes = [vp, vp, vp, i32, i32, f64, i32, vp, vp, vp, vp]
    lib.lslu_solve_fixed_pivots.restype = i32
    lib.lslu_spmv_config.argtypes = [vp] + [ctypes.POINTER(i32)] * 4
    lib.lslu_spmv_config.restype = i32
    lib.lslu_solve_optimal.argtypes = [vp, vp, i32, vp, i32, vp, vp]
    lib.lslu_solve_optimal.restype = i32
    lib.lslu_uq.argtypes = [vp, f64, f64, i32, vp, vp]
    lib.lslu_uq.restype = i32
    lib.lslu_set_spmv_shape.argtypes = [vp, i32, i32]
    lib.lslu_set_spmv_shape.restype = i32
    lib.lslu_tune_spmv.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), vp]
    lib.lslu_tune_spmv.restype = i32
    lib.lslu_solve_sampled.argtypes = [vp, vp, vp, i32, i32, f64, vp, i32, i32, vp, vp, vp, vp]
    lib.lslu_solve_sampled.restype = i32
    lib.lslu_solve_stopping.argtypes = [vp, vp, vp, i32, i32, f64, f64, i32, vp, vp, vp]
    lib.lslu_solve_stopping.restype = i32
    lib.lslu_adjoint.argtypes = [vp, vp, i32, vp, vp, vp]
    lib.lslu_adjoint.restype = i32
    lib.lslu_set_loop.argtypes = [vp, i32, i32, i64, i32]
    lib.lslu_set_loop.restype = i32
    lib.lslu_loop_config.argtypes = [vp] + [ctypes.POINTER(i32)] * 3
    lib.lslu_loop_config.restype = i32
    lib.lslu_destroy.argtypes = [vp]
    lib.lslu_destroy.restype = None
    _lib = lib
    return lib


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


LOOPS = {"graph": 0, "persistent": 1, "cluster": 2}


def _raise_unless_ok(handle, st):
    if st != OK:
        raise LsluError(st, handle.lib.lslu_error_string(handle.h).decode())
    return st


class _LoopControl:
    """Basis-loop execution of a handle (lslu_set_loop / lslu_loop_config)."""

    def set_loop(self, mode="persistent", blocks=0, wait_limit_ns=0, stall_first_barrier=False):
        _raise_unless_ok(self, self.lib.lslu_set_loop(self.h, LOOPS[mode], int(blocks),
                                                      int(wait_limit_ns),
                                                      int(bool(stall_first_barrier))))

    def loop_config(self):
        v = [ctypes.c_int32(0) for _ in range(3)]
        _raise_unless_ok(self, self.lib.lslu_loop_config(self.h, *[ctypes.byref(t) for t in v]))
        return dict(mode=[k for k, c in LOOPS.items() if c == v[0].value][0],
                    blocks=v[1].value, max_blocks=v[2].value)


class _SpmvControl:
    """Row shapes of a handle's sparse products (lslu_set_spmv_shape,
    lslu_spmv_config, lslu_tune_spmv); a batched handle has them too."""

    SHAPES = ("16x2", "32x1", "16x1", "8x1", "8x2", "4x1",
              "16x2/16-bit", "32x1/16-bit", "16x1/16-bit", "8x1/16-bit", "8x2/16-bit", "4x1/16-bit",
              "32x8e", "32x8e/16-bit", "32x4e", "32x4e/16-bit")

    def set_spmv_shape(self, shape_A, shape_AT=None):
        """Row shape of the sparse products (index into SHAPES)."""
        sa = int(shape_A)
        st = sa if shape_AT is None else int(shape_AT)
        _raise_unless_ok(self, self.lib.lslu_set_spmv_shape(self.h, sa, st))

    def spmv_config(self):
        """Row shapes and column formats of A and A^T."""
        v = [ctypes.c_int32(0) for _ in range(4)]
        _raise_unless_ok(self, self.lib.lslu_spmv_config(self.h, *[ctypes.byref(t) for t in v]))
        return dict(shape_A=self.SHAPES[v[0].value], shape_AT=self.SHAPES[v[1].value],
                    compressed_A=bool(v[2].value), compressed_AT=bool(v[3].value))

    def tune_spmv(self, reps=5):
        """Time every row shape on A and A^T and keep the fastest; returns the
        chosen shapes and the per-shape times (microseconds)."""
        a = ctypes.c_int32(0)
        t = ctypes.c_int32(0)
        ns = len(self.SHAPES)
        us = np.zeros(2 * ns)
        _raise_unless_ok(self, self.lib.lslu_tune_spmv(self.h, int(reps), ctypes.byref(a),
                                                       ctypes.byref(t), _ptr(us)))
        keep = lambda v: {k: x for k, x in zip(self.SHAPES, v.tolist()) if x >= 0}
        return dict(shape_A=a.value, shape_AT=t.value, us_A=keep(us[:ns]), us_AT=keep(us[ns:]))


class Solver(_LoopControl, _SpmvControl):
    """One LSLU handle on the current CUDA device.

    value_type: 'f64' (FP64 basis and accumulation), 'f32' or 'bf16' (A's
    values stored in that type, FP32 basis and accumulation).
    """

    def __init__(self, m, n, row_ptr, col_idx, vals, value_type="f32", max_iter=300,
                 stream=None, row_order=None, col_order=None):
        self.lib = load()
        self.m, self.n = int(m), int(n)
        self.value_type = value_type
        self.max_iter = int(max_iter)
        self.basis_dtype = np.float64 if value_type == "f64" else np.float32
        on_dev = not isinstance(row_ptr, np.ndarray)
        if not on_dev:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
            col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
            vals = np.ascontiguousarray(vals, dtype=np.float64)
        nnz = int(row_ptr[-1]) if not on_dev else int(row_ptr[-1].item())
        h = ctypes.c_void_p()
        self.ordered = row_order is not None or col_order is not None
        if self.ordered:  # lslu_create_ordered: orders live where the CSR arrays do
            if not on_dev:
                row_order = None if row_order is None else np.ascontiguousarray(row_order,
                                                                                dtype=np.int32)
                col_order = None if col_order is None else np.ascontiguousarray(col_order,
                                                                                dtype=np.int32)
            st = self.lib.lslu_create_ordered(
                self.m, self.n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(vals),
                VALUE_TYPES[value_type], self.max_iter,
                None if row_order is None else _ptr(row_order),
                None if col_order is None else _ptr(col_order),
                DEVICE if on_dev else HOST, stream, ctypes.byref(h))
        else:
            st = self.lib.lslu_create(self.m, self.n, nnz, _ptr(row_ptr), _ptr(col_idx),
                                      _ptr(vals), VALUE_TYPES[value_type], self.max_iter,
                                      DEVICE if on_dev else HOST, stream, ctypes.byref(h))
        if st != OK:
            raise LsluError(st, self.lib.lslu_error_string(None).decode())
        self.h = h
        self.epoch = 0  # bumped by every call that replaces the solve state

    def _check(self, st, allow_breakdown=False):
        if st == OK or (allow_breakdown and st in BREAKDOWNS):
            return st
        raise LsluError(st, self.lib.lslu_error_string(self.h).decode())

    def solve(self, b, K, rule="gcv", lam=0.0, x0=None, histories=False):
        """Host arrays in and out.  Returns a dict with x, pivots, histories,
        k_done and status (a breakdown is reported, not raised)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        x = np.zeros(self.n)
        gp = np.zeros(K, dtype=np.int32)
        tp = np.zeros(K + 1, dtype=np.int32)
        lh = np.zeros(K) if histories else None
        rh = np.zeros(K) if histories else None
        kd = ctypes.c_int32(0)
        self.epoch += 1
        st = self.lib.lslu_solve(self.h, _ptr(b), _ptr(x0), int(K), RULES[rule], float(lam), HOST,
                                 _ptr(x), _ptr(gp), _ptr(tp), _ptr(lh), _ptr(rh),
                                 ctypes.addressof(kd))
        self._check(st, allow_breakdown=True)
        return dict(x=x, gp=gp, tp=tp, lam_hist=lh, res_hist=rh, k_done=kd.value, status=st)

    def solve_device(self, b, x_out, K, rule="gcv", lam=0.0, x0=None, gp=None, tp=None,
                     lam_hist=None, res_hist=None, k_done=None):
        """Device buffers (torch tensors) in and out; returns the status."""
        self.epoch += 1
        st = self.lib.lslu_solve(self.h, _ptr(b), _ptr(x0), int(K), RULES[rule], float(lam),
                                 DEVICE, _ptr(x_out), _ptr(gp), _ptr(tp), _ptr(lam_hist),
                                 _ptr(res_hist), _ptr(k_done))
        return self._check(st, allow_breakdown=True)

    def state(self, k):
        """H, W, beta, L, D of the last solve (host copies); k = its k_done."""
        H = np.zeros((k, k + 1)) if k else np.zeros((0, 1))
        W = np.zeros((k, k))
        beta = np.zeros(1)
        L = np.zeros((k, self.n), dtype=self.basis_dtype)
        D = np.zeros((k + 1, self.m), dtype=self.basis_dtype)
        st = self.lib.lslu_get_state(self.h, HOST, _ptr(H), _ptr(W), _ptr(beta), _ptr(L), _ptr(D))
        self._check(st)
        return dict(H=H.T.copy(), W=W.T.copy(), beta=float(beta[0]), L=L.T.copy(), D=D.T.copy())

    def solve_fixed_pivots(self, b, K, gp, tp, rule="fixed", lam=0.0, x0=None):
        """Solve with the pivot lists replayed (host arrays)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        gp = np.ascontiguousarray(gp, dtype=np.int32)
        tp = np.ascontiguousarray(tp, dtype=np.int32)
        x = np.zeros(self.n)
        kd = ctypes.c_int32(0)
        self.epoch += 1
        st = self.lib.lslu_solve_fixed_pivots(self.h, _ptr(b), _ptr(x0), int(K), RULES[rule],
                                              float(lam), HOST, _ptr(gp), _ptr(tp), _ptr(x),
                                              ctypes.addressof(kd))
        self._check(st, allow_breakdown=True)
        return dict(x=x, k_done=kd.value, status=st)

    def solve_sampled(self, b, K, samples, rule="gcv", lam=0.0, x0=None):
        """Sampled pivoting (Section 2.2) with a host sample table of shape
        (2K+1, s); returns the same dict as solve (without histories)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        S = np.ascontiguousarray(samples, dtype=np.int32)
        x = np.zeros(self.n)
        gp = np.zeros(K, dtype=np.int32)
        tp = np.zeros(K + 1, dtype=np.int32)
        kd = ctypes.c_int32(0)
        self.epoch += 1
        st = self.lib.lslu_solve_sampled(self.h, _ptr(b), _ptr(x0), int(K), RULES[rule],
                                         float(lam), _ptr(S), int(S.shape[1]), HOST, _ptr(x),
                                         _ptr(gp), _ptr(tp), ctypes.addressof(kd))
        self._check(st, allow_breakdown=True)
        return dict(x=x, gp=gp, tp=tp, k_done=kd.value, status=st)

    def solve_stopping(self, b, K_max, rule="wgcv", lam=0.0, tol=1e-6, x0=None):
        """Solve with the stopping criterion G^(k) (host arrays): returns x at
        the stopping iteration, k_stop and the G history."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        x = np.zeros(self.n)
        g = np.zeros(K_max)
        ks = ctypes.c_int32(0)
        self.epoch += 1
        st = self.lib.lslu_solve_stopping(self.h, _ptr(b), _ptr(x0), int(K_max), RULES[rule],
                                          float(lam), float(tol), HOST, _ptr(x),
                                          ctypes.addressof(ks), _ptr(g))
        self._check(st)
        return dict(x=x, k_stop=ks.value, G=g)

    def adjoint(self, x_bar, want_x0=False):
        """Reverse-mode derivative of the last solve (pivots fixed): host
        x_bar -> dict(b_bar, lambda_bar[, x0_bar])."""
        x_bar = np.ascontiguousarray(x_bar, dtype=np.float64)
        bb = np.zeros(self.m)
        lb = np.zeros(1)
        xb = np.zeros(self.n) if want_x0 else None
        self._check(self.lib.lslu_adjoint(self.h, _ptr(x_bar), HOST, _ptr(bb), _ptr(lb),
                                          _ptr(xb)))
        out = dict(b_bar=bb, lambda_bar=float(lb[0]))
        if want_x0:
            out["x0_bar"] = xb
        return out

    def adjoint_device(self, x_bar, b_bar, lambda_bar=None, x0_bar=None):
        """Device tensors in and out (FP64)."""
        self._check(self.lib.lslu_adjoint(self.h, _ptr(x_bar), DEVICE, _ptr(b_bar),
                                          _ptr(lambda_bar), _ptr(x0_bar)))

    def spmv(self, transpose, x, y):
        """y = A x or y = A^T x on device tensors of the basis type."""
        self._check(self.lib.lslu_spmv(self.h, int(transpose), _ptr(x), _ptr(y)))

    def projected(self, H, beta, rule="gcv", lam=0.0, m=None):
        """Projected solve of Eq. (TSP) on the device for a host H ((k+1) x k)."""
        H = np.asfortranarray(H, dtype=np.float64)
        k = H.shape[1]
        y = np.zeros(k)
        sig = np.zeros(k)
        c = np.zeros(k + 1)
        lo = np.zeros(1)
        ro = np.zeros(1)
        self.epoch += 1
        st = self.lib.lslu_projected(self.h, k, _ptr(H), k + 1, float(beta), RULES[rule],
                                     float(lam), int(m or self.m), HOST, _ptr(y), _ptr(sig),
                                     _ptr(c), _ptr(lo), _ptr(ro))
        self._check(st)
        return dict(y=y, sigma=sig, c=c, lam=float(lo[0]), resid=float(ro[0]))

    def projected_history(self, H, beta, rule="gcv", lam=0.0, m=None):
        """lambda_k and the residual of the projected problem of every leading
        block H[:k+1, :k], k = 1..K, of a host H ((K+1) x K):
        dict(lam_hist, res_hist)."""
        H = np.asfortranarray(H, dtype=np.float64)
        K = H.shape[1]
        lh = np.zeros(K)
        rh = np.zeros(K)
        self.epoch += 1
        self._check(self.lib.lslu_projected_history(self.h, K, _ptr(H), K + 1, float(beta),
                                                    RULES[rule], float(lam), int(m or self.m),
                                                    HOST, _ptr(lh), _ptr(rh)))
        return dict(lam_hist=lh, res_hist=rh)

    def solve_optimal(self, b, K, x_true):
        """x_K with the optimal lambda (needs x_true): dict(x, lam)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        xt = np.ascontiguousarray(x_true, dtype=np.float64)
        x = np.zeros(self.n)
        lam = np.zeros(1)
        self.epoch += 1
        self._check(self.lib.lslu_solve_optimal(self.h, _ptr(b), int(K), _ptr(xt), HOST, _ptr(x),
                                                _ptr(lam)))
        return dict(x=x, lam=float(lam[0]))

    def uq(self, sigma2, lam, want_diag=True):
        """Low-rank posterior variances (Section 4.2) from the last solve:
        dict(var_diag (n) or None, var_sum)."""
        d = np.zeros(self.n) if want_diag else None
        tot = np.zeros(1)
        self._check(self.lib.lslu_uq(self.h, float(sigma2), float(lam), HOST, _ptr(d),
                                     _ptr(tot)))
        return dict(var_diag=d, var_sum=float(tot[0]))

    def profile(self, enable=True):
        self._check(self.lib.lslu_profile(self.h, int(enable)))

    def timing(self):
        n = ctypes.c_int32(0)
        ms = ctypes.c_double(0.0)
        self._check(self.lib.lslu_timing(self.h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def last_launch_count(self):
        return int(self.lib.lslu_last_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.lslu_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def torch_f64():
    import torch

    return torch.float64


def projected_noalloc(H, beta, rule, lam, m, y=None, sigma=None, c=None, lam_out=None,
                      resid_out=None, stream=None):
    """Allocation-free projected solve: H and every output are device tensors
    (torch, FP64); asynchronous on stream.  Raises LsluError on failure."""
    lib = load()
    k = H.shape[1]
    # the library sees raw pointers only: check the layouts it assumes here
    if H.dtype != torch_f64() or not H.is_cuda or H.dim() != 2 or H.stride(0) != 1 \
            or H.shape[0] < k + 1:
        raise ValueError("H must be a (k+1) x k column-major float64 CUDA tensor")
    for name, t, need in (("y", y, k), ("sigma", sigma, k), ("c", c, k + 1),
                          ("lam_out", lam_out, 1), ("resid_out", resid_out, 1)):
        if t is None:
            continue
        if t.dtype != torch_f64() or t.device != H.device or not t.is_contiguous() \
                or t.numel() < need:
            raise ValueError(f"{name} must be a contiguous float64 tensor on {H.device} "
                             f"with at least {need} entries")
    # a one-column H has no meaningful column stride: its leading dimension is
    # its row count
    ldh = H.stride(1) if k > 1 else H.shape[0]
    st = lib.lslu_projected_noalloc(k, _ptr(H), ldh, float(beta), RULES[rule],
                                    float(lam), int(m), _ptr(y), _ptr(sigma), _ptr(c),
                                    _ptr(lam_out), _ptr(resid_out), stream)
    if st != OK:
        raise LsluError(st, lib.lslu_error_string(None).decode())


def stack_orders(orders, k, off):
    """Global order of a batch from per-problem orders (entry k of each pair,
    None = identity) in the problems' own index spaces: problem p's index i
    goes to off[p] + order_p[i]."""
    return np.ascontiguousarray(np.concatenate([
        (np.arange(off[p + 1] - off[p]) if o[k] is None else np.asarray(o[k])) + off[p]
        for p, o in enumerate(orders)]), dtype=np.int32)


class BatchedSolver(_LoopControl, _SpmvControl):
    """One handle over several independent problems solved by one launch
    sequence (lslu_create_batched).  csr_list holds (m, n, row_ptr, col_idx,
    vals) per problem in the problem's own index space; they are stacked into
    one block-diagonal host CSR here (marshalling only).  orders: None, or one
    (row_order, col_order) pair per problem in its own index space (either may
    be None), stacked into the global orders of lslu_create_batched_ordered;
    with nrhs, one (row_order, col_order) pair for the shared matrix
    (lslu_create_shared_ordered)."""

    def __init__(self, csr_list, value_type="f32", max_iter=150, stream=None, nrhs=None,
                 orders=None):
        self.lib = load()
        if nrhs is not None:  # one matrix shared by nrhs right-hand sides
            m, n, rp, ci, vv = csr_list
            self._init_shared(int(m), int(n), rp, ci, vv, int(nrhs), value_type, max_iter,
                              stream, orders)
            return
        self.nprob = len(csr_list)
        self.value_type = value_type
        self.max_iter = int(max_iter)
        ms = [int(c[0]) for c in csr_list]
        ns = [int(c[1]) for c in csr_list]
        self.row_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
        self.col_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        rps, cis, vvs = [np.zeros(1, np.int64)], [], []
        base = 0
        for p, (m, n, rp, ci, vv) in enumerate(csr_list):
            rp = np.asarray(rp, dtype=np.int64)
            rps.append(rp[1:] + base)
            base += int(rp[-1])
            cis.append(np.asarray(ci, dtype=np.int64) + self.col_off[p])
            vvs.append(np.asarray(vv, dtype=np.float64))
        row_ptr = np.ascontiguousarray(np.concatenate(rps), dtype=np.int64)
        col_idx = np.ascontiguousarray(np.concatenate(cis), dtype=np.int32)
        vals = np.ascontiguousarray(np.concatenate(vvs), dtype=np.float64)
        h = ctypes.c_void_p()
        if orders is not None:
            ro, co = stack_orders(orders, 0, self.row_off), stack_orders(orders, 1, self.col_off)
            st = self.lib.lslu_create_batched_ordered(
                self.nprob, _ptr(self.row_off), _ptr(self.col_off), _ptr(row_ptr), _ptr(col_idx),
                _ptr(vals), VALUE_TYPES[value_type], self.max_iter, _ptr(ro), _ptr(co), stream,
                ctypes.byref(h))
        else:
            st = self.lib.lslu_create_batched(self.nprob, _ptr(self.row_off), _ptr(self.col_off),
                                              _ptr(row_ptr), _ptr(col_idx), _ptr(vals),
                                              VALUE_TYPES[value_type], self.max_iter, stream,
                                              ctypes.byref(h))
        if st != OK:
            raise LsluError(st, self.lib.lslu_error_string(None).decode())
        self.h = h

    def _init_shared(self, m, n, rp, ci, vv, nrhs, value_type, max_iter, stream, order=None):
        self.nprob = nrhs
        self.value_type = value_type
        self.max_iter = int(max_iter)
        self.row_off = (np.arange(nrhs + 1) * m).astype(np.int64)
        self.col_off = (np.arange(nrhs + 1) * n).astype(np.int64)
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        vv = np.ascontiguousarray(vv, dtype=np.float64)
        h = ctypes.c_void_p()
        if order is not None:
            ro, co = (None if o is None else np.ascontiguousarray(o, dtype=np.int32)
                      for o in order)
            st = self.lib.lslu_create_shared_ordered(m, n, _ptr(rp), _ptr(ci), _ptr(vv), nrhs,
                                                     VALUE_TYPES[value_type], self.max_iter,
                                                     _ptr(ro), _ptr(co), stream,
                                                     ctypes.byref(h))
        else:
            st = self.lib.lslu_create_shared(m, n, _ptr(rp), _ptr(ci), _ptr(vv), nrhs,
                                             VALUE_TYPES[value_type], self.max_iter, stream,
                                             ctypes.byref(h))
        if st != OK:
            raise LsluError(st, self.lib.lslu_error_string(None).decode())
        self.h = h

    def solve(self, b, K, rule="gcv", lam=0.0):
        """b: the problems' data concatenated (host).  Returns per-problem lists
        of x, g, t, k_done and status."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        P = self.nprob
        x = np.zeros(int(self.col_off[-1]))
        gp = np.zeros((P, K), dtype=np.int32)
        tp = np.zeros((P, K + 1), dtype=np.int32)
        kd = np.zeros(P, dtype=np.int32)
        sv = np.zeros(P, dtype=np.int32)
        st = self.lib.lslu_solve_batched(self.h, _ptr(b), int(K), RULES[rule], float(lam), HOST,
                                         _ptr(x), _ptr(gp), _ptr(tp), _ptr(kd), _ptr(sv))
        if st != OK:
            raise LsluError(st, self.lib.lslu_error_string(self.h).decode())
        co = self.col_off
        return dict(x=[x[co[p]:co[p + 1]] for p in range(P)], gp=gp, tp=tp, k_done=kd,
                    status=sv)

    def solve_device(self, b, x_out, K, rule="gcv", lam=0.0, gp=None, tp=None, k_done=None,
                     status=None):
        """Device buffers (torch tensors) in and out."""
        st = self.lib.lslu_solve_batched(self.h, _ptr(b), int(K), RULES[rule], float(lam),
                                         DEVICE, _ptr(x_out), _ptr(gp), _ptr(tp), _ptr(k_done),
                                         _ptr(status))
        if st != OK:
            raise LsluError(st, self.lib.lslu_error_string(self.h).decode())

    def last_launch_count(self):
        return int(self.lib.lslu_last_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.lslu_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


_autograd_fn = None


def _solve_function():
    """torch.autograd.Function around lslu_solve (forward, FIXED lambda) and
    lslu_adjoint (backward); built on first use so that importing this module
    does not import torch."""
    global _autograd_fn
    if _autograd_fn is not None:
        return _autograd_fn
    import torch

    class HybridLsluFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, b, log_lam, solver, K):
            lam = float(torch.exp(log_lam.detach()).item())
            x = torch.empty(solver.n, dtype=torch.float64, device=b.device)
            st = solver.solve_device(b.detach().to(torch.float64).contiguous(), x, K, "fixed", lam)
            if st != OK:
                raise LsluError(st, "breakdown in the forward solve: no derivative")
            ctx.solver, ctx.lam, ctx.epoch = solver, lam, solver.epoch
            return x

        @staticmethod
        def backward(ctx, x_bar):
            solver = ctx.solver
            if solver.epoch != ctx.epoch:
                raise RuntimeError("the handle solved again after this forward pass; the "
                                   "backward pass needs the state of its own solve")
            b_bar = torch.empty(solver.m, dtype=torch.float64, device=x_bar.device)
            lam_bar = torch.empty(1, dtype=torch.float64, device=x_bar.device)
            solver.adjoint_device(x_bar.detach().to(torch.float64).contiguous(), b_bar, lam_bar)
            # d/dlog(lambda) = lambda d/dlambda
            return b_bar, (lam_bar[0] * ctx.lam), None, None

    _autograd_fn = HybridLsluFn
    return HybridLsluFn


def hybrid_lslu(solver, b, log_lam, K):
    """x_K of Hybrid LSLU with fixed lambda = exp(log_lam) as a differentiable
    torch function of b (length m, CUDA) and log_lam (0-d tensor).  The
    backward pass is lslu_adjoint: the pivots of the forward solve are held
    fixed.  One backward per forward, before the handle solves again."""
    return _solve_function().apply(b, log_lam, solver, int(K))


def from_problems(Ps, value_type="f32", max_iter=150, stream=None, orders=None):
    """Batched solver over several tomography problems; orders as BatchedSolver's
    (e.g. [tomo.locality_order(P) for P in Ps])."""
    return BatchedSolver([(P.m, P.n, P.row_ptr, P.col_idx, P.vals) for P in Ps],
                         value_type=value_type, max_iter=max_iter, stream=stream, orders=orders)


def sample_table(K, s, m, n, seed):
    """Random sample indices for lslu_solve_sampled: 2K+1 rows of s indices,
    rows 0, 2, 4, ... in [0, m) and rows 1, 3, ... in [0, n) (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([rng.integers(0, m if t % 2 == 0 else n, size=s)
                     for t in range(2 * K + 1)]).astype(np.int32)


def shared_rhs(P, nrhs, value_type="f32", max_iter=150, stream=None, order=None):
    """Batched solver for nrhs right-hand sides of one tomography matrix; order:
    None or a (row_order, col_order) pair, e.g. tomo.locality_order(P)."""
    return BatchedSolver((P.m, P.n, P.row_ptr, P.col_idx, P.vals), value_type=value_type,
                         max_iter=max_iter, stream=stream, nrhs=nrhs, orders=order)


def from_problem(P, value_type="f32", max_iter=300, order=None):
    """Solver for a tomography problem (paper_2409_05239_gb300.tomo.TomoProblem).
    order: None (the matrix as numbered) or a (row_order, col_order) pair for
    lslu_create_ordered, e.g. tomo.locality_order(P)."""
    ro, co = (None, None) if order is None else order
    return Solver(P.m, P.n, P.row_ptr, P.col_idx, P.vals, value_type=value_type,
                  max_iter=max_iter, row_order=ro, col_order=co)
