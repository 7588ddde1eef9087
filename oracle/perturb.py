"""A second FP64 evaluation order of the same operator, for sensitivity runs.

TEST INFRASTRUCTURE ONLY.  PermutedOperator applies A and A^T with the rows
and columns of the CSR permuted (a different, equally valid summation order);
running the oracle on it measures how far two correct FP64 implementations of
Algorithm 4 drift apart, which bounds what GPU-versus-oracle parity can mean.
"""
import numpy as np


class PermutedOperator:
    def __init__(self, A, seed=1):
        rng = np.random.default_rng(seed)
        self.shape = A.shape
        self.pr = rng.permutation(A.shape[0])
        self.pc = rng.permutation(A.shape[1])
        self.Ap = A[self.pr][:, self.pc].tocsr()
        self.ApT = self.Ap.T.tocsr()
        self.ipr = np.argsort(self.pr)
        self.ipc = np.argsort(self.pc)

    def __matmul__(self, v):
        return (self.Ap @ v[self.pc])[self.ipr]

    @property
    def T(self):
        outer = self

        class _T:
            shape = (outer.shape[1], outer.shape[0])

            def __matmul__(self, u):
                return (outer.ApT @ u[outer.pr])[outer.ipc]

        return _T()


def first_difference(a, b):
    """Index of the first differing entry of two pivot lists (len if none)."""
    n = min(len(a), len(b))
    d = np.nonzero(np.asarray(a[:n]) != np.asarray(b[:n]))[0]
    return int(d[0]) if d.size else n
