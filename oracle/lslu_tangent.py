"""Forward-mode derivative (tangent) of Hybrid LSLU with the pivots held fixed.

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  It shares no code with the CUDA
library.

With the pivot lists g and t held fixed (replayed from a primal run), every
step of Algorithm 5 is a smooth map of the data, so the iterate
x_k(b, lambda) is differentiable.  The functions below run the steps of
Algorithm 4 in the paper's order, carrying for every quantity v its tangent
dv, the directional derivative along (db, dlambda):

  r0 = b - A x0                      dr0 = db - A dx0
  beta = r0(t_1)                     dbeta = dr0(t_1)
  d_1 = r0 / beta                    dd_1 = (dr0 - d_1 dbeta) / beta
  q = A^T d_k;  W(j,k) = q(g_j);  q <- q - W(j,k) l_j        (j < k, in order)
      dq = A^T dd_k;  dW(j,k) = dq(g_j);  dq <- dq - dW(j,k) l_j - W(j,k) dl_j
  W(k,k) = q(g_k);  l_k = q / W(k,k)
      dl_k = (dq - l_k dW(k,k)) / W(k,k)
  the same for u = A l_k against d_1 .. d_k, H(j,k), d_{k+1};
  y solves the regularised normal equations of Eq. (TSP),
      (H^T H + lam^2 I) y = H^T (beta e1),
  so  (H^T H + lam^2 I) dy = dH^T (beta e1 - H y) + H^T (dbeta e1 - dH y)
                             - 2 lam dlam y;
  x = x0 + L y,  dx = dx0 + dL y + L dy.

The primal part repeats the oracle's own steps with the given pivots; the
tests pin it to lslu_oracle.hybrid_lslu (same pivots, same x) and the tangent
to central differences, to Euler's identity for the 1-homogeneous map
b -> x and to the exact derivative of a consistent full-basis problem.
"""
from __future__ import annotations

import numpy as np


def hybrid_lslu_tangent(A, b, db, lam, dlam, K, gp, tp, x0=None, dx0=None):
    """x_K and its directional derivative dx along (db, dlam) [, dx0].

    A: m x n (scipy sparse or dense); b, db: length m; lam >= 0 the fixed
    Tikhonov parameter and dlam its tangent; gp (K) and tp (K+1) the pivot
    rows of a primal run (Algorithm 4).  Returns (x, dx, aux) where aux holds
    L, D, H, W, beta, y and their tangents.
    """
    m, n = A.shape
    b = np.asarray(b, dtype=np.float64)
    db = np.asarray(db, dtype=np.float64)
    r0 = b.copy()
    dr0 = db.copy()
    if x0 is not None:
        r0 = r0 - A @ np.asarray(x0, dtype=np.float64)
        if dx0 is not None:
            dr0 = dr0 - A @ np.asarray(dx0, dtype=np.float64)
    L = np.zeros((n, K))
    dL = np.zeros((n, K))
    D = np.zeros((m, K + 1))
    dD = np.zeros((m, K + 1))
    H = np.zeros((K + 1, K))
    dH = np.zeros((K + 1, K))
    W = np.zeros((K, K))
    dW = np.zeros((K, K))

    beta = float(r0[tp[0]])
    dbeta = float(dr0[tp[0]])
    D[:, 0] = r0 / beta
    dD[:, 0] = (dr0 - D[:, 0] * dbeta) / beta
    for k in range(K):
        q = np.asarray(A.T @ D[:, k], dtype=np.float64).reshape(-1)
        dq = np.asarray(A.T @ dD[:, k], dtype=np.float64).reshape(-1)
        for j in range(k):
            W[j, k] = q[gp[j]]
            dW[j, k] = dq[gp[j]]
            q = q - W[j, k] * L[:, j]
            dq = dq - dW[j, k] * L[:, j] - W[j, k] * dL[:, j]
        W[k, k] = q[gp[k]]
        dW[k, k] = dq[gp[k]]
        L[:, k] = q / W[k, k]
        dL[:, k] = (dq - L[:, k] * dW[k, k]) / W[k, k]

        u = np.asarray(A @ L[:, k], dtype=np.float64).reshape(-1)
        du = np.asarray(A @ dL[:, k], dtype=np.float64).reshape(-1)
        for j in range(k + 1):
            H[j, k] = u[tp[j]]
            dH[j, k] = du[tp[j]]
            u = u - H[j, k] * D[:, j]
            du = du - dH[j, k] * D[:, j] - H[j, k] * dD[:, j]
        H[k + 1, k] = u[tp[k + 1]]
        dH[k + 1, k] = du[tp[k + 1]]
        D[:, k + 1] = u / H[k + 1, k]
        dD[:, k + 1] = (du - D[:, k + 1] * dH[k + 1, k]) / H[k + 1, k]

    # projected problem (Eq. TSP) through its regularised normal equations
    M = H.T @ H + lam * lam * np.eye(K)
    e1 = np.zeros(K + 1)
    e1[0] = 1.0
    y = np.linalg.solve(M, H.T @ (beta * e1))
    rhs = dH.T @ (beta * e1 - H @ y) + H.T @ (dbeta * e1 - dH @ y) - 2.0 * lam * dlam * y
    dy = np.linalg.solve(M, rhs)

    x = L @ y
    dx = dL @ y + L @ dy
    if x0 is not None:
        x = x + np.asarray(x0, dtype=np.float64)
        if dx0 is not None:
            dx = dx + np.asarray(dx0, dtype=np.float64)
    aux = dict(L=L, dL=dL, D=D, dD=dD, H=H, dH=dH, W=W, dW=dW, beta=beta, dbeta=dbeta,
               y=y, dy=dy)
    return x, dx, aux


def loss_and_directional(A, b, lam, K, gp, tp, x_true, db, dloglam):
    """J = ||x_K - x_true||^2 and its directional derivative along
    (db, d log lambda) with the pivots fixed: dJ = 2 (x - x_true)^T dx,
    dlam = lam * dloglam."""
    x, dx, _ = hybrid_lslu_tangent(A, b, db, lam, lam * dloglam, K, gp, tp)
    r = x - x_true
    return float(r @ r), float(2.0 * r @ dx)
