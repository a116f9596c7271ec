"""CPU FP64 oracle of deflated, right-Jacobi-preconditioned restarted GMRES
(PDGMRES) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module.  It restates the method of the paper's Section 3.2
(restarted GMRES with deflation, right preconditioning) with the
subdomain-levelset deflation vectors of Section 3.2.2 fixed before the
iteration (so the harmonic-Ritz construction of Section 3.2.1 is skipped):

  E = Z^T A Z,  P1 = I - A Z E^{-1} Z^T,  P2 = I - Z E^{-1} Z^T A,
  x* = Z E^{-1} Z^T b  (eq. (defsplit) with A in place of A M^{-1}: the
  paper's remark on right preconditioning),
  GMRES(m) on  P1 A M^{-1} u = P1 b  (M = diag A, x~ = M^{-1} u),
  x = P2 x~ + x*.

Since b - A x = P1 (b - A x~), the GMRES residual is the true residual of x.
The Arnoldi step orthogonalises with modified Gram-Schmidt, the least-squares
problem is reduced by Givens rotations, and a cycle stops early when the
residual estimate reaches tol ||b|| or the new basis vector vanishes.  The
coarse solve and the small triangular solve use numpy.linalg as library
steps.  Plain and slow by design.
"""
from __future__ import annotations

import numpy as np

from . import coarse, restrict

OK, NOT_CONVERGED = 0, 3


class GmresResult:
    def __init__(self, x, iterations, cycles, relres_est, true_relres, status, hist, arnoldi):
        self.x, self.iterations, self.cycles = x, iterations, cycles
        self.relres_est, self.true_relres, self.status = relres_est, true_relres, status
        self.hist, self.arnoldi = hist, arnoldi


def pdgmres(A, label=None, d=0, b=None, m=20, tol=1e-6, maxiter=5000, record=False) -> GmresResult:
    """Solve A x = b (A: the oracle's CSR matrix, b defaults to its rhs).

    label/d: the deflation columns (indicators of label values 0..d-1), or
    d = 0 for plain right-Jacobi GMRES(m).  hist: the residual estimate
    ||b - A x|| / ||b|| after every Arnoldi step (index 0: the start).
    record: also return (V, Hbar, defl_op) of the first cycle."""
    n = A.n
    b = A.b if b is None else np.asarray(b, dtype=np.float64)
    dia = A.diag()
    defl = d > 0
    if defl:
        E, _ = coarse(A, label, d)
        lab = np.asarray(label)

        def coarse_solve(v):  # y = E^{-1} Z^T v
            return np.linalg.solve(E, restrict(label, d, v))

        def P1(w):  # w - A Z E^{-1} Z^T w
            return w - A.spmv(coarse_solve(w)[lab])

        xstar = coarse_solve(b)[lab]
    else:
        def P1(w):
            return w

        xstar = np.zeros(n)

    def op(v):  # P1 A M^{-1} v
        return P1(A.spmv(v / dia))

    bnorm = float(np.linalg.norm(b))
    xt = np.zeros(n)
    hist = []
    arnoldi = None
    its = 0
    cycles = 0
    converged = False
    if bnorm == 0.0:
        return GmresResult(np.zeros(n), 0, 0, 0.0, 0.0, OK, [0.0], None)
    while True:
        r = P1(b - A.spmv(xt))
        beta = float(np.linalg.norm(r))
        if not hist:
            hist.append(beta / bnorm)
        if beta <= tol * bnorm:
            converged = True
            break
        if its >= maxiter:
            break
        cycles += 1
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        R = np.zeros((m + 1, m))  # H with the rotations applied
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = op(V[j])
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            # the earlier rotations on column j, then a new one for row j+1
            col = H[: j + 2, j].copy()
            for i in range(j):
                t = cs[i] * col[i] + sn[i] * col[i + 1]
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1]
                col[i] = t
            rho = float(np.hypot(col[j], col[j + 1]))
            cs[j], sn[j] = (1.0, 0.0) if rho == 0.0 else (col[j] / rho, col[j + 1] / rho)
            col[j] = rho
            col[j + 1] = 0.0
            R[: j + 2, j] = col
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or H[j + 1, j] == 0.0 or its >= maxiter:
                break
        if record and arnoldi is None:
            arnoldi = (V[: k + 1].copy(), H[: k + 1, :k].copy(), op)
        u = np.linalg.solve(R[:k, :k], g[:k]) if k > 0 else np.zeros(0)
        xt = xt + (u @ V[:k]) / dia
    if defl:
        x = xt - coarse_solve(A.spmv(xt))[lab] + xstar
    else:
        x = xt
    true_rel = float(np.linalg.norm(b - A.spmv(x)) / bnorm)
    return GmresResult(x, its, cycles, hist[-1], true_rel, OK if converged else NOT_CONVERGED, np.array(hist),
                       arnoldi)
