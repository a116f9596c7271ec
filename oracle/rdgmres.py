"""CPU FP64 oracle of restarted GMRES with harmonic-Ritz deflation (RDGMRES)
-- TEST INFRASTRUCTURE ONLY (only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import it).

Section 3.2.1 and its algorithm: right-preconditioned GMRES(m) (M = diag A)
whose first cycle runs without deflation; from that cycle's Arnoldi data the
d harmonic Ritz vectors of the smallest harmonic Ritz values are formed
(the Petrov-Galerkin condition (A V_m)^T (A z - theta z) = 0, solved as the
eigenproblem (H_m + h_{m+1,m}^2 H_m^{-T} e_m e_m^T) y = theta y, z = V_m y;
a complex-conjugate pair is replaced by its real and imaginary parts), the
deflation operators are fixed with them, and the remaining cycles run
deflated.

Reading of the restart (the algorithm leaves the spaces implicit): the
Krylov vectors, hence Z, live in the preconditioned variable u (x = M^{-1} u),
so the deflation uses B = A M^{-1} (the algorithm's A_p):
  E = Z^T B Z, P1 = I - B Z E^{-1} Z^T, P2 = I - Z E^{-1} Z^T B.
After the first cycle (iterate u1, residual r1 = b - B u1) the correction
delta with B delta = r1 is found by GMRES(m) on P1 B t = P1 r1 and
delta = P2 t + Z E^{-1} Z^T r1; x = M^{-1} (u1 + delta).  As for PDGMRES,
b - A x = P1 (r1 - B t), so the GMRES residual is the true residual.

Library steps: numpy.linalg.eig for the m x m harmonic Ritz problem,
numpy.linalg.solve for E and the small triangular systems.
"""
from __future__ import annotations

import numpy as np

OK, NOT_CONVERGED = 0, 3


class RdgmresResult:
    def __init__(self, x, iterations, cycles, true_relres, status, hist, Z, theta):
        self.x, self.iterations, self.cycles = x, iterations, cycles
        self.true_relres, self.status, self.hist = true_relres, status, hist
        self.Z, self.theta = Z, theta


def _cycle(op, r0, m, tol_abs, its, maxiter, hist, bnorm):
    """One GMRES(m) cycle on op from residual r0 (modified Gram-Schmidt,
    Givens).  Returns (V, Hbar, k, u, its)."""
    n = r0.size
    beta = float(np.linalg.norm(r0))
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    R = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[0] = r0 / beta
    k = 0
    for j in range(m):
        w = op(V[j])
        for i in range(j + 1):
            H[i, j] = float(w @ V[i])
            w = w - H[i, j] * V[i]
        H[j + 1, j] = float(np.linalg.norm(w))
        if H[j + 1, j] > 0.0:
            V[j + 1] = w / H[j + 1, j]
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
        if abs(g[j + 1]) <= tol_abs or H[j + 1, j] == 0.0 or its >= maxiter:
            break
    u = np.linalg.solve(R[:k, :k], g[:k]) if k > 0 else np.zeros(0)
    return V, H, k, u, its


def harmonic_ritz(V, H, d):
    """The d harmonic Ritz vectors (columns, real basis) of the smallest
    |theta| from an Arnoldi cycle of m steps (H: (m+1) x m), and the values."""
    m = H.shape[1]
    Hm = H[:m, :m]
    em = np.zeros(m)
    em[-1] = 1.0
    F = Hm + H[m, m - 1] ** 2 * np.linalg.solve(Hm.T, em)[:, None] * em[None, :]
    theta, Y = np.linalg.eig(F)
    order = np.argsort(np.abs(theta))
    cols, vals = [], []
    i = 0
    while len(cols) < d and i < m:
        k = order[i]
        y = Y[:, k]
        if abs(theta[k].imag) > 0 and len(cols) + 2 <= d:
            cols += [y.real, y.imag]  # the pair's real and imaginary parts span its space
            vals += [theta[k], np.conj(theta[k])]
            i += 2 if i + 1 < m and np.isclose(theta[order[i + 1]], np.conj(theta[k])) else 1
            continue
        cols.append(y.real)
        vals.append(theta[k])
        i += 1
    Yr = np.stack(cols[:d], axis=1)
    return V[:m].T @ Yr, np.array(vals[:d])


def rdgmres(A, d=3, b=None, m=30, tol=1e-6, maxiter=5000) -> RdgmresResult:
    n = A.n
    b = A.b if b is None else np.asarray(b, dtype=np.float64)
    dia = A.diag()

    def B(v):
        return A.spmv(v / dia)

    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return RdgmresResult(np.zeros(n), 0, 0, 0.0, OK, np.array([0.0]), None, None)
    hist = [1.0]
    tol_abs = tol * bnorm
    # first cycle: plain GMRES(m) from u = 0
    V, H, k, y, its = _cycle(B, b.copy(), m, tol_abs, 0, maxiter, hist, bnorm)
    u1 = y @ V[:k]
    r1 = b - B(u1)
    cycles = 1
    if np.linalg.norm(r1) <= tol_abs or its >= maxiter or k < m:
        x = u1 / dia
        tr = float(np.linalg.norm(b - A.spmv(x)) / bnorm)
        return RdgmresResult(x, its, cycles, tr, OK if np.linalg.norm(r1) <= tol_abs else NOT_CONVERGED,
                             np.array(hist), None, None)
    Z, theta = harmonic_ritz(V, H, d)
    BZ = np.stack([B(Z[:, k]) for k in range(Z.shape[1])], axis=1)
    E = Z.T @ BZ

    def P1(w):
        return w - BZ @ np.linalg.solve(E, Z.T @ w)

    def op(v):
        return P1(B(v))

    t = np.zeros(n)
    converged = False
    while True:
        r = P1(r1 - B(t))
        if np.linalg.norm(r) <= tol_abs:
            converged = True
            break
        if its >= maxiter:
            break
        cycles += 1
        V, H, k, y, its = _cycle(op, r, m, tol_abs, its, maxiter, hist, bnorm)
        t = t + y @ V[:k]
    delta = t - Z @ np.linalg.solve(E, Z.T @ B(t)) + Z @ np.linalg.solve(E, Z.T @ r1)
    x = (u1 + delta) / dia
    tr = float(np.linalg.norm(b - A.spmv(x)) / bnorm)
    return RdgmresResult(x, its, cycles, tr, OK if converged else NOT_CONVERGED, np.array(hist), Z, theta)
