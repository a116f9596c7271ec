"""Pins for the CPU oracle: each test checks the oracle against something other
than itself (closed forms, hand-derived fixtures, dense linear algebra,
SciPy's CG, dense eigenvalues, brute-force recounts).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from paper_1510_02148_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lognormal(shape, seed, sigma=1.0):
    return np.exp(sigma * np.random.default_rng(seed).standard_normal(shape))


# --------------------------------------------------------------------------
# Assembly (a1): hand-derived fixtures, closed forms, structure
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["tpfa_3cell.json", "tpfa_4cell.json"])
def test_golden_tpfa(oracle_mod, name):
    g = json.load(open(os.path.join(GOLDEN, name)))
    K = np.array(g["K"]).reshape(g["nz"], g["ny"], g["nx"])
    q = np.array(g["q"]).reshape(K.shape)
    A = oracle_mod.assemble(K, q, g["bc_type"], g["bc_value"])
    np.testing.assert_allclose(A.dense(), np.array(g["A"]), rtol=1e-15, atol=0)
    np.testing.assert_allclose(A.b, np.array(g["b"]), rtol=1e-15, atol=0)
    r = oracle_mod.dpcg(A, None, 0, tol=1e-14)
    np.testing.assert_allclose(r.x, np.array(g["x"]), rtol=1e-13, atol=1e-15)


def test_series_resistance_column(oracle_mod):
    """1-D column with Dirichlet ends: the flux equals the pressure drop over
    the sum of half-cell resistances 1/(2K) (series resistors); the pressure
    falls by flux * resistance across each face.  An arithmetic-mean face
    coefficient fails this."""
    K = np.array([0.3, 5.0, 0.01, 2.0, 7.5, 1e-3, 1.0])
    A = oracle_mod.assemble(K.reshape(1, 1, -1))
    r = oracle_mod.dpcg(A, None, 0, tol=1e-15)
    R = 1.0 / (2 * K[:-1]) + 1.0 / (2 * K[1:])
    F = 1.0 / R.sum()
    expect = 1.0 - F * np.concatenate([[0.0], np.cumsum(R)])
    np.testing.assert_allclose(r.x, expect, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("kind", ["homogeneous", "layered"])
def test_linear_pressure_closed_form(oracle_mod, kind):
    """K independent of x with Dirichlet x-faces and no-flow elsewhere: the
    discrete solution is exactly p = 1 - ix/(nx-1) (two-point flux is exact
    for linear fields; z-fluxes vanish because p does not vary in z)."""
    nx, ny, nz = 12, 5, 8
    if kind == "homogeneous":
        K = np.full((nz, ny, nx), 2.5)
        tol = 1e-13
    else:
        K = W.layered(nx, ny, nz, 4, 1.0, 1e-6)
        tol = 1e-14
    A = oracle_mod.assemble(K)
    lab = oracle_mod.labels(K, (2, 1, 2), (1e-3,), 2)
    r = oracle_mod.dpcg(A, lab, 8, tol=tol)
    exact = np.broadcast_to(1.0 - np.arange(nx) / (nx - 1), K.shape).reshape(-1)
    assert np.linalg.norm(r.x - exact) / np.linalg.norm(exact) < 1e-9
    assert r.true_relres < 1e-12


def test_layered_sandwich_32_closed_form(oracle_mod):
    """The 32^3 layered workload itself (K depends on z only, BC on x only,
    q = 0) has the same closed-form linear solution."""
    P = W.layered_sandwich()
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
    exact = np.broadcast_to(1.0 - np.arange(32) / 31.0, P.K.shape).reshape(-1)
    # at the workload's tolerance the error is bounded by cond(A) * 1e-9
    r = oracle_mod.dpcg(A, lab, P.d, tol=P.tol)
    assert r.true_relres <= 1.01e-9
    assert np.linalg.norm(r.x - exact) / np.linalg.norm(exact) < 1e-5
    # and it converges to the closed form as the tolerance tightens
    r = oracle_mod.dpcg(A, lab, P.d, tol=1e-13)
    assert np.linalg.norm(r.x - exact) / np.linalg.norm(exact) < 1e-9


def test_matrix_structure(oracle_mod):
    K = _lognormal((4, 5, 6), 3, 2.0)
    A = oracle_mod.assemble(K)
    D = A.dense()
    assert np.array_equal(D, D.T)                     # symmetric, bitwise
    assert np.all(np.linalg.eigvalsh(D) > 0)          # SPD
    isd = A.is_dirichlet.astype(bool)
    # Dirichlet rows are identity rows
    assert np.array_equal(D[isd][:, isd], np.eye(isd.sum()))
    # rows of free cells away from Dirichlet cells sum to zero
    # (x-Dirichlet faces: the cells with ix in {0, 1, nx-2, nx-1})
    ix = np.broadcast_to(np.arange(6), K.shape).reshape(-1)
    assert np.array_equal(isd, (ix == 0) | (ix == 5))
    near = (ix <= 1) | (ix >= 4)
    rs = D[~near].sum(axis=1)
    assert np.max(np.abs(rs)) <= 1e-13 * np.max(np.abs(D))
    # the off-diagonal of a face is minus the harmonic mean
    i, j = 1 + 0 * 6, 2  # cells (1,0,0) and (2,0,0), both free
    Ki, Kj = K.reshape(-1)[1], K.reshape(-1)[2]
    assert D[1, 2] == -(2 * Ki * Kj) / (Ki + Kj)


def test_dense_direct_solve(oracle_mod):
    K = _lognormal((4, 5, 6), 7, 2.0)
    q = np.random.default_rng(8).standard_normal(K.shape)
    A = oracle_mod.assemble(K, q)
    lab = oracle_mod.labels(K, (2, 2, 2), (1.0,), 2)
    r = oracle_mod.dpcg(A, lab, 16, tol=1e-14)
    xd = np.linalg.solve(A.dense(), A.b)
    assert np.linalg.norm(r.x - xd) / np.linalg.norm(xd) < 1e-10


# --------------------------------------------------------------------------
# Labels (a2): brute-force recount
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape,S,L", [((3, 5, 7), (3, 2, 2), 3), ((8, 8, 8), (2, 2, 2), 2),
                                       ((1, 1, 9), (4, 1, 1), 2), ((5, 4, 6), (6, 4, 5), 1)])
def test_labels_bruteforce(oracle_mod, shape, S, L):
    nz, ny, nx = shape
    K = _lognormal(shape, 11, 3.0)
    tau = np.sort(np.random.default_rng(12).lognormal(0, 2, L - 1))
    if L > 1:
        K.reshape(-1)[0] = tau[0]  # a tie goes to the upper class
    lab = oracle_mod.labels(K, S, tau, L).reshape(shape)
    Sx, Sy, Sz = S
    expect = np.full(shape, -1)
    # subdomain s along an axis of n cells holds the cells with
    # s*n/S <= i < (s+1)*n/S, i.e. ceil(s*n/S) <= i < ceil((s+1)*n/S)
    cls = np.searchsorted(tau, K, side="right") if L > 1 else np.zeros(shape, int)
    for sz in range(Sz):
        for sy in range(Sy):
            for sx in range(Sx):
                zs = slice(-(-sz * nz // Sz), -(-(sz + 1) * nz // Sz))
                ys = slice(-(-sy * ny // Sy), -(-(sy + 1) * ny // Sy))
                xs = slice(-(-sx * nx // Sx), -(-(sx + 1) * nx // Sx))
                expect[zs, ys, xs] = ((sz * Sy + sy) * Sx + sx) * L + cls[zs, ys, xs]
    assert np.array_equal(lab, expect)
    if L > 1:
        assert lab.reshape(-1)[0] % L == 1


# --------------------------------------------------------------------------
# Coarse matrix (a3): dense Z^T A Z, symmetry, SPD, pinned empty columns
# --------------------------------------------------------------------------
def test_coarse_matrix_dense(oracle_mod):
    K = _lognormal((6, 5, 7), 21, 2.5)
    A = oracle_mod.assemble(K)
    d = 2 * 2 * 3 * 2
    lab = oracle_mod.labels(K, (2, 2, 3), (1.0,), 2)
    Zd = np.random.default_rng(22).standard_normal((K.size, 3))
    E, Lc = oracle_mod.coarse(A, lab, d, Zd)
    Z = np.concatenate([np.eye(d)[lab], Zd], axis=1)
    Ed = Z.T @ A.dense() @ Z
    empty = np.bincount(lab, minlength=d) == 0
    Ed[np.flatnonzero(empty), np.flatnonzero(empty)] = 1.0
    np.testing.assert_allclose(E, Ed, rtol=1e-12, atol=1e-12 * np.abs(Ed).max())
    np.testing.assert_allclose(E, E.T, rtol=1e-12, atol=1e-13 * np.abs(E).max())
    assert Lc is not None
    np.testing.assert_allclose(Lc @ Lc.T, E, rtol=1e-10, atol=1e-12 * np.abs(E).max())


def test_coarse_face_rule(oracle_mod):
    """Faces inside one label contribute nothing to E; a face between labels k
    and l adds T to E_kk and E_ll and -T to E_kl; a free-Dirichlet face adds T
    at the free cell's label only; a Dirichlet cell adds 1 at its label."""
    K = np.array([1.0, 3.0, 2.0, 1.0, 4.0]).reshape(1, 1, 5)
    A = oracle_mod.assemble(K)
    lab = np.array([0, 0, 1, 1, 1], dtype=np.int32)
    E, _ = oracle_mod.coarse(A, lab, 2)
    T = lambda a, b: 2 * a * b / (a + b)
    T01, T12 = T(1.0, 3.0), T(3.0, 2.0)
    T34 = T(1.0, 4.0)
    # label 0 = {Dirichlet cell 0, free cell 1}; label 1 = {free 2, free 3, Dirichlet 4}
    E00 = 1.0 + T01 + T12          # Dirichlet identity + free-Dirichlet face + crossing face
    E11 = 1.0 + T12 + T34          # crossing face + free-Dirichlet face + Dirichlet identity
    np.testing.assert_allclose(E, [[E00, -T12], [-T12, E11]], rtol=1e-15)


def test_cholesky(oracle_mod):
    rng = np.random.default_rng(5)
    B = rng.standard_normal((9, 9))
    E = B @ B.T + 9 * np.eye(9)
    np.testing.assert_allclose(oracle_mod.cholesky(E), np.linalg.cholesky(E), rtol=1e-12)
    E[3, 3] = -1.0
    assert oracle_mod.cholesky(E) is None


# --------------------------------------------------------------------------
# Deflation operator and iteration (a4-a7)
# --------------------------------------------------------------------------
def test_projection_invariants(oracle_mod):
    K = W.lognormal_layered(8, 8, 8, 4, 1.0, 1e-4, 1.0, seed=3)
    A = oracle_mod.assemble(K, W.point_source(8, 8, 8))
    lab = oracle_mod.labels(K, (2, 2, 2), (1e-2,), 2)
    E, _ = oracle_mod.coarse(A, lab, 16)
    Z = np.eye(16)[lab]
    Ad = A.dense()
    AZ = Ad @ Z
    P = np.eye(A.n) - AZ @ np.linalg.solve(E, Z.T)
    assert np.linalg.norm(P @ AZ) / np.linalg.norm(AZ) < 1e-12        # P A Z = 0
    assert np.linalg.norm(Z.T @ P) / np.linalg.norm(Z) < 1e-12        # Z^T P = 0
    r = oracle_mod.dpcg(A, lab, 16, tol=1e-10, history=True)
    assert r.ztr_max < 1e-13                                          # Z^T r_k = 0
    assert r.true_relres < 2e-10
    # the recursive residual equals the true residual of the recovered x
    assert abs(r.hist[-1] - r.true_relres) < 1e-11


def test_invariant_subspace_deflates_exactly(oracle_mod):
    """With Z spanning exact eigenvectors, P A has d zero eigenvalues and the
    remaining spectrum is that of A minus those eigenvalues (Def. 3.1
    discussion: deflating d eigenvalues to zero)."""
    K = _lognormal((3, 4, 5), 31, 1.0)
    A = oracle_mod.assemble(K)
    Ad = A.dense()
    lam, V = np.linalg.eigh(Ad)
    Zd = V[:, :3]
    E, _ = oracle_mod.coarse(A, None, 0, Zd)
    P = np.eye(A.n) - Ad @ Zd @ np.linalg.solve(E, Zd.T)
    mu = np.sort(np.linalg.eigvalsh(0.5 * (P @ Ad + (P @ Ad).T)))
    assert np.all(np.abs(mu[:3]) < 1e-10 * lam[-1])
    np.testing.assert_allclose(mu[3:], lam[3:], rtol=1e-9)
    r = oracle_mod.dpcg(A, None, 0, tol=1e-12, Zd=Zd)
    xd = np.linalg.solve(Ad, A.b)
    assert np.linalg.norm(r.x - xd) / np.linalg.norm(xd) < 1e-10


def test_d0_is_jacobi_pcg(oracle_mod):
    """Without deflation vectors the iteration is textbook Jacobi-PCG."""
    import scipy.sparse.linalg as sla
    K = _lognormal((6, 7, 8), 41, 1.5)
    A = oracle_mod.assemble(K, W.point_source(8, 7, 6))
    r = oracle_mod.dpcg(A, None, 0, tol=1e-10)
    S = A.to_scipy()
    dinv = 1.0 / A.diag()
    M = sla.LinearOperator(S.shape, matvec=lambda v: dinv * v)
    count = [0]
    x, info = sla.cg(S, A.b, rtol=1e-10, atol=0.0, M=M, maxiter=5000,
                     callback=lambda xk: count.__setitem__(0, count[0] + 1))
    assert info == 0
    assert abs(count[0] - r.iterations) <= 1
    assert np.linalg.norm(r.x - x) / np.linalg.norm(x) < 1e-8


def test_single_label_and_empty_labels(oracle_mod):
    K = _lognormal((4, 4, 4), 51, 1.0)
    A = oracle_mod.assemble(K)
    xd = np.linalg.solve(A.dense(), A.b)
    one = np.zeros(K.size, dtype=np.int32)
    r1 = oracle_mod.dpcg(A, one, 1, tol=1e-12)
    assert np.linalg.norm(r1.x - xd) / np.linalg.norm(xd) < 1e-9
    # labels 0 and 2 used, 1 and 3 empty: E pinned, same solution
    lab = np.where(np.arange(K.size) % 2 == 0, 0, 2).astype(np.int32)
    r2 = oracle_mod.dpcg(A, lab, 4, tol=1e-12)
    assert np.linalg.norm(r2.x - xd) / np.linalg.norm(xd) < 1e-9


# --------------------------------------------------------------------------
# Spectral claims (Theorem 3.1) and jump independence
# --------------------------------------------------------------------------
def _scaled(Ad):
    s = 1.0 / np.sqrt(np.diag(Ad))
    return s[:, None] * Ad * s[None, :]


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_theorem31_eigen_count(oracle_mod, eps):
    """Theorem 3.1 (cf. Vuik99): the diagonally scaled matrix has as many O(eps)
    eigenvalues as there are high-permeability layers lying between
    low-permeability layers (no-flow everywhere, Dirichlet on top).  Layers
    bottom to top: H L H L H L, the top L touching the Dirichlet face, so 3
    floating high layers.  With one subdomain per layer (SLD), deflation removes
    all of them; with one subdomain (levelset only) two remain."""
    P = W.sandwich_theorem(eps=eps)
    A = oracle_mod.assemble(P.K, None, P.bc_type, P.bc_value)
    Ad = A.dense()
    lam = np.sort(np.linalg.eigvalsh(_scaled(Ad)))
    small = lam[lam < 100 * eps]
    assert len(small) == 3
    assert np.all(small > 0.01 * eps)        # O(eps), not smaller

    sc = 1.0 / np.sqrt(np.diag(Ad))

    def deflated_spectrum(S, d):
        lab = oracle_mod.labels(P.K, S, P.tau, P.L)
        E, _ = oracle_mod.coarse(A, lab, d)
        Z = np.eye(d)[lab]
        PA = Ad - Ad @ Z @ np.linalg.solve(E, Z.T @ Ad)
        mu = np.sort(np.linalg.eigvalsh(sc[:, None] * (0.5 * (PA + PA.T)) * sc[None, :]))
        used = int(np.count_nonzero(np.bincount(lab, minlength=d)))
        return mu, used

    mu, nzc = deflated_spectrum(P.S, P.d)            # one subdomain per layer
    assert np.all(np.abs(mu[:nzc]) < 1e-9)
    assert mu[nzc] > 1e3 * eps                       # no O(eps) eigenvalue left
    mu1, nz1 = deflated_spectrum((1, 1, 1), 2)      # levelset only
    rest = mu1[nz1:]
    assert np.sum(rest < 100 * eps) == 2


def test_jump_independence(oracle_mod):
    """DPCG iteration counts stay flat as the contrast grows, PCG's grow
    (Section 1: convergence of deflated CG independent of the jump size).
    Layered field with no-flow sides and a Dirichlet top, so the high layers
    float (the Theorem 3.1 setting), and a point source near the bottom."""
    it_d, it_p = [], []
    for eps in (1e-2, 1e-4, 1e-6, 1e-8):
        P = W.sandwich_theorem(16, 16, 16, 8, eps)
        q = W.point_source(16, 16, 16, 1.0, at=(5, 9, 1))
        A = oracle_mod.assemble(P.K, q, P.bc_type, P.bc_value)
        lab = oracle_mod.labels(P.K, (1, 1, 8), P.tau, 2)
        it_d.append(oracle_mod.dpcg(A, lab, 16, tol=1e-9).iterations)
        it_p.append(oracle_mod.dpcg(A, None, 0, tol=1e-9).iterations)
    # deflated counts do not grow with the contrast (they settle), PCG's do
    assert max(it_d) <= it_d[0] + 4, it_d
    assert it_p[-1] > 1.3 * it_p[0], it_p
    assert all(a <= b for a, b in zip(it_d, it_p)), (it_d, it_p)


def test_restrict_is_z_transpose_times_v(oracle_mod):
    """oracle.restrict(label, d, v) = Z^T v, with Z the explicit indicator
    matrix of the labels (dense on a small grid), and with extra dense
    columns appended; empty labels give exact zeros."""
    rng = np.random.default_rng(31)
    n, d, k = 300, 11, 3
    lab = rng.integers(0, d - 2, n).astype(np.int32)  # labels d-2, d-1 never used
    v = rng.standard_normal(n)
    Z = np.zeros((n, d))
    Z[np.arange(n), lab] = 1.0
    s = oracle_mod.restrict(lab, d, v)
    np.testing.assert_allclose(s, Z.T @ v, rtol=1e-13, atol=1e-13)
    assert s[d - 2] == 0.0 and s[d - 1] == 0.0
    Zd = rng.standard_normal((n, k))
    s2 = oracle_mod.restrict(lab, d, v, Zd=Zd)
    np.testing.assert_allclose(s2, np.concatenate([Z.T @ v, Zd.T @ v]), rtol=1e-12, atol=1e-12)
    # a mistake that swaps labels or drops cells would change these sums
    np.testing.assert_allclose(np.sum(s), np.sum(v), rtol=1e-12)
