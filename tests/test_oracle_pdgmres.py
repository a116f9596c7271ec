"""Pins for the PDGMRES oracle (deflated, right-Jacobi-preconditioned
restarted GMRES, Section 3.2 with the subdomain-levelset vectors of Section
3.2.2): against dense direct solves, the minimal-residual definition of a
GMRES iterate solved by dense least squares on an explicit Krylov basis,
SciPy's restarted GMRES on the same (deflated, right-preconditioned)
operator, the Arnoldi relation, finite termination, and the projection
identities.  CPU only."""
import numpy as np
import pytest

from paper_1510_02148_gb300 import workloads as W


@pytest.fixture(scope="module")
def gm():
    import oracle
    from oracle import pdgmres
    oracle.build()
    return oracle, pdgmres


def _case(oracle, shape=(6, 7, 8), seed=3, S=(2, 2, 2), contrast=1e-4):
    nz, ny, nx = shape
    K = W.lognormal_layered(nx, ny, nz, 4, 1.0, contrast, 1.0, seed=seed)
    A = oracle.assemble(K, W.point_source(nx, ny, nz))
    lab = oracle.labels(K, S, (1e-2,), 2)
    d = 2 * S[0] * S[1] * S[2]
    return K, A, lab, d


@pytest.mark.parametrize("m", [5, 20])
@pytest.mark.parametrize("defl", [False, True])
def test_matches_dense_direct_solve(gm, m, defl):
    oracle, P = gm
    K, A, lab, d = _case(oracle)
    r = P.pdgmres(A, lab if defl else None, d if defl else 0, m=m, tol=1e-11, maxiter=20000)
    assert r.status == P.OK
    xd = np.linalg.solve(A.dense(), A.b)
    assert np.linalg.norm(r.x - xd) / np.linalg.norm(xd) < 1e-7
    assert r.true_relres <= 2e-11


@pytest.mark.parametrize("defl", [False, True])
def test_iterates_minimise_the_residual_over_the_krylov_space(gm, defl):
    """GMRES by definition: after j steps of the first cycle the residual is
    the minimum of ||r0 - B K_j c|| over c, B = P1 A M^{-1}, K_j the explicit
    (unorthogonalised) Krylov basis [r0, B r0, ..., B^{j-1} r0]; here by
    dense least squares."""
    oracle, P = gm
    K, A, lab, d = _case(oracle, shape=(4, 5, 6), seed=7)
    Ad = A.dense()
    Minv = 1.0 / A.diag()
    if defl:
        Z = np.eye(d)[lab]
        E = Z.T @ Ad @ Z
        P1 = np.eye(A.n) - Ad @ Z @ np.linalg.solve(E, Z.T)
    else:
        P1 = np.eye(A.n)
    B = P1 @ Ad @ np.diag(Minv)
    r0 = P1 @ A.b
    res = P.pdgmres(A, lab if defl else None, d if defl else 0, m=8, tol=1e-14, maxiter=8)
    bn = np.linalg.norm(A.b)
    Kry = [r0]
    for j in range(1, 7):
        Kry.append(B @ Kry[-1])
        Kj = np.stack(Kry[:j], axis=1)
        c, *_ = np.linalg.lstsq(B @ Kj, r0, rcond=None)
        best = np.linalg.norm(r0 - B @ Kj @ c) / bn
        assert abs(res.hist[j] - best) <= 1e-9 * max(best, 1e-3), (j, res.hist[j], best)


def test_arnoldi_relation_and_orthonormal_basis(gm):
    oracle, P = gm
    K, A, lab, d = _case(oracle)
    r = P.pdgmres(A, lab, d, m=12, tol=1e-14, maxiter=12, record=True)
    V, H, op = r.arnoldi
    k = H.shape[1]
    BV = np.stack([op(V[j]) for j in range(k)], axis=1)
    assert np.linalg.norm(BV - V.T @ H) / np.linalg.norm(BV) < 1e-12
    G = V @ V.T
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-10


def test_residual_history_and_true_residual(gm):
    """Within a cycle the estimates never increase; at the end the estimate
    is the true residual of x = P2 x~ + x*  (b - A x = P1 (b - A x~))."""
    oracle, P = gm
    K, A, lab, d = _case(oracle, contrast=1e-6)
    r = P.pdgmres(A, lab, d, m=30, tol=1e-10, maxiter=30)
    h = r.hist
    assert np.all(np.diff(h) <= 1e-13)
    assert abs(h[-1] - r.true_relres) <= 1e-9 * max(h[-1], 1e-12) + 1e-15


def test_finite_termination(gm):
    """Without restarts GMRES ends within dim of the Krylov space: n steps for
    the full-rank operator, at most n - d + 1 for the deflated one (P1 A has
    rank n - d)."""
    oracle, P = gm
    K = np.exp(np.random.default_rng(5).standard_normal((2, 3, 4)))
    A = oracle.assemble(K, W.point_source(4, 3, 2))
    n = A.n
    r0 = P.pdgmres(A, None, 0, m=n, tol=1e-10, maxiter=n)
    assert r0.status == P.OK and r0.iterations <= n
    lab = oracle.labels(K, (2, 1, 1), (), 1)
    r1 = P.pdgmres(A, lab, 2, m=n, tol=1e-10, maxiter=n)
    assert r1.status == P.OK and r1.iterations <= n - 2 + 1


def test_deflation_cuts_iterations_on_layered_contrast(gm):
    """The paper's observation (Section 4, PDGMRES vs GMRES): physics-based
    vectors at the permeability jumps take out the slow modes."""
    oracle, P = gm
    K, A, lab, d = _case(oracle, shape=(16, 16, 16), seed=11, contrast=1e-6)
    plain = P.pdgmres(A, None, 0, m=20, tol=1e-6, maxiter=4000)
    defl = P.pdgmres(A, lab, d, m=20, tol=1e-6, maxiter=4000)
    assert defl.status == P.OK
    assert defl.iterations < 0.7 * plain.iterations, (defl.iterations, plain.iterations)


def test_zero_rhs_and_iteration_cap(gm):
    oracle, P = gm
    K, A, lab, d = _case(oracle)
    r = P.pdgmres(A, lab, d, b=np.zeros(A.n), m=10)
    assert r.iterations == 0 and not np.any(r.x)
    capped = P.pdgmres(A, lab, d, m=10, tol=1e-14, maxiter=3)
    assert capped.status == P.NOT_CONVERGED and capped.iterations == 3
    assert np.all(np.isfinite(capped.x)) and capped.true_relres < 1.0


@pytest.mark.parametrize("defl", [False, True])
def test_history_matches_scipy_gmres_on_the_same_operator(gm, defl):
    """SciPy's restarted GMRES (no preconditioner of its own) on the operator
    B = P1 A M^{-1} with right-hand side P1 b minimises the same residual as
    PDGMRES; its per-step residual norms (callback 'pr_norm', relative to
    ||P1 b||) match the oracle's first cycles."""
    import scipy.sparse.linalg as sla
    oracle, P = gm
    K, A, lab, d = _case(oracle, shape=(6, 7, 8), seed=9)
    Ad = A.dense()
    Minv = 1.0 / A.diag()
    if defl:
        Z = np.eye(d)[lab]
        P1 = np.eye(A.n) - Ad @ Z @ np.linalg.solve(Z.T @ Ad @ Z, Z.T)
    else:
        P1 = np.eye(A.n)
    B = P1 @ Ad * Minv[None, :]
    rhs = P1 @ A.b
    hist = []
    sla.gmres(sla.aslinearoperator(B), rhs, rtol=1e-12, atol=0.0, restart=10, maxiter=3,
              callback=lambda r: hist.append(r), callback_type="pr_norm")
    res = P.pdgmres(A, lab if defl else None, d if defl else 0, m=10, tol=1e-12, maxiter=30)
    bn = np.linalg.norm(A.b)
    ours = res.hist[1:1 + len(hist)] * bn / np.linalg.norm(rhs)
    k = min(len(hist), 25)
    np.testing.assert_allclose(ours[:k], np.array(hist[:k]), rtol=1e-6, atol=1e-13)
