"""Pins for the RDGMRES oracle (restarted GMRES with harmonic-Ritz
deflation, Section 3.2.1): the dense direct solve, the first cycle equal to
plain GMRES, the Petrov-Galerkin condition of the harmonic Ritz pairs, exact
eigenvalues when the Krylov space is the whole space, and the deflation gain
the paper reports for cycles long enough.  CPU only."""
import numpy as np
import pytest

from paper_1510_02148_gb300 import workloads as W


@pytest.fixture(scope="module")
def rd():
    import oracle
    from oracle import pdgmres, rdgmres
    oracle.build()
    return oracle, pdgmres, rdgmres


def _A(oracle, shape=(6, 7, 8), seed=3, contrast=1e-4):
    nz, ny, nx = shape
    K = W.lognormal_layered(nx, ny, nz, 4, 1.0, contrast, 1.0, seed=seed)
    return oracle.assemble(K, W.point_source(nx, ny, nz))


def test_matches_dense_direct_solve(rd):
    oracle, PG, RD = rd
    A = _A(oracle)
    r = RD.rdgmres(A, d=3, m=20, tol=1e-11, maxiter=20000)
    assert r.status == RD.OK and r.cycles > 1 and r.Z is not None
    xd = np.linalg.solve(A.dense(), A.b)
    assert np.linalg.norm(r.x - xd) / np.linalg.norm(xd) < 1e-7
    assert r.true_relres <= 2e-11


def test_first_cycle_is_plain_gmres(rd):
    oracle, PG, RD = rd
    A = _A(oracle, seed=4)
    m = 15
    r = RD.rdgmres(A, d=2, m=m, tol=1e-12, maxiter=m)
    p = PG.pdgmres(A, None, 0, m=m, tol=1e-12, maxiter=m)
    np.testing.assert_allclose(r.hist[: m + 1], p.hist[: m + 1], rtol=1e-12, atol=1e-15)


def test_harmonic_ritz_petrov_galerkin(rd):
    """(B V_m)^T (B z - theta z) = 0 for the real harmonic Ritz pairs."""
    oracle, PG, RD = rd
    A = _A(oracle, seed=5)
    m = 12
    p = PG.pdgmres(A, None, 0, m=m, tol=1e-14, maxiter=m, record=True)
    V, H, op = p.arnoldi
    Z, theta = RD.harmonic_ritz(V, H, 4)
    Bd = A.dense() / A.diag()[None, :]
    BV = Bd @ V[:m].T
    for k in range(Z.shape[1]):
        if abs(theta[k].imag) > 0:
            continue
        z = Z[:, k]
        res = BV.T @ (Bd @ z - theta[k].real * z)
        assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(BV) * np.linalg.norm(Bd @ z)


def test_invariant_krylov_space_gives_exact_eigenvalues(rd):
    """When the Krylov space of the start vector is invariant (Arnoldi breaks
    down, h_{k+1,k} = 0), the harmonic Ritz values are exact eigenvalues of
    B = A M^{-1}: for a generic start, its distinct eigenvalues.  (The
    Dirichlet rows give B the eigenvalue 1 many times over, so the space has
    fewer dimensions than n.)  The Arnoldi steps here are the test's own,
    dense, with full reorthogonalisation."""
    oracle, PG, RD = rd
    K = np.exp(np.random.default_rng(7).standard_normal((2, 3, 4)))
    A = oracle.assemble(K, W.point_source(4, 3, 2))
    n = A.n
    Bd = A.dense() / A.diag()[None, :]
    v = np.random.default_rng(8).standard_normal(n)
    V = [v / np.linalg.norm(v)]
    H = np.zeros((n + 1, n))
    k = 0
    for j in range(n):
        w = Bd @ V[j]
        for _ in range(2):
            for i in range(j + 1):
                c = w @ V[i]
                H[i, j] += c
                w = w - c * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        k = j + 1
        if H[j + 1, j] < 1e-10 * np.linalg.norm(H[: j + 2, : j + 1]):
            H[j + 1, j] = 0.0
            V.append(np.zeros(n))
            break
        V.append(w / H[j + 1, j])
    assert k < n
    _, theta = RD.harmonic_ritz(np.array(V), H[: k + 1, :k], 3)
    ev = np.linalg.eigvals(Bd).real
    distinct = np.unique(np.round(ev, 9))
    expect = distinct[np.argsort(np.abs(distinct))][:3]
    np.testing.assert_allclose(np.sort(np.abs(theta)), np.sort(np.abs(expect)), rtol=1e-7)


def test_deflation_gain_with_long_cycles(rd):
    """The paper's observation: with cycles long enough for the harmonic Ritz
    vectors to settle, RDGMRES(m, d) needs fewer steps than GMRES(m)."""
    oracle, PG, RD = rd
    A = _A(oracle, shape=(16, 16, 16), seed=11, contrast=1e-6)
    plain = PG.pdgmres(A, None, 0, m=30, tol=1e-8, maxiter=20000)
    defl = RD.rdgmres(A, d=3, m=30, tol=1e-8, maxiter=20000)
    assert defl.status == RD.OK and plain.status == PG.OK
    assert defl.iterations < plain.iterations, (defl.iterations, plain.iterations)
