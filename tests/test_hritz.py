"""The harmonic Ritz routine of the C library (sld_harmonic_ritz, host code:
Francis double-shift QR and inverse iteration) against numpy's dense
eigensolver on the same matrix and against the RDGMRES oracle's harmonic
Ritz vectors on real Arnoldi data.  CPU only (no GPU call)."""
import numpy as np
import pytest

from paper_1510_02148_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_1510_02148_gb300 import _build, sld
    try:
        path = _build.build()
    except RuntimeError as e:  # no nvcc here
        pytest.skip(str(e))
    sld.load(path)
    return sld


def _F(H):
    m = H.shape[1]
    em = np.zeros(m)
    em[-1] = 1.0
    return H[:m, :m] + H[m, m - 1] ** 2 * np.linalg.solve(H[:m, :m].T, em)[:, None] * em[None, :]


@pytest.mark.parametrize("seed", range(6))
def test_random_hessenberg_against_numpy(lib, seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(3, 30))
    H = np.triu(rng.standard_normal((m + 1, m)), -1)
    d = min(4, m)
    Y, theta = lib.harmonic_ritz(H, d)
    F = _F(H)
    ev = np.linalg.eigvals(F)
    ev = ev[np.argsort(np.abs(ev))]
    # the smallest |theta| agree with numpy's (a conjugate pair counts twice)
    np.testing.assert_allclose(np.sort(np.abs(theta)), np.sort(np.abs(ev[:d])), rtol=1e-8, atol=1e-12)
    # each real column (theta real) is an eigenvector of F
    for k in range(d):
        if theta[k].imag == 0:
            y = Y[:, k]
            assert np.linalg.norm(F @ y - theta[k].real * y) <= 1e-8 * np.linalg.norm(F) * np.linalg.norm(y)


def test_complex_pair_spans_the_invariant_subspace(lib):
    # a rotation block with eigenvalues 0.1 +- 0.5i, the rest far away
    m = 6
    F = np.diag([5.0, 6.0, 7.0, 8.0, 0.0, 0.0])
    F[4:, 4:] = [[0.1, 0.5], [-0.5, 0.1]]
    F = np.triu(F + np.triu(np.ones((m, m)), 1) * 0.01, -1)
    H = np.vstack([F, np.zeros((1, m))])  # h_{m+1,m} = 0: F = H_m
    Y, theta = lib.harmonic_ritz(H, 2)
    ev = np.linalg.eigvals(F)
    pair = ev[np.argsort(np.abs(ev))][:2]  # 0.1 +- i sqrt(0.51 * 0.5)
    assert np.allclose(np.sort(theta.imag), np.sort(pair.imag)) and np.allclose(theta.real, pair.real)
    # span(Y) is invariant under F
    Q, _ = np.linalg.qr(Y)
    assert np.linalg.norm(F @ Q - Q @ (Q.T @ F @ Q)) <= 1e-9 * np.linalg.norm(F)


def test_same_space_as_the_oracle_on_arnoldi_data(lib):
    import oracle
    from oracle import pdgmres, rdgmres
    oracle.build()
    K = W.lognormal_layered(8, 7, 6, 4, 1.0, 1e-4, 1.0, seed=5)
    A = oracle.assemble(K, W.point_source(8, 7, 6))
    p = pdgmres.pdgmres(A, None, 0, m=12, tol=1e-14, maxiter=12, record=True)
    V, H, _ = p.arnoldi
    Zo, th_o = rdgmres.harmonic_ritz(V, H, 3)
    Y, th = lib.harmonic_ritz(H, 3)
    np.testing.assert_allclose(np.sort(np.abs(th)), np.sort(np.abs(th_o)), rtol=1e-8)
    Zg = V[:12].T @ Y
    Qo, _ = np.linalg.qr(Zo)
    Qg, _ = np.linalg.qr(Zg)
    s = np.linalg.svd(Qo.T @ Qg, compute_uv=False)
    assert np.all(s > 1 - 1e-8)  # the same 3-dimensional space


def test_argument_errors(lib):
    with pytest.raises(lib.SldError, match="INVALID_ARG"):
        lib.harmonic_ritz(np.zeros((2, 1)), 1)


def test_all_pairs_span_the_whole_space(lib):
    """d = m: every eigenvalue of F once (a conjugate pair as two values) and
    a basis of the whole space."""
    rng = np.random.default_rng(11)
    m = 9
    H = np.triu(rng.standard_normal((m + 1, m)), -1)
    Y, theta = lib.harmonic_ritz(H, m)
    ev = np.linalg.eigvals(_F(H))
    np.testing.assert_allclose(np.sort_complex(theta), np.sort_complex(ev), rtol=1e-8, atol=1e-12)
    assert np.linalg.matrix_rank(Y, tol=1e-8 * np.linalg.norm(Y)) == m


def test_largest_cycle(lib):
    rng = np.random.default_rng(12)
    m = 64
    H = np.triu(rng.standard_normal((m + 1, m)), -1) + 4.0 * np.eye(m + 1, m)
    Y, theta = lib.harmonic_ritz(H, 5)
    ev = np.linalg.eigvals(_F(H))
    np.testing.assert_allclose(np.sort(np.abs(theta)), np.sort(np.abs(ev))[:5], rtol=1e-8)


def test_singular_and_non_finite_hessenberg(lib):
    m = 5
    H = np.triu(np.ones((m + 1, m)), -1)
    H[:, 2] = 0.0   # H_m singular while h_{m+1,m} != 0: F is undefined
    with pytest.raises(lib.SldError, match="BREAKDOWN"):
        lib.harmonic_ritz(H, 2)
    H = np.triu(np.ones((m + 1, m)), -1) + np.eye(m + 1, m)
    H[1, 3] = np.nan
    with pytest.raises(lib.SldError):
        lib.harmonic_ritz(H, 2)
    with pytest.raises(lib.SldError, match="INVALID_ARG"):
        lib.harmonic_ritz(np.triu(np.ones((66, 65)), -1), 2)
    with pytest.raises(lib.SldError, match="INVALID_ARG"):
        lib.harmonic_ritz(np.triu(np.ones((5, 4)), -1), 5)


@pytest.mark.parametrize("scale", [2.0 ** -560, 1e-170, 1e150])
def test_tiny_and_huge_hessenberg(lib, scale):
    """Entries near 1e-170: unscaled, the products that form h^2 and the
    bulge-chase 3-vectors underflow to exact zeros (the reflector step then
    has nothing to act on); near 1e150 they overflow.  The eigenvalues scale
    with H and the eigenvectors do not, so the result is the unit-scale one
    times `scale`."""
    rng = np.random.default_rng(21)
    m = 12
    H = np.triu(rng.standard_normal((m + 1, m)), -1) + 2.0 * np.eye(m + 1, m)
    Y1, th1 = lib.harmonic_ritz(H, 4)
    Ys, ths = lib.harmonic_ritz(H * scale, 4)
    np.testing.assert_allclose(ths.real, th1.real * scale, rtol=1e-10, atol=1e-12 * scale)
    np.testing.assert_allclose(ths.imag, th1.imag * scale, rtol=1e-10, atol=1e-12 * scale)
    Q1, _ = np.linalg.qr(Y1)
    Qs, _ = np.linalg.qr(Ys)
    assert np.all(np.linalg.svd(Q1.T @ Qs, compute_uv=False) > 1 - 1e-9)


def test_bulge_with_zero_column_keeps_chasing(lib):
    """A block whose leading part is already upper triangular to rounding in
    the first column (h_21 = 0 exactly, h_31 = 0): the active block splits
    there, and the Francis steps of the lower block still converge."""
    m = 8
    rng = np.random.default_rng(3)
    H = np.triu(rng.standard_normal((m + 1, m)), -1) + 3.0 * np.eye(m + 1, m)
    H[1, 0] = 0.0
    ev = np.linalg.eigvals(_F(H))
    Y, theta = lib.harmonic_ritz(H, m)
    np.testing.assert_allclose(np.sort_complex(theta), np.sort_complex(ev), rtol=1e-8, atol=1e-12)
