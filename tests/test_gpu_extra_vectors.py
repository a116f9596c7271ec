"""Extra dense deflation columns (Z = [Z_lab, Z_extra], Section 3.1, Def. 3.1
with a general full-rank Z) through the C ABI, against the CPU oracle run
with the same columns (the FP32-rounded values the library deflates with)."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from paper_1510_02148_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sld():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1510_02148_gb300 import _build, sld as mod
    _build.build()
    mod.load()
    return mod


def _smooth_columns(shape, k, seed):
    """k smooth fields (products of low-frequency sines with random phases)."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cols = []
    for _ in range(k):
        fx, fy, fz = rng.uniform(0.3, 1.5, 3)
        px, py, pz = rng.uniform(0, np.pi, 3)
        f = (np.sin(np.pi * fx * x / nx + px) * np.sin(np.pi * fy * y / ny + py) *
             np.sin(np.pi * fz * z / nz + pz))
        cols.append(f.reshape(-1))
    return np.stack(cols, axis=1)


def _relerr(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def _energy_relerr(A, x, y):
    e = x - y
    return np.sqrt(max(e @ A.spmv(e), 0.0) / (y @ A.spmv(y)))


def _setup(oracle_mod, P):
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
    return A, lab


CASE = W.lognormal_point_source(64, 48, 40, 8, (4, 3, 2), seed=2)


def test_extra_coarse_matrix(sld, oracle_mod):
    P = CASE
    A, lab = _setup(oracle_mod, P)
    Z = _smooth_columns(P.shape, 3, 5).astype(np.float32)
    s = sld.from_problem(P)
    s.build_deflation(P.d, Zextra=Z)
    assert s.deflation_info() == (P.d, 3, 3)
    E, Einv = s.get_coarse()
    Eo, Lo = oracle_mod.coarse(A, lab, P.d, Z.astype(np.float64))
    assert Lo is not None
    d = P.d
    for blk in (np.s_[:d, :d], np.s_[:d, d:], np.s_[d:, d:]):
        scale = np.max(np.abs(Eo[blk]))
        assert np.max(np.abs(E[blk] - Eo[blk])) <= 1e-12 * scale, blk
    assert np.allclose(E, E.T, rtol=0, atol=1e-13 * np.max(np.abs(E)))
    I = Einv @ Eo
    assert np.max(np.abs(I - np.eye(d + 3))) <= 1e-6
    s.close()


@pytest.mark.parametrize("zdtype", [np.float64, np.float32])
def test_extra_fp64_parity(sld, oracle_mod, zdtype):
    """FP64: the oracle's iteration with the same Z: solution within 1e-7, iterations within 2."""
    P = CASE
    A, lab = _setup(oracle_mod, P)
    Z = _smooth_columns(P.shape, 4, 7).astype(zdtype)
    Z32 = Z.astype(np.float32).astype(np.float64)  # the columns the library keeps
    ref = oracle_mod.dpcg(A, lab, P.d, tol=P.tol, Zd=Z32)
    assert ref.status == 0
    s = sld.from_problem(P)
    s.build_deflation(P.d, Zextra=Z)
    x, info = s.solve(precision=0, tol=P.tol)
    assert info.kernel_path == 1
    assert _relerr(x, ref.x) <= 1e-7
    assert abs(info.iterations - ref.iterations) <= 2, (info.iterations, ref.iterations)
    assert info.true_relres <= 1.5e-9
    s.close()


def test_extra_fp32ir(sld, oracle_mod):
    """FP32 inner / FP64 refinement with extra columns reaches the FP64
    residual; against the exact discrete solution its 2-norm error is within
    max(1e-7, 3x the FP64 oracle's) and its energy-norm error within 5x."""
    P = CASE
    A, lab = _setup(oracle_mod, P)
    Z = _smooth_columns(P.shape, 8, 9).astype(np.float32)
    Zd = Z.astype(np.float64)
    ref = oracle_mod.dpcg(A, lab, P.d, tol=P.tol, Zd=Zd)
    tight = oracle_mod.dpcg(A, lab, P.d, tol=1e-13, Zd=Zd)
    s = sld.from_problem(P)
    s.build_deflation(P.d, Zextra=Z)
    x, info = s.solve(precision=1, tol=P.tol)
    assert info.true_relres <= 1e-9
    assert _energy_relerr(A, x, tight.x) <= max(1e-9, 5 * _energy_relerr(A, ref.x, tight.x))
    assert _relerr(x, tight.x) <= max(1e-7, 3 * _relerr(ref.x, tight.x))
    s.close()


def test_extra_device_input_and_repeat(sld):
    import torch
    P = CASE
    Z = torch.from_numpy(_smooth_columns(P.shape, 2, 3)).cuda()
    s = sld.from_problem(P)
    s.build_deflation(P.d, Zextra=Z)
    x1, i1 = s.solve(precision=1)
    x2, i2 = s.solve(precision=1)
    assert i1.iterations == i2.iterations and np.array_equal(x1, x2)
    s.close()


def test_extra_dependent_columns_dropped(sld, oracle_mod):
    """A column inside span(Z_lab) makes E singular: the extra columns are
    dropped and the label deflation alone is used."""
    P = CASE
    A, lab = _setup(oracle_mod, P)
    Z = np.stack([(lab == 0).astype(np.float64), _smooth_columns(P.shape, 1, 2)[:, 0]], axis=1)
    s = sld.from_problem(P)
    _, plain = s.solve(precision=0)
    s.build_deflation(P.d, Zextra=Z)
    assert s.deflation_info() == (P.d, 2, 0)
    x, info = s.solve(precision=0)
    assert info.iterations == plain.iterations and info.true_relres <= 1.5e-9
    s.close()


def test_extra_rejects(sld):
    P = CASE
    s = sld.from_problem(P)
    with pytest.raises(sld.SldError, match="k must be"):
        s.build_deflation(P.d, Zextra=np.zeros((P.n, 9)))
    Z = _smooth_columns(P.shape, 2, 1)
    Z[5, 1] = np.nan
    with pytest.raises(sld.SldError, match="non-finite"):
        s.build_deflation(P.d, Zextra=Z)
    s.build_deflation(P.d, Zextra=_smooth_columns(P.shape, 2, 1))
    _, info = s.solve(precision=2, raise_on_error=False)
    assert info.status == sld.ERR_INVALID_ARG
    s.close()
    Q = W.lognormal_point_source(30, 24, 16, 4, (2, 2, 2), seed=1)  # nx % 8 != 0
    s = sld.from_problem(Q)
    s.build_deflation(Q.d, Zextra=_smooth_columns(Q.shape, 2, 1))
    _, info = s.solve(precision=0, raise_on_error=False)
    assert info.status == sld.ERR_INVALID_ARG and b"TMA" in sld.load().sld_last_error()
    s.close()


def test_eigenvectors_cut_iterations(sld, oracle_mod):
    """Appending the eigenvectors of the smallest nonzero eigenvalues of the
    label-deflated, Jacobi-preconditioned operator removes them from the
    spectrum the CG sees: fewer iterations to the same tolerance."""
    P = W.lognormal_point_source(32, 24, 16, 6, (2, 2, 2), seed=4)
    A, lab = _setup(oracle_mod, P)
    As = A.to_scipy().tocsr()
    n, d = A.n, P.d
    Zs = np.eye(d)[lab]
    E = Zs.T @ (As @ Zs)
    Dm = 1.0 / np.sqrt(A.diag())
    Q, _ = np.linalg.qr(Zs / Dm[:, None])  # basis of the null space of H below

    def H(h):  # D^{-1/2} (A - A Z E^{-1} Z^T A) D^{-1/2} h, plus a shift on its null space
        t = Dm * h
        u = As @ t
        u = u - As @ (Zs @ np.linalg.solve(E, Zs.T @ u))
        return Dm * u + 10.0 * (Q @ (Q.T @ h))

    op = sla.LinearOperator((n, n), matvec=H, dtype=np.float64)
    vals, vecs = sla.eigsh(op, k=6, which="SA", tol=1e-10, maxiter=20000)
    V = (Dm[:, None] * vecs)  # eigenvectors of M^{-1} P A
    s = sld.from_problem(P)
    _, plain = s.solve(precision=0)
    s.build_deflation(d, Zextra=V)
    assert s.deflation_info()[2] == 6
    _, info = s.solve(precision=0)
    ref = oracle_mod.dpcg(A, lab, d, tol=P.tol, Zd=V.astype(np.float32).astype(np.float64))
    print(f"iterations: labels {plain.iterations}, labels + 6 eigenvectors {info.iterations} "
          f"(oracle {ref.iterations}); eigenvalues {vals}")
    assert abs(info.iterations - ref.iterations) <= 2
    assert info.iterations < plain.iterations
    assert info.true_relres <= 1.5e-9
    s.close()
