"""Parity at the benchmark sizes, in the launch configuration bench.py times,
checked through quantities the oracle computes at any size: the labels
(bit-exact), and the FP64 true residual of the GPU solution evaluated with the
oracle's own assembled matrix.  Plus the coarse sizes above the per-warp
accumulator limit (d > 256) against the full oracle solve on a smaller grid,
and the next rows at their bench sizes: PDGMRES, the automatic labels, the
SPE10-shaped workload."""
import numpy as np
import pytest

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


def _true_relres(A, x):
    return np.linalg.norm(A.b - A.spmv(x)) / np.linalg.norm(A.b)


def test_lognormal_256x256x128(sld, oracle_mod):
    """The bench workload (8.4M cells, d = 128) against the full oracle solve
    (about 90 s on 16 host cores): the FP64 solution within 1e-7 of the
    oracle's and the iteration count within 2; the FP32-inner and
    BF16-coefficient solutions within 1e-7 of the oracle's as well (at this
    size both the oracle's and the mixed forms' own errors are a few 1e-8);
    every true residual through the oracle's matrix."""
    import torch
    P = W.lognormal_point_source()
    s = sld.System(torch.from_numpy(P.K.reshape(-1)).cuda(), torch.from_numpy(P.q.reshape(-1)).cuda(),
                   P.bc_type, P.bc_value, stream=torch.cuda.current_stream().cuda_stream, shape=P.shape)
    lab = s.make_labels(P.S, P.tau, P.L)
    assert np.array_equal(lab, oracle_mod.labels(P.K, P.S, P.tau, P.L))
    s.build_deflation(P.d)
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    ref = oracle_mod.dpcg(A, lab, P.d, tol=P.tol)
    assert ref.status == 0
    x32, i32 = s.solve(precision=sld.FP32_IR)
    x16, i16 = s.solve(precision=sld.BF16COEF_IR)
    x64, i64 = s.solve(precision=sld.FP64)
    for name, x, info in (("fp32_ir", x32, i32), ("bf16", x16, i16), ("fp64", x64, i64)):
        t = _true_relres(A, x)
        err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        print(f"256x256x128 {name}: iterations {info.iterations} (oracle {ref.iterations}), "
              f"rel.err vs oracle {err:.2e}, true relres {t:.2e}")
        assert info.kernel_path == 1
        assert t <= 1.5e-9 and abs(t - info.true_relres) <= 1e-3 * t + 1e-12, (t, info.true_relres)
        assert err <= 1e-7, (name, err)
    assert abs(i64.iterations - ref.iterations) <= 2
    s.close()


def test_inclusions_512x512x256_bf16(sld, oracle_mod):
    """The BF16-coefficient workload (67M cells, d = 1536: label sums in the
    global per-warp rows): labels bit-exact, the true residual through the
    oracle's matrix."""
    import torch
    P, _ = W.inclusion_field()
    s = sld.System(torch.from_numpy(P.K.reshape(-1)).cuda(), None, P.bc_type, P.bc_value, shape=P.shape)
    lab = s.make_labels(P.S, P.tau, P.L)
    assert np.array_equal(lab, oracle_mod.labels(P.K, P.S, P.tau, P.L))
    s.build_deflation(P.d)
    x, info = s.solve(precision=sld.BF16COEF_IR)
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    t = _true_relres(A, x)
    assert t <= 1e-9 and abs(t - info.true_relres) <= 1e-3 * t + 1e-12, (t, info.true_relres)
    s.close()


def test_large_d_parity(sld, oracle_mod):
    """d = 512 label columns (above the per-warp accumulator limit of 256):
    FP64 within 1e-7 of the oracle, iterations within 2; FP32 inner reaches 1e-9."""
    P = W.lognormal_point_source(64, 64, 32, 8, (8, 8, 4), seed=6)
    assert P.d == 512
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
    ref = oracle_mod.dpcg(A, lab, P.d, tol=P.tol)
    s = sld.from_problem(P)
    x, info = s.solve(precision=sld.FP64)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    assert abs(info.iterations - ref.iterations) <= 2
    x32, i32 = s.solve(precision=sld.FP32_IR)
    assert _true_relres(A, x32) <= 1e-9
    with pytest.raises(sld.SldError, match="d must be"):
        s.build_deflation(4097)
    s.close()


def test_pdgmres_fullsize(sld, oracle_mod):
    """PDGMRES(20) on the bench workload at the paper's tolerance: the
    residual through the oracle's matrix, and the Givens estimate equal to it."""
    P = W.lognormal_point_source()
    s = sld.from_problem(P)
    x, info = s.solve_gmres(m=20, tol=1e-6, maxiter=20000)
    s.close()
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    t = _true_relres(A, x)
    assert t <= 1e-6 and abs(t - info.true_relres) <= 1e-3 * t
    assert abs(info.relres_estimate - t) <= 1e-3 * t


def test_automatic_labels_fullsize(sld, oracle_mod):
    """The automatic labels of the bench workload bit-exact against the
    oracle's, and the FP32-inner solve with them to 1e-9 through the
    oracle's matrix."""
    from oracle import sld_cc
    P = W.lognormal_point_source()
    ref, dref = sld_cc.cc_labels(P.K, P.S, P.tau, P.L)
    s = sld.System(P.K.reshape(-1), P.q.reshape(-1), P.bc_type, P.bc_value, shape=P.shape)
    lab, d = s.make_labels_cc(P.S, P.tau, P.L)
    assert d == dref and np.array_equal(lab, ref)
    s.build_deflation(d)
    x, info = s.solve(precision=sld.FP32_IR)
    s.close()
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    assert _true_relres(A, x) <= 1e-9


def test_spe10_like_fullsize(sld, oracle_mod):
    """The SPE10-shaped sweep's workload (180x220x85) with d = 64: labels
    bit-exact, the FP32-inner solve to 1e-9 through the oracle's matrix."""
    P = W.spe10_like(S=(4, 4, 4))
    s = sld.System(P.K.reshape(-1), P.q.reshape(-1), P.bc_type, P.bc_value, shape=P.shape)
    lab = s.make_labels(P.S, P.tau, P.L)
    assert np.array_equal(lab, oracle_mod.labels(P.K, P.S, P.tau, P.L))
    s.build_deflation(P.d)
    x, info = s.solve(precision=sld.FP32_IR)
    s.close()
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    assert _true_relres(A, x) <= 1e-9
