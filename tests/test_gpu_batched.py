"""Batched persistent solves (one cooperative launch, one team of CTAs per
system, captured in a CUDA graph) against the CPU oracle and against
one-at-a-time solves."""
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


def _energy_relerr(A, x, y):
    e = x - y
    return np.sqrt(max(e @ A.spmv(e), 0.0) / (y @ A.spmv(y)))


def _small_batch():
    probs = W.batch(count=9, side_range=(12, 40), seed=5)
    probs.append(W.lognormal_point_source(37, 21, 17, 4, (3, 2, 2), seed=4))
    probs.append(W.lognormal_point_source(64, 48, 40, 8, (4, 3, 4), seed=2))
    return probs


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_batched_matches_oracle(sld, oracle_mod, precision):
    probs = _small_batch()
    systems = [sld.from_problem(P) for P in probs]
    bt = sld.Batch(systems, precision=precision)
    print(bt.describe())
    xs, infos = bt.solve()
    for P, x, info in zip(probs, xs, infos):
        A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
        lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
        ref = oracle_mod.dpcg(A, lab, P.d, tol=P.tol)
        true = np.linalg.norm(A.b - A.spmv(x)) / np.linalg.norm(A.b)
        assert info.kernel_path == 2 and info.status == 0
        assert abs(true - info.true_relres) <= 1e-3 * true + 1e-12
        if precision == 0:
            assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-7, P.name
            assert abs(info.iterations - ref.iterations) <= 2, (P.name, info.iterations, ref.iterations)
            assert true <= 1.5e-9
        else:
            tight = oracle_mod.dpcg(A, lab, P.d, tol=1e-13)
            assert true <= 1e-9
            assert _energy_relerr(A, x, tight.x) <= max(1e-9, 5 * _energy_relerr(A, ref.x, tight.x)), P.name
            e_gpu = np.linalg.norm(x - tight.x) / np.linalg.norm(tight.x)
            e_ref = np.linalg.norm(ref.x - tight.x) / np.linalg.norm(tight.x)
            assert e_gpu <= max(1e-7, 3 * e_ref), (P.name, e_gpu, e_ref)
    bt.close()
    for s in systems:
        s.close()


def test_batched_equals_single_solves(sld):
    probs = _small_batch()
    systems = [sld.from_problem(P) for P in probs]
    bt = sld.Batch(systems, precision=0)
    xs, infos = bt.solve()
    xs2, infos2 = bt.solve()  # the graph runs again from a reset state
    for s, x, x2, info, info2 in zip(systems, xs, xs2, infos, infos2):
        xs1, i1 = s.solve(precision=0)
        assert abs(info.iterations - i1.iterations) <= 2
        assert np.linalg.norm(x - xs1) / np.linalg.norm(xs1) <= 1e-7
        assert info2.iterations == info.iterations and np.array_equal(x, x2)
    bt.close()
    for s in systems:
        s.close()


def test_batched_given_rhs_device(sld, oracle_mod):
    import torch
    probs = _small_batch()[:4]
    systems = [sld.from_problem(P) for P in probs]
    rng = np.random.default_rng(3)
    bs = [rng.standard_normal(P.n) for P in probs]
    bd = [torch.from_numpy(b).cuda() for b in bs]
    xd = [torch.empty(P.n, dtype=torch.float64, device="cuda") for P in probs]
    bt = sld.Batch(systems, precision=0, ctas_per_sm=1)
    _, infos = bt.solve(bd, xd)
    for P, b, x, info in zip(probs, bs, xd, infos):
        A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
        lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
        ref = oracle_mod.dpcg(A, lab, P.d, b=b, tol=P.tol)
        assert np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    bt.close()
    for s in systems:
        s.close()


def test_batched_rejects(sld):
    P = W.layered_sandwich(16, 16, 16, 4, (2, 2, 2))
    s = sld.from_problem(P)
    with pytest.raises(sld.SldError) as e:
        sld.Batch([s, s])
    assert e.value.status == sld.ERR_INVALID_ARG
    with pytest.raises(sld.SldError) as e:
        sld.Batch([s], precision=sld.BF16COEF_IR)
    assert e.value.status == sld.ERR_INVALID_ARG
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_batched_large_d_repeatable(sld, oracle_mod, precision):
    """A batch whose largest d (512) takes the global per-warp label rows:
    each system matches the oracle and a second launch repeats bit for bit."""
    probs = [W.lognormal_point_source(64, 64, 32, 4, (8, 8, 4), seed=21),
             W.lognormal_point_source(48, 40, 24, 4, (2, 2, 2), seed=22)]
    systems = [sld.from_problem(P) for P in probs]
    bt = sld.Batch(systems, precision=precision)
    xs1, infos1 = bt.solve()
    xs1 = [x.copy() for x in xs1]
    xs2, infos2 = bt.solve()
    for P, x1, x2, i1, i2 in zip(probs, xs1, xs2, infos1, infos2):
        assert i1.iterations == i2.iterations and np.array_equal(x1, x2), P.name
        A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
        lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
        ref = oracle_mod.dpcg(A, lab, P.d, tol=P.tol)
        if precision == 0:
            assert np.linalg.norm(x1 - ref.x) / np.linalg.norm(ref.x) <= 1e-7
            assert abs(i1.iterations - ref.iterations) <= 2
        else:
            tight = oracle_mod.dpcg(A, lab, P.d, tol=1e-13)
            e = np.linalg.norm(x1 - tight.x) / np.linalg.norm(tight.x)
            assert e <= max(1e-7, 3 * np.linalg.norm(ref.x - tight.x) / np.linalg.norm(tight.x))
    bt.close()
    for s in systems:
        s.close()
