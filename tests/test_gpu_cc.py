"""Automatic subdomain-levelset labels on the GPU (sld_make_labels_cc)
against the oracle: labels bit-exact (the canonical numbering makes them
unique), the too-many-components error, and the deflated solve with the
component labels against the oracle solve with the same labels."""
import numpy as np
import pytest

from paper_1510_02148_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from oracle import sld_cc
    from paper_1510_02148_gb300 import _build, sld
    _build.build()
    sld.load()
    oracle.build()
    return sld, oracle, sld_cc


def _sys(sld, P):
    return sld.System(P.K.reshape(-1), P.q.reshape(-1), P.bc_type, P.bc_value, shape=P.shape)


FIELDS = [
    ("lognormal layered 40x28x24", lambda: W.lognormal_point_source(40, 28, 24, 6, (2, 2, 2), seed=3), None),
    ("ragged 23x17x11, 3 classes", lambda: W.lognormal_point_source(23, 17, 11, 4, (3, 2, 1), seed=8),
     ((1e-3, 1e-1), 3)),
    ("rough lognormal 32^3", None, None),
]


def _rough(seed=5):
    rng = np.random.default_rng(seed)
    K = np.exp(2.0 * rng.standard_normal((32, 32, 32)))
    return W.Problem("rough32", K, W.point_source(32, 32, 32), *W.X_DIRICHLET, S=(2, 2, 2), tau=(1.0,), L=2)


@pytest.mark.parametrize("field", FIELDS, ids=[f[0] for f in FIELDS])
def test_labels_bit_exact(env, field):
    sld, oracle, C = env
    P = field[1]() if field[1] else _rough()
    tau, L = field[2] if field[2] else (P.tau, P.L)
    ref, dref = C.cc_labels(P.K, P.S, tau, L)
    s = _sys(sld, P)
    lab, d = s.make_labels_cc(P.S, tau, L)
    s.close()
    assert d == dref
    assert np.array_equal(lab, ref)


def test_too_many_components(env):
    sld, oracle, C = env
    z, y, x = np.meshgrid(np.arange(16), np.arange(20), np.arange(24), indexing="ij")
    K = np.where((x + y + z) % 2 == 0, 1.0, 1e-6)  # every cell its own component: 7680 > 4096
    P = W.Problem("checker", K, W.point_source(24, 20, 16), *W.X_DIRICHLET, S=(1, 1, 1), tau=(1e-3,), L=2)
    s = _sys(sld, P)
    with pytest.raises(sld.SldError, match="INVALID_ARG"):
        s.make_labels_cc(P.S, P.tau, P.L)
    assert s.cc_components == K.size
    s.close()


def test_solve_with_component_labels(env):
    """FP64 deflated CG with the component labels: the oracle's solve with
    the same labels (solution 1e-7, iterations within 2); fewer iterations
    than with the plain SLD labels on this layered field."""
    sld, oracle, C = env
    P = W.lognormal_point_source(48, 40, 32, 8, (2, 2, 2), seed=4)
    A = oracle.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab, d = C.cc_labels(P.K, P.S, P.tau, P.L)
    ref = oracle.dpcg(A, lab, d, tol=1e-9)
    plain = oracle.dpcg(A, oracle.labels(P.K, P.S, P.tau, P.L), P.d, tol=1e-9)
    s = _sys(sld, P)
    glab, gd = s.make_labels_cc(P.S, P.tau, P.L)
    assert gd == d and np.array_equal(glab, lab)
    s.build_deflation(gd)
    x, info = s.solve(precision=sld.FP64, tol=1e-9)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    assert abs(info.iterations - ref.iterations) <= 2
    x32, i32 = s.solve(precision=sld.FP32_IR, tol=1e-9)
    assert i32.true_relres <= 1e-9
    s.close()
    assert d > P.d and ref.iterations < plain.iterations, (d, ref.iterations, plain.iterations)
