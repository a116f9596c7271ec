"""RDGMRES on the GPU (sld_solve_rdgmres) against the CPU oracle of the same
method (harmonic-Ritz deflation from the first cycle, Section 3.2.1): the
solution, the step count, the residual, the first-cycle branch, errors."""
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
    from oracle import pdgmres, rdgmres
    from paper_1510_02148_gb300 import _build, sld
    _build.build()
    sld.load()
    oracle.build()
    return sld, oracle, pdgmres, rdgmres


def _sys(sld, P):
    return sld.System(P.K.reshape(-1), P.q.reshape(-1), P.bc_type, P.bc_value, shape=P.shape)


def test_parity_with_oracle(env):
    """32^3 lognormal-layered: the oracle takes 330 steps (11 cycles of 30,
    unchanged under 1e-15 perturbations of b), plain GMRES(30) 372."""
    sld, oracle, PG, RD = env
    P = W.lognormal_point_source(32, 32, 32, 8, (2, 2, 2), seed=2)
    A = oracle.assemble(P.K, P.q, P.bc_type, P.bc_value)
    ref = RD.rdgmres(A, d=3, m=30, tol=1e-8, maxiter=20000)
    assert ref.status == RD.OK
    s = _sys(sld, P)
    x, info = s.solve_rdgmres(m=30, d=3, tol=1e-8, maxiter=20000)
    _, plain = s.solve_gmres(m=30, deflate=False, tol=1e-8, maxiter=20000)
    s.close()
    assert info.true_relres <= 1.5e-8
    assert abs(info.relres_estimate - info.true_relres) <= 1e-3 * info.true_relres
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-5
    assert abs(info.iterations - ref.iterations) <= max(5, int(0.05 * ref.iterations)), \
        (info.iterations, ref.iterations)
    assert info.iterations < plain.iterations, (info.iterations, plain.iterations)


def test_converged_in_the_first_cycle(env):
    """A loose tolerance met inside the first cycle: plain GMRES(m) steps."""
    sld, oracle, PG, RD = env
    P = W.lognormal_point_source(24, 20, 16, 4, (2, 2, 2), seed=5)
    A = oracle.assemble(P.K, P.q, P.bc_type, P.bc_value)
    ref = PG.pdgmres(A, None, 0, m=30, tol=5e-2, maxiter=30)  # 11 steps
    assert ref.status == PG.OK and ref.iterations < 30
    s = _sys(sld, P)
    x, info = s.solve_rdgmres(m=30, d=3, tol=5e-2, maxiter=20000)
    s.close()
    assert info.iterations == ref.iterations and info.cycles == 1
    assert info.true_relres <= 5e-2


def test_errors(env):
    sld, oracle, PG, RD = env
    P = W.lognormal_point_source(16, 16, 16, 4, (2, 2, 2), seed=5)
    s = _sys(sld, P)
    for bad in (dict(m=1), dict(m=32), dict(d=0), dict(d=9), dict(m=4, d=5), dict(tol=0.0), dict(maxiter=0)):
        with pytest.raises(sld.SldError, match="INVALID_ARG"):
            s.solve_rdgmres(**bad)
    x, info = s.solve_rdgmres(m=20, d=2, tol=1e-14, maxiter=25, raise_on_error=False)
    assert info.status == 3 and info.iterations == 25 and np.all(np.isfinite(x))
    s.close()
