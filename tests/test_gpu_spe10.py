"""The SPE10-shaped synthetic with plain subdomain deflation (L = 1,
d = Sx*Sy*Sz), the sweep of the paper's SPE10 runs on the deflated-CG path:
labels bit-exact and the FP64 solve against the oracle at a reduced size of
the same generator, for d = 1, 8, 27, 64."""
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
    from paper_1510_02148_gb300 import _build, sld
    _build.build()
    sld.load()
    oracle.build()
    P = W.spe10_like(30, 44, 17, seed=2)
    A = oracle.assemble(P.K, P.q, P.bc_type, P.bc_value)
    return sld, oracle, P, A


@pytest.mark.parametrize("S", [(1, 1, 1), (2, 2, 2), (3, 3, 3), (4, 4, 4)])
def test_subdomain_deflation_sweep(env, S):
    sld, oracle, P, A = env
    d = S[0] * S[1] * S[2]
    lab = oracle.labels(P.K, S, (), 1)
    ref = oracle.dpcg(A, lab, d, tol=1e-9)
    s = sld.System(P.K.reshape(-1), P.q.reshape(-1), P.bc_type, P.bc_value, shape=P.shape)
    glab = s.make_labels(S, (), 1)
    assert np.array_equal(glab, lab)
    s.build_deflation(d)
    x, info = s.solve(precision=sld.FP64, tol=1e-9)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    assert abs(info.iterations - ref.iterations) <= 2
    x32, i32 = s.solve(precision=sld.FP32_IR, tol=1e-9)
    assert i32.true_relres <= 1e-9
    s.close()
