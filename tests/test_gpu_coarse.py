"""The coarse solve at large d (Def. 3.1, eq. (E); Remark 3.1: E = Z^T A Z
with the unpreconditioned A).  The library factors E once by Cholesky and
applies E^{-1} = L^{-T} L^{-1}, formed from that factor, as a distributed
FP64 matrix-vector product in every iteration, instead of a forward and a
back triangular solve (2d dependent steps per iteration).

Checked here at d = 512 (lognormal layers) and d = 1536 (inclusions, the
512x512x256 workload's coarse size, 8x8x8 subdomains x 3 levelsets):
  * E from the GPU against the oracle's dense-product Z^T (A Z);
  * cond(E) reported;
  * y = E^{-1} s through the GPU's explicit inverse against Cholesky
    forward/back solves with E's own factor (LAPACK) and with the oracle's
    factor of its E, for random s and for s = Z^T A p: the explicit inverse
    must agree with the triangular solves to within 10 cond(E) eps, the
    accuracy either attains;
  * the whole FP64 solve at d = 1536 against the oracle (1e-7, +-2
    iterations)."""
import numpy as np
import pytest
import scipy.linalg as sl

from paper_1510_02148_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def sld():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1510_02148_gb300 import _build, sld as mod
    _build.build()
    mod.load()
    return mod


def _cases():
    return [
        ("d512_lognormal", W.lognormal_point_source(128, 128, 64, 8, (8, 8, 4), seed=7)),
        ("d1536_inclusions", W.inclusion_field(128, 128, 64, (8, 8, 8), 0.2, 1, (8, 48))[0]),
    ]


CASES = _cases()


@pytest.mark.parametrize("name,P", CASES, ids=[c[0] for c in CASES])
def test_explicit_inverse_against_triangular_solves(sld, oracle_mod, name, P):
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
    E_o, L_o = oracle_mod.coarse(A, lab, P.d)
    assert L_o is not None
    s = sld.from_problem(P)
    E, Einv = s.get_coarse()
    assert E.shape == (P.d, P.d)
    # E: the same sums as the oracle's product, up to summation order
    assert np.max(np.abs(E - E_o)) <= 1e-12 * np.max(np.abs(E_o))
    cond = np.linalg.cond(E_o)
    cf = sl.cho_factor(E, lower=True)
    rng = np.random.default_rng(3)
    p = rng.standard_normal(A.n)
    rhs = [rng.standard_normal(P.d) for _ in range(3)] + [oracle_mod.restrict(lab, P.d, A.spmv(p))]
    worst_own = worst_oracle = 0.0
    for r in rhs:
        y_inv = Einv @ r                              # what the iteration applies
        y_tri = sl.cho_solve(cf, r)                   # forward/back solves, E's own factor
        y_o = sl.solve_triangular(L_o.T, sl.solve_triangular(L_o, r, lower=True), lower=False)
        worst_own = max(worst_own, np.linalg.norm(y_inv - y_tri) / np.linalg.norm(y_tri))
        worst_oracle = max(worst_oracle, np.linalg.norm(y_inv - y_o) / np.linalg.norm(y_o))
    print(f"{name}: d={P.d} cond(E)={cond:.2e} (cond*eps {cond * EPS:.1e}); explicit inverse vs "
          f"triangular solves {worst_own:.2e}, vs the oracle's factor {worst_oracle:.2e}")
    assert worst_own <= 10 * cond * EPS
    assert worst_oracle <= 10 * cond * EPS
    s.close()


def test_fp64_solve_at_d1536(sld, oracle_mod):
    """The whole FP64 iteration with the explicit inverse at d = 1536 matches
    the oracle's (explicit Z, Cholesky solves) to 1e-7, iterations within 2."""
    P = dict(CASES)["d1536_inclusions"]
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
    ref = oracle_mod.dpcg(A, lab, P.d, tol=P.tol)
    s = sld.from_problem(P)
    x, info = s.solve(precision=0, tol=P.tol)
    err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    print(f"d1536 FP64: iterations {info.iterations} (oracle {ref.iterations}), rel.err {err:.2e}, "
          f"{info.solve_ms:.1f} ms")
    assert err <= 1e-7
    assert abs(info.iterations - ref.iterations) <= 2
    s.close()
