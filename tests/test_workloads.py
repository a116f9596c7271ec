"""The seeded input recipes: same seed, same field; the shapes, value ranges
and structure each generator's docstring states (layer formula, inclusion
fraction, batch size ranges, the two zones of the SPE10-shaped field).  CPU
only."""
import math

import numpy as np
import pytest

from paper_1510_02148_gb300 import workloads as W


def test_layered_layer_formula_and_bottom_high():
    K = W.layered(3, 2, 10, 4, 1.0, 1e-6)
    assert K.shape == (10, 2, 3) and K.dtype == np.float64
    for iz in range(10):
        layer = iz * 4 // 10
        assert np.all(K[iz] == (1.0 if layer % 2 == 0 else 1e-6))
    Kt = W.layered(3, 2, 10, 4, 1.0, 1e-6, bottom_high=False)
    assert np.all(Kt[0] == 1e-6)


def test_lognormal_layered_seeded_and_log_spread():
    a = W.lognormal_layered(16, 16, 16, 4, 1.0, 1e-4, 1.0, seed=3)
    b = W.lognormal_layered(16, 16, 16, 4, 1.0, 1e-4, 1.0, seed=3)
    c = W.lognormal_layered(16, 16, 16, 4, 1.0, 1e-4, 1.0, seed=4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    base = W.layered(16, 16, 16, 4, 1.0, 1e-4)
    xi = np.log(a / base)
    assert abs(xi.mean()) < 0.1 and abs(xi.std() - 1.0) < 0.05


def test_point_source_single_unit_cell():
    q = W.point_source(5, 6, 7)
    assert q.sum() == 1.0 and np.count_nonzero(q) == 1 and q[3, 3, 2] == 1.0
    q2 = W.point_source(5, 6, 7, value=-2.0, at=(0, 1, 2))
    assert q2[2, 1, 0] == -2.0 and np.count_nonzero(q2) == 1


def test_inclusions_reach_the_fraction_and_are_binary():
    K, f = W.inclusions(48, 40, 32, frac=0.2, a_range=(6, 14), seed=2)
    assert K.shape == (32, 40, 48)
    assert set(np.unique(K).tolist()) <= {1.0, 1e-6}
    assert f >= 0.2 and abs(np.mean(K == 1e-6) - f) < 1e-12
    K2, f2 = W.inclusions(48, 40, 32, frac=0.2, a_range=(6, 14), seed=2)
    assert np.array_equal(K, K2) and f == f2


def test_rotations_are_orthonormal():
    rng = np.random.default_rng(0)
    for _ in range(5):
        R = W._random_rotation(rng)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1.0) < 1e-12


def test_batch_recipe_ranges():
    probs = W.batch(count=12, side_range=(8, 20), seed=5)
    assert len(probs) == 12
    for p in probs:
        nz, ny, nx = p.K.shape
        assert nx == ny == nz and 8 <= nx <= 20
        assert p.S[0] == p.S[1] == p.S[2] and 2 <= p.S[0] <= 4
        assert p.L == 2 and p.tau == (1e-2,)
        assert set(np.unique(p.K).tolist()) <= {1.0, 1e-4}
    assert [p.K.shape for p in probs] == [p.K.shape for p in W.batch(count=12, side_range=(8, 20), seed=5)]


def test_learned_field_threshold_between_the_medians():
    p = W.learned_field(7, n=16)
    assert p.K.shape == (16, 16, 16) and p.S == (4, 4, 2) and p.L == 2
    t = p.tau[0]
    # threshold is the geometric mean of the medians 1 and 10^-c, c in [4, 6]
    assert 1e-3 <= t <= 1e-2
    assert W.learned_field(7, n=16).tau == p.tau


def test_sandwich_theorem_boundary():
    p = W.sandwich_theorem()
    assert p.bc_type == (W.NOFLOW,) * 5 + (W.DIRICHLET,)
    assert p.S == (1, 1, 6) and p.tau == (math.sqrt(1e-6),)


@pytest.mark.parametrize("seed", [1, 2])
def test_spe10_like_zones_and_range(seed):
    nx, ny, nz = 30, 44, 17
    p = W.spe10_like(nx, ny, nz, seed=seed)
    K = p.K
    assert K.shape == (nz, ny, nx)
    assert K.min() >= 1e-3 and K.max() <= 10.0 ** 4.5
    ntop = int(round(nz * 35 / 85))
    top, bottom = np.log10(K[nz - ntop:]), np.log10(K[: nz - ntop])
    # top: smooth lognormal around 10^1 with a spread of several decades
    assert 0.0 < np.median(top) < 2.0 and top.max() - top.min() > 3.0
    # bottom: ~1e-2 background with ~1e3 channels, nothing in between
    chan = bottom > 1.5
    assert 0.02 < chan.mean() < 0.8
    assert np.all((bottom < -0.5) | chan)
    assert p.L == 1 and p.tau == () and p.bc_type == W.X_DIRICHLET[0]
    assert np.array_equal(K, W.spe10_like(nx, ny, nz, seed=seed).K)
