"""Pins of the network oracle (oracle/net_oracle.py) against facts that do not
come from it: scipy's correlation, adjoint identities, finite differences of
the whole network and of the subspace loss, closed-form loss values and the
first Adam step."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import net_oracle as N


def _rng(s):
    return np.random.default_rng(s)


def test_conv_single_channel_matches_scipy_correlate():
    x = _rng(0).standard_normal((5, 6, 7))
    k = _rng(1).standard_normal((3, 3, 3))
    w = k.reshape(27, 1, 1)  # tap (dz+1)*9 + (dy+1)*3 + (dx+1)
    y = N.conv3d(x[..., None], w)[..., 0]
    ref = ndi.correlate(x, k, mode="constant", cval=0.0)
    assert np.allclose(y, ref, rtol=0, atol=1e-12)


def test_conv_bias_and_channels():
    x = _rng(2).standard_normal((4, 4, 4, 3))
    w = _rng(3).standard_normal((27, 5, 3))
    b = _rng(4).standard_normal(5)
    y = N.conv3d(x, w, b)
    # brute force at one interior and one corner cell
    for p in [(1, 2, 1), (0, 0, 3)]:
        ref = b.copy()
        for t, (dz, dy, dx) in enumerate(N.taps()):
            q = (p[0] + dz, p[1] + dy, p[2] + dx)
            if all(0 <= q[a] < 4 for a in range(3)):
                ref += w[t] @ x[q]
        assert np.allclose(y[p], ref, atol=1e-12)


def test_adjoints():
    x = _rng(5).standard_normal((4, 6, 8, 3))
    g = _rng(6).standard_normal((4, 6, 8, 5))
    w = _rng(7).standard_normal((27, 5, 3))
    lhs = np.sum(N.conv3d(x, w) * g)
    assert np.isclose(lhs, np.sum(x * N.conv3d_dgrad(g, w)), rtol=1e-12)
    assert np.isclose(lhs, np.sum(w * N.conv3d_wgrad(g, x)), rtol=1e-12)
    a = _rng(8).standard_normal((2, 3, 4, 2))
    bb = _rng(9).standard_normal((4, 6, 8, 2))
    assert np.isclose(np.sum(N.up(a) * bb), np.sum(a * N.up_bwd(bb)), rtol=1e-12)
    assert np.isclose(np.sum(N.pool(bb) * a), np.sum(bb * N.pool_bwd(a)), rtol=1e-12)


def test_features():
    logK = _rng(10).standard_normal((8, 8, 8)) * 2 - 3
    f = N.features(logK)
    assert abs(f[..., 0].mean()) < 1e-12 and abs(f[..., 0].std() - 1) < 1e-12
    assert np.allclose(f[0, 0, :, 1], (2 * np.arange(8) + 1) / 8 - 1)
    assert np.all(f[..., 4:] == 0)
    assert np.all(N.features(np.full((8, 8, 8), 2.0))[..., 0] == 0)


def test_backward_matches_finite_differences():
    rng = _rng(11)
    params = N.init_params(3)
    for i in range(1, len(params), 2):
        params[i] = rng.standard_normal(params[i].shape) * 0.1  # nonzero biases
    f = N.features(rng.standard_normal((8, 8, 8)))
    out, cache = N.forward(params, f)
    R = rng.standard_normal(out.shape)
    grads = N.backward(params, cache, R)

    def L(ps):
        return np.sum(N.forward(ps, f)[0] * R)

    h = 1e-6
    for li in range(len(params)):
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in params[li].shape)
            pp = [p.copy() for p in params]
            pm = [p.copy() for p in params]
            pp[li][idx] += h
            pm[li][idx] -= h
            fd = (L(pp) - L(pm)) / (2 * h)
            an = grads[li][idx]
            assert abs(fd - an) <= 1e-5 * (abs(an) + 1e-3), (li, idx, fd, an)


def test_subspace_loss_values_and_gradient():
    rng = _rng(12)
    n, k = 200, 3
    D = rng.uniform(0.5, 2.0, n)
    V = rng.standard_normal((n, k))
    L0, g0 = N.subspace_loss(V @ rng.standard_normal((k, k)), V, D)  # same span
    assert abs(L0) <= 1e-9 * np.sum(D[:, None] * V * V) and np.max(np.abs(g0)) <= 1e-8
    Y = rng.standard_normal((n, 2))
    Vp = V - Y @ np.linalg.solve(Y.T @ (D[:, None] * Y), Y.T @ (D[:, None] * V))  # D-orthogonal to Y
    L1, _ = N.subspace_loss(Y, Vp, D)
    assert np.isclose(L1, np.sum(D[:, None] * Vp * Vp), rtol=1e-10)
    L, g = N.subspace_loss(Y, V, D)
    h = 1e-6
    for _ in range(6):
        i, j = rng.integers(0, n), rng.integers(0, 2)
        Yp, Ym = Y.copy(), Y.copy()
        Yp[i, j] += h
        Ym[i, j] -= h
        fd = (N.subspace_loss(Yp, V, D)[0] - N.subspace_loss(Ym, V, D)[0]) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-5 * (abs(g[i, j]) + 1e-6)


def test_adam_first_step():
    g = np.array([0.5, -2.0, 1e-3])
    p = np.zeros(3)
    m, v = np.zeros(3), np.zeros(3)
    p1 = N.adam(p, g, m, v, 1, lr=0.01)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8))


def test_param_flatten_roundtrip():
    p = N.init_params(0)
    flat = N.flatten(p)
    assert flat.size == sum(27 * ci * co + co for ci, co in N.LAYERS)
    q = N.unflatten(flat)
    assert all(np.array_equal(a, b) for a, b in zip(p, q))


def test_pool_and_up_values():
    """Pooling is the mean of each 2x2x2 block (not the sum) and upsampling
    repeats each value into its 2x2x2 block: checked cell by cell on random
    data, and on a constant field (the mean of a constant is the constant)."""
    rng = _rng(21)
    x = rng.standard_normal((4, 6, 8, 3))
    p = N.pool(x)
    assert p.shape == (2, 3, 4, 3)
    for z in range(2):
        for y in range(3):
            for xx in range(4):
                blk = x[2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * xx:2 * xx + 2, :]
                np.testing.assert_allclose(p[z, y, xx], blk.reshape(-1, 3).mean(axis=0), rtol=1e-14)
    np.testing.assert_allclose(N.pool(np.full((4, 4, 4, 2), 3.5)), 3.5, rtol=0, atol=0)
    a = rng.standard_normal((2, 3, 4, 2))
    u = N.up(a)
    assert u.shape == (4, 6, 8, 2)
    for z in range(4):
        for y in range(6):
            for xx in range(8):
                assert np.array_equal(u[z, y, xx], a[z // 2, y // 2, xx // 2])
    # pooling after upsampling gives the coarse field back
    np.testing.assert_allclose(N.pool(u), a, rtol=1e-14)
