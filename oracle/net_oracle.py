"""CPU FP64 oracle of the deflation-vector network -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module.  It restates, in plain numpy, what
the CUDA network kernels compute: a small 3-D U-net that maps a
log-permeability field to k extra deflation vectors (appended to the
subdomain-levelset columns of Z, Section 3.1, Def. 3.1 with a general Z),
its backward pass, and the subspace loss that trains it against eigenvectors
of the deflated, Jacobi-preconditioned operator M^{-1} P A (the vectors
Section 3.1 says deflation should ideally remove).

Layout: activations are channels-last arrays [nz, ny, nx, C]; a 3x3x3
convolution has weights [27, Cout, Cin] with tap t = (dz+1)*9 + (dy+1)*3 +
(dx+1) reading the input at offset (dz, dy, dx), zero outside the grid.
"""
from __future__ import annotations

import numpy as np

# (Cin, Cout) of the nine 3x3x3 convolutions, in parameter order
LAYERS = [(16, 16), (16, 16), (16, 32), (32, 48), (48, 64), (64, 48), (48, 32), (32, 16), (16, 8)]
K_OUT = 8
IN_CH = 16  # standardised log10 K, three coordinates, twelve zero channels


def taps():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, off):
    """out[p] = x[p + off] (zero where p + off is outside the grid)."""
    dz, dy, dx = off
    nz, ny, nx = x.shape[:3]
    out = np.zeros_like(x)
    zs, ys, xs = [slice(max(0, -o), min(n, n - o)) for o, n in ((dz, nz), (dy, ny), (dx, nx))]
    zt, yt, xt = [slice(max(0, o), min(n, n + o)) for o, n in ((dz, nz), (dy, ny), (dx, nx))]
    out[zs, ys, xs] = x[zt, yt, xt]
    return out


def conv3d(x, w, b=None):
    """y[p, co] = b[co] + sum_t sum_ci w[t, co, ci] x[p + off_t, ci]."""
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for t, off in enumerate(taps()):
        y += shift(x, off) @ w[t].T
    if b is not None:
        y += b
    return y


def conv3d_dgrad(g, w):
    """dx[p, ci] = sum_t sum_co w[t, co, ci] g[p - off_t, co]."""
    dx = np.zeros(g.shape[:3] + (w.shape[2],))
    for t, off in enumerate(taps()):
        dx += shift(g, tuple(-o for o in off)) @ w[t]
    return dx


def conv3d_wgrad(g, x):
    """dw[t, co, ci] = sum_p g[p, co] x[p + off_t, ci]."""
    C = g.shape[3]
    gf = g.reshape(-1, C)
    return np.stack([gf.T @ shift(x, off).reshape(-1, x.shape[3]) for off in taps()])


def pool(x):
    nz, ny, nx, c = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(1, 3, 5))


def pool_bwd(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_bwd(g):
    nz, ny, nx, c = g.shape
    return g.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).sum(axis=(1, 3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def features(logK):
    """Input channels: (log10 K - mean) / std over the field (std 1 if the
    field is constant), and the cell-centre coordinates mapped to (-1, 1)."""
    nz, ny, nx = logK.shape
    m = logK.mean()
    sd = logK.std()
    f = np.zeros((nz, ny, nx, IN_CH))
    f[..., 0] = (logK - m) / (sd if sd > 0 else 1.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f[..., 1] = 2.0 * (x + 0.5) / nx - 1.0
    f[..., 2] = 2.0 * (y + 0.5) / ny - 1.0
    f[..., 3] = 2.0 * (z + 0.5) / nz - 1.0
    return f


def init_params(seed=0):
    """He-normal weights, zero biases (flat FP32 order: w0, b0, w1, b1, ...)."""
    rng = np.random.default_rng(seed)
    p = []
    for cin, cout in LAYERS:
        p.append(rng.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin)))
        p.append(np.zeros(cout))
    return p


def flatten(params):
    return np.concatenate([a.reshape(-1) for a in params])


def unflatten(flat):
    out, o = [], 0
    for cin, cout in LAYERS:
        n = 27 * cout * cin
        out.append(flat[o:o + n].reshape(27, cout, cin))
        o += n
        out.append(flat[o:o + cout].copy())
        o += cout
    return out


def _ident(a):
    return a


def forward(params, f, rnd=_ident):
    """The U-net: two convolutions at full resolution, three average-pool
    levels (16, 32, 48, 64 channels), nearest-neighbour upsampling with
    additive skips, and a linear 3x3x3 output convolution to K_OUT channels.

    rnd: applied to every stored activation (the input channels, each conv
    and pool output except the network output).  The identity gives the FP64
    network; rounding to BF16 reproduces where a BF16-storage implementation
    rounds, so that both sides take the same ReLU mask decisions."""
    W = params[0::2]
    B = params[1::2]
    c = {"f": rnd(f)}
    c["a0"] = rnd(relu(conv3d(c["f"], W[0], B[0])))
    c["e0"] = rnd(relu(conv3d(c["a0"], W[1], B[1])))
    c["p1"] = rnd(pool(c["e0"]))
    c["e1"] = rnd(relu(conv3d(c["p1"], W[2], B[2])))
    c["p2"] = rnd(pool(c["e1"]))
    c["e2"] = rnd(relu(conv3d(c["p2"], W[3], B[3])))
    c["p3"] = rnd(pool(c["e2"]))
    c["b3"] = rnd(relu(conv3d(c["p3"], W[4], B[4])))
    c["u2"] = up(c["b3"])
    c["d2"] = rnd(relu(conv3d(c["u2"], W[5], B[5]) + c["e2"]))
    c["u1"] = up(c["d2"])
    c["d1"] = rnd(relu(conv3d(c["u1"], W[6], B[6]) + c["e1"]))
    c["u0"] = up(c["d1"])
    c["d0"] = rnd(relu(conv3d(c["u0"], W[7], B[7]) + c["e0"]))
    out = conv3d(c["d0"], W[8], B[8])
    return out, c


def backward(params, c, dout, rnd=_ident):
    """Gradients of a scalar with d(scalar)/d(out) = dout, by the chain rule
    through forward(); returns them in parameter order.  rnd: applied to the
    masked gradient of each convolution output before it enters that
    convolution's weight and data gradients (the identity for FP64)."""
    W = params[0::2]
    gW = [None] * 9
    gB = [None] * 9

    def conv_back(i, g, x):
        gr = rnd(g)
        gW[i] = conv3d_wgrad(gr, x)
        gB[i] = g.sum(axis=(0, 1, 2))
        return conv3d_dgrad(gr, W[i])

    dd0 = conv_back(8, dout, c["d0"])
    g7 = dd0 * (c["d0"] > 0)
    de0 = g7.copy()
    dd1 = up_bwd(conv_back(7, g7, c["u0"]))
    g6 = dd1 * (c["d1"] > 0)
    de1 = g6.copy()
    dd2 = up_bwd(conv_back(6, g6, c["u1"]))
    g5 = dd2 * (c["d2"] > 0)
    de2 = g5.copy()
    db3 = up_bwd(conv_back(5, g5, c["u2"]))
    g4 = db3 * (c["b3"] > 0)
    de2 += pool_bwd(conv_back(4, g4, c["p3"]))
    g3 = de2 * (c["e2"] > 0)
    de1 += pool_bwd(conv_back(3, g3, c["p2"]))
    g2 = de1 * (c["e1"] > 0)
    de0 += pool_bwd(conv_back(2, g2, c["p1"]))
    g1 = de0 * (c["e0"] > 0)
    da0 = conv_back(1, g1, c["a0"])
    g0 = da0 * (c["a0"] > 0)
    conv_back(0, g0, c["f"])
    out = []
    for i in range(9):
        out += [gW[i], gB[i]]
    return out


def subspace_loss(Y, V, D):
    """Squared D-norm of the part of V outside span(Y):
    L = tr(V^T D V) - tr(C^T G^{-1} C), G = Y^T D Y, C = Y^T D V.
    Y: n x k network output, V: n x m targets, D: n weights (diag A).
    Returns L and dL/dY = -2 D (V - Y G^{-1} C) C^T G^{-1}."""
    DY = D[:, None] * Y
    DV = D[:, None] * V
    G = Y.T @ DY
    C = Y.T @ DV
    GiC = np.linalg.solve(G, C)
    L = np.sum(V * DV) - np.sum(C * GiC)
    grad = -2.0 * (DV - DY @ GiC) @ GiC.T
    return L, grad


def adam(param, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), in place on m and v; returns the new param."""
    m[:] = b1 * m + (1 - b1) * grad
    v[:] = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return param - lr * mh / (np.sqrt(vh) + eps)
