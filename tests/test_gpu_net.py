"""The deflation-vector network's CUDA kernels (BF16 tensor-core convolutions,
their gradients, pooling, the subspace loss, Adam) and the GPU Lanczos
routine, through the C ABI, against the FP64 oracles on the same inputs."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import net_oracle as N
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


def _bf16(a):
    """Round FP64/FP32 values to BF16 (nearest even), returned as FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _params(seed):
    rng = np.random.default_rng(seed)
    p = N.init_params(seed)
    for i in range(1, len(p), 2):
        p[i] = rng.standard_normal(p[i].shape) * 0.05
    return p


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


SHAPE = (16, 24, 32)  # nz, ny, nx


def _field(seed=1):
    return np.exp(2.0 * np.random.default_rng(seed).standard_normal(SHAPE))


def _oracle_params(p):
    """The parameters as the GPU uses them: weights rounded to BF16, biases FP32."""
    q = []
    for i, a in enumerate(p):
        q.append(_bf16(a) if i % 2 == 0 else a.astype(np.float32).astype(np.float64))
    return q


def test_forward_matches_oracle(sld):
    """The FP64 oracle with BF16 rounding where the kernels store BF16 (same
    ReLU decisions on both sides); weights rounded to BF16 as the kernels use them."""
    p = _params(0)
    K = _field()
    net = sld.Net(SHAPE)
    net.set_params(N.flatten(p).astype(np.float32))
    y = net.forward(K.reshape(-1)).astype(np.float64)
    f = N.features(np.log10(K))
    ref = N.forward(_oracle_params(p), f, rnd=_bf16)[0].reshape(-1, 8)
    err = _rel(y, ref)
    print(f"forward: rel err vs BF16-storage oracle {err:.2e}, "
          f"vs FP64 oracle {_rel(y, N.forward(_oracle_params(p), f)[0].reshape(-1, 8)):.2e}")
    # BF16 storage (unit roundoff 2^-9) at about ten successive activations
    assert err <= 1e-2
    net.close()


def test_backward_matches_oracle(sld):
    p = _params(1)
    K = _field(2)
    net = sld.Net(SHAPE)
    net.set_params(N.flatten(p).astype(np.float32))
    net.forward(K.reshape(-1))
    R = np.random.default_rng(3).standard_normal((K.size, 8))
    net.backward(R.astype(np.float32))
    g = N.unflatten(net.get_grads().astype(np.float64))
    po = _oracle_params(p)
    _, cache = N.forward(po, N.features(np.log10(K)), rnd=_bf16)
    ref = N.backward(po, cache, R.reshape(SHAPE + (8,)), rnd=_bf16)
    for i, (a, b) in enumerate(zip(g, ref)):
        err = _rel(a, b)
        print(f"param {i}: rel err vs BF16-storage oracle {err:.2e}")
        assert err <= 2e-2, i
    net.close()


def test_loss_and_its_gradient(sld):
    p = _params(4)
    K = _field(5)
    net = sld.Net(SHAPE)
    net.set_params(N.flatten(p).astype(np.float32))
    rng = np.random.default_rng(6)
    V = rng.standard_normal((K.size, 6)).astype(np.float32)
    D = rng.uniform(0.1, 3.0, K.size)
    Y = net.forward(K.reshape(-1)).astype(np.float64)
    loss = net.loss_backward(V, D)
    L, dY = N.subspace_loss(Y, V.astype(np.float64), D)
    vv = np.sum(D[:, None] * V.astype(np.float64) ** 2)
    assert abs(loss - L / vv) <= 1e-6 * max(1.0, L / vv)
    g1 = net.get_grads()
    net.backward((dY / vv).astype(np.float32))  # the same gradient through the plain backward
    g2 = net.get_grads()
    assert _rel(g1, g2) <= 1e-3
    net.close()


def test_adam_step(sld):
    p = N.flatten(_params(7)).astype(np.float32)
    K = _field(8)
    net = sld.Net(SHAPE)
    net.set_params(p)
    net.forward(K.reshape(-1))
    net.backward(np.random.default_rng(9).standard_normal((K.size, 8)).astype(np.float32))
    g = net.get_grads().astype(np.float64)
    net.adam(1e-3, 1)
    m, v = np.zeros_like(g), np.zeros_like(g)
    ref = N.adam(p.astype(np.float64), g, m, v, 1, 1e-3)
    assert np.max(np.abs(net.get_params() - ref)) <= 1e-6
    net.close()


def test_training_reduces_the_loss(sld):
    """A few Adam steps on one field and fixed targets lower the loss."""
    K = _field(10)
    net = sld.Net(SHAPE)
    net.set_params(N.flatten(_params(11)).astype(np.float32))
    z, y, x = np.meshgrid(*[np.arange(s) for s in SHAPE], indexing="ij")
    V = np.stack([np.sin(np.pi * (k + 1) * (x + 0.5) / SHAPE[2]) * np.cos(np.pi * k * (z + 0.5) / SHAPE[0])
                  for k in range(4)], axis=-1).reshape(-1, 4).astype(np.float32)
    D = np.ones(K.size)
    losses = []
    for step in range(1, 41):
        net.forward(K.reshape(-1), keep=True)
        losses.append(net.loss_backward(V, D))
        net.adam(3e-3, step)
    print("loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.5 * losses[0]
    net.close()


def test_lanczos_matches_scipy(sld, oracle_mod):
    P = W.lognormal_point_source(32, 24, 16, 6, (2, 2, 2), seed=4)
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
    As = A.to_scipy().tocsr()
    n, d = A.n, P.d
    Zs = np.eye(d)[lab]
    E = Zs.T @ (As @ Zs)
    Dg = A.diag()
    Dm = 1.0 / np.sqrt(Dg)
    Q, _ = np.linalg.qr(Zs / Dm[:, None])

    def H(h):
        u = As @ (Dm * h)
        u = u - As @ (Zs @ np.linalg.solve(E, Zs.T @ u))
        return Dm * u + 10.0 * (Q @ (Q.T @ h))

    ref = sla.eigsh(sla.LinearOperator((n, n), matvec=H, dtype=np.float64), k=4, which="SA", tol=1e-12,
                    maxiter=50000)[0]
    s = sld.from_problem(P)
    vals, vecs, res = sld.lanczos_eigvecs(s, k=4, m=40)
    print("lanczos", vals, "scipy", ref, "residuals", res)
    assert np.allclose(vals, np.sort(ref), rtol=1e-6)
    assert np.all(res <= 1e-6)
    V = vecs.astype(np.float64)
    G = V.T @ (Dg[:, None] * V)  # D-orthonormal
    assert np.max(np.abs(G - np.eye(4))) <= 1e-5
    # M^{-1} P A v = theta v
    for j in range(4):
        v = V[:, j]
        u = As @ v
        u = u - As @ (Zs @ np.linalg.solve(E, Zs.T @ u))
        r = u / Dg - vals[j] * v
        assert np.sqrt(np.sum(Dg * r * r)) <= 1e-4 * max(vals[j], 1e-12) + 1e-6, j
    s.close()
