"""The learned part end to end at a small scale: GPU Lanczos targets, training
of the BF16 tensor-core network on them, and the gain of its vectors over
label deflation alone on held-out fields, with the solution still meeting
the FP64 tolerance (the deflated solve is exact for any full-rank Z)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1510_02148_gb300 import _build, learned, sld
    _build.build()
    sld.load()
    return learned, sld


def test_learned_vectors_cut_iterations(env, oracle_mod):
    learned, sld = env
    n = 32
    data = [learned.make_sample(s, n, m=40) for s in range(16)]
    res = np.array([d["res"] for d in data])
    print("Lanczos residuals: max of the smallest pair", res[:, 0].max(), "median of the largest", np.median(res.max(1)))
    assert np.all(np.isfinite(res)) and res[:, 0].max() <= 1e-6
    net = sld.Net((n, n, n))
    net.set_params(learned.init_params(0))
    hist = learned.train(net, data, epochs=20, lr=2e-3)
    print("loss", hist[0], "->", hist[-1])
    assert hist[-1] < 0.6 * hist[0]
    rows = learned.evaluate(net, range(learned.EVAL_SEED0, learned.EVAL_SEED0 + 4), n)
    summ = learned.summarize(rows)
    print(summ)
    assert summ["fields_with_columns_dropped"] == 0
    assert summ["max_learned_relres"] <= 1e-9
    assert summ["mean_iteration_reduction"] >= 0.10
    assert summ["fields_with_fewer_iterations"] >= 3
    # the learned deflation's solution against the oracle's with the same Z (FP64 solve)
    import torch
    P = learned.field(learned.EVAL_SEED0, n)
    Y = net.forward(torch.from_numpy(P.K.reshape(-1)).cuda().contiguous())
    s = learned.build_system(P)
    s.build_deflation(P.d, Zextra=Y)
    x, info = s.solve(precision=sld.FP64)
    A = oracle_mod.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle_mod.labels(P.K, P.S, P.tau, P.L)
    ref = oracle_mod.dpcg(A, lab, P.d, tol=P.tol, Zd=Y.astype(np.float64))
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    assert abs(info.iterations - ref.iterations) <= 2
    s.close()
    net.close()


def _splitmix_order(n, seed):
    """The field order sld_learned_train documents: Fisher-Yates with the
    SplitMix64 generator (Steele, Lea and Flood 2014) seeded by seed + epoch."""
    M = (1 << 64) - 1
    st = seed & M
    order = list(range(n))

    def nxt():
        nonlocal st
        st = (st + 0x9E3779B97F4A7C15) & M
        z = st
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    for i in range(n - 1, 0, -1):
        j = nxt() % (i + 1)
        order[i], order[j] = order[j], order[i]
    return order


def test_learned_train_is_the_documented_loop(env):
    """sld_learned_train in one call gives the parameters of the per-step
    calls (forward, loss and gradient, Adam) run in its documented order and
    learning-rate schedule -- to rounding, since the loss sums and weight
    gradients are accumulated with floating-point atomics -- and not those
    of another order."""
    learned, sld = env
    n = 16
    data = [learned.make_sample(s, n, m=12) for s in range(5)]
    Ks, Vs, Ds = [d["K"] for d in data], [d["V"] for d in data], [d["D"] for d in data]
    p0 = learned.init_params(3)
    epochs, lr, decay, every, seed = 4, 3e-3, 0.5, 2, 11
    a = sld.Net((n, n, n))
    a.set_params(p0)
    hist = a.train(Ks, Vs, Ds, epochs=epochs, lr=lr, lr_decay=decay, decay_every=every, seed=seed)
    def loop(order_of):
        b = sld.Net((n, n, n))
        b.set_params(p0)
        step = 0
        means = []
        for ep in range(epochs):
            lr_ep = np.float32(lr) * np.float32(decay) ** np.float32(ep // every)
            losses = []
            for i in order_of(ep):
                b.forward(Ks[i], keep=True)
                losses.append(b.loss_backward(Vs[i], Ds[i]))
                step += 1
                b.adam(float(lr_ep), step)
            means.append(np.mean(losses))
        p = b.get_params()
        b.close()
        return np.array(means), p

    means, pb = loop(lambda ep: _splitmix_order(len(data), seed + ep))
    _, pw = loop(lambda ep: list(range(len(data)))[::-1])  # another order
    pa = a.get_params()
    np.testing.assert_allclose(hist, means, rtol=1e-3)
    # The weight gradients are summed with atomics in no fixed order and the
    # activations are stored in BF16: the atomics' rounding noise now and
    # then tips a BF16 rounding, and Adam steps carry such differences on,
    # so two runs of the same loop end close but not equal.  The documented
    # order must still be far closer than another order.
    d_same, d_other = np.linalg.norm(pa - pb), np.linalg.norm(pa - pw)
    print(f"parameters: documented loop {d_same:.2e} apart, another order {d_other:.2e} apart")
    assert d_same <= 0.1 * d_other
    assert hist[-1] < hist[0]
    with pytest.raises(sld.SldError):
        a.train(Ks, Vs, Ds, epochs=0)
    a.close()


def test_learned_infer_equals_forward_and_build(env):
    """sld_learned_infer (the network on the system's own K, appended to its
    labels) builds the same deflation as sld_net_forward followed by
    sld_build_deflation with those columns."""
    import torch
    learned, sld = env
    n = 32
    P = learned.field(learned.EVAL_SEED0 + 3, n)
    net = sld.Net((n, n, n))
    net.set_params(learned.init_params(5))
    s1 = learned.build_system(P)
    Y1 = torch.empty((P.n, 8), dtype=torch.float32, device="cuda")
    net.infer(s1, out=Y1)
    Y2 = net.forward(torch.from_numpy(P.K.reshape(-1)).cuda())
    assert np.array_equal(Y1.cpu().numpy(), Y2)
    s2 = learned.build_system(P)
    s2.build_deflation(P.d, Zextra=Y2)
    assert s1.deflation_info() == s2.deflation_info()
    # E is assembled with FP64 atomics: two builds agree to rounding
    E1, _ = s1.get_coarse()
    E2, _ = s2.get_coarse()
    assert np.max(np.abs(E1 - E2)) <= 1e-13 * np.max(np.abs(E1))
    x1, i1 = s1.solve(precision=sld.FP64)
    x2, i2 = s2.solve(precision=sld.FP64)
    assert abs(i1.iterations - i2.iterations) <= 1
    assert np.linalg.norm(x1 - x2) <= 1e-9 * np.linalg.norm(x2)
    other = sld.Net((n, n, n // 2))
    with pytest.raises(sld.SldError):
        other.infer(s1)
    other.close()
    for s in (s1, s2):
        s.close()
    net.close()
