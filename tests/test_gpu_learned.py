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
