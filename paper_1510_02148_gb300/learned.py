"""Learned extra deflation vectors: dataset, training and evaluation driver.

Pipeline (every numerical step runs in libsld's CUDA kernels; this module
only moves device buffers between the C-ABI calls):
  1. seeded lognormal-layered fields (contrast 10^c, c ~ U[4, 6]);
  2. for each field: assemble, subdomain-levelset labels, the label
     deflation, then the 8 eigenvectors of the smallest eigenvalues of
     M^{-1} P A by shift-invert Lanczos -- the vectors the paper's Section 3.1
     says deflation should remove, and its harmonic-Ritz discussion finds too
     costly to compute per system;
  3. the U-net (BF16 tensor-core convolutions) is trained with Adam on the
     subspace loss against those eigenvectors;
  4. on held-out seeds, its output is appended to Z (sld_build_deflation)
     and the deflated solve is compared with label deflation alone.

    python -m paper_1510_02148_gb300.learned --n 128 --train 200 --eval 20
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import time

import numpy as np

from . import sld, workloads as W

TRAIN_SEED0 = 0        # training fields use seeds 0 .. ntrain-1
EVAL_SEED0 = 10_000    # held-out fields use seeds 10000 ..


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the learned-deflation pipeline needs a CUDA GPU")
    return torch


def field(seed, n):
    S = (4, 4, 2) if n >= 64 else (2, 2, 2)
    return W.learned_field(seed, n=n, S=S)


def build_system(P, stream=None):
    torch = _torch()
    s = sld.System(torch.from_numpy(P.K.reshape(-1)).cuda(), None, P.bc_type, P.bc_value, stream=stream,
                   shape=P.shape)
    s.make_labels(P.S, P.tau, P.L)
    s.build_deflation(P.d)
    return s


def make_sample(seed, n, k=8, m=30):
    """(K, V, D) on the device for one training field, plus diagnostics."""
    torch = _torch()
    P = field(seed, n)
    s = build_system(P)
    V = torch.empty((P.n, k), dtype=torch.float32, device="cuda")
    vals, _, res = sld.lanczos_eigvecs(s, k=k, m=m, vecs=V)
    D = torch.from_numpy(s.get_operator()["diag"]).cuda()
    K = torch.from_numpy(P.K.reshape(-1)).cuda()
    s.close()
    return {"seed": seed, "K": K, "V": V, "D": D, "vals": vals, "res": res}


def init_params(seed=0):
    """He-normal weights, zero biases, in the flat order of sld_net.h."""
    rng = np.random.default_rng(seed)
    out = []
    for cin, cout in [(16, 16), (16, 16), (16, 32), (32, 48), (48, 64), (64, 48), (48, 32), (32, 16), (16, 8)]:
        out.append(rng.standard_normal(27 * cout * cin) * np.sqrt(2.0 / (27 * cin)))
        out.append(np.zeros(cout))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == sld.net_num_params()
    return p


def train(net, data, epochs, lr=2e-3, seed=0, log=None, lr_decay=0.5, decay_every=None):
    """Adam on the subspace loss, one field per step, shuffled each epoch:
    one sld_learned_train call.  Returns the mean loss of each epoch."""
    hist = net.train([d["K"] for d in data], [d["V"] for d in data], [d["D"] for d in data], epochs=epochs,
                     lr=lr, lr_decay=lr_decay, decay_every=decay_every or 0, seed=seed)
    if log:
        for ep, h in enumerate(hist):
            log(f"epoch {ep}: mean loss {h:.4f}")
    return [float(h) for h in hist]


def evaluate(net, seeds, n, precision=sld.FP32_IR, tol=1e-9, auto_labels=False):
    """Label deflation alone vs label + learned columns on each field; with
    auto_labels also the automatic (connected-component) labels alone and
    with the learned columns appended."""
    torch = _torch()
    out = []
    for seed in seeds:
        P = field(seed, n)
        s = build_system(P)
        x = torch.empty(P.n, dtype=torch.float64, device="cuda")
        s.solve(x=x, precision=precision, tol=tol)  # warm-up
        _, plain = s.solve(x=x, precision=precision, tol=tol)
        t0 = time.perf_counter()
        net.infer(s)  # network on the system's own K, columns appended to its labels
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        _, ku = s.deflation_info()[1:]
        s.solve(x=x, precision=precision, tol=tol)
        _, lrn = s.solve(x=x, precision=precision, tol=tol)
        row = {"seed": seed, "plain_its": plain.iterations, "plain_ms": plain.solve_ms,
               "learned_its": lrn.iterations, "learned_ms": lrn.solve_ms, "k_used": ku,
               "learned_relres": lrn.true_relres, "plain_relres": plain.true_relres,
               "net_and_deflation_setup_ms": setup_ms}
        if auto_labels:  # the automatic labels (connected components), alone and with the learned columns
            _, dcc = s.make_labels_cc(P.S, P.tau, P.L)
            s.build_deflation(dcc)
            s.solve(x=x, precision=precision, tol=tol)
            _, cc = s.solve(x=x, precision=precision, tol=tol)
            net.infer(s)
            kcc = s.deflation_info()[2]
            s.solve(x=x, precision=precision, tol=tol)
            _, ccl = s.solve(x=x, precision=precision, tol=tol)
            row.update({"auto_d": dcc, "auto_its": cc.iterations, "auto_ms": cc.solve_ms,
                        "auto_learned_its": ccl.iterations, "auto_learned_ms": ccl.solve_ms,
                        "auto_learned_k_used": kcc, "auto_learned_relres": ccl.true_relres})
        out.append(row)
        s.close()
    return out


def summarize(rows):
    def med(key):
        return statistics.median(r[key] for r in rows)
    its_gain = [1 - r["learned_its"] / r["plain_its"] for r in rows]
    t_gain = [r["plain_ms"] / r["learned_ms"] for r in rows]
    return {"fields": len(rows), "median_plain_its": med("plain_its"), "median_learned_its": med("learned_its"),
            "mean_iteration_reduction": float(np.mean(its_gain)),
            "fields_with_fewer_iterations": int(sum(g > 0 for g in its_gain)),
            "median_plain_ms": med("plain_ms"), "median_learned_ms": med("learned_ms"),
            "median_time_ratio_plain_over_learned": float(np.median(t_gain)),
            "max_learned_relres": max(r["learned_relres"] for r in rows),
            "fields_with_columns_dropped": int(sum(r["k_used"] == 0 for r in rows)),
            **({"median_auto_its": med("auto_its"), "median_auto_ms": med("auto_ms"),
                "median_auto_learned_its": med("auto_learned_its"), "median_auto_learned_ms": med("auto_learned_ms"),
                "max_auto_learned_relres": max(r["auto_learned_relres"] for r in rows)}
               if rows and "auto_its" in rows[0] else {})}


def save_params(path, params, meta):
    np.savez(path, params=params, meta=json.dumps(meta))


def load_params(path):
    z = np.load(path)
    return z["params"], json.loads(str(z["meta"]))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--eval", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lanczos-steps", type=int, default=30)
    ap.add_argument("--out", default=None, help="write the trained parameters (.npz)")
    ap.add_argument("--json", default=None, help="write the results (.json)")
    a = ap.parse_args(argv)
    _torch()
    sld.load()
    log = lambda m: print(m, flush=True)  # noqa: E731
    t0 = time.perf_counter()
    data = [make_sample(TRAIN_SEED0 + i, a.n, m=a.lanczos_steps) for i in range(a.train)]
    t_data = time.perf_counter() - t0
    log(f"eigenvector dataset: {a.train} fields of {a.n}^3 in {t_data:.1f} s; "
        f"max residual {max(float(np.max(d['res'])) for d in data):.1e}")
    net = sld.Net((a.n, a.n, a.n))
    net.set_params(init_params(0))
    t0 = time.perf_counter()
    hist = train(net, data, a.epochs, lr=a.lr, log=log)
    t_train = time.perf_counter() - t0
    rows = evaluate(net, range(EVAL_SEED0, EVAL_SEED0 + a.eval), a.n, auto_labels=True)
    summ = summarize(rows)
    res = {"n": a.n, "train_fields": a.train, "eval_fields": a.eval, "epochs": a.epochs,
           "dataset_s": t_data, "train_s": t_train, "loss_history": hist, "summary": summ, "rows": rows}
    log(json.dumps(summ, indent=1))
    if a.out:
        save_params(a.out, net.get_params(), {"n": a.n, "train_fields": a.train, "epochs": a.epochs})
    if a.json:
        with open(a.json, "w") as f:
            json.dump(res, f, indent=1)
    net.close()
    return res


if __name__ == "__main__":
    main()
