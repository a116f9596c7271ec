"""Writes ref_iterations.json: the CPU oracle's FP64 deflated-CG iteration
count to the tolerance of each benchmark workload, by a full oracle solve.
The reference arm of bench.py scales its bounded timing sample to this
count.  Calls only the oracle and the seeded input generators.

    python tests/golden/make_ref_iterations.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1510_02148_gb300 import workloads as W  # noqa: E402


def main():
    oracle.build()
    out = {}
    P = W.lognormal_point_source()
    A = oracle.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle.labels(P.K, P.S, P.tau, P.L)
    t0 = time.perf_counter()
    r = oracle.dpcg(A, lab, P.d, tol=P.tol)
    out[P.name] = {"iterations": r.iterations, "status": r.status, "true_relres": r.true_relres,
                   "tol": P.tol, "d": P.d, "oracle_seconds": round(time.perf_counter() - t0, 1),
                   "threads": oracle.max_threads()}
    with open(os.path.join(HERE, "ref_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
