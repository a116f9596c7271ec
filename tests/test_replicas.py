"""The multi-GPU run's host logic on CPU: world size 2 over gloo.

The solve has no data-path exchange between GPUs (replicas only), so what
runs across ranks is the bench's bookkeeping: joining the group, the barrier
around the timed region, the maximum of the per-rank step times, one seeded
field per rank, and rank 0 alone printing (the reference arm's other ranks
exit without work)."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
from paper_1510_02148_gb300 import replicas
world, rank, local = replicas.init(cuda=False)
replicas.barrier(cuda=False)
m = replicas.max_over_ranks(10.0 + 5.0 * rank, cuda=False)
replicas.barrier(cuda=False)
print(world, rank, local, m, replicas.replica_seed(rank), flush=True)
replicas.finish()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_max_step_time():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(out.split())
    assert [o[:3] for o in outs] == [["2", "0", "0"], ["2", "1", "1"]]
    assert all(float(o[3]) == 15.0 for o in outs)  # max over ranks, seen by both
    assert [int(o[4]) for o in outs] == [1, 2]  # each replica its own field


def test_single_rank_needs_no_group():
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    script = RANK_SCRIPT.format(root=ROOT)
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["1", "0", "0", "10.0", "1"]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
