"""Host-side arithmetic of the benchmark line (no GPU): the PDGMRES byte
count against a step-by-step tally of its passes, the clock-record parser
and the peak lookup."""
import json
import os

import pytest

import bench


def _tally(n, m, its, deflated):
    """Step by step: a cycle's residual pass, then per Arnoldi step with basis
    size j+1 the apply, the deflation, two dot and two orthogonalisation
    passes over the basis; the pass that writes the next raw vector (the
    residual copy, the second orthogonalisation) also reads 1/diag and
    writes M^-1 of it."""
    tot, left = 0, its
    while left > 0:
        k = min(m, left)
        left -= k
        tot += (68 + 52 + 16 + 16) if deflated else (68 + 16 + 16 - 4)
        for j in range(k):
            dot = (j + 1) * 8 + 8     # basis and w read
            orth = (j + 1) * 8 + 16   # basis read, w read and written
            step = 68 + 2 * dot + 2 * orth + 16
            if deflated:
                step += 52
            else:
                step -= 4  # no label read in the apply
            tot += step
    return n * tot


@pytest.mark.parametrize("deflated", [False, True])
@pytest.mark.parametrize("m,its", [(20, 20), (20, 47), (5, 1), (30, 90)])
def test_gmres_bytes_matches_step_tally(deflated, m, its):
    cycles = -(-its // m)
    assert bench.gmres_bytes(1000, m, its, cycles, deflated) == _tally(1000, m, its, deflated)


def test_clock_summary_parses_nvidia_smi_lines():
    c = bench.ClockSampler()
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1100.4, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_clock_summary_empty():
    s = bench.ClockSampler().summary()
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["reasons"] == []


def test_peaks_from_measured_file():
    p = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    val, kind = bench._peaks()
    if os.path.exists(p):
        assert kind == "measured" and val == float(json.load(open(p))["hbm_gbs"])
    else:
        assert (val, kind) == (6800.0, "fallback")


def _fake_smi(tmp_path, body):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text("#!/bin/sh\n" + body)
    f.chmod(0o755)
    return str(d)


def test_clock_sampler_opens_after_the_first_sample(tmp_path, monkeypatch):
    """The sampler returns from __enter__ once nvidia-smi has printed its
    first line (its start-up happens before the timed region), and keeps
    collecting afterwards."""
    import time
    line = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    fake = _fake_smi(tmp_path, f"sleep 0.3\nwhile true; do echo '{line}'; sleep 0.05; done\n")
    monkeypatch.setenv("PATH", fake + os.pathsep + os.environ.get("PATH", ""))
    t0 = time.perf_counter()
    with bench.ClockSampler() as c:
        waited = time.perf_counter() - t0
        assert c.lines and waited >= 0.25
        time.sleep(0.2)
    assert len(c.lines) >= 2 and c.summary()["sm_mhz"] == 2070


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    """No nvidia-smi, or one that exits at once: no wait, an empty record."""
    import time
    monkeypatch.setenv("PATH", str(tmp_path))
    t0 = time.perf_counter()
    with bench.ClockSampler() as c:
        pass
    assert time.perf_counter() - t0 < 2.0 and c.summary()["samples"] == 0
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, "exit 0\n") + os.pathsep + os.environ.get("PATH", ""))
    t0 = time.perf_counter()
    with bench.ClockSampler() as c:
        pass
    assert time.perf_counter() - t0 < 2.0 and c.summary()["samples"] == 0
