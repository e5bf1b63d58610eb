"""CPU checks of bench.py's host-side pieces: the clock record taken during
the timed region, the code hash that keys a DRAM-traffic capture, and the
oracle sample behind the CPU baseline."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(HERE, "..", "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_record_median_and_throttle_reasons():
    b = _bench()
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample
        "0, 2040, 2070, 1100.0, 0x0, Not Active, Active, Not Active, Not Active",
    ]
    s = b.ClockSampler(0)
    s.proc = _FakeSmi("\n".join(lines) + "\n")
    r = s.stop()
    assert r["samples"] == 4
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0      # upper median of 1980, 2040, 2070, 2070
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_record_without_nvidia_smi():
    b = _bench()
    s = b.ClockSampler(0)
    r = s.stop()
    assert r["samples"] == 0 and r["sm_mhz"] is None


def test_source_hash_ignores_comments_and_whitespace(tmp_path):
    b = _bench()
    a = tmp_path / "a.cu"
    a.write_text("__global__ void k(int* x) {\n  x[0] = 1;  // store\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("/* a kernel */\n__global__ void k(int* x)\n{ x[0] = 1; }\n")
    d = tmp_path / "d.cu"
    d.write_text("__global__ void k(int* x) { x[0] = 2; }\n")
    assert b.source_hash(str(a)) == b.source_hash(str(c))
    assert b.source_hash(str(a)) != b.source_hash(str(d))


def test_oracle_sample_and_cpu_baseline_block():
    """The CPU baseline's sample is a well-formed symmetric kNN graph on a
    prefix of the benchmark body, and its throughput counts E x L per step."""
    b = _bench()
    from oracle import xmgn_oracle as O
    s = b.oracle_sample(400)
    rp, col = np.asarray(s["rp"]), np.asarray(s["col"])
    assert s["n"] == 400 and len(rp) == 401 and rp[-1] == len(col) == s["E"]
    assert np.all(np.diff(rp) >= b.WL["k"]) and col.min() >= 0 and col.max() < 400
    recv = np.repeat(np.arange(400), np.diff(rp))
    assert set(zip(recv.tolist(), col.tolist())) == set(zip(col.tolist(), recv.tolist()))   # undirected
    assert len(s["params"]) == O.param_count(b.WL["H"], b.WL["L"], b.WL["in_node"], b.WL["out"])
    cb = b.cpu_baseline_block(s, 2.0, 4)
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["unit"] == b.UNIT
    assert abs(cb["value"] - s["E"] * b.WL["L"] * 4 / 2.0) < 1e-9 * cb["value"]
