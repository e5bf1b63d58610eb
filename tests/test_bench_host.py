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


def test_oracle_patch_and_cpu_baseline_block():
    """The CPU baseline's sample is a contiguous patch of the oracle's graph:
    the first nodes in breadth-first order from node 0 with their induced,
    still undirected subgraph; its throughput counts E x L per step."""
    b = _bench()
    from oracle import xmgn_oracle as O
    from paper_2411_17164_gb300 import synth
    xyz, nrm = synth.car_body(2000, 2)
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, 3)
    params = synth.init_params(128, 15, 6, 4, 4)
    rp, col = b.oracle_graph(xyz)
    rp2, col2, _, _ = O.symmetrise(O.knn(xyz, 6), 2000)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    s = b.oracle_patch(xyz, nin, tgt, params, rp, col, n_points=400)
    prp, pcol = np.asarray(s["rp"]), np.asarray(s["col"])
    assert s["n"] == 400 and len(prp) == 401 and prp[-1] == len(pcol) == s["E"]
    assert pcol.min() >= 0 and pcol.max() < 400
    recv = np.repeat(np.arange(400), np.diff(prp))
    assert set(zip(recv.tolist(), pcol.tolist())) == set(zip(pcol.tolist(), recv.tolist()))   # undirected
    assert np.all(O.bfs_hops(prp, pcol, [0], 400) >= 0)                                          # one piece
    assert len(s["params"]) == O.param_count(128, 15, 6, 4)
    cb = b.cpu_baseline_block(s, 2.0, 4, 15, "a test body")
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["unit"] == b.UNIT
    assert abs(cb["value"] - s["E"] * 15 * 4 / 2.0) < 1e-9 * cb["value"]


def test_rank_share_of_batched_partitions():
    """Under torchrun the batched workload's partitions are dealt to ranks by
    edges; every partition lands on exactly one rank."""
    from paper_2411_17164_gb300.dist import assign_partitions
    edges = [int(x) for x in np.random.default_rng(0).integers(10_000, 500_000, 64)]
    for world in (1, 2, 4, 8):
        share = assign_partitions(edges, world)
        assert sorted(sum(share, [])) == list(range(64))
        loads = [sum(edges[p] for p in r) for r in share]
        assert max(loads) - min(loads) <= max(edges)
