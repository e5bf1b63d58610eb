#!/usr/bin/env python3
"""fwd+bwd edge-updates/s per message-passing layer of X-MeshGraphNet on GB300,
BF16 batched against FP32 per partition, with the error against the FP64
oracle.

Default workload (batched64; seeded, synthetic, standing in for the paper's
DrivAerML surface clouds): four car-like bodies of 1,000,000 surface points
each (ellipsoid + two boxes, primitive sizes jittered by up to 10 %), their
symmetrised 6-nearest-neighbour graph, 64 breadth-first regions with
log-uniform inner sizes in [5k, 80k] as halo partitions with 15-hop halos
(Sec. III-A), all concatenated into one batch; MeshGraphNet with hidden
width 128, 15 processor layers, 6 node inputs, 4 outputs, MSE loss over the
inner nodes against a smooth 8-mode Fourier target field.  The whole BF16
training step is one CUDA graph; launch shapes come from the project's
autotuner.  Compared against FP32, one partition after another.

One step = encoders + 15 processor layers + decoder + loss forward, then the
full backward with per-layer activation recomputation and the summed
parameter gradient.  value = batch edges x layers / step time (whole job,
every rank; halo edges count, as they are processed; "useful" counts only
full-graph edges into inner nodes).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batched64|car200k|h512]

car200k: one unpartitioned 200,000-point body (the full-graph step); h512:
the same body at the paper's hidden width 512.  Under torchrun (N > 1) the
64 partitions of the batched workload are dealt to the ranks by edge count;
each rank runs its share as one batch, and the gradient is summed over ranks
once per step (compensated, rank order).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (a contiguous 3,000-point surface patch of the first body, same
model) on the host cores: there is no reference implementation to run, the
oracle is the baseline.  Under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd edge-updates/s per MP layer"
UNIT = "edge-updates/s"
SAMPLE_POINTS = 3000
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
B64 = dict(workload="batched64_regions_4x1M_bodies_k6_H128_L15", points=1_000_000, k=6, H=128, L=15, in_node=6,
           out=4, regions=64, lo=5e3, hi=8e4, seed_regions=505, seed_tgt=505, seed_params=105,
           offsets=[(-2.4, -1.1), (2.4, -1.1), (-2.4, 1.1), (2.4, 1.1)], seed_body0=51)
C2 = dict(workload="car_body_200k_k6_H128_L15", N=200_000, k=6, H=128, L=15, in_node=6, out=4,
          seed_xyz=2, seed_tgt=202, seed_params=102)
WL = C2  # the unpartitioned body's constants (car200k and h512)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def source_hash(path):
    """sha256 prefix of a CUDA source's code: comments and whitespace are
    dropped first, so that a comment edit does not invalidate a capture."""
    with open(path, encoding="utf-8") as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = re.sub(r"\s+", " ", text).strip()
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def load_traffic(kernel_key):
    """DRAM bytes per edge of one launch from the committed ncu summary
    (profiles/traffic.json), if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e:
        return None
    src = os.path.join(ROOT, e["source"])
    if not os.path.exists(src) or source_hash(src) != e["source_sha256_16"]:
        return None
    return e


# ---------------------------------------------------------------------------
# workloads (seeded inputs; no method arithmetic here)
# ---------------------------------------------------------------------------
def batched64_inputs():
    """Four jittered 1M-point bodies placed apart (no kNN edge joins two),
    node inputs, targets and parameters of the batched workload."""
    import numpy as np

    from paper_2411_17164_gb300 import synth
    pts, nrms = [], []
    for b_, (cx, cy) in enumerate(B64["offsets"]):
        p, nr = synth.car_body(B64["points"], B64["seed_body0"] + b_, jitter=0.1)
        pts.append(p + np.array([cx, cy, 0.0], np.float32))
        nrms.append(nr)
    xyz = np.concatenate(pts)
    nin = synth.node_inputs(xyz, np.concatenate(nrms))
    tgt = synth.fourier_targets(xyz, B64["seed_tgt"])
    params = synth.init_params(B64["H"], B64["L"], B64["in_node"], B64["out"], B64["seed_params"])
    return xyz, nin, tgt, params


def c2_inputs(rank=0):
    from paper_2411_17164_gb300 import synth
    xyz, nrm = synth.car_body(C2["N"], C2["seed_xyz"] + 1000 * rank)
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, C2["seed_tgt"])
    params = synth.init_params(C2["H"], C2["L"], C2["in_node"], C2["out"], C2["seed_params"])
    return xyz, nin, tgt, params


# ---------------------------------------------------------------------------
# oracle legs: CPU baseline / reference arm sample, sampled parity
# ---------------------------------------------------------------------------
def oracle_graph(xyz, k=6):
    """The oracle's symmetrised kNN graph (row_ptr, col) of a large cloud."""
    from oracle import xmgn_oracle as O
    rp, col, _, _ = O.symmetrise(O.knn_tree(xyz, k), len(xyz), csc=False)
    return rp, col


def oracle_patch(xyz, nin, tgt, params, rp, col, n_points=SAMPLE_POINTS):
    """A contiguous surface patch: the first n_points nodes in breadth-first
    order (hop, then id) from node 0, with their induced subgraph, built by
    the oracle from the oracle's graph (rp, col) of the cloud."""
    import numpy as np

    from oracle import xmgn_oracle as O
    d = O.bfs_hops(rp, col, [0], 200)
    reach = np.nonzero(d >= 0)[0]
    ids = reach[np.lexsort((reach, d[reach]))][:n_points]
    lrp, lcol = O.induced_subgraph(rp, col, ids)
    return dict(xyz=xyz[ids], nin=nin[ids], tgt=tgt[ids], params=params.astype(np.float64), rp=lrp, col=lcol,
                E=int(len(lcol)), n=len(ids))


def oracle_step(s, H, L, in_node, out):
    from oracle import xmgn_oracle as O
    t0 = time.perf_counter()
    O.loss_and_grad(s["params"], (H, L, in_node, out), s["rp"], s["col"], s["nin"], s["xyz"], s["tgt"])
    return time.perf_counter() - t0


def cpu_baseline_block(s, secs, steps, L, what):
    v = s["E"] * L * steps / secs
    return {"value": v, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": f"FP64 numpy oracle fwd+bwd, {steps} step(s) on a contiguous {s['n']}-point patch of "
                      f"{what} ({s['E']} directed edges, H=128, L={L})"}


def timed_oracle(s, H, L, in_node, out, budget_s=12.0, max_steps=8):
    """The oracle as it stands on the sample, for about budget_s seconds."""
    secs, steps = 0.0, 0
    while steps < max_steps and (steps == 0 or secs < budget_s):
        secs += oracle_step(s, H, L, in_node, out)
        steps += 1
    return secs, steps


def _sampled_gpu(X, model_graph, xyz, nin, tgt, params, S, n_norm, H, L, dtype):
    """The library's outputs y at the sampled nodes S found among the graph's
    inner nodes (rows of a [len(S), 4] array, NaN where absent; the library
    writes y by global id), the parameter gradient and the loss of the loss
    restricted to them (every other node marked halo)."""
    import numpy as np
    import torch
    dev = model_graph["row_ptr"].device
    gg = dict(model_graph)
    if "gid" in model_graph:
        gid = model_graph["gid"].cpu().numpy()
        sel = (model_graph["hop"].cpu().numpy() == 0) & np.isin(gid, S)
        gg["hop"] = torch.from_numpy(np.where(sel, 0, 1).astype(np.uint8)).to(dev)
        here = set(int(g) for g in gid[sel])
    else:
        hop = np.ones(len(xyz), np.uint8)
        hop[S] = 0
        gg["hop"] = torch.from_numpy(hop).to(dev)
        here = set(int(g) for g in S)
    m = X.Model(H, L, gg, dtype=dtype, n_norm=n_norm)
    tp = torch.from_numpy(params).to(dev)
    ni, xz, tt = (torch.from_numpy(a).to(dev) for a in (nin, xyz, tgt))
    y = torch.zeros((len(xyz), 4), device=dev)  # rows by global id, inner (here: sampled) nodes written
    lo = torch.zeros((), device=dev)
    m.forward(tp, ni, xz, targets=tt, y=y, loss=lo)
    dpp = torch.zeros_like(tp)
    m.backward(tp, ni, xz, tt, dpp)
    torch.cuda.synchronize()
    X.check_device()
    ya = y.cpu().numpy()
    yg = np.full((len(S), 4), np.nan)
    for k, g in enumerate(S):
        if int(g) in here:
            yg[k] = ya[int(g)]
    gd, lg = dpp.cpu().numpy().astype(np.float64), float(lo)
    del m, y, dpp
    torch.cuda.empty_cache()
    return yg, gd, lg


def parity_sampled(X, model_graph, rp, col, xyz, nin, tgt, params, S, n_norm, H, L, dtype="bf16"):
    """Library loss restricted to the sampled nodes S (every other node marked
    halo) vs the oracle on exactly their L-hop neighbourhood in the oracle's
    full graph (rp, col): the same quantity by the locality of L-layer
    message passing (Sec. II-D) and halo depth L (Sec. III-A).  model_graph
    may be a list of partition graphs (the per-partition FP32 form): each
    contributes the sampled nodes among its inner nodes, and the losses and
    gradients add up (Sec. III-A)."""
    import numpy as np

    from oracle import xmgn_oracle as O
    graphs = model_graph if isinstance(model_graph, list) else [model_graph]
    yg = np.full((len(S), 4), np.nan)
    gd, lg = 0.0, 0.0
    for gp in graphs:
        if isinstance(model_graph, list):
            inner = gp["gid"].cpu().numpy()[gp["hop"].cpu().numpy() == 0]
            if not np.isin(S, inner).any():
                continue
        y1, g1, l1 = _sampled_gpu(X, gp, xyz, nin, tgt, params, S, n_norm, H, L, dtype)
        yg = np.where(np.isnan(yg), y1, yg)
        gd = gd + g1
        lg += l1
    if np.isnan(yg).any():
        raise RuntimeError("sampled node not found among the graphs' inner nodes")
    dist_ = O.bfs_hops(rp, col, S, L)
    sub = np.concatenate([S, np.setdiff1d(np.nonzero(dist_ >= 0)[0], S)])
    lrp, lcol = O.induced_subgraph(rp, col, sub)
    mask = np.zeros(len(sub))
    mask[:len(S)] = 1
    lo_o, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, nin.shape[1], 4), lrp, lcol, nin[sub],
                                   xyz[sub], tgt[sub], mask, n_norm)
    rel = lambda a, b: float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))
    return {"y_rel_l2": rel(yg, yo[:len(S)]), "grad_rel_l2": rel(gd, go),
            "y_max_abs": float(np.abs(yg - yo[:len(S)]).max()), "grad_max_abs": float(np.abs(gd - go).max()),
            "loss_rel": abs(lg - lo_o) / abs(lo_o), "tolerance": 2e-2 if dtype == "bf16" else 1e-4,
            "reference": f"FP64 oracle on the {L}-hop neighbourhood ({len(sub)} nodes) of {len(S)} sampled "
                         f"inner nodes, on the oracle's own kNN graph"}


# ---------------------------------------------------------------------------
# roofline of the dominant kernel (the fused edge-MLP backward)
# ---------------------------------------------------------------------------
def roofline_block(probes, E, n, H, peak_info):
    """Edge-MLP backward: bytes the method must move per launch (read e and
    the incoming edge gradient, write the outgoing one: 3 bf16 rows of H per
    edge; 6H bytes per node for the node terms), divided by the mean launch
    time that CUDA events on the launch stream measured in the timed region.
    Also: the kernel's own design bytes (it also writes dZ1 for the node-level
    sums and reads two 4-byte ids per edge), the DRAM traffic ncu measured
    (profiles/traffic.json, per edge, scaled to this launch), and the tensor
    view (12 H^2 flop per edge with the factorised first layer)."""
    pk, src = peak_info
    peak = float(pk["hbm_gbs"])
    nl, tot = probes["edge_bwd"]
    ms = tot / max(nl, 1)
    alg = 6 * H * E + 6 * H * n
    design = (8 * H + 8) * E + 6 * H * n
    achieved = alg / (ms * 1e-3) / 1e9
    tr = load_traffic("edge_bwd")
    traffic = None if tr is None else int(tr["dram_bytes_per_edge"] * E)
    tflops = 12 * H * H * E / (ms * 1e-3) / 1e12
    sust = float(pk.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]))
    return {"kernel": "edge_bwd_kernel (fused edge-MLP backward with recompute)", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{src} hbm_gbs (of {src})", "traffic": traffic,
            "algorithmic_bytes_per_launch": alg,
            "algorithmic_bytes_rule": "6H per edge (e, incoming and outgoing edge gradient, bf16) + 6H per node",
            "design_bytes_per_launch": design, "design_frac": design / (ms * 1e-3) / 1e9 / peak,
            "traffic_frac": None if traffic is None else traffic / (ms * 1e-3) / 1e9 / peak,
            "avg_launch_ms": ms, "launches": nl, "edges_per_launch": E, "nodes_per_launch": n,
            "tensor_tflops": tflops, "tensor_frac_of_sustained_bf16": tflops / sust}


def kernel_block(probes, E, n, H, L, step_ms, graph, steps, peak):
    nf, totf = probes["edge_fwd"]
    fwd_ms = totf / max(nf, 1)
    nb, totb = probes["edge_bwd"]
    bwd_ms = totb / max(nb, 1)
    fwd_alg = 4 * H * E + 4 * H * n  # read e, write e' (bf16) + node terms
    out = {
        "edge_fwd": {"avg_ms": fwd_ms, "achieved_gbs": fwd_alg / (fwd_ms * 1e-3) / 1e9,
                     "frac_hbm": fwd_alg / (fwd_ms * 1e-3) / 1e9 / peak,
                     "tensor_tflops": E * 4 * H * H / (fwd_ms * 1e-3) / 1e12},
        "edge_bwd": {"avg_ms": bwd_ms},
        "node_fwd": {"avg_ms": probes["node_fwd"][1] / max(probes["node_fwd"][0], 1)},
        "node_bwd": {"avg_ms": probes["node_bwd"][1] / max(probes["node_bwd"][0], 1)},
        "share_of_step": {k: probes[k][1] / (step_ms * (1 if graph else steps)) for k in probes},
    }
    return out


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def capture(torch, fn, dev):
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.graph(graph, stream=side):
        fn()
    return graph


def tune_gain(torch, xmgn, step, dev, stream, ms_tuned, tuned, steps=3, rounds=3):
    """The autotuner's measured effect: the step as a CUDA graph with the tuned
    table and as one with every launch on candidate 0, timed in alternating
    blocks of `steps` replays (no clock sampler running, so both see the same
    conditions); the tuned table is restored afterwards.  `ms_tuned` is the
    headline's own figure, kept beside for reference."""
    import tempfile
    import numpy as np
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        xmgn.tune_save(path)
        graphs = {}
        try:
            for name in ("tuned", "untuned"):
                if name == "untuned":
                    xmgn.tune_clear()
                for _ in range(2):
                    step()
                graphs[name] = capture(torch, step, dev)
                for _ in range(2):
                    graphs[name].replay()
            torch.cuda.synchronize()
            t = {"tuned": [], "untuned": []}
            for _ in range(rounds):
                for name in ("tuned", "untuned"):
                    t[name].append(event_time(torch, stream, graphs[name].replay, steps))
            del graphs
        finally:
            xmgn.tune_clear()
            xmgn.tune_load(path)
    xmgn.check_device()
    mt, mu = float(np.median(t["tuned"])), float(np.median(t["untuned"]))
    return {"untuned_ms_per_step": mu, "tuned_ms_per_step": mt, "speedup": mu / mt,
            "headline_ms_per_step": ms_tuned, "non_default": {k: v for k, v in tuned.items() if v},
            "method": f"median of {rounds} alternating blocks of {steps} graph replays each"}


_SIDE = {}


def side_stream(torch, dev):
    if dev not in _SIDE:
        _SIDE[dev] = torch.cuda.Stream(dev)
    return _SIDE[dev]


def upload(torch, hosts, dev):
    """Copies pinned host tensors to the device: the first on the current
    stream, the others on a side stream (the caller makes the current stream
    wait for it before their first use).  Returns (first, [others])."""
    cur = torch.cuda.current_stream(dev)
    first = hosts[0].to(dev, non_blocking=True)
    side = side_stream(torch, dev)
    side.wait_stream(cur)
    with torch.cuda.stream(side):
        rest = [t.to(dev, non_blocking=True) for t in hosts[1:]]
    for t in rest:
        t.record_stream(cur)  # used on the current stream: not reused before that work is done
    return first, rest


def event_time(torch, stream, fn, steps):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


# ---------------------------------------------------------------------------
# reference arm: the oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def reference_sample(workload):
    """The oracle's patch sample of the workload's first body."""
    import numpy as np

    from paper_2411_17164_gb300 import synth
    if workload == "batched64":
        (cx, cy) = B64["offsets"][0]
        xyz, nrm = synth.car_body(B64["points"], B64["seed_body0"], jitter=0.1)
        xyz = xyz + np.array([cx, cy, 0.0], np.float32)
        nin = synth.node_inputs(xyz, nrm)
        tgt = synth.fourier_targets(xyz, B64["seed_tgt"])
        params = synth.init_params(B64["H"], B64["L"], B64["in_node"], B64["out"], B64["seed_params"])
        what = "the first 1M-point body of the batched workload"
    else:
        xyz, nin, tgt, params = c2_inputs()
        what = "the 200k-point body"
    rp, col = oracle_graph(xyz)
    return oracle_patch(xyz, nin, tgt, params, rp, col), what


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    W = B64 if args.workload == "batched64" else C2
    s, what = reference_sample(args.workload)
    dims = (W["H"], W["L"], W["in_node"], W["out"])
    for _ in range(args.warmup):
        oracle_step(s, *dims)
    t = sum(oracle_step(s, *dims) for _ in range(args.steps))
    value = s["E"] * W["L"] * args.steps / t
    cb = cpu_baseline_block(s, t, args.steps, W["L"], what)
    cfg = {"workload": W["workload"], "parallelism": f"dp{args.gpus}" if args.gpus > 1 else "single-gpu",
           "sample_nodes": s["n"], "sample_edges": s["E"], "hidden": W["H"], "layers": W["L"]}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "strong" if args.workload == "batched64" else "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# batched64 (default): 64 halo partitions, BF16 batched vs FP32 per partition
# ---------------------------------------------------------------------------
def run_batched64(args):
    import numpy as np
    import torch

    from paper_2411_17164_gb300 import synth, xmgn
    from paper_2411_17164_gb300.dist import allreduce_gradient, assign_partitions, rank_batch
    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, L, k = B64["H"], B64["L"], B64["k"]

    xyz, nin, tgt, params = batched64_inputs()
    N = len(xyz)
    txyz, tnin, ttgt, tp = (torch.from_numpy(a).to(dev) for a in (xyz, nin, tgt, params))
    g = xmgn.build_knn(txyz, k)
    # the regions are grown on the oracle's graph, which the library's must equal
    rp_o, col_o = oracle_graph(xyz, k)
    graph_exact = bool(np.array_equal(g["row_ptr"].cpu().numpy(), rp_o) and
                       np.array_equal(g["col"].cpu().numpy(), col_o))
    region = synth.bfs_regions(rp_o, col_o, B64["regions"], B64["lo"], B64["hi"], B64["seed_regions"])
    n_inner = int((region >= 0).sum())
    full = xmgn.partition_halo(g, txyz, B64["regions"], L, part_in=torch.from_numpy(region).to(dev))
    part_edges = [full["edge_ptr"][p + 1] - full["edge_ptr"][p] for p in range(B64["regions"])]
    mine = assign_partitions(part_edges, world)[rank]
    my_region = rank_batch(region, mine) if world > 1 else region.astype(np.int32)
    b = full if world == 1 else xmgn.partition_halo(g, txyz, len(mine), L,
                                                     part_in=torch.from_numpy(my_region).to(dev))
    if world > 1:
        del full
    Eb, nb = b["E"], b["n"]
    useful_E = int(np.diff(rp_o)[np.isin(my_region, np.arange(len(mine)))].sum())
    dp = torch.zeros_like(tp)
    loss = torch.zeros((), device=dev)
    model = xmgn.Model(H, L, b, dtype="bf16", n_norm=n_inner)
    tuned = None if args.no_tune else model.autotune(tp, tnin, txyz, ttgt, iters=1)

    def step():
        dp.zero_()
        model.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
        model.backward(tp, tnin, txyz, ttgt, dp)
        if dist is not None:
            allreduce_gradient(dp)  # gradient aggregation across ranks (Sec. III-A), rank order

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    xmgn.check_device()
    graph, launches_per_step = None, None
    if world == 1:  # the whole step as one CUDA graph, kernel probes recorded into it
        xmgn.probe_enable(True)
        for q in range(4):
            xmgn.probe_read(q, reset=True)
        c0 = xmgn.launch_count()
        graph = capture(torch, step, dev)
        launches_per_step = xmgn.launch_count() - c0
        xmgn.probe_enable(False)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        xmgn.check_device()
    run = graph.replay if graph is not None else step

    stream = torch.cuda.current_stream(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if graph is None:
        xmgn.probe_enable(True)
        for q in range(4):
            xmgn.probe_read(q, reset=True)
    n0 = xmgn.launch_count()
    ms = event_time(torch, stream, run, args.steps)
    n1 = xmgn.launch_count()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    xmgn.probe_enable(False)
    probes = {name: xmgn.probe_read(q, reset=True) for q, name in
              enumerate(["edge_fwd", "edge_bwd", "node_fwd", "node_bwd"])}
    xmgn.check_device()
    edges_all = Eb
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t)
        t = torch.tensor([Eb, useful_E], device=dev, dtype=torch.float64)
        dist.all_reduce(t)
        edges_all, useful_E = int(t[0]), int(t[1])
    value = edges_all * L / (ms * 1e-3)
    gpu_launches = (n1 - n0) if graph is None else launches_per_step * args.steps
    had_graph = graph is not None
    del graph
    tuning = tune_gain(torch, xmgn, step, dev, stream, ms, tuned) if had_graph and tuned else None
    del model
    torch.cuda.empty_cache()

    # ---- end to end through the public API with host buffers: every step
    # copies points, features, targets, parameters and the region ids in,
    # builds the kNN graph and this rank's halo partitions, runs forward and
    # backward (and the rank-order gradient sum), copies loss and gradient out
    hosts = [torch.from_numpy(a).pin_memory() for a in (xyz, nin, tgt, params, my_region)]
    h_loss = torch.zeros((), dtype=torch.float32).pin_memory()
    h_grad = torch.zeros(len(params), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hosts)
    d2h = 4 + h_grad.numel() * 4
    P_mine = len(mine)

    def e2e_step():
        # the points first; the other inputs travel on a side stream while the kNN graph is built
        d_xyz, (d_nin, d_tgt, d_par, d_reg) = upload(torch, hosts, dev)
        gg = xmgn.build_knn(d_xyz, k)
        torch.cuda.current_stream(dev).wait_stream(side_stream(torch, dev))
        bb = xmgn.partition_halo(gg, d_xyz, P_mine, L, part_in=d_reg)
        m = xmgn.Model(H, L, bb, dtype="bf16", n_norm=n_inner)
        lo = torch.zeros((), device=dev)
        gr = torch.zeros_like(d_par)
        m.forward(d_par, d_nin, d_xyz, targets=d_tgt, loss=lo)
        m.backward(d_par, d_nin, d_xyz, d_tgt, gr)
        if dist is not None:
            allreduce_gradient(gr)
        h_loss.copy_(lo, non_blocking=True)
        h_grad.copy_(gr, non_blocking=True)
        return bb["E"]

    e2e_steps = max(3, args.steps // 6)
    e2e_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    ee = 0
    for _ in range(e2e_steps):
        ee = e2e_step()
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    ee_all = ee
    if dist is not None:
        t = torch.tensor([t_e2e, float(ee)], device=dev, dtype=torch.float64)
        tt_ = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
        dist.all_reduce(tt_, op=dist.ReduceOp.MAX)
        dist.all_reduce(t)
        t_e2e, ee_all = float(tt_), int(t[1])
    e2e = {"value": ee_all * L / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": 1e3 * t_e2e,
           "includes": "pinned H2D of points/features/targets/params/region ids, kNN graph build, halo "
                       "partitioning, model workspace, fwd, bwd, D2H of loss and gradient"}
    torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    pk = peaks()
    roof = roofline_block(probes, Eb, nb, H, pk) if world == 1 else None
    kernels = kernel_block(probes, Eb, nb, H, L, ms, True, args.steps, float(pk[0]["hbm_gbs"])) if world == 1 else None

    # ---- FP32, one partition at a time (its own graph, workspace and launches)
    fp32 = None
    if world == 1 and not args.skip_fp32:
        parts = xmgn.split_batch(b)

        def step32():
            dp.zero_()
            for gp in parts:
                m = xmgn.Model(H, L, gp, dtype="fp32", n_norm=n_inner)
                m.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
                m.backward(tp, tnin, txyz, ttgt, dp)
                del m

        step32()
        torch.cuda.synchronize()
        ms32 = event_time(torch, stream, step32, 1)
        xmgn.check_device()
        fp32 = {"value": Eb * L / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32, "bf16_speedup": ms32 / ms,
                "form": "FP32 on CUDA cores, the 64 partitions one after another (own graph, workspace and "
                        "launches each), 1 timed step"}
        if not args.skip_parity:  # the same sampled check as the BF16 line's err, through the partitions
            S32 = np.sort(np.random.default_rng(55).choice(np.nonzero(region >= 0)[0], 8, replace=False))
            fp32["err"] = parity_sampled(xmgn, parts, rp_o, col_o, xyz, nin, tgt, params, S32, n_inner, H, L,
                                         dtype="fp32")
        del parts
        torch.cuda.empty_cache()

    # ---- parity at this workload: sampled inner nodes vs the oracle
    err = None
    if world == 1 and not args.skip_parity:
        S = np.sort(np.random.default_rng(55).choice(np.nonzero(region >= 0)[0], 8, replace=False))
        err = parity_sampled(xmgn, b, rp_o, col_o, xyz, nin, tgt, params, S, n_inner, H, L)
        err["graph_bit_exact"] = graph_exact

    # ---- CPU baseline: the oracle on a bounded sample, on this host's cores
    cb = None
    if world == 1 and not args.skip_cpu:
        s = oracle_patch(xyz[:B64["points"]], nin[:B64["points"]], tgt[:B64["points"]], params,
                         *(_body0_graph(rp_o, col_o)))
        secs, steps = timed_oracle(s, H, L, B64["in_node"], B64["out"])
        cb = cpu_baseline_block(s, secs, steps, L, "the first 1M-point body of the batched workload")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": B64["workload"], "partitions": B64["regions"], "inner_nodes": n_inner,
                       "batch_nodes": nb, "batch_edges": Eb, "halo_hops": L, "hidden": H, "layers": L,
                       "partitions_per_rank": P_mine,
                       "parallelism": f"dp{world} (partitions dealt to ranks by edges)" if world > 1 else "single-gpu",
                       "cuda_graph": world == 1, "tuned": tuned, "tuning": tuning,
                       "l2": "inputs larger than L2 (edge states 5.2 GB per layer, no flush)"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(gpu_launches), "roofline": roof,
            "cpu_baseline": cb, "err": err, "fp32_per_partition": fp32, "kernels": kernels,
            "useful": {"value": useful_E * L / (ms * 1e-3), "unit": UNIT,
                       "note": "full-graph edges into inner nodes; halo edges not counted"}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _body0_graph(rp, col):
    """The oracle graph restricted to the first body (bodies are separate
    components, so this is the first body's own kNN graph)."""
    n0 = B64["points"]
    col0 = col[:rp[n0]]
    if col0.size and int(col0.max()) >= n0:
        raise RuntimeError("the first body shares an edge with another body")
    return rp[:n0 + 1].copy(), col0.copy()


# ---------------------------------------------------------------------------
# car200k: one unpartitioned 200k-point body (the full-graph step)
# ---------------------------------------------------------------------------
def run_car200k(args):
    import numpy as np
    import torch

    from paper_2411_17164_gb300 import xmgn
    from paper_2411_17164_gb300.dist import allreduce_gradient
    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, L, k = C2["H"], C2["L"], C2["k"]
    # each rank its own body sample (weak scaling), replicated weights
    xyz, nin, tgt, params = c2_inputs(rank)
    txyz, tnin, ttgt, tp = (torch.from_numpy(a).to(dev) for a in (xyz, nin, tgt, params))
    g = xmgn.build_knn(txyz, k)
    E, N = g["E"], C2["N"]
    model = xmgn.Model(H, L, g, dtype="bf16")
    dp = torch.zeros_like(tp)
    loss = torch.zeros((), device=dev)
    tuned = None if args.no_tune else model.autotune(tp, tnin, txyz, ttgt, iters=2)

    def step():
        dp.zero_()
        model.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
        model.backward(tp, tnin, txyz, ttgt, dp)
        if dist is not None:
            allreduce_gradient(dp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    xmgn.check_device()
    graph, launches_per_step = None, None
    if world == 1 and not args.no_graph:
        xmgn.probe_enable(True)
        for q in range(4):
            xmgn.probe_read(q, reset=True)
        c0 = xmgn.launch_count()
        graph = capture(torch, step, dev)
        launches_per_step = xmgn.launch_count() - c0
        xmgn.probe_enable(False)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        xmgn.check_device()
    run = graph.replay if graph is not None else step
    stream = torch.cuda.current_stream(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if graph is None:
        xmgn.probe_enable(True)
        for q in range(4):
            xmgn.probe_read(q, reset=True)
    n0 = xmgn.launch_count()
    ms = event_time(torch, stream, run, args.steps)
    n1 = xmgn.launch_count()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    xmgn.probe_enable(False)
    probes = {name: xmgn.probe_read(q, reset=True) for q, name in
              enumerate(["edge_fwd", "edge_bwd", "node_fwd", "node_bwd"])}
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t)
    value = world * E * L / (ms * 1e-3)
    gpu_launches = (n1 - n0) if graph is None else launches_per_step * args.steps
    xmgn.check_device()
    tuning = tune_gain(torch, xmgn, step, dev, stream, ms, tuned, steps=10) if graph is not None and tuned else None

    fwd_only = None
    if world == 1:
        def fstep():
            model.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
        frun = fstep if args.no_graph else capture(torch, fstep, dev).replay
        for _ in range(args.warmup):
            frun()
        torch.cuda.synchronize()
        fms = event_time(torch, stream, frun, args.steps)
        fwd_only = {"value": E * L / (fms * 1e-3), "unit": "edge-updates/s (forward only)", "ms_per_step": fms}
        xmgn.check_device()

    offload = None
    if world == 1:  # activation-checkpoint offload: edge states in page-locked host memory
        mo = xmgn.Model(H, L, g, dtype="bf16", offload=True)

        def ostep():
            dp.zero_()
            mo.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
            mo.backward(tp, tnin, txyz, ttgt, dp)
        orun = ostep if args.no_graph else capture(torch, ostep, dev).replay
        for _ in range(args.warmup):
            orun()
        torch.cuda.synchronize()
        oms = event_time(torch, stream, orun, args.steps)
        xmgn.check_device()
        offload = {"value": E * L / (oms * 1e-3), "unit": UNIT, "ms_per_step": oms,
                   "device_ckpt_bytes": int(mo.ckpt.numel()), "host_ckpt_bytes": int(mo.host_ckpt.numel()),
                   "device_ckpt_bytes_without_offload": int(model.ckpt.numel()),
                   "note": "edge-state checkpoints copied to page-locked host memory during the forward and "
                           "back one layer ahead in the backward, on a copy stream"}
        del mo
        torch.cuda.empty_cache()

    hosts = [torch.from_numpy(a).pin_memory() for a in (xyz, nin, tgt, params)]
    h_loss = torch.zeros((), dtype=torch.float32).pin_memory()
    h_grad = torch.zeros(len(params), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hosts)
    d2h = 4 + h_grad.numel() * 4

    def e2e_step():
        d_xyz, (d_nin, d_tgt, d_par) = upload(torch, hosts, dev)
        gg = xmgn.build_knn(d_xyz, k)
        torch.cuda.current_stream(dev).wait_stream(side_stream(torch, dev))
        m = xmgn.Model(H, L, gg, dtype="bf16")
        lo = torch.zeros((), device=dev)
        gr = torch.zeros_like(d_par)
        m.forward(d_par, d_nin, d_xyz, targets=d_tgt, loss=lo)
        m.backward(d_par, d_nin, d_xyz, d_tgt, gr)
        if dist is not None:
            allreduce_gradient(gr)
        h_loss.copy_(lo, non_blocking=True)
        h_grad.copy_(gr, non_blocking=True)
        return gg["E"]

    e2e_steps = max(3, args.steps // 3)
    e2e_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    ee = 0
    for _ in range(e2e_steps):
        ee = e2e_step()
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        t = torch.tensor([t_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t)
    e2e = {"value": world * ee * L / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * t_e2e,
           "includes": "pinned H2D of points/features/targets/params, kNN graph build, fwd, bwd, D2H of loss and "
                       "gradient"}
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    pk = peaks()
    roof = roofline_block(probes, E, N, H, pk)
    kernels = kernel_block(probes, E, N, H, L, ms, graph is not None, args.steps, float(pk[0]["hbm_gbs"]))
    rp_o, col_o = oracle_graph(xyz, k) if not (args.skip_parity and args.skip_cpu) else (None, None)
    graph_exact = None if rp_o is None else bool(np.array_equal(g["row_ptr"].cpu().numpy(), rp_o) and
                                                 np.array_equal(g["col"].cpu().numpy(), col_o))
    S = np.sort(np.random.default_rng(5).choice(N, 8, replace=False))
    err = None
    if not args.skip_parity:
        del model
        torch.cuda.empty_cache()
        err = parity_sampled(xmgn, g, rp_o, col_o, xyz, nin, tgt, params, S, N, H, L)
        err["graph_bit_exact"] = graph_exact

    fp32 = None
    if not args.skip_fp32:
        torch.cuda.empty_cache()
        m32 = xmgn.Model(H, L, g, dtype="fp32")

        def step32():
            dp.zero_()
            m32.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
            m32.backward(tp, tnin, txyz, ttgt, dp)

        step32()
        torch.cuda.synchronize()
        ms32 = event_time(torch, stream, step32, 2)
        fp32 = {"value": E * L / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32, "bf16_speedup": ms32 / ms}
        del m32
        torch.cuda.empty_cache()
        if not args.skip_parity:
            fp32["err"] = parity_sampled(xmgn, g, rp_o, col_o, xyz, nin, tgt, params, S, N, H, L, dtype="fp32")

    cb = None
    if world == 1 and not args.skip_cpu:
        s = oracle_patch(xyz, nin, tgt, params, rp_o, col_o)
        secs, steps = timed_oracle(s, H, L, C2["in_node"], C2["out"])
        cb = cpu_baseline_block(s, secs, steps, L, "the 200k-point body")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": C2["workload"], "nodes": N, "k": k, "hidden": H, "layers": L,
                       "node_inputs": C2["in_node"], "outputs": C2["out"], "edges": E,
                       "parallelism": f"dp{world}" if world > 1 else "single-gpu", "cuda_graph": graph is not None,
                       "tuned": tuned, "tuning": tuning, "l2": "inputs larger than L2 (edge states 361 MB per layer, no flush)"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(gpu_launches), "roofline": roof,
            "cpu_baseline": cb, "fp32_plain": fp32, "err": err, "kernels": kernels,
            "forward_only": fwd_only, "offload": offload,
            "useful": {"value": value, "unit": UNIT,
                       "note": "full graph, no halo edges: every processed edge is useful"}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def wide_gemm_flops(H, L, E, N, in_node, out):
    """GEMM flops of one wide-path fwd+bwd step (2 M K N per product): per MLP
    the forward X W1 and A1 W2, the backward's recompute of both (the decoder,
    without LayerNorm, recomputes only X W1), A1^T dZ2, dZ2 W2^T, X^T dZ1 and,
    except for the encoders, dZ1 W1^T."""
    def mlp(M, K, o, ln=True, dx=True):
        f = 2 * M * (K * H + H * o)
        b = 2 * M * K * H + (2 * M * H * o if ln else 0) + 2 * M * H * o + 2 * M * o * H + 2 * M * K * H
        return f + b + (2 * M * H * K if dx else 0)
    return (mlp(N, in_node, H, dx=False) + mlp(E, 4, H, dx=False) + L * (mlp(E, 3 * H, H) + mlp(N, 2 * H, H)) +
            mlp(N, H, out, ln=False))


def run_h512(args):
    """The paper's production width: H=512 on the 200k-node body (k=6,
    L=15), the wide BF16 path (every product on this project's tcgen05 GEMM
    with bf16 operands, fp32 activations), against the FP32 plain path timed
    on one step.  One GPU; prints one JSON line with the GEMM's roofline
    (tensor-bound: GEMM flops of the step over the summed device time of its
    GEMM launches, CUDA-event probes on the launch stream)."""
    import torch

    from paper_2411_17164_gb300 import synth, xmgn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    H, L = 512, C2["L"]
    xyz, nrm = synth.car_body(C2["N"], C2["seed_xyz"])
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, C2["seed_tgt"])
    params = synth.init_params(H, L, C2["in_node"], C2["out"], C2["seed_params"])
    txyz, tnin, ttgt, tp = (torch.from_numpy(a).to(dev) for a in (xyz, nin, tgt, params))
    g = xmgn.build_knn(txyz, C2["k"])
    E = g["E"]

    def timed(model, steps, warmup, probe=False):
        dp = torch.zeros_like(tp)
        loss = torch.zeros((), device=dev)

        def step():
            dp.zero_()
            model.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
            model.backward(tp, tnin, txyz, ttgt, dp)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        if probe:
            xmgn.probe_enable(True)
            xmgn.probe_read(xmgn.PROBE_WIDE_GEMM, reset=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            step()
        b.record()
        torch.cuda.synchronize()
        xmgn.check_device()
        pr = None
        if probe:
            xmgn.probe_enable(False)
            pr = xmgn.probe_read(xmgn.PROBE_WIDE_GEMM, reset=True)
        return a.elapsed_time(b) / steps, pr

    model = xmgn.Model(H, L, g, dtype="bf16")
    steps = max(1, min(args.steps, 5))
    sampler = ClockSampler(0)
    sampler.start()
    ms, (n_gemm, gemm_ms) = timed(model, steps, args.warmup, probe=True)
    clocks = sampler.stop()
    del model
    torch.cuda.empty_cache()
    fp32 = None
    if not args.skip_fp32:
        m32 = xmgn.Model(H, L, g, dtype="fp32")
        ms32, _ = timed(m32, 1, 1)
        fp32 = {"value": E * L / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32, "bf16_speedup": ms32 / ms,
                "form": "FP32 plain path, CUDA cores, 1 timed step"}
        del m32
        torch.cuda.empty_cache()
    err = None
    if not args.skip_parity:  # eight sampled nodes: the FP64 oracle at width 512 on their 15-hop neighbourhoods
        import numpy as np
        rp_o, col_o = oracle_graph(xyz, C2["k"])
        S = np.sort(np.random.default_rng(77).choice(C2["N"], 8, replace=False))
        err = parity_sampled(xmgn, g, rp_o, col_o, xyz, nin, tgt, params, S, C2["N"], H, L)
        err["graph_bit_exact"] = bool(np.array_equal(g["row_ptr"].cpu().numpy(), rp_o) and
                                      np.array_equal(g["col"].cpu().numpy(), col_o))
    flops = wide_gemm_flops(H, L, E, C2["N"], C2["in_node"], C2["out"])
    pk, src = peaks()
    peak = float(pk.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]))
    gemm_step_ms = gemm_ms / steps
    achieved = flops / (gemm_step_ms * 1e-3) / 1e12
    roof = {"kernel": "wg_kernel (tcgen05 GEMM of the wide path, all launches of a step)", "bound": "tensor",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": f"{src} bf16_tflops_sustained (of {src}; the GEMMs run inside a long step)",
            "traffic": None, "flop_per_step": flops, "gemm_ms_per_step": gemm_step_ms,
            "gemm_launches_per_step": n_gemm / steps, "gemm_share_of_step": gemm_step_ms / ms}
    line = {"metric": METRIC, "value": E * L / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "car_body_200k_k6_H512_L15", "nodes": C2["N"], "edges": E, "hidden": H,
                       "layers": L, "parallelism": "single-gpu",
                       "path": "wide (tcgen05 GEMMs of this project, bf16 operands, fp32 elementwise)",
                       "l2": "inputs larger than L2 (edge states 2.9 GB per layer, no flush)"},
            "clocks": clocks, "roofline": roof,
            "tensor_work": {"tflop_per_step": flops / 1e12, "achieved_tflops_over_step": flops / (ms * 1e-3) / 1e12,
                            "note": "GEMM flops of the step over its whole duration"},
            "fp32_plain": fp32, "err": err}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--skip-parity", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="car200k: launch the step's kernels directly")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner (candidate 0 everywhere)")
    ap.add_argument("--workload", choices=["batched64", "car200k", "h512"], default="batched64",
                    help="batched64: 64 halo partitions on four 1M-point bodies, BF16 batched vs FP32 per "
                         "partition; car200k: the 200k-node full-graph step; h512: the 200k-node body at "
                         "hidden width 512")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    from paper_2411_17164_gb300 import build
    build.build()
    if args.workload == "car200k":
        return run_car200k(args)
    if args.workload == "h512":
        return run_h512(args)
    return run_batched64(args)


if __name__ == "__main__":
    sys.exit(main())
