#!/usr/bin/env python3
"""fwd+bwd edge-updates/s per message-passing layer of X-MeshGraphNet on GB300.

Workload (seeded, synthetic; stands in for the paper's DrivAerML surface
clouds): a 200,000-point car-like body surface (ellipsoid + two boxes),
6-nearest-neighbour graph symmetrised (E measured, ~1.41M directed edges),
MeshGraphNet with hidden width 128, 15 processor layers, 6 node inputs,
4 outputs, MSE loss against a smooth 8-mode Fourier target field.

One step = encoder + 15 processor layers + decoder + loss forward, then the
full backward with per-layer activation recomputation and the parameter
gradient.  value = edges x layers / step time (whole job over all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (a contiguous 3,000-point surface patch, same model) on the host
cores: there is no reference implementation to run, the oracle is the
baseline.  Under torchrun only rank 0 runs it.
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

WL = dict(workload="car_body_200k_k6_H128_L15", N=200_000, k=6, H=128, L=15, in_node=6, out=4,
          seed_xyz=2, seed_tgt=202, seed_params=102)
METRIC = "fwd+bwd edge-updates/s per MP layer"
UNIT = "edge-updates/s"
SAMPLE_POINTS = 3000
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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


# ---------------------------------------------------------------------------
# oracle sample (cpu baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(n_points=SAMPLE_POINTS):
    """Contiguous surface patch of the workload: the first n_points of the
    Morton-ordered body cloud, with its own kNN graph, built by the oracle."""
    import numpy as np

    from oracle import xmgn_oracle as O
    from paper_2411_17164_gb300 import synth
    xyz, nrm = synth.car_body(WL["N"], WL["seed_xyz"])
    xyz, nrm = xyz[:n_points], nrm[:n_points]
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, WL["seed_tgt"])
    params = synth.init_params(WL["H"], WL["L"], WL["in_node"], WL["out"], WL["seed_params"]).astype(np.float64)
    rp, col, _, _ = O.symmetrise(O.knn(xyz, WL["k"]), n_points)
    return dict(xyz=xyz, nin=nin, tgt=tgt, params=params, rp=rp, col=col, E=int(len(col)), n=n_points)


def oracle_step(s):
    from oracle import xmgn_oracle as O
    dims = (WL["H"], WL["L"], WL["in_node"], WL["out"])
    t0 = time.perf_counter()
    O.loss_and_grad(s["params"], dims, s["rp"], s["col"], s["nin"], s["xyz"], s["tgt"])
    return time.perf_counter() - t0


def cpu_baseline_block(s, secs, steps):
    v = s["E"] * WL["L"] * steps / secs
    return {"value": v, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": f"FP64 numpy oracle fwd+bwd, {steps} step(s) on a contiguous {s['n']}-point patch of the "
                      f"200k-point body ({s['E']} directed edges, H=128, L=15)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    s = oracle_sample()
    for _ in range(args.warmup):
        oracle_step(s)
    t = sum(oracle_step(s) for _ in range(args.steps))
    value = s["E"] * WL["L"] * args.steps / t
    cb = cpu_baseline_block(s, t, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(None, args.gpus, sample=s),
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_block(E, n_gpus, sample=None):
    c = {"workload": WL["workload"], "nodes": WL["N"], "k": WL["k"], "hidden": WL["H"], "layers": WL["L"],
         "node_inputs": WL["in_node"], "outputs": WL["out"], "edges": E,
         "parallelism": f"dp{n_gpus}" if n_gpus > 1 else "single-gpu",
         "l2": "inputs larger than L2 (edge states 361 MB per layer, no flush)"}
    if sample is not None:
        c["sample_nodes"] = sample["n"]
        c["sample_edges"] = sample["E"]
    return c


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
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
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source."""
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


def run_ours(args):
    import numpy as np
    import torch

    from paper_2411_17164_gb300 import synth, xmgn
    from paper_2411_17164_gb300.dist import allreduce_gradient

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # workload (each rank its own body sample: weak scaling; replicated weights)
    xyz, nrm = synth.car_body(WL["N"], WL["seed_xyz"] + 1000 * rank)
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, WL["seed_tgt"])
    params = synth.init_params(WL["H"], WL["L"], WL["in_node"], WL["out"], WL["seed_params"])
    txyz, tnin, ttgt, tp = (torch.from_numpy(a).to(dev) for a in (xyz, nin, tgt, params))
    g = xmgn.build_knn(txyz, WL["k"])
    E = g["E"]
    H, L = WL["H"], WL["L"]
    model = xmgn.Model(H, L, g, dtype="bf16")
    dp = torch.zeros_like(tp)
    loss = torch.zeros((), device=dev)
    # launch shapes from the autotuner (untimed; every candidate keeps parity)
    tuned = None if args.no_tune else model.autotune(tp, tnin, txyz, ttgt, iters=2)

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

    # ---- the whole step as one CUDA graph (single rank): the library's
    # launches are recorded once and replayed; the kernel probes (CUDA event
    # pairs around the fused kernels) are recorded into the graph as well.
    graph, launches_per_step = None, None
    if world == 1 and not args.no_graph:
        xmgn.probe_enable(True)
        for k in range(4):
            xmgn.probe_read(k, reset=True)
        c0 = xmgn.launch_count()
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.graph(graph, stream=side):
            step()
        launches_per_step = xmgn.launch_count() - c0
        xmgn.probe_enable(False)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        xmgn.check_device()
    run = graph.replay if graph is not None else step

    # ---- timed region (device time, CUDA events on the launch stream)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if graph is None:
        xmgn.probe_enable(True)
        for k in range(4):
            xmgn.probe_read(k, reset=True)
    n0 = xmgn.launch_count()
    e0.record(stream)
    for _ in range(args.steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    n1 = xmgn.launch_count()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    xmgn.probe_enable(False)
    # with a graph the probes hold the last replayed step; without, every step
    probes = {name: xmgn.probe_read(k, reset=True) for k, name in
              enumerate(["edge_fwd", "edge_bwd", "node_fwd", "node_bwd"])}
    ms = e0.elapsed_time(e1) / args.steps
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t)
    value = world * E * L / (ms * 1e-3)
    gpu_launches = (n1 - n0) if graph is None else launches_per_step * args.steps
    xmgn.check_device()

    # ---- forward only (encoders, 15 layers, decoder, loss), same timing rules
    fwd_only = None
    if world == 1:
        def fstep():
            model.forward(tp, tnin, txyz, targets=ttgt, loss=loss)

        frun = fstep
        if not args.no_graph:
            fgraph = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.graph(fgraph, stream=side):
                fstep()
            frun = fgraph.replay
        for _ in range(args.warmup):
            frun()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            frun()
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / args.steps
        fwd_only = {"value": E * L / (fms * 1e-3), "unit": "edge-updates/s (forward only)", "ms_per_step": fms}
        xmgn.check_device()

    # ---- activation-checkpoint offload: edge states in page-locked host memory
    offload = None
    if world == 1:
        mo = xmgn.Model(H, L, g, dtype="bf16", offload=True)

        def ostep():
            dp.zero_()
            mo.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
            mo.backward(tp, tnin, txyz, ttgt, dp)

        orun = ostep
        if not args.no_graph:
            ograph = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.graph(ograph, stream=side):
                ostep()
            orun = ograph.replay
        for _ in range(args.warmup):
            orun()
        torch.cuda.synchronize()
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for _ in range(args.steps):
            orun()
        o1.record(stream)
        torch.cuda.synchronize()
        oms = o0.elapsed_time(o1) / args.steps
        xmgn.check_device()
        offload = {"value": E * L / (oms * 1e-3), "unit": UNIT, "ms_per_step": oms,
                   "device_ckpt_bytes": int(mo.ckpt.numel()), "host_ckpt_bytes": int(mo.host_ckpt.numel()),
                   "device_ckpt_bytes_without_offload": int(model.ckpt.numel()),
                   "note": "edge-state checkpoints copied to page-locked host memory during the forward and "
                           "back one layer ahead in the backward, on a copy stream"}
        del mo
        torch.cuda.empty_cache()

    # ---- end to end through the public API with host buffers
    h_xyz = torch.from_numpy(xyz).pin_memory()
    h_nin = torch.from_numpy(nin).pin_memory()
    h_tgt = torch.from_numpy(tgt).pin_memory()
    h_par = torch.from_numpy(params).pin_memory()
    h_loss = torch.zeros((), dtype=torch.float32).pin_memory()
    h_grad = torch.zeros_like(h_par).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_xyz, h_nin, h_tgt, h_par))
    d2h = h_loss.numel() * 4 + h_grad.numel() * 4

    def e2e_step():
        d_xyz = h_xyz.to(dev, non_blocking=True)
        d_nin = h_nin.to(dev, non_blocking=True)
        d_tgt = h_tgt.to(dev, non_blocking=True)
        d_par = h_par.to(dev, non_blocking=True)
        gg = xmgn.build_knn(d_xyz, WL["k"])
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
           "includes": "pinned H2D of points/features/targets/params, kNN graph build, fwd, bwd, D2H of loss and gradient"}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (edge-MLP backward), live device times
    pk, pk_src = peaks()
    n_nodes = WL["N"]
    nl, tot = probes["edge_bwd"]
    bwd_ms = tot / max(nl, 1)
    # algorithmic bytes per launch: every edge reads e and de' (bf16), writes
    # de and dZ1 (bf16), reads its two ids; node arrays P (bf16, 2H) and d a
    # (bf16, H) read once.
    bytes_bwd = E * (2 * H + 2 * H + 2 * H + 2 * H + 8) + n_nodes * (2 * 2 * H + 2 * H)
    achieved = bytes_bwd / (bwd_ms * 1e-3) / 1e9
    peak = float(pk["hbm_gbs"])
    tr = load_traffic("edge_bwd")
    roof = {"kernel": "edge_bwd_kernel (fused edge-MLP backward)", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{pk_src} hbm_gbs", "algorithmic_bytes_per_launch": bytes_bwd,
            "avg_launch_ms": bwd_ms, "launches": nl,
            "traffic": None if tr is None else tr["dram_bytes_per_launch_scaled"]}
    nf, totf = probes["edge_fwd"]
    fwd_ms = totf / max(nf, 1)
    # forward: every edge reads e (bf16) and its two ids and writes e' (bf16;
    # not stored by the last layer); node arrays P (bf16, 2H) read once and
    # the aggregate a (bf16, H) written once.
    L = WL["L"]
    bytes_fwd = E * (2 * H + 2 * H * (L - 1) / L + 8) + n_nodes * (2 * 2 * H + 2 * H)
    kernels = {
        "edge_fwd": {"avg_ms": fwd_ms, "achieved_gbs": bytes_fwd / (fwd_ms * 1e-3) / 1e9,
                     "frac_hbm": bytes_fwd / (fwd_ms * 1e-3) / 1e9 / peak,
                     "tensor_tflops": E * 4 * H * H / (fwd_ms * 1e-3) / 1e12},
        "edge_bwd": {"avg_ms": bwd_ms, "achieved_gbs": achieved, "frac_hbm": achieved / peak,
                     "tensor_tflops": E * 12 * H * H / (bwd_ms * 1e-3) / 1e12},
        "node_fwd": {"avg_ms": probes["node_fwd"][1] / max(probes["node_fwd"][0], 1)},
        "node_bwd": {"avg_ms": probes["node_bwd"][1] / max(probes["node_bwd"][0], 1)},
        "share_of_step": {k: probes[k][1] / (ms * (1 if graph is not None else args.steps)) for k in probes},
    }

    # ---- FP32 plain comparator on the same graph
    fp32 = None
    if not args.skip_fp32:
        del model
        torch.cuda.empty_cache()
        m32 = xmgn.Model(H, L, g, dtype="fp32")

        def step32():
            dp.zero_()
            m32.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
            m32.backward(tp, tnin, txyz, ttgt, dp)

        step32()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(2):
            step32()
        b.record(stream)
        torch.cuda.synchronize()
        ms32 = a.elapsed_time(b) / 2
        fp32 = {"value": E * L / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32,
                "bf16_speedup": (E * L / (ms * 1e-3)) / (E * L / (ms32 * 1e-3))}
        del m32
        torch.cuda.empty_cache()

    # ---- parity at the bench workload (sampled nodes, oracle on their 15-hop neighbourhood)
    err = parity_sampled(g, xyz, nin, tgt, params, dev) if not args.skip_parity else None

    # ---- CPU baseline: the oracle on a bounded sample, on this host's cores
    cb = None
    if world == 1 and not args.skip_cpu:
        s = oracle_sample()
        secs = oracle_step(s)
        cb = cpu_baseline_block(s, secs, 1)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": dict(config_block(E, world), cuda_graph=graph is not None, tuned=tuned),
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


def parity_sampled(g, xyz, nin, tgt, params, dev, n_seeds=8):
    """GPU loss restricted to a few sampled nodes (all other nodes marked halo)
    vs the oracle on exactly their 15-hop neighbourhood: identical by the
    locality of L-layer message passing (Sec. II-D)."""
    import numpy as np
    import torch

    from oracle import xmgn_oracle as O
    from paper_2411_17164_gb300 import xmgn
    N, H, L = WL["N"], WL["H"], WL["L"]
    S = np.sort(np.random.default_rng(5).choice(N, n_seeds, replace=False))
    hop = np.ones(N, np.uint8)
    hop[S] = 0
    gg = dict(g)
    gg["hop"] = torch.from_numpy(hop).to(dev)
    m = xmgn.Model(H, L, gg, dtype="bf16", n_norm=N)
    tp = torch.from_numpy(params).to(dev)
    ni, xz, tt = (torch.from_numpy(a).to(dev) for a in (nin, xyz, tgt))
    y = torch.zeros((N, WL["out"]), device=dev)
    lo = torch.zeros((), device=dev)
    m.forward(tp, ni, xz, targets=tt, y=y, loss=lo)
    dpp = torch.zeros_like(tp)
    m.backward(tp, ni, xz, tt, dpp)
    torch.cuda.synchronize()
    rp, col = g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy()
    dist_ = O.bfs_hops(rp, col, S, L)
    sub = np.nonzero(dist_ >= 0)[0]
    sub = np.concatenate([S, np.setdiff1d(sub, S)])
    lrp, lcol = O.induced_subgraph(rp, col, sub)
    mask = np.zeros(len(sub))
    mask[:len(S)] = 1
    lo_o, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, WL["in_node"], WL["out"]), lrp, lcol,
                                   nin[sub], xyz[sub], tgt[sub], mask, N)
    yg = y.cpu().numpy()[S]
    gd = dpp.cpu().numpy()
    rel = lambda a, b: float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))
    return {"y_rel_l2": rel(yg, yo[:len(S)]), "grad_rel_l2": rel(gd, go),
            "y_max_abs": float(np.abs(yg - yo[:len(S)]).max()), "grad_max_abs": float(np.abs(gd - go).max()),
            "loss_rel": abs(float(lo) - lo_o) / abs(lo_o), "tolerance": 2e-2,
            "reference": f"FP64 oracle on the 15-hop neighbourhood ({len(sub)} nodes) of {len(S)} sampled nodes"}


def run_h512(args):
    """The paper's production width: H=512 on the 200k-node body (k=6,
    L=15), the wide BF16 path (every product on the tensor cores with bf16
    operands, fp32 activations), against the FP32 plain path timed on one
    step.  One GPU; prints one JSON line."""
    import torch

    from paper_2411_17164_gb300 import synth, xmgn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    H, L = 512, WL["L"]
    xyz, nrm = synth.car_body(WL["N"], WL["seed_xyz"])
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, WL["seed_tgt"])
    params = synth.init_params(H, L, WL["in_node"], WL["out"], WL["seed_params"])
    txyz, tnin, ttgt, tp = (torch.from_numpy(a).to(dev) for a in (xyz, nin, tgt, params))
    g = xmgn.build_knn(txyz, WL["k"])
    E = g["E"]

    def timed(model, steps, warmup):
        dp = torch.zeros_like(tp)
        loss = torch.zeros((), device=dev)

        def step():
            dp.zero_()
            model.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
            model.backward(tp, tnin, txyz, ttgt, dp)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            step()
        b.record()
        torch.cuda.synchronize()
        xmgn.check_device()
        return a.elapsed_time(b) / steps

    model = xmgn.Model(H, L, g, dtype="bf16")
    steps = max(1, min(args.steps, 5))
    sampler = ClockSampler(0)
    sampler.start()
    ms = timed(model, steps, args.warmup)
    clocks = sampler.stop()
    del model
    torch.cuda.empty_cache()
    fp32 = None
    if not args.skip_fp32:
        m32 = xmgn.Model(H, L, g, dtype="fp32")
        ms32 = timed(m32, 1, 1)
        fp32 = {"value": E * L / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32, "bf16_speedup": ms32 / ms,
                "form": "FP32 plain path, CUDA cores, 1 timed step"}
    # products per edge-update at H: edge MLP 2(3H*H + H*H), node MLP 2(2H*H + H*H)/d, x3 with recompute + grads
    d = E / WL["N"]
    flops = 3 * (8 * H * H + 6 * H * H / d) * E * L
    line = {"metric": METRIC, "value": E * L / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "car_body_200k_k6_H512_L15", "nodes": WL["N"], "edges": E, "hidden": H,
                       "layers": L, "parallelism": "single-gpu", "path": "wide (library bf16 GEMMs, fp32 elementwise)",
                       "l2": "inputs larger than L2 (edge states 2.9 GB per layer, no flush)"},
            "clocks": clocks,
            "tensor_work": {"tflop_per_step": flops / 1e12, "achieved_tflops": flops / (ms * 1e-3) / 1e12,
                            "note": "GEMM flops of the step over its whole duration"},
            "fp32_plain": fp32}
    print(json.dumps(line), flush=True)
    return 0


def run_batched64(args):
    """Batched-partition workload: 64 breadth-first regions with log-uniform
    inner sizes in [5k, 80k] on four 1M-point bodies, 15-hop halos, BF16 with
    the whole step in one CUDA graph, against an FP32 loop that runs the
    partitions one at a time.  One GPU; prints one JSON line."""
    import numpy as np
    import torch

    from paper_2411_17164_gb300 import synth, xmgn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    H, L = WL["H"], WL["L"]
    pts = []
    for b_, (cx, cy) in enumerate([(-2.4, -1.1), (2.4, -1.1), (-2.4, 1.1), (2.4, 1.1)]):
        p, nr = synth.car_body(1_000_000, 51 + b_, jitter=0.1)
        pts.append((p + np.array([cx, cy, 0.0], np.float32), nr))
    xyz = np.concatenate([p for p, _ in pts])
    nin = synth.node_inputs(xyz, np.concatenate([nr for _, nr in pts]))
    tgt = synth.fourier_targets(xyz, 505)
    params = synth.init_params(H, L, WL["in_node"], WL["out"], 105)
    txyz, tnin, ttgt, tp = (torch.from_numpy(a).to(dev) for a in (xyz, nin, tgt, params))
    g = xmgn.build_knn(txyz, WL["k"])
    rp, col = g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy()
    region = synth.bfs_regions(rp, col, 64, 5e3, 8e4, 505)
    b = xmgn.partition_halo(g, txyz, 64, L, part_in=torch.from_numpy(region).to(dev))
    n_inner = int((region >= 0).sum())
    useful_E = int(np.diff(rp)[region >= 0].sum())  # full-graph edges into inner nodes
    Eb = b["E"]
    dp = torch.zeros_like(tp)
    loss = torch.zeros((), device=dev)
    model = xmgn.Model(H, L, b, dtype="bf16", n_norm=n_inner)
    tuned = None if args.no_tune else model.autotune(tp, tnin, txyz, ttgt, iters=1)

    def step():
        dp.zero_()
        model.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
        model.backward(tp, tnin, txyz, ttgt, dp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    c0 = xmgn.launch_count()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.graph(graph, stream=side):
        step()
    launches = xmgn.launch_count() - c0
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    xmgn.check_device()
    del graph, model
    torch.cuda.empty_cache()

    # FP32, one partition at a time (its own graph, workspace and launches)
    fp32 = None
    if not args.skip_fp32:
        parts = []
        brp, bcol, brecv, bperm = b["row_ptr"], b["col"], b["recv"], b["csc_perm"]
        for p_ in range(64):
            n0, n1 = b["node_ptr"][p_], b["node_ptr"][p_ + 1]
            q0, q1 = b["edge_ptr"][p_], b["edge_ptr"][p_ + 1]
            parts.append(dict(n=n1 - n0, E=q1 - q0, row_ptr=(brp[n0:n1 + 1] - q0).contiguous(),
                              col=(bcol[q0:q1] - n0).contiguous(), recv=(brecv[q0:q1] - n0).contiguous(),
                              csc_perm=(bperm[q0:q1] - q0).contiguous(), gid=b["gid"][n0:n1].contiguous(),
                              hop=b["hop"][n0:n1].contiguous(), n_global=b["n_global"]))

        def step32():
            dp.zero_()
            for gp in parts:
                m = xmgn.Model(H, L, gp, dtype="fp32", n_norm=n_inner)
                m.forward(tp, tnin, txyz, targets=ttgt, loss=loss)
                m.backward(tp, tnin, txyz, ttgt, dp)
                del m

        step32()
        torch.cuda.synchronize()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step32()
        c.record(stream)
        torch.cuda.synchronize()
        ms32 = a.elapsed_time(c)
        fp32 = {"value": Eb * L / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32,
                "bf16_speedup": ms32 / ms, "form": "FP32, one partition after another, 1 timed step"}
        xmgn.check_device()
    line = {"metric": METRIC, "value": Eb * L / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "batched64_regions_4x1M_bodies_k6_H128_L15", "partitions": 64,
                       "inner_nodes": n_inner, "batch_nodes": b["n"], "batch_edges": Eb, "halo_hops": L,
                       "parallelism": "single-gpu", "cuda_graph": True, "tuned": tuned,
                       "l2": "inputs larger than L2 (edge states 5.2 GB per layer, no flush)"},
            "clocks": clocks, "gpu_launches": int(launches * args.steps),
            "useful": {"value": useful_E * L / (ms * 1e-3), "unit": UNIT,
                       "note": "full-graph edges into inner nodes; halo edges not counted"},
            "fp32_per_partition": fp32}
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
    ap.add_argument("--no-graph", action="store_true", help="launch the step's kernels directly (no CUDA graph)")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner (candidate 0 everywhere)")
    ap.add_argument("--workload", choices=["car200k", "batched64", "h512"], default="car200k",
                    help="car200k: the 200k-node full-graph step; batched64: 64 halo partitions, BF16 batched "
                         "vs FP32 per-partition loop; h512: the 200k-node body at hidden width 512")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    from paper_2411_17164_gb300 import build
    build.build()
    if args.workload == "batched64":
        return run_batched64(args)
    if args.workload == "h512":
        return run_h512(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
