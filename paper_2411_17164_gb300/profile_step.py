"""Plain driver for profilers: builds a synthetic workload and runs BF16
forward+backward steps of the model through the public API.

    python -m paper_2411_17164_gb300.profile_step [--nodes N] [--layers L] [--steps S] [--hidden H]
                                                  [--tune NAME=CHOICE ...] [--batched64]

Defaults are the 200,000-point car body (k = 6, H = 128, L = 15, two
steps); other hidden widths run the wide BF16 path.  --batched64 runs the
64-partition batch instead (four jittered 1M-point bodies, 64 breadth-first
regions with log-uniform inner sizes in [5k, 80k], 15-hop halos; --nodes is
then ignored).  Prints the loss so that a run can be checked for completion.
"""
import argparse

import numpy as np
import torch

from . import build, synth, xmgn


def batched64(layers):
    pts, nrms = [], []
    for b_, (cx, cy) in enumerate([(-2.4, -1.1), (2.4, -1.1), (-2.4, 1.1), (2.4, 1.1)]):
        p, nr = synth.car_body(1_000_000, 51 + b_, jitter=0.1)
        pts.append(p + np.array([cx, cy, 0.0], np.float32))
        nrms.append(nr)
    xyz = np.concatenate(pts)
    nin = synth.node_inputs(xyz, np.concatenate(nrms))
    g = xmgn.build_knn(torch.from_numpy(xyz).cuda(), 6)
    region = synth.bfs_regions(g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy(), 64, 5e3, 8e4, 505)
    b = xmgn.partition_halo(g, torch.from_numpy(xyz).cuda(), 64, layers, part_in=torch.from_numpy(region).cuda())
    return xyz, nin, synth.fourier_targets(xyz, 505), b, int((region >= 0).sum())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nodes", type=int, default=200_000)
    ap.add_argument("--layers", type=int, default=15)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--hidden", type=int, default=128)
    ap.add_argument("--tune", action="append", default=[],
                    help="launch-shape choice NAME=CHOICE for every size (see xmgn_tune_op_name)")
    ap.add_argument("--batched64", action="store_true")
    args = ap.parse_args()
    build.build()
    ops = xmgn.tune_ops()
    for item in args.tune:
        name, choice = item.split("=")
        for rows in (1 << b for b in range(40)):
            xmgn.tune_set(ops[name][0], rows, int(choice))
    H = args.hidden
    if args.batched64:
        xyz, nin, tgt, g, n_norm = batched64(args.layers)
    else:
        xyz, nrm = synth.car_body(args.nodes, 2)
        nin = synth.node_inputs(xyz, nrm)
        tgt = synth.fourier_targets(xyz, 202)
        g = xmgn.build_knn(torch.from_numpy(xyz).cuda(), 6)
        n_norm = None
    params = synth.init_params(H, args.layers, 6, 4, 102)
    tp = torch.from_numpy(params).cuda()
    ni, xz, tt = (torch.from_numpy(a).cuda() for a in (nin, xyz, tgt))
    m = xmgn.Model(H, args.layers, g, dtype="bf16", n_norm=n_norm)
    dp = torch.zeros_like(tp)
    loss = torch.zeros((), device="cuda")
    for _ in range(args.steps):
        m.forward(tp, ni, xz, targets=tt, loss=loss)
        m.backward(tp, ni, xz, tt, dp)
    torch.cuda.synchronize()
    xmgn.check_device()
    print("ok", g["E"], float(loss))


if __name__ == "__main__":
    main()
