"""Plain driver for profilers: builds the synthetic car-body graph and runs
BF16 forward+backward steps of the model through the public API.

    python -m paper_2411_17164_gb300.profile_step [--nodes N] [--layers L] [--steps S] [--hidden H]
                                                  [--tune NAME=CHOICE ...]

Defaults are the benchmark workload (200,000 points, k = 6, H = 128, L = 15,
two steps).  Other hidden widths run the wide BF16 path.  Prints the loss so
that a run can be checked for completion.
"""
import argparse

import torch

from . import build, synth, xmgn


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nodes", type=int, default=200_000)
    ap.add_argument("--layers", type=int, default=15)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--hidden", type=int, default=128)
    ap.add_argument("--tune", action="append", default=[],
                    help="launch-shape choice NAME=CHOICE for every size (see xmgn_tune_op_name)")
    args = ap.parse_args()
    build.build()
    ops = xmgn.tune_ops()
    for item in args.tune:
        name, choice = item.split("=")
        for rows in (1 << b for b in range(40)):
            xmgn.tune_set(ops[name][0], rows, int(choice))
    H = args.hidden
    xyz, nrm = synth.car_body(args.nodes, 2)
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, 202)
    params = synth.init_params(H, args.layers, 6, 4, 102)
    g = xmgn.build_knn(torch.from_numpy(xyz).cuda(), 6)
    tp = torch.from_numpy(params).cuda()
    ni, xz, tt = (torch.from_numpy(a).cuda() for a in (nin, xyz, tgt))
    m = xmgn.Model(H, args.layers, g, dtype="bf16")
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
