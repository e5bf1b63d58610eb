"""Shared helpers for the GPU parity tests (inputs come from the seeded
generators; expected values from the FP64 oracle)."""
import numpy as np

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case(kind, n, seed, jitter=0.0):
    if kind == "sphere":
        xyz, nrm = synth.sphere_cloud(n, seed)
    else:
        xyz, nrm = synth.car_body(n, seed, jitter=jitter)
    return xyz, synth.node_inputs(xyz, nrm)


def to_np_graph(g):
    """device graph dict -> numpy (row_ptr, col)"""
    return g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy()


def oracle_graph(xyz, k=6):
    nbr = O.knn(xyz, k)
    rp, col, cp, cperm = O.symmetrise(nbr, len(xyz))
    return nbr, rp, col, cperm
