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


def tree_graph(xyz, k=6):
    """The oracle's symmetrised kNN graph of a cloud too large for the
    brute-force search (exact kNN through knn_tree): row_ptr, col, csc_perm."""
    rp, col, _, cperm = O.symmetrise(O.knn_tree(xyz, k), len(xyz))
    return rp, col, cperm


def assert_same_graph(g, rp, col, cperm=None):
    """A device graph from the library equals the oracle's, bit for bit; the
    oracle's arrays are then the ones every further oracle call receives."""
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    np.testing.assert_array_equal(g["recv"].cpu().numpy(), O.edge_receivers(rp))
    if cperm is not None:
        np.testing.assert_array_equal(g["csc_perm"].cpu().numpy(), cperm)


def sampled_parity(X, model_graph, rp, col, xyz, nin, tgt, params, S, n_norm, H, L, dtype="bf16"):
    """Outputs of the sampled nodes S and the gradient of a loss restricted to
    them, from the library run on ``model_graph`` (the full graph, or a batch
    of halo partitions in which each node of S is inner in exactly one part),
    against the oracle run on exactly the L-hop neighbourhood of S in the full
    graph (rp, col): by the locality of L-layer message passing (Sec. II-D)
    and halo depth L (Sec. III-A) the two are the same quantity.
    Returns (rel L2 of y[S], rel L2 of the gradient, loss, oracle loss,
    neighbourhood size)."""
    import torch
    dev = "cuda"
    gg = dict(model_graph)
    if "gid" in model_graph:
        gid = model_graph["gid"].cpu().numpy()
        sel = (model_graph["hop"].cpu().numpy() == 0) & np.isin(gid, S)
        assert sel.sum() == len(S)  # every sampled node is inner in exactly one part
        gg["hop"] = torch.from_numpy(np.where(sel, 0, 1).astype(np.uint8)).to(dev)
    else:
        hop = np.ones(len(xyz), np.uint8)
        hop[S] = 0
        gg["hop"] = torch.from_numpy(hop).to(dev)
    m = X.Model(H, L, gg, dtype=dtype, n_norm=n_norm)
    tp = torch.from_numpy(params).to(dev)
    ni, xz, tt = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (nin, xyz, tgt))
    y = torch.zeros((len(xyz), 4), device=dev)
    loss = torch.zeros((), device=dev)
    m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
    dp = torch.zeros_like(tp)
    m.backward(tp, ni, xz, tt, dp)
    torch.cuda.synchronize()
    X.check_device()
    del m
    dist = O.bfs_hops(rp, col, S, L)
    sub = np.concatenate([S, np.setdiff1d(np.nonzero(dist >= 0)[0], S)])
    lrp, lcol = O.induced_subgraph(rp, col, sub)
    mask = np.zeros(len(sub))
    mask[:len(S)] = 1
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, nin.shape[1], 4), lrp, lcol, nin[sub],
                                 xyz[sub], tgt[sub], mask, n_norm)
    return (rel_l2(y.cpu().numpy()[S], yo[:len(S)]), rel_l2(dp.cpu().numpy(), go), float(loss), lo, len(sub))


def halo_part_exact(b, p, rp, col, part, hops):
    """Part p of a library batch (xmgn_partition_halo) against the oracle's
    halo partition of that part: global ids, hops, inner count, local CSR."""
    pt = O.halo_partition(rp, col, np.where(np.asarray(part) == p, 0, -1), 1, hops)[0]
    n0, n1 = b["node_ptr"][p], b["node_ptr"][p + 1]
    e0, e1 = b["edge_ptr"][p], b["edge_ptr"][p + 1]
    np.testing.assert_array_equal(b["gid"][n0:n1].cpu().numpy(), pt["gid"])
    np.testing.assert_array_equal(b["hop"][n0:n1].cpu().numpy(), pt["hop"])
    assert b["inner_cnt"][p] == pt["n_inner"]
    np.testing.assert_array_equal(b["row_ptr"][n0:n1 + 1].cpu().numpy() - e0, pt["row_ptr"])
    np.testing.assert_array_equal(b["col"][e0:e1].cpu().numpy() - n0, pt["col"])
    return len(pt["gid"])
