"""World-size-2 CPU test (gloo) of the multi-rank path: each rank runs its
share of the halo partitions (here with the FP64 oracle standing in for the
per-rank device computation), gradients are aggregated across ranks, and the
result equals the full-graph gradient (Sec. III-A "Gradient Aggregation")."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2411_17164_gb300.dist import allreduce_gradient, assign_partitions, rank_batch


def _neumaier(dst, src, comp=None):
    """Host stand-in for one compensated addition of xmgn_grad_accumulate
    (the device kernel is checked against exact sums on the GPU)."""
    if comp is None:
        dst += src
        return
    t = dst + src
    big = dst.abs() >= src.abs()
    comp += torch.where(big, (dst - t) + src, (src - t) + dst)
    dst.copy_(t)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    from oracle import xmgn_oracle as O
    from paper_2411_17164_gb300 import synth
    xyz, nrm = synth.car_body(600, 77)
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, 78)
    rp, col, _, _ = O.symmetrise(O.knn(xyz, 6), 600)
    part = O.rcb(xyz, 5)
    dims = (8, 2, 6, 4)
    params = synth.init_params(8, 2, 6, 4, 79, perturb_ln=True).astype(np.float64)
    parts = O.halo_partition(rp, col, part, 5, 2)
    return xyz, nin, tgt, rp, col, dims, params, parts


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from oracle import xmgn_oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    xyz, nin, tgt, rp, col, dims, params, parts = _case()
    mine = assign_partitions([len(p["col"]) for p in parts], world)[rank]
    # this rank's partitions, rebuilt from the renumbered part ids it would hand the library
    part = rank_batch(O.rcb(xyz, 5), mine)
    own = O.halo_partition(rp, col, part, len(mine), 2)
    for q, p in enumerate(mine):
        np.testing.assert_array_equal(own[q]["gid"], parts[p]["gid"])
    g = torch.zeros(len(params), dtype=torch.float64)
    for pt in own:
        _, gp = O.partitioned_step(params, dims, [pt], nin, xyz, tgt, len(xyz))[1:]
        g += torch.from_numpy(gp)
    allreduce_gradient(g, accumulate=_neumaier)
    out[rank] = g.numpy().copy()
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_to_full_graph_gradient():
    from oracle import xmgn_oracle as O
    xyz, nin, tgt, rp, col, dims, params, parts = _case()
    _, g_full, _ = O.loss_and_grad(params, dims, rp, col, nin, xyz, tgt)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        g0, g1 = out[0], out[1]
    np.testing.assert_array_equal(g0, g1)                    # identical on every rank
    np.testing.assert_allclose(g0, g_full, rtol=1e-9, atol=1e-12 * np.abs(g_full).max())


def test_rank_batch_renumbers_own_parts():
    part = np.array([3, 0, -1, 2, 3, 1, 0])
    np.testing.assert_array_equal(rank_batch(part, [0, 3]), [1, 0, -1, -1, 1, -1, 0])
    np.testing.assert_array_equal(rank_batch(part, []), [-1] * 7)


def test_compensated_rank_sum_beats_plain_sum():
    """The rank-order compensated sum (host stand-in of the library step)
    recovers the exact sum of many float32 gradients far better than plain
    float32 addition."""
    rng = np.random.default_rng(3)
    parts = [torch.from_numpy((rng.standard_normal(4096) * 10.0 ** rng.integers(-3, 4, 4096)).astype(np.float32))
             for _ in range(16)]
    exact = sum(p.double() for p in parts)
    acc, comp, plain = parts[0].clone(), torch.zeros(4096), parts[0].clone()
    for p in parts[1:]:
        _neumaier(acc, p, comp)
        plain += p
    e_c = float((acc.double() + comp.double() - exact).norm())
    e_p = float((plain.double() - exact).norm())
    assert e_c <= 1e-3 * e_p


def test_assign_partitions_balanced_and_deterministic():
    counts = [50, 10, 40, 30, 30, 20, 5]
    a = assign_partitions(counts, 3)
    assert sorted(sum(a, [])) == list(range(7))
    loads = [sum(counts[p] for p in r) for r in a]
    assert max(loads) - min(loads) <= max(counts)
    assert a == assign_partitions(counts, 3)
    assert assign_partitions(counts, 1) == [list(range(7))]


def _worker_dropout(rank, world, port, out):
    """Rank 1 leaves before the gradient exchange; rank 0 must get an error
    from the collective within the process-group timeout instead of hanging."""
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        out[rank] = "left"
        return  # leaves between steps, with nothing in flight
    g = torch.ones(16, dtype=torch.float64)
    try:
        allreduce_gradient(g, accumulate=_neumaier)
        out[rank] = "no error"
    except Exception as e:  # the peer is gone: the collective fails
        out[rank] = "error: " + type(e).__name__


def test_rank_that_leaves_surfaces_as_an_error():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker_dropout, args=(2, _free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        assert out[1] == "left"
        assert out[0].startswith("error"), out[0]
