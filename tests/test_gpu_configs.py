"""BF16 parity at the sizes of the partitioned and batched workloads.

Outputs of sampled inner nodes and the gradient of a loss restricted to them
are compared with the oracle run on the sampled nodes' exact L-hop
neighbourhoods in the full graph: with halo depth L the partitioned (Sec.
III-A) result of an inner node equals the full-graph result, and L-layer
message passing only reaches L hops (Sec. II-D)."""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu
TOL = 2e-2
H, L = 128, 15


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


def _sampled_batch_parity(X, xyz, nin, tgt, params, g, b, S, n_norm):
    dev = "cuda"
    gid = b["gid"].cpu().numpy()
    hop = b["hop"].cpu().numpy()
    sel = (hop == 0) & np.isin(gid, S)
    assert sel.sum() == len(S)  # every sampled node is inner in exactly one part
    bb = dict(b)
    bb["hop"] = torch.from_numpy(np.where(sel, 0, 1).astype(np.uint8)).to(dev)  # loss on the sampled nodes only
    m = X.Model(H, L, bb, dtype="bf16", n_norm=n_norm)
    tp = torch.from_numpy(params).to(dev)
    ni, xz, tt = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (nin, xyz, tgt))
    y = torch.zeros((len(xyz), 4), device=dev)
    loss = torch.zeros((), device=dev)
    m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
    dp = torch.zeros_like(tp)
    m.backward(tp, ni, xz, tt, dp)
    torch.cuda.synchronize()
    X.check_device()
    y = y.cpu().numpy()
    dp = dp.cpu().numpy()
    rp, col = g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy()
    dist = O.bfs_hops(rp, col, S, L)
    sub = np.concatenate([S, np.setdiff1d(np.nonzero(dist >= 0)[0], S)])
    lrp, lcol = O.induced_subgraph(rp, col, sub)
    mask = np.zeros(len(sub))
    mask[:len(S)] = 1
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, 6, 4), lrp, lcol, nin[sub], xyz[sub],
                                 tgt[sub], mask, n_norm)
    ey, eg = rel_l2(y[S], yo[:len(S)]), rel_l2(dp, go)
    print(f"batch {b['n']} nodes {b['E']} edges; oracle on {len(sub)} nodes: rel L2 y {ey:.3e} grad {eg:.3e} "
          f"loss {float(loss):.6e} vs {lo:.6e}")
    assert ey <= TOL and eg <= TOL
    assert abs(float(loss) - lo) <= TOL * abs(lo)


def test_partitioned_2m_rcb16_sampled_parity(X):
    """2M-point body, 16 RCB partitions with 15-hop halos, BF16, gradients
    summed over partitions."""
    N = 2_000_000
    xyz, nrm = synth.car_body(N, 3)
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, 303)
    params = synth.init_params(H, L, 6, 4, 103, perturb_ln=True)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), 16, L)
    assert b["n"] > N  # halos duplicate boundary nodes
    S = np.sort(np.random.default_rng(33).choice(N, 8, replace=False))
    _sampled_batch_parity(X, xyz, nin, tgt, params, g, b, S, N)


def test_batched_64_regions_four_bodies_sampled_parity(X):
    """64 breadth-first regions with log-uniform inner sizes in [5k, 80k] on
    four 1M-point bodies (primitive sizes jittered by up to 10 %), 15-hop
    halos, one batched launch per kernel; nodes outside every region appear
    only as halo."""
    parts = []
    for b_, (cx, cy) in enumerate([(-2.4, -1.1), (2.4, -1.1), (-2.4, 1.1), (2.4, 1.1)]):
        p, nr = synth.car_body(1_000_000, 51 + b_, jitter=0.1)
        parts.append((p + np.array([cx, cy, 0.0], np.float32), nr))
    xyz = np.concatenate([p for p, _ in parts])
    nin = synth.node_inputs(xyz, np.concatenate([nr for _, nr in parts]))
    tgt = synth.fourier_targets(xyz, 505)
    params = synth.init_params(H, L, 6, 4, 105, perturb_ln=True)
    N = len(xyz)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    rp, col = g["row_ptr"].cpu().numpy(), g["col"].cpu().numpy()
    body = np.arange(N) // 1_000_000
    assert np.all(body[np.repeat(np.arange(N), np.diff(rp))] == body[col])  # bodies are separate components
    region = synth.bfs_regions(rp, col, 64, 5e3, 8e4, 505)
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), 64, L, part_in=torch.from_numpy(region).cuda())
    n_inner = int((region >= 0).sum())
    assert sum(b["inner_cnt"]) == n_inner
    S = np.sort(np.random.default_rng(55).choice(np.nonzero(region >= 0)[0], 8, replace=False))
    _sampled_batch_parity(X, xyz, nin, tgt, params, g, b, S, n_inner)


def test_multiscale_3_levels_rcb8_sampled_parity(X):
    """Three nested levels of 50k, 250k and 1.25M points (Sec. III-C): kNN
    within each level plus 3 links from every finer point to the coarser
    level; 8 RCB partitions with 15-hop halos.  Sampled rows of the graph are
    checked bit-exactly against the oracle's kNN, then the model."""
    sizes = [50_000, 250_000, 1_250_000]
    xyz, nrm = synth.nested_levels(sizes, 4)
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, 404)
    params = synth.init_params(H, L, 6, 4, 104, perturb_ln=True)
    N = len(xyz)
    g = X.build_multiscale(torch.from_numpy(xyz).cuda(), sizes, want_nbr=True)
    nbr = g["nbr"].cpu().numpy()
    rng = np.random.default_rng(44)
    for lv, n_l in enumerate(sizes):
        rows = rng.choice(n_l, 3, replace=False)
        np.testing.assert_array_equal(nbr[rows, 6 * lv:6 * lv + 6], O.knn(xyz[:n_l], 6, rows=rows))
        if lv:
            rows = rng.integers(sizes[lv - 1], n_l, 3)
            np.testing.assert_array_equal(nbr[rows, 18:], O.knn_among(xyz, rows, sizes[lv - 1], 3))
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), 8, L)
    # coarse links make 15-hop neighbourhoods large (~16k nodes each): 3 samples
    S = np.sort(rng.choice(N, 3, replace=False))
    _sampled_batch_parity(X, xyz, nin, tgt, params, g, b, S, N)
