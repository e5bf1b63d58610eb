"""The partitioned and batched workloads at their full sizes (2M-point body
in 16 RCB parts; three nested levels of 50k / 250k / 1.25M points in 8 RCB
parts; 64 breadth-first regions on four 1M-point bodies; all with 15-hop
halos, H = 128, L = 15).

Integer work is compared bit for bit with the oracle at these sizes: the
whole kNN (or multi-scale) graph, every RCB part id, and the halo sets (global
ids, hops, inner counts, local CSR) of several parts or regions.

BF16 model parity: outputs of sampled inner nodes and the gradient of a loss
restricted to them, against the oracle run on the sampled nodes' exact L-hop
neighbourhoods in the full graph: with halo depth L the partitioned (Sec.
III-A) result of an inner node equals the full-graph result, and L-layer
message passing only reaches L hops (Sec. II-D).  Two independent draws per
workload, each within the tolerance."""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import assert_same_graph, halo_part_exact, sampled_parity, tree_graph

pytestmark = pytest.mark.gpu
TOL = 2e-2
H, L = 128, 15


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


def _parity_draws(X, b, rp, col, xyz, nin, tgt, params, pool, n_norm, draws, per_draw, seed):
    rng = np.random.default_rng(seed)
    for d in range(draws):
        S = np.sort(rng.choice(pool, per_draw, replace=False))
        ey, eg, loss, lo, ns = sampled_parity(X, b, rp, col, xyz, nin, tgt, params, S, n_norm, H, L)
        print(f"batch {b['n']} nodes {b['E']} edges, draw {d}: oracle on {ns} nodes; rel L2 y {ey:.3e} "
              f"grad {eg:.3e} loss rel {abs(loss - lo) / abs(lo):.2e}")
        assert ey <= TOL and eg <= TOL
        assert abs(loss - lo) <= TOL * abs(lo)


# --------------------------------------------------------------- 2M points, 16 RCB parts
@pytest.fixture(scope="module")
def C3(X):
    N = 2_000_000
    xyz, nrm = synth.car_body(N, 3)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    rp, col, cperm = tree_graph(xyz)
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), 16, L)
    return dict(N=N, xyz=xyz, nin=synth.node_inputs(xyz, nrm), g=g, rp=rp, col=col, cperm=cperm, b=b)


def test_partitioned_2m_graph_rcb_and_halos_exact(C3):
    assert_same_graph(C3["g"], C3["rp"], C3["col"], C3["cperm"])
    part = O.rcb(C3["xyz"], 16)
    np.testing.assert_array_equal(C3["b"]["part"].cpu().numpy(), part)
    for p in (0, 7, 15):
        n = halo_part_exact(C3["b"], p, C3["rp"], C3["col"], part, L)
        assert n > C3["b"]["inner_cnt"][p]  # a 15-hop halo around every part
    assert C3["b"]["n"] > C3["N"]


def test_partitioned_2m_rcb16_sampled_parity(X, C3):
    """Gradients summed over the 16 partitions of one batch."""
    tgt = synth.fourier_targets(C3["xyz"], 303)
    params = synth.init_params(H, L, 6, 4, 103, perturb_ln=True)
    _parity_draws(X, C3["b"], C3["rp"], C3["col"], C3["xyz"], C3["nin"], tgt, params, C3["N"], C3["N"], 2, 8, 33)


# --------------------------------------------------------------- 64 regions on four bodies
@pytest.fixture(scope="module")
def C5(X):
    parts = []
    for b_, (cx, cy) in enumerate([(-2.4, -1.1), (2.4, -1.1), (-2.4, 1.1), (2.4, 1.1)]):
        p, nr = synth.car_body(1_000_000, 51 + b_, jitter=0.1)
        parts.append((p + np.array([cx, cy, 0.0], np.float32), nr))
    xyz = np.concatenate([p for p, _ in parts])
    nin = synth.node_inputs(xyz, np.concatenate([nr for _, nr in parts]))
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    rp, col, cperm = tree_graph(xyz)
    region = synth.bfs_regions(rp, col, 64, 5e3, 8e4, 505)
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), 64, L, part_in=torch.from_numpy(region).cuda())
    return dict(xyz=xyz, nin=nin, g=g, rp=rp, col=col, cperm=cperm, region=region, b=b)


def test_batched_64_regions_graph_and_halos_exact(C5):
    assert_same_graph(C5["g"], C5["rp"], C5["col"], C5["cperm"])
    N = len(C5["xyz"])
    body = np.arange(N) // 1_000_000
    assert np.all(body[O.edge_receivers(C5["rp"])] == body[C5["col"]])  # bodies are separate components
    region = C5["region"]
    assert sum(C5["b"]["inner_cnt"]) == int((region >= 0).sum())
    sizes = np.bincount(region[region >= 0], minlength=64)
    for p in (int(np.argmin(sizes)), int(np.argmax(sizes))):  # the smallest and the largest region
        halo_part_exact(C5["b"], p, C5["rp"], C5["col"], region, L)


def test_batched_64_regions_four_bodies_sampled_parity(X, C5):
    """One batched launch per kernel over all 64 regions; nodes outside every
    region appear only as halo."""
    tgt = synth.fourier_targets(C5["xyz"], 505)
    params = synth.init_params(H, L, 6, 4, 105, perturb_ln=True)
    region = C5["region"]
    n_inner = int((region >= 0).sum())
    _parity_draws(X, C5["b"], C5["rp"], C5["col"], C5["xyz"], C5["nin"], tgt, params,
                  np.nonzero(region >= 0)[0], n_inner, 2, 8, 55)


# --------------------------------------------------------------- multi-scale, 8 RCB parts
def test_multiscale_3_levels_rcb8_exact_and_sampled_parity(X):
    """Three nested levels of 50k, 250k and 1.25M points (Sec. III-C): kNN
    within each level plus 3 links from every finer point to the coarser
    level, checked whole against the oracle; 8 RCB partitions with 15-hop
    halos (part ids and one part's halo exact), then the model."""
    sizes = [50_000, 250_000, 1_250_000]
    xyz, nrm = synth.nested_levels(sizes, 4)
    nin = synth.node_inputs(xyz, nrm)
    tgt = synth.fourier_targets(xyz, 404)
    params = synth.init_params(H, L, 6, 4, 104, perturb_ln=True)
    N = len(xyz)
    g = X.build_multiscale(torch.from_numpy(xyz).cuda(), sizes)
    rp, col, _, cperm = O.multiscale_graph(xyz, sizes, tree=True)
    assert_same_graph(g, rp, col, cperm)
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), 8, L)
    part = O.rcb(xyz, 8)
    np.testing.assert_array_equal(b["part"].cpu().numpy(), part)
    halo_part_exact(b, 3, rp, col, part, L)
    # coarse links make 15-hop neighbourhoods large (~16k nodes each): 3 samples per draw
    _parity_draws(X, b, rp, col, xyz, nin, tgt, params, N, N, 2, 3, 44)
