"""FP32 plain path vs the FP64 oracle (relative L2 <= 1e-4 on outputs and
gradients), on one full graph and on halo-partitioned batches."""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import assert_same_graph, case, oracle_graph, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


def _run(X, xyz, nin, H, L, seed, dtype="fp32", P=None, hops=None, tgt_seed=7, perturb=True):
    dev = "cuda"
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    _, rp, col, cperm = oracle_graph(xyz)
    assert_same_graph(g, rp, col, cperm)
    g["orp"], g["ocol"] = rp, col
    graph = g if P is None else X.partition_halo(g, torch.from_numpy(xyz).cuda(), P, hops)
    params = synth.init_params(H, L, 6, 4, seed, perturb_ln=perturb)
    tgt = synth.fourier_targets(xyz, tgt_seed)
    m = X.Model(H, L, graph, dtype=dtype, n_norm=len(xyz))
    tp = torch.from_numpy(params).to(dev)
    y = torch.zeros((len(xyz), 4), device=dev)
    loss = torch.zeros((), device=dev)
    ni, xz, tt = (torch.from_numpy(a).to(dev) for a in (nin, xyz, tgt))
    m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
    dp = torch.zeros_like(tp)
    m.backward(tp, ni, xz, tt, dp)
    torch.cuda.synchronize()
    X.check_device()
    return g, y.cpu().numpy(), float(loss), dp.cpu().numpy(), params, tgt


def test_forward_c1_sphere_2000(X):
    """Plain forward, 2000-node sphere, H=64, L=4 (the small full-graph case)."""
    xyz, nin = case("sphere", 2000, 1)
    g, y, loss, _, params, tgt = _run(X, xyz, nin, 64, 4, 101, perturb=False)
    rp, col = g["orp"], g["ocol"]
    yo = O.forward(params.astype(np.float64), (64, 4, 6, 4), rp, col, nin, xyz)
    assert rel_l2(y, yo) <= TOL, rel_l2(y, yo)
    lo, _ = O.mse_loss(yo, tgt, np.ones(2000), 2000)
    assert abs(loss - lo) <= TOL * abs(lo)


def test_forward_backward_body(X):
    xyz, nin = case("body", 3000, 3)
    g, y, loss, dp, params, tgt = _run(X, xyz, nin, 64, 3, 5)
    rp, col = g["orp"], g["ocol"]
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (64, 3, 6, 4), rp, col, nin, xyz, tgt)
    assert rel_l2(y, yo) <= TOL
    assert abs(loss - lo) <= TOL * abs(lo)
    assert rel_l2(dp, go) <= TOL, rel_l2(dp, go)


def test_partitioned_batch_equals_full_graph_oracle(X):
    """Sec. III-A: halo depth = L and gradient aggregation reproduce the full graph."""
    xyz, nin = case("body", 2500, 8)
    H, L = 32, 3
    g, y, loss, dp, params, tgt = _run(X, xyz, nin, H, L, 9, P=4, hops=L)
    rp, col = g["orp"], g["ocol"]
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, 6, 4), rp, col, nin, xyz, tgt)
    assert rel_l2(y, yo) <= TOL
    assert abs(loss - lo) <= TOL * abs(lo)
    assert rel_l2(dp, go) <= TOL, rel_l2(dp, go)


def test_deterministic_repeat(X):
    xyz, nin = case("body", 1500, 4)
    a = _run(X, xyz, nin, 64, 2, 3)
    b = _run(X, xyz, nin, 64, 2, 3)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[3], b[3])
