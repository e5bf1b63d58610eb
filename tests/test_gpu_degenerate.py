"""Degenerate graphs through the model on the GPU, against the FP64 oracle:
a hub whose 299 incoming edges span three 128-edge tiles (aggregation
partials across several tile boundaries, a long receiver run in the
backward sums), isolated nodes (zero messages), and a graph without edges."""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu
H = 128


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


def _graph(n, undirected_pairs):
    """CSR (receiver-major, senders ascending) with the CSC permutation."""
    pairs = sorted({(i, j) for a, b in undirected_pairs for i, j in ((a, b), (b, a)) if i != j})
    recv = np.array([p[0] for p in pairs], np.int32)
    col = np.array([p[1] for p in pairs], np.int32)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, recv.astype(np.int64) + 1, 1)
    rp = np.cumsum(rp)
    csc = np.lexsort((recv, col)).astype(np.int32)  # by sender, then receiver
    dev = "cuda"
    E = len(pairs)
    g = dict(n=n, E=E, row_ptr=torch.from_numpy(rp).to(dev), col=torch.from_numpy(col).to(dev),
             recv=torch.from_numpy(recv).to(dev), csc_perm=torch.from_numpy(csc).to(dev))
    return g, rp, col


def _hub_graph(n=400):
    pairs = [(0, j) for j in range(1, 300)]               # hub: 299 edges each way
    pairs += [(j, j + 1) for j in range(300, n - 2)]       # a chain
    pairs += [(5, 6), (17, 301), (250, 320)]
    return _graph(n, pairs)                                # node n-1 stays isolated


def _run(X, g, xyz, nin, tgt, params, L, dtype):
    dev = "cuda"
    m = X.Model(H, L, g, dtype=dtype)
    m.validate()
    tp = torch.from_numpy(params).to(dev)
    ni, xz, tt = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (nin, xyz, tgt))
    y = torch.zeros((g["n"], 4), device=dev)
    loss = torch.zeros((), device=dev)
    m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
    dp = torch.zeros_like(tp)
    m.backward(tp, ni, xz, tt, dp)
    torch.cuda.synchronize()
    X.check_device()
    return y.cpu().numpy(), float(loss), dp.cpu().numpy()


@pytest.mark.parametrize("dtype,tol", [("bf16", 2e-2), ("fp32", 1e-4)])
@pytest.mark.parametrize("kind", ["hub", "no_edges"])
def test_degenerate_graphs_match_oracle(X, kind, dtype, tol):
    n = 400 if kind == "hub" else 50
    g, rp, col = _hub_graph(n) if kind == "hub" else _graph(n, [])
    rng = np.random.default_rng(71)
    xyz = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    nrm = xyz / np.linalg.norm(xyz, axis=1, keepdims=True)
    nin = synth.node_inputs(xyz, nrm.astype(np.float32))
    tgt = synth.fourier_targets(xyz, 72)
    L = 3
    params = synth.init_params(H, L, 6, 4, 73, perturb_ln=True)
    y, loss, dp = _run(X, g, xyz, nin, tgt, params, L, dtype)
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, 6, 4), rp, col, nin, xyz, tgt)
    ey, eg = rel_l2(y, yo), rel_l2(dp, go)
    print(f"{kind} {dtype}: E={g['E']} rel L2 y {ey:.3e} grad {eg:.3e} loss {loss:.6f} vs {lo:.6f}")
    assert ey <= tol and eg <= tol
    assert abs(loss - lo) <= tol * abs(lo)
    if kind == "hub":
        assert int(rp[1] - rp[0]) == 299 and rp[n] - rp[n - 1] == 0  # the run spans three tiles; n-1 isolated
