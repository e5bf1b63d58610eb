"""BF16 tensor-core path vs the FP64 oracle: relative L2 <= 2e-2 on outputs
and parameter gradients (bf16 operands, fp32 accumulation)."""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import assert_same_graph, case, oracle_graph, rel_l2

pytestmark = pytest.mark.gpu
TOL = 2e-2
H = 128


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


def _gpu(X, graph, xyz, nin, tgt, params, L, dtype="bf16", n_norm=None):
    dev = "cuda"
    m = X.Model(H, L, graph, dtype=dtype, n_norm=n_norm if n_norm is not None else len(xyz))
    tp = torch.from_numpy(params).to(dev)
    ni, xz, tt = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (nin, xyz, tgt))
    y = torch.zeros((len(xyz), 4), device=dev)
    loss = torch.zeros((), device=dev)
    m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
    dp = torch.zeros_like(tp)
    m.backward(tp, ni, xz, tt, dp)
    torch.cuda.synchronize()
    X.check_device()
    return y.cpu().numpy(), float(loss), dp.cpu().numpy()


def _setup(X, kind, n, seed, L):
    """Seeded case; the library's graph is checked against the oracle's, whose
    arrays (rp, col) then feed the oracle."""
    xyz, nin = case(kind, n, seed)
    tgt = synth.fourier_targets(xyz, seed + 1)
    params = synth.init_params(H, L, 6, 4, seed + 2, perturb_ln=True)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    _, rp, col, cperm = oracle_graph(xyz)
    assert_same_graph(g, rp, col, cperm)
    g["orp"], g["ocol"] = rp, col
    return xyz, nin, tgt, params, g


@pytest.mark.parametrize("kind,n,L", [("sphere", 700, 2), ("body", 3000, 3)])
def test_bf16_forward_backward_vs_oracle(X, kind, n, L):
    xyz, nin, tgt, params, g = _setup(X, kind, n, 11, L)
    y, loss, dp = _gpu(X, g, xyz, nin, tgt, params, L)
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, 6, 4), g["orp"], g["ocol"], nin, xyz, tgt)
    ey, eg = rel_l2(y, yo), rel_l2(dp, go)
    print(f"bf16 {kind} n={n} L={L}: rel L2 y {ey:.3e} grad {eg:.3e} loss {loss:.6f} vs {lo:.6f}")
    assert ey <= TOL and eg <= TOL
    assert abs(loss - lo) <= TOL * abs(lo)
    # every parameter block gets a gradient close to the oracle's
    off = 0
    for name, shape in O.param_shapes(H, L, 6, 4):
        sz = int(np.prod(shape))
        e = rel_l2(dp[off:off + sz], go[off:off + sz])
        assert e <= 0.1, (name, e)
        off += sz


def test_bf16_partitioned_batch_matches_full_graph_oracle(X):
    L = 3
    xyz, nin, tgt, params, g = _setup(X, "body", 2500, 21, L)
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), 4, L)
    y, loss, dp = _gpu(X, b, xyz, nin, tgt, params, L)
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, 6, 4), g["orp"], g["ocol"], nin, xyz, tgt)
    assert rel_l2(y, yo) <= TOL and rel_l2(dp, go) <= TOL
    assert abs(loss - lo) <= TOL * abs(lo)


def test_bf16_deterministic(X):
    L = 2
    xyz, nin, tgt, params, g = _setup(X, "body", 2000, 31, L)
    a = _gpu(X, g, xyz, nin, tgt, params, L)
    b = _gpu(X, g, xyz, nin, tgt, params, L)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[2], b[2])


def test_bf16_close_to_fp32_path(X):
    L = 2
    xyz, nin, tgt, params, g = _setup(X, "body", 1500, 41, L)
    yb, lb, gb = _gpu(X, g, xyz, nin, tgt, params, L, "bf16")
    yf, lf, gf = _gpu(X, g, xyz, nin, tgt, params, L, "fp32")
    assert rel_l2(yb, yf) <= TOL and rel_l2(gb, gf) <= TOL


@pytest.mark.parametrize("dtype,tol", [("bf16", TOL), ("fp32", 1e-4)])
def test_fourier_inputs_fused_in_node_encoder(X, dtype, tol):
    """24 node-encoder inputs (Sec. IV-D): xyz, normal and 18 Fourier features
    computed by the encoder from the coordinates; the oracle gets them
    precomputed."""
    L = 2
    xyz, nin = case("body", 2500, 61)
    tgt = synth.fourier_targets(xyz, 62)
    params = synth.init_params(H, L, 24, 4, 63, perturb_ln=True)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    _, rp, col, cperm = oracle_graph(xyz)
    assert_same_graph(g, rp, col, cperm)
    m = X.Model(H, L, g, dtype=dtype, fourier=3)
    tp = torch.from_numpy(params).cuda()
    ni, xz, tt = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (nin, xyz, tgt))
    y = torch.zeros((len(xyz), 4), device="cuda")
    loss = torch.zeros((), device="cuda")
    m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
    dp = torch.zeros_like(tp)
    m.backward(tp, ni, xz, tt, dp)
    torch.cuda.synchronize()
    X.check_device()
    x24 = np.concatenate([nin.astype(np.float64), O.fourier_features(xyz, 3)], axis=1)
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, 24, 4), rp, col, x24, xyz, tgt)
    ey, eg = rel_l2(y.cpu().numpy(), yo), rel_l2(dp.cpu().numpy(), go)
    print(f"fourier {dtype}: rel L2 y {ey:.3e} grad {eg:.3e}")
    assert ey <= tol and eg <= tol


def test_checkpoint_offload_bit_identical_and_capturable(X):
    """Edge-state checkpoints in page-locked host memory (Sec. IV-E):
    outputs and gradient within the BF16 tolerance of the FP64 oracle, the
    same bits as the device-resident run, a smaller device checkpoint, and a
    CUDA graph of forward + backward replays to the same result."""
    L = 4
    xyz, nin, tgt, params, g = _setup(X, "body", 3000, 71, L)
    dev = "cuda"
    tp = torch.from_numpy(params).to(dev)
    ni, xz, tt = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (nin, xyz, tgt))

    def run(m):
        y = torch.zeros((len(xyz), 4), device=dev)
        loss = torch.zeros((), device=dev)
        dp = torch.zeros_like(tp)
        m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
        m.backward(tp, ni, xz, tt, dp)
        torch.cuda.synchronize()
        X.check_device()
        return y.cpu().numpy(), float(loss), dp.cpu().numpy()

    ref = run(X.Model(H, L, g, dtype="bf16"))
    mo = X.Model(H, L, g, dtype="bf16", offload=True)
    got = run(mo)
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (H, L, 6, 4), g["orp"], g["ocol"], nin, xyz, tgt)
    ey, eg = rel_l2(got[0], yo), rel_l2(got[2], go)
    print(f"offload bf16 vs oracle: rel L2 y {ey:.3e} grad {eg:.3e} loss {got[1]:.6f} vs {lo:.6f}")
    assert ey <= TOL and eg <= TOL and abs(got[1] - lo) <= TOL * abs(lo)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[2], ref[2])
    assert mo.ckpt.numel() < X.Model(H, L, g, dtype="bf16").ckpt.numel()
    assert mo.host_ckpt.numel() >= L * g["E"] * H * 2
    # the offloaded step as one CUDA graph
    y = torch.zeros((len(xyz), 4), device=dev)
    loss = torch.zeros((), device=dev)
    dp = torch.zeros_like(tp)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        mo.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
        mo.backward(tp, ni, xz, tt, dp)
    for _ in range(2):
        dp.zero_()
        graph.replay()
    torch.cuda.synchronize()
    X.check_device()
    np.testing.assert_array_equal(dp.cpu().numpy(), ref[2])
