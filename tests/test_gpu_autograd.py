"""The autograd wrapper (XMGNLoss, a torch.autograd.Function around
xmgn_forward / xmgn_backward) checked on the GPU:

* its FP32 gradient against the FP64 oracle's hand-written gradient;
* central finite differences of the GPU's own FP32 loss, along random and
  gradient-mixed directions and for one parameter of every block (weights,
  biases, LayerNorm gain and shift of every MLP);
* the BF16 directional derivative against the oracle's;
* a second forward on the same model before backward is refused.

Differentiated: the message-passing model of Sec. II-B..II-D (eqs. 1-4) and
its MSE loss (Sec. IV-C), with the per-layer activation recomputation of the
backward pass.

Finite-difference tolerance (FP32).  Each derivative is the Richardson
combination (4 D(s/2) - D(s)) / 3 of two central differences, whose
truncation error is O(s^4): below 3e-5 relative on this model for the steps
used (measured on the FP64 oracle).  What remains is the FP32 rounding of the
loss (about 1e-6 of its value, uncorrelated between the perturbed points),
divided by the step: about 1e-3 of the smallest derivative checked, so the
bound is 5e-3 relative.  The comparator is the GPU gradient dotted with the
perturbation actually applied (the perturbed parameters are rounded to FP32).
"""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import case, rel_l2

pytestmark = pytest.mark.gpu
H, L = 128, 3
FD_TOL = 5e-3


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


@pytest.fixture(scope="module")
def C(X):
    """A 1,500-point car-body graph, H = 128, L = 3, LayerNorm gains and
    shifts perturbed away from 1 and 0; the oracle's loss and gradient."""
    xyz, nin = case("body", 1500, 81)
    tgt = synth.fourier_targets(xyz, 82)
    params = synth.init_params(H, L, 6, 4, 83, perturb_ln=True)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    rp, col, _, _ = O.symmetrise(O.knn(xyz, 6), len(xyz))
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    lo, go, _ = O.loss_and_grad(params.astype(np.float64), (H, L, 6, 4), rp, col, nin, xyz, tgt)
    dev = "cuda"
    t = dict(ni=torch.from_numpy(nin).to(dev), xz=torch.from_numpy(xyz).to(dev), tt=torch.from_numpy(tgt).to(dev))
    return dict(g=g, params=params, lo=lo, go=go, **t)


def _grad(X, C, dtype, scale=1.0):
    """Parameter gradient of scale * loss through torch.autograd."""
    m = X.Model(H, L, C["g"], dtype=dtype)
    tp = torch.from_numpy(C["params"]).cuda().requires_grad_(True)
    loss = X.XMGNLoss.apply(tp, m, C["ni"], C["xz"], C["tt"])
    (scale * loss).backward()
    torch.cuda.synchronize()
    X.check_device()
    return float(loss), tp.grad.double().cpu().numpy()


def test_autograd_fp32_gradient_matches_oracle(X, C):
    loss, g = _grad(X, C, "fp32")
    e = rel_l2(g, C["go"])
    print(f"XMGNLoss fp32: loss {loss:.7f} (oracle {C['lo']:.7f}), gradient rel L2 {e:.3e}")
    assert abs(loss - C["lo"]) <= 1e-4 * abs(C["lo"])
    assert e <= 1e-4
    # the incoming gradient scales the result (chain rule through the Function)
    _, g3 = _grad(X, C, "fp32", scale=-3.0)
    np.testing.assert_allclose(g3, -3.0 * g, rtol=1e-6, atol=0)


def _loss_at(X, m, C, theta32):
    out = torch.zeros((), device="cuda")
    m.forward(torch.from_numpy(theta32).cuda(), C["ni"], C["xz"], targets=C["tt"], loss=out)
    torch.cuda.synchronize()
    return float(out)


def _richardson(X, m, C, g, v, s):
    """(4 D(s/2) - D(s)) / 3 of the GPU loss along v, and the same
    combination of g . (theta+ - theta-) / (2 step) with the rounded steps."""
    th = C["params"].astype(np.float64)
    fd, an = [], []
    for step in (s, s / 2):
        tp = (th + step * v).astype(np.float32)
        tm = (th - step * v).astype(np.float32)
        fd.append((_loss_at(X, m, C, tp) - _loss_at(X, m, C, tm)) / (2 * step))
        an.append(float(g @ (tp.astype(np.float64) - tm.astype(np.float64))) / (2 * step))
    return (4 * fd[1] - fd[0]) / 3, (4 * an[1] - an[0]) / 3


def test_fp32_central_differences_of_gpu_loss(X, C):
    _, g = _grad(X, C, "fp32")
    m = X.Model(H, L, C["g"], dtype="fp32")
    n = len(C["params"])
    rng = np.random.default_rng(91)
    worst = 0.0
    # 4 random unit directions (derivatives ~1e-2) and 4 directions half
    # along the oracle's gradient (derivatives ~15)
    gu = C["go"] / np.linalg.norm(C["go"])
    dirs = []
    for k in range(4):
        z = rng.standard_normal(n)
        dirs.append((z / np.linalg.norm(z), 0.5))
    for k in range(4):
        z = rng.standard_normal(n)
        dirs.append(((gu + z / np.linalg.norm(z)) / np.sqrt(2.0), 2e-3))
    for v, s in dirs:
        fd, an = _richardson(X, m, C, g, v, s)
        err = abs(fd - an) / abs(an)
        worst = max(worst, err)
        assert err <= FD_TOL, (fd, an, err)
    # one parameter per block: the entry with the largest oracle derivative
    off = 0
    blocks = 0
    for name, shape in O.param_shapes(H, L, 6, 4):
        sz = int(np.prod(shape))
        i = off + int(np.argmax(np.abs(C["go"][off:off + sz])))
        v = np.zeros(n)
        v[i] = 1.0
        fd, an = _richardson(X, m, C, g, v, 0.05)
        err = abs(fd - an) / abs(an)
        worst = max(worst, err)
        assert err <= FD_TOL, (name, fd, an, err)
        off += sz
        blocks += 1
    assert blocks == len(O.param_shapes(H, L, 6, 4)) >= 16
    print(f"fp32 central differences: {len(dirs)} directions, {blocks} single parameters, worst rel err {worst:.2e}")


def test_bf16_directional_derivatives_match_oracle(X, C):
    _, g = _grad(X, C, "bf16")
    go = C["go"]
    n = len(go)
    rng = np.random.default_rng(92)
    gu = go / np.linalg.norm(go)
    errs = []
    for k in range(6):
        z = rng.standard_normal(n)
        v = (gu + z / np.linalg.norm(z)) / np.sqrt(2.0)
        d_gpu, d_or = float(g @ v), float(go @ v)
        errs.append(abs(d_gpu - d_or) / abs(d_or))
    print("bf16 directional derivative rel errors", ", ".join(f"{e:.2e}" for e in errs))
    assert max(errs) <= 2e-2
    assert rel_l2(g, go) <= 2e-2


def test_backward_after_a_second_forward_is_refused(X, C):
    m = X.Model(H, L, C["g"], dtype="fp32")
    tp = torch.from_numpy(C["params"]).cuda().requires_grad_(True)
    loss = X.XMGNLoss.apply(tp, m, C["ni"], C["xz"], C["tt"])
    m.forward(tp.detach() * 0.5, C["ni"], C["xz"], targets=C["tt"], loss=torch.zeros((), device="cuda"))
    with pytest.raises(RuntimeError, match="another forward"):
        loss.backward()
