"""GPU test of xmgn_mse_loss_static, the loss entry point that allocates
nothing (for callers that may not allocate device memory, e.g. inside a
framework whose allocator owns the device).  Its result must match the loss
that xmgn_forward computes with caller workspace, on two calls in a row with
different sizes, so that contents left in its shared scratch by the first
call cannot leak into the second; and, on seeded predictions, it must match
the oracle's masked MSE.  This file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2411_17164_gb300 import synth
from tests.helpers import case

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    fn = xmgn.lib().xmgn_mse_loss_static
    P = C.c_void_p
    fn.restype = C.c_int32
    fn.argtypes = [P, C.c_int64, C.c_int32, P, P, P, C.c_int64, P, P]
    return xmgn, fn


def _forward_loss(xmgn, g, xyz, nin, tgt, params, L=2):
    m = xmgn.Model(64, L, g, dtype="fp32", n_norm=len(xyz))
    dev = "cuda"
    y = torch.zeros((len(xyz), 4), device=dev)
    loss = torch.zeros((), device=dev)
    ni, xz, tt, tp = (torch.from_numpy(a).to(dev) for a in (nin, xyz, tgt, params))
    m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
    torch.cuda.synchronize()
    return y, tt, float(loss)


def _static_loss(xmgn, fn, y, tt, n_norm, hop=None):
    out = torch.full((), -1.0, device="cuda")
    st = fn(C.c_void_p(y.data_ptr()), y.shape[0], y.shape[1], C.c_void_p(tt.data_ptr()), None,
            None if hop is None else C.c_void_p(hop.data_ptr()), n_norm, C.c_void_p(out.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, xmgn.lib().xmgn_last_error()
    torch.cuda.synchronize()
    return float(out)


def test_static_loss_matches_forward_loss_twice(X):
    xmgn, fn = X
    # call 1: a 1,500-node sphere, every node counted
    xyz, nin = case("sphere", 1500, 3)
    tgt = synth.fourier_targets(xyz, 4)
    params = synth.init_params(64, 2, 6, 4, 5)
    g = xmgn.build_knn(torch.from_numpy(xyz).cuda(), 6)
    y, tt, ref = _forward_loss(xmgn, g, xyz, nin, tgt, params)
    got = _static_loss(xmgn, fn, y, tt, len(xyz))
    assert abs(got - ref) <= TOL * abs(ref), (got, ref)
    # call 2: a larger body (several scratch blocks), only a subset of nodes counted
    xyz, nin = case("body", 5000, 6)
    tgt = synth.fourier_targets(xyz, 7)
    g = xmgn.build_knn(torch.from_numpy(xyz).cuda(), 6)
    hop = (np.arange(5000) % 3 != 0).astype(np.uint8)   # one node in three counts
    gg = dict(g)
    gg["hop"] = torch.from_numpy(hop).cuda()
    y, tt, ref = _forward_loss(xmgn, gg, xyz, nin, tgt, params)
    got = _static_loss(xmgn, fn, y, tt, len(xyz), hop=gg["hop"])
    assert abs(got - ref) <= TOL * abs(ref), (got, ref)


def test_static_loss_rejects_oversize(X):
    xmgn, fn = X
    y = torch.zeros((4, 4), device="cuda")
    out = torch.zeros((), device="cuda")
    st = fn(C.c_void_p(y.data_ptr()), 4_194_305, 4, C.c_void_p(y.data_ptr()), None, None, 1,
            C.c_void_p(out.data_ptr()), None)
    assert st == 4 and b"at most" in xmgn.lib().xmgn_last_error()


def test_static_loss_matches_oracle_mse(X):
    """The same entry point against the oracle's masked MSE (Sec. IV-C loss
    over inner nodes, Sec. III-D) on seeded predictions and targets, twice in
    a row: 70,000 rows with one row in three counted, then 3,000 rows with
    row ids mapped through gid and every row counted."""
    from oracle import xmgn_oracle as O
    xmgn, fn = X
    rng = np.random.default_rng(17)
    for n, n_glob, every in ((70_000, 70_000, 3), (3_000, 9_000, 1)):
        y = rng.standard_normal((n, 4)).astype(np.float32)
        t = rng.standard_normal((n_glob, 4)).astype(np.float32)
        gid = rng.permutation(n_glob)[:n].astype(np.int32)
        hop = (np.arange(n) % every != 0).astype(np.uint8) if every > 1 else np.zeros(n, np.uint8)
        out = torch.full((), -1.0, device="cuda")
        dy, dt, dg, dh = (torch.from_numpy(a).cuda() for a in (y, t, gid, hop))
        st = fn(C.c_void_p(dy.data_ptr()), n, 4, C.c_void_p(dt.data_ptr()), C.c_void_p(dg.data_ptr()),
                C.c_void_p(dh.data_ptr()), n_glob, C.c_void_p(out.data_ptr()),
                C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, xmgn.lib().xmgn_last_error()
        torch.cuda.synchronize()
        want, _ = O.mse_loss(y.astype(np.float64), t[gid], (hop == 0).astype(np.float64), n_glob)
        assert abs(float(out) - want) <= TOL * abs(want), (float(out), want)
