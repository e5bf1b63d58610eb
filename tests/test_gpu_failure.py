"""Failure handling on the GPU without a fault: a device-side wait that can
never complete gives up after its bound, the host reads XMGN_ERR_TIMEOUT, the
error word is cleared, and the context keeps working."""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import assert_same_graph, case, oracle_graph, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


def test_bounded_wait_reports_timeout_and_context_survives(X):
    L = X.lib()
    st = L.xmgn_selftest_wait_timeout(X._stream())
    assert st == 6, X.lib().xmgn_last_error().decode()  # XMGN_ERR_TIMEOUT
    assert b"bounded" in L.xmgn_last_error()
    X.check_device()  # the error word was cleared
    # the context still runs the model correctly
    xyz, nin = case("sphere", 600, 3)
    tgt = synth.fourier_targets(xyz, 4)
    params = synth.init_params(128, 2, 6, 4, 5)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    m = X.Model(128, 2, g, dtype="bf16")
    y = torch.zeros((600, 4), device="cuda")
    m.forward(torch.from_numpy(params).cuda(), torch.from_numpy(nin).cuda(), torch.from_numpy(xyz).cuda(), y=y)
    torch.cuda.synchronize()
    X.check_device()
    _, rp, col, cperm = oracle_graph(xyz)
    assert_same_graph(g, rp, col, cperm)
    lo, go, yo = O.loss_and_grad(params.astype(np.float64), (128, 2, 6, 4), rp, col, nin, xyz, tgt)
    assert rel_l2(y.cpu().numpy(), yo) <= 2e-2
