"""Gradient aggregation across partitions (Sec. III-A "Gradient
Aggregation"), one partition per call: the 16 RCB parts (3-hop halos) of a
4,000-point body each run as their own graph through xmgn_forward /
xmgn_backward in FP32, and their gradients are summed into one buffer in
part order with the library's Neumaier compensation (dcomp).

* The summed gradient, the assembled inner-node outputs and the summed loss
  match the oracle's partitioned step (which equals its full-graph step):
  relative L2 <= 1e-4.
* The compensated sum is checked against the exact (float64) sum of the 16
  per-part gradients the library returned: its error is at most 1 % of the
  error of plain float32 accumulation of the same gradients.
* xmgn_grad_accumulate (the step the rank-order all-reduce uses) gives the
  same bits as the accumulation inside xmgn_backward."""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import assert_same_graph, case, oracle_graph, rel_l2

pytestmark = pytest.mark.gpu
H, L, N, P = 128, 3, 4000, 16


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


def test_sixteen_partition_calls_compensated_sum(X):
    dev = "cuda"
    xyz, nin = case("body", N, 12)
    tgt = synth.fourier_targets(xyz, 13)
    params = synth.init_params(H, L, 6, 4, 14, perturb_ln=True)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    _, rp, col, cperm = oracle_graph(xyz)
    assert_same_graph(g, rp, col, cperm)
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), P, L)
    part = O.rcb(xyz, P)
    np.testing.assert_array_equal(b["part"].cpu().numpy(), part)
    tp = torch.from_numpy(params).to(dev)
    ni, xz, tt = (torch.from_numpy(a).to(dev) for a in (nin, xyz, tgt))
    y = torch.zeros((N, 4), device=dev)
    acc = torch.zeros_like(tp)
    comp = torch.zeros_like(tp)
    plain = torch.zeros_like(tp)
    acc2 = torch.zeros_like(tp)
    comp2 = torch.zeros_like(tp)
    exact = np.zeros(len(params))
    loss_sum = 0.0
    for gp in X.split_batch(b):
        m = X.Model(H, L, gp, dtype="fp32", n_norm=N)
        loss = torch.zeros((), device=dev)
        m.forward(tp, ni, xz, targets=tt, y=y, loss=loss)
        m.backward(tp, ni, xz, tt, acc, comp)     # compensated accumulation in the call
        m.forward(tp, ni, xz, targets=tt)
        m.backward(tp, ni, xz, tt, plain)         # plain float32 accumulation
        m.forward(tp, ni, xz, targets=tt)
        one = torch.zeros_like(tp)
        m.backward(tp, ni, xz, tt, one)           # this part alone
        X.grad_accumulate(acc2, one, comp2)       # the same step through xmgn_grad_accumulate
        torch.cuda.synchronize()
        X.check_device()
        exact += one.double().cpu().numpy()
        loss_sum += float(loss)
    total = acc.double().cpu().numpy() + comp.double().cpu().numpy()
    e_comp = np.linalg.norm(total - exact)
    e_plain = np.linalg.norm(plain.double().cpu().numpy() - exact)
    print(f"16 partition calls: |compensated - exact| {e_comp:.3e}, |plain - exact| {e_plain:.3e} "
          f"(|exact| {np.linalg.norm(exact):.3e})")
    assert e_plain > 0 and e_comp <= 0.01 * e_plain
    np.testing.assert_array_equal(acc2.cpu().numpy(), acc.cpu().numpy())
    np.testing.assert_array_equal(comp2.cpu().numpy(), comp.cpu().numpy())
    parts = O.halo_partition(rp, col, part, P, L)
    yo, lo, go = O.partitioned_step(params.astype(np.float64), (H, L, 6, 4), parts, nin, xyz, tgt, N)
    ey, eg = rel_l2(y.cpu().numpy(), yo), rel_l2(total, go)
    print(f"vs oracle partitioned step: rel L2 y {ey:.3e} grad {eg:.3e}, loss {loss_sum:.7f} vs {lo:.7f}")
    assert ey <= 1e-4 and eg <= 1e-4 and abs(loss_sum - lo) <= 1e-4 * abs(lo)
