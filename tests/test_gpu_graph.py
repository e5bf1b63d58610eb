"""GPU parity of the graph builders (Sec. III-B kNN, Sec. III-A partitioning)
against the FP64 oracle: bit-exact integer outputs."""
import numpy as np
import pytest
import torch

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import case

pytestmark = pytest.mark.gpu
S64 = 1.0 / 64.0


@pytest.fixture(scope="module")
def X():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn


def _knn_exact(X, xyz, k=6):
    g = X.build_knn(torch.from_numpy(xyz).cuda(), k, want_nbr=True)
    nbr, rp, col, cperm = None, None, None, None
    nbr = O.knn(xyz, k)
    rp, col, _, cperm = O.symmetrise(nbr, len(xyz))
    np.testing.assert_array_equal(g["nbr"].cpu().numpy(), nbr)
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    np.testing.assert_array_equal(g["recv"].cpu().numpy(), O.edge_receivers(rp))
    np.testing.assert_array_equal(g["csc_perm"].cpu().numpy(), cperm)
    return g


def test_knn_sphere_2000(X):
    xyz, _ = case("sphere", 2000, 1)
    g = _knn_exact(X, xyz)
    assert 6 * 2000 <= g["E"] <= 12 * 2000


def test_knn_body_morton_8000(X):
    xyz, _ = case("body", 8000, 2)
    _knn_exact(X, xyz)


@pytest.mark.parametrize("k", [1, 3, 6, 16])
def test_knn_k_values(X, k):
    xyz, _ = case("body", 1500, 9)
    _knn_exact(X, xyz, k)


def test_knn_exact_ties_lattice_and_duplicates(X):
    g = np.arange(6) * S64
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    x = np.concatenate([x, x[:20]])  # coincident duplicates
    _knn_exact(X, x)


def test_knn_minimum_size(X):
    x = np.array([[0, 0, 0], [S64, 0, 0], [0, 2 * S64, 0]], np.float32)
    _knn_exact(X, x, k=2)


def test_knn_full_size_sampled_rows(X):
    """200k-node car body (the full-graph workload): sampled rows vs brute force."""
    xyz, _ = case("body", 200_000, 2)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6, want_nbr=True)
    rows = np.random.default_rng(0).choice(200_000, 200, replace=False)
    np.testing.assert_array_equal(g["nbr"].cpu().numpy()[rows], O.knn(xyz, 6, rows=rows))
    rp = g["row_ptr"].cpu().numpy()
    col = g["col"].cpu().numpy()
    perm = g["csc_perm"].cpu().numpy()
    recv = g["recv"].cpu().numpy()
    assert np.all(np.diff(rp) >= 6) and rp[-1] == g["E"]
    # symmetric, sorted rows, csc_perm maps each edge to its reverse
    assert np.all(col[perm] == recv) and np.all(recv[perm] == col)
    d = np.diff(col)
    assert np.all((d > 0) | (np.diff(recv) > 0))


def test_knn_range_error(X):
    x = np.zeros((10, 3), np.float32)
    x[3, 1] = 9.0
    with pytest.raises(X.XmgnError) as e:
        X.build_knn(torch.from_numpy(x).cuda(), 2)
    assert e.value.status == 2


def _partition_exact(X, xyz, P, hops, part_in=None):
    nbr = O.knn(xyz, 6)
    rp, col, _, _ = O.symmetrise(nbr, len(xyz))
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    pin = None if part_in is None else torch.from_numpy(part_in.astype(np.int32)).cuda()
    b = X.partition_halo(g, torch.from_numpy(xyz).cuda(), P, hops, part_in=pin)
    part = O.rcb(xyz, P) if part_in is None else part_in
    np.testing.assert_array_equal(b["part"].cpu().numpy(), part)
    parts = O.halo_partition(rp, col, part, P, hops)
    gid = b["gid"].cpu().numpy()
    hop = b["hop"].cpu().numpy()
    brp = b["row_ptr"].cpu().numpy()
    bcol = b["col"].cpu().numpy()
    for p, pt in enumerate(parts):
        n0, n1 = b["node_ptr"][p], b["node_ptr"][p + 1]
        e0, e1 = b["edge_ptr"][p], b["edge_ptr"][p + 1]
        np.testing.assert_array_equal(gid[n0:n1], pt["gid"])
        np.testing.assert_array_equal(hop[n0:n1], pt["hop"])
        assert b["inner_cnt"][p] == pt["n_inner"]
        np.testing.assert_array_equal(brp[n0:n1 + 1] - e0, pt["row_ptr"])
        np.testing.assert_array_equal(bcol[e0:e1] - n0, pt["col"])
    perm = b["csc_perm"].cpu().numpy()
    recv = b["recv"].cpu().numpy()
    assert np.all(bcol[perm] == recv) and np.all(recv[perm] == bcol)
    return b


@pytest.mark.parametrize("P,hops", [(1, 2), (3, 2), (4, 3), (8, 4)])
def test_partition_rcb_halo_exact(X, P, hops):
    xyz, _ = case("body", 3000, 5)
    _partition_exact(X, xyz, P, hops)


def test_partition_given_parts(X):
    xyz, _ = case("body", 2500, 6)
    part = (np.arange(2500) * 7 // 2500).astype(np.int32)   # seven contiguous id ranges
    _partition_exact(X, xyz, 7, 3, part_in=part)


def test_partition_given_regions_with_unassigned_nodes(X):
    """Breadth-first regions that leave nodes outside every part (-1): those
    nodes appear only as halo, exactly as the oracle's halo sets say."""
    xyz, _ = case("body", 3000, 8)
    rp, col, _, _ = O.symmetrise(O.knn(xyz, 6), len(xyz))
    part = synth.bfs_regions(rp, col, 6, 60, 400, 9)
    assert (part < 0).any() and (part >= 0).any()
    _partition_exact(X, xyz, 6, 3, part_in=part)


@pytest.mark.parametrize("sizes", [[400], [300, 1500], [250, 1000, 4000]])
def test_multiscale_graph_exact(X, sizes):
    """Multi-scale graph (Sec. III-C): bit-exact CSR, CSC permutation and
    per-slot neighbour lists against the oracle."""
    xyz, _ = synth.nested_levels(sizes, 21)
    rp, col, _, cperm = O.multiscale_graph(xyz, sizes)
    g = X.build_multiscale(torch.from_numpy(xyz).cuda(), sizes, want_nbr=True)
    np.testing.assert_array_equal(g["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(g["col"].cpu().numpy(), col)
    np.testing.assert_array_equal(g["csc_perm"].cpu().numpy(), cperm)
    nbr = g["nbr"].cpu().numpy()
    for lv, n_l in enumerate(sizes):
        np.testing.assert_array_equal(nbr[:n_l, 6 * lv:6 * lv + 6], O.knn(xyz[:n_l], 6))
        assert np.all(nbr[n_l:, 6 * lv:6 * lv + 6] == -1)
    if len(sizes) > 1:
        c0 = 6 * len(sizes)
        assert np.all(nbr[:sizes[0], c0:] == -1)
        for lv in range(1, len(sizes)):
            rows = np.arange(sizes[lv - 1], sizes[lv])
            np.testing.assert_array_equal(nbr[rows, c0:], O.knn_among(xyz, rows, sizes[lv - 1], 3))


def _partition_raw(X, g, xyz, P, hops, part_in, ws, emit_fn, sizes=None):
    """One call of the partition ABI (sizing when sizes is None, else an emit
    call into fresh outputs); returns (status, host arrays, device outputs)."""
    import ctypes as C
    L = X.lib()
    N, E = g["n"], g["E"]
    node_ptr, edge_ptr, inner = (C.c_int64 * (P + 1))(), (C.c_int64 * (P + 1))(), (C.c_int64 * P)()
    if sizes is not None:
        node_ptr[:], edge_ptr[:], inner[:] = sizes
    part = torch.empty(N, dtype=torch.int32, device="cuda")
    args = (X._ptr(g["row_ptr"]), X._ptr(g["col"]), N, E, X._ptr(xyz), 0.0, P, hops, X._ptr(part_in),
            X._ptr(ws), ws.numel(), X._ptr(part), node_ptr, edge_ptr, inner)
    if sizes is None:
        st = L.xmgn_partition_halo(*args, None, None, None, None, None, None, 0, 0, X._stream())
        return st, (list(node_ptr), list(edge_ptr), list(inner)), None
    nb, eb = node_ptr[P], edge_ptr[P]
    out = dict(gid=torch.full((nb,), -7, dtype=torch.int32, device="cuda"),
               hop=torch.full((nb,), 7, dtype=torch.uint8, device="cuda"),
               rp=torch.full((nb + 1,), -7, dtype=torch.int64, device="cuda"),
               col=torch.full((eb,), -7, dtype=torch.int32, device="cuda"),
               recv=torch.full((eb,), -7, dtype=torch.int32, device="cuda"),
               perm=torch.full((eb,), -7, dtype=torch.int32, device="cuda"))
    fn = getattr(L, emit_fn)
    st = fn(*args, *(X._ptr(out[k]) for k in ("gid", "hop", "rp", "col", "recv", "perm")), nb, eb, X._stream())
    torch.cuda.synchronize()
    return st, None, out


def test_partition_emit_pass_resumes_and_checks_its_stamp(X):
    """xmgn_partition_halo_emit after a sizing call gives the same batch as a
    full second call; without a matching sizing pass in the workspace it is
    rejected on the host and writes nothing."""
    import ctypes as C
    xyz, _ = case("body", 3000, 5)
    g = X.build_knn(torch.from_numpy(xyz).cuda(), 6)
    dxyz = torch.from_numpy(xyz).cuda()
    P, hops = 4, 3
    wsb = C.c_size_t()
    assert X.lib().xmgn_partition_halo_ws(g["n"], g["E"], P, C.byref(wsb)) == 0
    ws = torch.zeros(wsb.value, dtype=torch.uint8, device="cuda")
    st, sizes, _ = _partition_raw(X, g, dxyz, P, hops, None, ws, None)
    assert st == 0
    st, _, full = _partition_raw(X, g, dxyz, P, hops, None, ws, "xmgn_partition_halo", sizes)
    assert st == 0
    st, sizes2, _ = _partition_raw(X, g, dxyz, P, hops, None, ws, None)
    assert st == 0 and sizes2 == sizes
    st, _, res = _partition_raw(X, g, dxyz, P, hops, None, ws, "xmgn_partition_halo_emit", sizes)
    assert st == 0
    for k in full:
        assert torch.equal(full[k], res[k]), k
    # the completed emit cleared the stamp: a second resume is refused, outputs untouched
    st, _, again = _partition_raw(X, g, dxyz, P, hops, None, ws, "xmgn_partition_halo_emit", sizes)
    assert st == 1 and b"no sizing pass" in X.lib().xmgn_last_error()
    assert int(again["gid"].min()) == -7 and int(again["gid"].max()) == -7
    # a sizing pass with other halo depth does not match
    st, _, _ = _partition_raw(X, g, dxyz, P, hops + 1, None, ws, None)
    assert st == 0
    st, _, _ = _partition_raw(X, g, dxyz, P, hops, None, ws, "xmgn_partition_halo_emit", sizes)
    assert st == 1
