"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Every test here runs on the CPU.  None of them compares the oracle with
itself: each checks a hand-worked fixture (tests/golden), a library routine
on a special case (scipy cKDTree, networkx BFS, torch float64 functional ops,
scipy sparse products), a closed form, an invariant, central finite
differences, or the paper's halo-equivalence statement (Sec. II-D, III-A).
"""
import os

import numpy as np
import pytest

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
S64 = 1.0 / 64.0


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([list(map(float, part.split())) for part in line.split("|")])
    return rows


def _graph(n, seed, k=6):
    xyz, nrm = synth.sphere_cloud(n, seed)
    nbr = O.knn(xyz, k)
    rp, col, cp, cperm = O.symmetrise(nbr, n)
    return xyz, synth.node_inputs(xyz, nrm), rp, col, cp, cperm


# ---------------------------------------------------------------------------
# kNN (Sec. III-B)
# ---------------------------------------------------------------------------
def test_knn_golden_line():
    rows = _read_golden("knn_line.txt")
    x = np.array([[r[0][0] * S64, 0, 0] for r in rows], np.float32)
    want = np.array([r[1] for r in rows], np.int64)
    np.testing.assert_array_equal(O.knn(x, 2), want)


def test_knn_cubic_lattice_axis_neighbours():
    g = np.arange(5) * S64
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    nbr = O.knn(x, 6)
    idx = np.arange(125).reshape(5, 5, 5)
    for i in range(1, 4):
        for j in range(1, 4):
            for k in range(1, 4):
                want = sorted([idx[i - 1, j, k], idx[i + 1, j, k], idx[i, j - 1, k], idx[i, j + 1, k],
                               idx[i, j, k - 1], idx[i, j, k + 1]])
                assert list(nbr[idx[i, j, k]]) == want  # six ties at one spacing, index order


def test_knn_matches_kdtree_on_random_cloud():
    spatial = pytest.importorskip("scipy.spatial")
    xyz, _ = synth.sphere_cloud(1500, 7)
    nbr = O.knn(xyz, 6)
    d, ref = spatial.cKDTree(xyz.astype(np.float64)).query(xyz.astype(np.float64), k=7)
    ref = ref[:, 1:]
    bad = 0
    for i in range(len(xyz)):
        if set(nbr[i]) != set(ref[i]):
            # only a near tie at the k-th place (within lattice rounding) may differ
            assert d[i, 6] - d[i, 5] < 4.0 / 2 ** 21 or abs(d[i, 7 - 1] - d[i, 6 - 1]) < 4.0 / 2 ** 21
            bad += 1
    assert bad <= 2
    # nearest-first ordering by distance
    dd = np.linalg.norm(xyz[nbr].astype(np.float64) - xyz[:, None, :].astype(np.float64), axis=2)
    assert np.all(np.diff(dd, axis=1) >= -1e-6)


def test_knn_duplicates_and_self_exclusion():
    x = np.array([[0, 0, 0], [0, 0, 0], [S64, 0, 0], [0, 0, 0]], np.float32)
    nbr = O.knn(x, 2)
    np.testing.assert_array_equal(nbr, [[1, 3], [0, 3], [0, 1], [0, 1]])


def test_knn_range_and_arg_errors():
    with pytest.raises(ValueError):
        O.knn(np.array([[9.0, 0, 0], [0, 0, 0]], np.float32), 1)
    with pytest.raises(ValueError):
        O.knn(np.zeros((3, 3), np.float32), 3)


@pytest.mark.parametrize("k", [1, 3, 6, 16])
def test_knn_tree_matches_brute_force(k):
    """knn_tree (k-d tree candidates, exact decision) equals the brute-force
    definition on random clouds and on a lattice with exact ties plus many
    coincident points (31 copies of one point force the widening step)."""
    pytest.importorskip("scipy.spatial")
    g = np.arange(6) * S64
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    lat = np.concatenate([lat, lat[:20]] + [lat[5:6]] * 30)
    for x in (synth.sphere_cloud(1500, 7)[0], synth.car_body(2500, 3)[0], lat):
        np.testing.assert_array_equal(O.knn_tree(x, k), O.knn(x, k))
    rows = np.array([0, 5, 17, len(lat) - 1])
    np.testing.assert_array_equal(O.knn_tree(lat, k, rows=rows), O.knn(lat, k)[rows])


def test_knn_tree_among_and_multiscale_match_brute_force():
    pytest.importorskip("scipy.spatial")
    xyz, _ = synth.nested_levels([300, 1500], 21)
    rows = np.arange(300, 1500)
    np.testing.assert_array_equal(O.knn_tree(xyz, 3, n_ref=300, rows=rows), O.knn_among(xyz, rows, 300, 3))
    dup = np.concatenate([xyz[:40]] * 3 + [xyz[:10]])  # ties at every distance
    rows = np.arange(40, len(dup))
    np.testing.assert_array_equal(O.knn_tree(dup, 3, n_ref=40, rows=rows), O.knn_among(dup, rows, 40, 3))
    for u, v in zip(O.multiscale_graph(xyz, [300, 1500], tree=True), O.multiscale_graph(xyz, [300, 1500])):
        np.testing.assert_array_equal(u, v)


def test_quantize_round_half_even():
    x = np.array([[0.5 / 2 ** 21, 1.5 / 2 ** 21, -2.5 / 2 ** 21]], np.float32)
    np.testing.assert_array_equal(O.quantize(x), [[0, 2, -2]])


# ---------------------------------------------------------------------------
# Symmetrised CSR
# ---------------------------------------------------------------------------
def test_symmetrise_matches_set_definition():
    xyz, _, rp, col, cp, cperm = _graph(300, 3)
    nbr = O.knn(xyz, 6)
    edges = set()
    for i in range(300):
        for j in nbr[i]:
            edges.add((i, int(j)))
            edges.add((int(j), i))
    got = [(i, int(col[e])) for i in range(300) for e in range(rp[i], rp[i + 1])]
    assert got == sorted(edges)                       # receiver-major, senders ascending, unique
    assert all(a != b for a, b in got)                # no self loops
    assert np.all(np.diff(rp) >= 6)
    # CSC: a permutation listing edges sender-major, receivers ascending
    recv = np.repeat(np.arange(300), np.diff(rp))
    assert sorted(cperm.tolist()) == list(range(len(col)))
    pairs = list(zip(col[cperm].tolist(), recv[cperm].tolist()))
    assert pairs == sorted(pairs)
    np.testing.assert_array_equal(cp, rp)             # symmetric graph: same degrees


def test_symmetrise_pairs_set_definition_with_self_loops_and_repeats():
    """Directed pairs with repeats, both orientations and self pairs: the
    result is the undirected set without self loops (eq. (2)'s
    neighbourhoods exclude the node itself)."""
    recv = [0, 0, 1, 2, 2, 3, 3, 4, 4]
    send = [1, 1, 0, 2, 4, 3, 0, 0, 2]   # (0,1) twice, (1,0), self pairs (2,2), (3,3)
    rp, col, cp, cperm = O.symmetrise_pairs(recv, send, 5)
    want = sorted({(a, b) for a, b in zip(recv, send) if a != b} | {(b, a) for a, b in zip(recv, send) if a != b})
    got = [(i, int(col[e])) for i in range(5) for e in range(rp[i], rp[i + 1])]
    assert got == want
    assert want == [(0, 1), (0, 3), (0, 4), (1, 0), (2, 4), (3, 0), (4, 0), (4, 2)]


# ---------------------------------------------------------------------------
# RCB + halo (Sec. III-A)
# ---------------------------------------------------------------------------
def test_rcb_golden_plane():
    rows = _read_golden("rcb_plane.txt")
    x = np.array([[r[0][1] * S64, r[0][2] * S64, 0.0] for r in rows], np.float32)
    want = np.array([r[1][0] for r in rows], np.int64)
    np.testing.assert_array_equal(O.rcb(x, 4), want)


@pytest.mark.parametrize("P", [1, 3, 5, 6, 8, 16])
def test_rcb_balance_and_cover(P):
    """Every point in exactly one part, and the parts balanced to one point
    for any P (splits proportional to the part counts on each side)."""
    xyz, _ = synth.car_body(4001, 11)
    part = O.rcb(xyz, P)
    sizes = np.bincount(part, minlength=P)
    assert sizes.sum() == 4001 and len(sizes) == P
    assert sizes.max() - sizes.min() <= 1


def test_halo_hops_match_networkx_bfs():
    nx = pytest.importorskip("networkx")
    xyz, _, rp, col, _, _ = _graph(600, 5)
    part = O.rcb(xyz, 4)
    parts = O.halo_partition(rp, col, part, 4, 3)
    G = nx.Graph()
    G.add_nodes_from(range(600))
    recv = np.repeat(np.arange(600), np.diff(rp))
    G.add_edges_from(zip(recv.tolist(), col.tolist()))
    for p, pt in enumerate(parts):
        inner = np.nonzero(part == p)[0]
        G2 = G.copy()
        G2.add_node(-1)
        G2.add_edges_from((-1, int(v)) for v in inner)
        dist = nx.single_source_shortest_path_length(G2, -1, cutoff=4)
        want = sorted((d - 1, v) for v, d in dist.items() if v != -1 and d - 1 <= 3)
        got = sorted(zip(pt["hop"].tolist(), pt["gid"].tolist()))
        assert got == want
        np.testing.assert_array_equal(pt["gid"][:pt["n_inner"]], inner)
        halo = list(zip(pt["hop"][pt["n_inner"]:].tolist(), pt["gid"][pt["n_inner"]:].tolist()))
        assert halo == sorted(halo)                                  # halo by (hop, id)
        sub = G.subgraph(pt["gid"].tolist())
        lrecv = np.repeat(np.arange(len(pt["gid"])), np.diff(pt["row_ptr"]))
        ledges = {(int(pt["gid"][a]), int(pt["gid"][b])) for a, b in zip(lrecv, pt["col"])}
        assert ledges == {(a, b) for a, b in sub.edges()} | {(b, a) for a, b in sub.edges()}
        for r in range(len(pt["gid"])):                               # senders by global id
            g = pt["gid"][pt["col"][pt["row_ptr"][r]:pt["row_ptr"][r + 1]]]
            assert np.all(np.diff(g) > 0)


def test_bfs_hops_and_induced_subgraph_match_networkx():
    """The neighbourhood selection of the sampled parity checks: hop
    distances from a source set up to a limit, and the induced subgraph in a
    given node order, against networkx."""
    nx = pytest.importorskip("networkx")
    xyz, _, rp, col, _, _ = _graph(500, 9)
    recv = np.repeat(np.arange(500), np.diff(rp))
    G = nx.Graph()
    G.add_nodes_from(range(500))
    G.add_edges_from(zip(recv.tolist(), col.tolist()))
    src = [3, 77, 250]
    got = O.bfs_hops(rp, col, src, 4)
    G.add_edges_from((-1, v) for v in src)
    dist = nx.single_source_shortest_path_length(G, -1, cutoff=5)
    want = np.full(500, -1)
    for v, d in dist.items():
        if v != -1:
            want[v] = d - 1
    np.testing.assert_array_equal(got, want)
    G.remove_node(-1)
    gid = np.nonzero(got >= 0)[0][::-1]                       # any order: local ids follow it
    lrp, lcol = O.induced_subgraph(rp, col, gid)
    lrecv = np.repeat(np.arange(len(gid)), np.diff(lrp))
    edges = {(int(gid[a]), int(gid[b])) for a, b in zip(lrecv, lcol)}
    sub = G.subgraph(gid.tolist())
    assert edges == {(a, b) for a, b in sub.edges()} | {(b, a) for a, b in sub.edges()}
    assert len(edges) == len(lcol)
    for r in range(len(gid)):                                 # senders by ascending global id
        assert np.all(np.diff(gid[lcol[lrp[r]:lrp[r + 1]]]) > 0)


# ---------------------------------------------------------------------------
# MLP pieces against library routines / closed forms
# ---------------------------------------------------------------------------
def test_layernorm_silu_match_torch_float64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    v = rng.standard_normal((37, 16)) * 3
    g = rng.standard_normal(16)
    b = rng.standard_normal(16)
    y, _ = O.layer_norm(v, g, b)
    ref = torch.nn.functional.layer_norm(torch.from_numpy(v), (16,), torch.from_numpy(g), torch.from_numpy(b), eps=1e-5)
    np.testing.assert_allclose(y, ref.numpy(), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(O.silu(v), torch.nn.functional.silu(torch.from_numpy(v)).numpy(), rtol=1e-14, atol=1e-15)
    # SiLU derivative against central differences of torch's SiLU
    t = torch.from_numpy(v).requires_grad_(True)
    torch.nn.functional.silu(t).sum().backward()
    np.testing.assert_allclose(O.silu_grad(v), t.grad.numpy(), rtol=1e-13, atol=1e-14)


def test_layernorm_two_feature_closed_form():
    a, b = 0.7, -1.9
    y, _ = O.layer_norm(np.array([[a, b]]), np.ones(2), np.zeros(2))
    half = (a - b) / 2
    want = np.array([half, -half]) / np.sqrt(half * half + 1e-5)
    np.testing.assert_allclose(y[0], want, rtol=1e-15)


def test_mse_loss_matches_torch_mean():
    """Sec. IV-C MSE: with every node inner and the normaliser n, the loss is
    torch's mean squared error over all n x out entries and dL/dy its
    autograd gradient; with a mask it is the mean over the masked rows when
    the normaliser is their count (halo rows contribute nothing)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    y = rng.standard_normal((23, 4))
    t = rng.standard_normal((23, 4)).astype(np.float32)
    loss, dy = O.mse_loss(y, t, np.ones(23), 23)
    ty = torch.from_numpy(y).requires_grad_(True)
    ref = torch.nn.functional.mse_loss(ty, torch.from_numpy(t.astype(np.float64)))
    ref.backward()
    assert abs(loss - ref.item()) <= 1e-14 * abs(ref.item())
    np.testing.assert_allclose(dy, ty.grad.numpy(), rtol=1e-14, atol=1e-16)
    mask = (np.arange(23) % 4 != 1).astype(np.float64)
    sel = mask > 0
    loss_m, dy_m = O.mse_loss(y, t, mask, int(sel.sum()))
    ref_m = torch.nn.functional.mse_loss(torch.from_numpy(y[sel]), torch.from_numpy(t[sel].astype(np.float64)))
    assert abs(loss_m - ref_m.item()) <= 1e-14 * abs(ref_m.item())
    assert np.all(dy_m[~sel] == 0.0)


def test_edge_features_golden():
    rows = _read_golden("edge_features.txt")
    xyz = np.array([[0, 0, 0], [3, 0, 4]], np.float32)
    rp = np.array([0, 1, 2])
    col = np.array([1, 0])
    f = O.edge_inputs(xyz, rp, col)
    for t, r in enumerate(rows):
        assert (int(r[0][0]), int(r[0][1])) == (t, int(col[t]))
        np.testing.assert_array_equal(f[t], r[1])


# ---------------------------------------------------------------------------
# Model special cases (eqs. 1-4)
# ---------------------------------------------------------------------------
DIMS = (8, 2, 6, 4)


def _params(seed, dims=DIMS, perturb=True):
    H, L, i, o = dims
    return synth.init_params(H, L, i, o, seed, perturb_ln=perturb).astype(np.float64)


def _set(flat, dims, name, value):
    H, L, i, o = dims
    off = 0
    for nm, shape in O.param_shapes(H, L, i, o):
        sz = int(np.prod(shape))
        if nm == name:
            flat[off:off + sz] = np.broadcast_to(value, shape).reshape(-1)
            return flat
        off += sz
    raise KeyError(name)


def _blocks(flat, dims):
    return O.unpack(flat, *dims)


def test_message_roles_reduce_to_sparse_products():
    """With only the sender block of the first message layer non-zero,
    m_ij depends on h_j alone and sum aggregation gives A f(H) (scipy sparse);
    with only the receiver block it gives deg_i f(h_i)."""
    sp = pytest.importorskip("scipy.sparse")
    H, L, i, o = dims = (8, 1, 6, 4)
    xyz, nin, rp, col, _, _ = _graph(200, 9)
    n = 200
    A = sp.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
    for block in ("send", "recv"):
        flat = _params(4, dims)
        p = _blocks(flat, dims)
        W1 = p["e0.W1"].copy()
        if block == "send":
            W1[:H] = 0
        else:
            W1[H:2 * H] = 0
        W1[2 * H:] = 0
        _set(flat, dims, "e0.W1", W1)
        # probe: node update reads only the aggregated message; decoder = identity-ish
        Wn = _blocks(flat, dims)["n0.W1"].copy()
        Wn[:H] = 0
        _set(flat, dims, "n0.W1", Wn)
        y, cache = O.forward(flat, dims, rp, col, nin, xyz, keep=True)
        p = _blocks(flat, dims)
        h0 = cache["c_ne"]
        h0 = O.layer_norm(O.silu(nin.astype(np.float64) @ p["ne.W1"] + p["ne.b1"]) @ p["ne.W2"] + p["ne.b2"], p["ne.g"], p["ne.be"])[0]
        f = lambda hh: O.layer_norm(O.silu(hh @ W1[:H] + p["e0.b1"]) @ p["e0.W2"] + p["e0.b2"], p["e0.g"], p["e0.be"])[0] \
            if block == "recv" else O.layer_norm(O.silu(hh @ W1[H:2 * H] + p["e0.b1"]) @ p["e0.W2"] + p["e0.b2"], p["e0.g"], p["e0.be"])[0]
        fh = f(h0)
        agg_want = A @ fh if block == "send" else np.diff(rp)[:, None] * fh
        x_node = cache["caches"][0][1][0]
        np.testing.assert_allclose(x_node[:, H:], agg_want, rtol=1e-12, atol=1e-12)


def test_constant_messages_closed_form():
    """W2 = 0 and a feature-constant b2 make each LayerNorm input a constant
    row (zero variance), so every processor MLP output is exactly beta:
    e^{l+1} = e^l + beta_e, agg_i = deg_i beta_e, h^{l+1} = h^l + beta_n."""
    H, L, i, o = dims = (8, 3, 6, 4)
    xyz, nin, rp, col, _, _ = _graph(150, 2)
    flat = _params(6, dims)
    for l in range(L):
        _set(flat, dims, f"e{l}.W2", 0.0)
        _set(flat, dims, f"n{l}.W2", 0.0)
        _set(flat, dims, f"e{l}.b2", 0.375)
        _set(flat, dims, f"n{l}.b2", -1.25)
    y, cache = O.forward(flat, dims, rp, col, nin, xyz, keep=True)
    p = _blocks(flat, dims)
    h = cache["c_ne"]
    h0 = O.layer_norm(O.silu(nin.astype(np.float64) @ p["ne.W1"] + p["ne.b1"]) @ p["ne.W2"] + p["ne.b2"], p["ne.g"], p["ne.be"])[0]
    e0 = O.layer_norm(O.silu(O.edge_inputs(xyz, rp, col) @ p["ee.W1"] + p["ee.b1"]) @ p["ee.W2"] + p["ee.b2"], p["ee.g"], p["ee.be"])[0]
    hL = h0 + sum(p[f"n{l}.be"] for l in range(L))
    for l in range(L):
        c_e, c_n = cache["caches"][l]
        e_l = e0 + sum(p[f"e{t}.be"] for t in range(l))
        np.testing.assert_allclose(c_e[0][:, 2 * H:], e_l, rtol=0, atol=1e-12)
        np.testing.assert_allclose(c_n[0][:, H:], np.diff(rp)[:, None] * p[f"e{l}.be"], rtol=0, atol=1e-12)
    want_y = O.silu(hL @ p["d.W1"] + p["d.b1"]) @ p["d.W2"] + p["d.b2"]
    np.testing.assert_allclose(y, want_y, rtol=1e-12, atol=1e-12)


def test_isolated_node_gets_zero_message():
    H, L, i, o = dims = (8, 2, 6, 4)
    xyz, nin, rp, col, _, _ = _graph(120, 4)
    # append an isolated node far from the others
    xyz2 = np.concatenate([xyz, [[3.0, 3.0, 3.0]]]).astype(np.float32)
    nin2 = np.concatenate([nin, [[3, 3, 3, 1, 0, 0]]]).astype(np.float32)
    rp2 = np.concatenate([rp, [rp[-1]]])
    flat = _params(8, dims)
    y, cache = O.forward(flat, dims, rp2, col, nin2, xyz2, keep=True)
    for l in range(L):
        assert np.all(cache["caches"][l][1][0][-1, H:] == 0.0)
    y_alone = O.forward(flat, dims, np.array([0, 0]), np.zeros(0, np.int64), nin2[-1:], xyz2[-1:])
    np.testing.assert_allclose(y[-1], y_alone[0], rtol=1e-14, atol=1e-15)  # BLAS row blocking may differ by an ulp
    np.testing.assert_allclose(y[:-1], O.forward(flat, dims, rp, col, nin, xyz), rtol=1e-13, atol=1e-13)


def test_node_permutation_equivariance():
    dims = DIMS
    xyz, nin, rp, col, _, _ = _graph(250, 12)
    flat = _params(3, dims)
    y = O.forward(flat, dims, rp, col, nin, xyz)
    perm = np.random.default_rng(1).permutation(250)          # new id -> old id
    inv = np.empty_like(perm)
    inv[perm] = np.arange(250)
    recv = np.repeat(np.arange(250), np.diff(rp))
    r2, s2 = inv[recv], inv[col]
    key = np.lexsort((s2, r2))
    r2, s2 = r2[key], s2[key]
    rp2 = np.zeros(251, np.int64)
    np.cumsum(np.bincount(r2, minlength=250), out=rp2[1:])
    y2 = O.forward(flat, dims, rp2, s2, nin[perm], xyz[perm])
    np.testing.assert_allclose(y2, y[perm], rtol=1e-12, atol=1e-12)


def test_forward_matches_torch_functional_float64():
    """Library cross-check: the same network assembled from torch float64
    functional ops (linear, silu, layer_norm, index_add_)."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    H, L, i, o = dims = (8, 2, 6, 4)
    xyz, nin, rp, col, _, _ = _graph(180, 21)
    flat = _params(5, dims)
    p = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in _blocks(flat, dims).items()}
    recv = torch.from_numpy(np.repeat(np.arange(180), np.diff(rp)))
    send = torch.from_numpy(col.astype(np.int64))
    X = torch.from_numpy(xyz.astype(np.float64))

    def mlp(x, pre, ln=True):
        z = F.linear(F.silu(F.linear(x, p[pre + "W1"].T, p[pre + "b1"])), p[pre + "W2"].T, p[pre + "b2"])
        return F.layer_norm(z, (z.shape[1],), p[pre + "g"], p[pre + "be"], eps=1e-5) if ln else z

    h = mlp(torch.from_numpy(nin.astype(np.float64)), "ne.")
    d = X[send] - X[recv]
    e = mlp(torch.cat([d, d.norm(dim=1, keepdim=True)], 1), "ee.")
    for l in range(L):
        m = mlp(torch.cat([h[recv], h[send], e], 1), f"e{l}.")
        e = e + m
        agg = torch.zeros(180, H, dtype=torch.float64).index_add_(0, recv, m)
        h = h + mlp(torch.cat([h, agg], 1), f"n{l}.")
    yt = mlp(h, "d.", ln=False).numpy()
    np.testing.assert_allclose(O.forward(flat, dims, rp, col, nin, xyz), yt, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------------------
# Backward: central finite differences
# ---------------------------------------------------------------------------
def test_backward_central_differences():
    dims = (6, 2, 6, 4)
    H, L, i, o = dims
    xyz, nin, rp, col, _, _ = _graph(60, 13, k=4)
    tgt = synth.fourier_targets(xyz, 3)
    flat = _params(11, dims)
    mask = (np.arange(60) % 3 != 0).astype(np.float64)   # loss on a subset only
    loss, grad, _ = O.loss_and_grad(flat, dims, rp, col, nin, xyz, tgt, mask, 60)
    f = lambda th: O.mse_loss(O.forward(th, dims, rp, col, nin, xyz), tgt, mask, 60)[0]
    rng = np.random.default_rng(0)
    idx = rng.choice(len(flat), 48, replace=False)
    # include every kind of parameter: first entries of each block
    off = 0
    for _, shape in O.param_shapes(H, L, i, o):
        idx = np.append(idx, off)
        off += int(np.prod(shape))
    for j in idx:
        st = 1e-6 * max(1.0, abs(flat[j]))
        a, b = flat.copy(), flat.copy()
        a[j] += st
        b[j] -= st
        fd = (f(a) - f(b)) / (2 * st)
        assert abs(fd - grad[j]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max()), (j, fd, grad[j])
    # directional derivative along a random direction
    v = rng.standard_normal(len(flat))
    st = 1e-6
    fd = (f(flat + st * v) - f(flat - st * v)) / (2 * st)
    assert abs(fd - grad @ v) <= 1e-6 * abs(fd)


# ---------------------------------------------------------------------------
# Halo partitioning equivalence (Sec. II-D, III-A), loss filter (Sec. III-D)
# ---------------------------------------------------------------------------
def _halo_case(n=700, P=4, L=3, H=8, seed=31):
    xyz, nrm = synth.car_body(n, seed)
    nin = synth.node_inputs(xyz, nrm)
    nbr = O.knn(xyz, 6)
    rp, col, _, _ = O.symmetrise(nbr, n)
    part = O.rcb(xyz, P)
    tgt = synth.fourier_targets(xyz, seed + 1)
    dims = (H, L, 6, 4)
    flat = _params(seed + 2, dims)
    return xyz, nin, rp, col, part, tgt, dims, flat


def test_halo_depth_L_reproduces_full_graph():
    xyz, nin, rp, col, part, tgt, dims, flat = _halo_case()
    n = len(xyz)
    loss_f, grad_f, y_f = O.loss_and_grad(flat, dims, rp, col, nin, xyz, tgt)
    parts = O.halo_partition(rp, col, part, 4, dims[1])
    y_p, loss_p, grad_p = O.partitioned_step(flat, dims, parts, nin, xyz, tgt, n)
    assert sum(pt["n_inner"] for pt in parts) == n
    np.testing.assert_allclose(y_p, y_f, rtol=1e-13, atol=1e-14)
    assert abs(loss_p - loss_f) <= 1e-12 * abs(loss_f)
    np.testing.assert_allclose(grad_p, grad_f, rtol=1e-9, atol=1e-12 * np.abs(grad_f).max())


def test_halo_depth_below_L_differs():
    xyz, nin, rp, col, part, tgt, dims, flat = _halo_case()
    n = len(xyz)
    y_f = O.forward(flat, dims, rp, col, nin, xyz)
    parts = O.halo_partition(rp, col, part, 4, dims[1] - 1)
    y_p, _, _ = O.partitioned_step(flat, dims, parts, nin, xyz, tgt, n, with_grad=False)
    assert np.abs(y_p - y_f).max() > 1e-6


def test_halo_targets_do_not_affect_loss_or_grad():
    xyz, nin, rp, col, part, tgt, dims, flat = _halo_case(n=400, P=3, L=2)
    parts = O.halo_partition(rp, col, part, 3, 2)
    pt = parts[0]
    gid = pt["gid"]
    mask = np.zeros(len(gid))
    mask[:pt["n_inner"]] = 1
    t = tgt[gid].copy()
    l1, g1, _ = O.loss_and_grad(flat, dims, pt["row_ptr"], pt["col"], nin[gid], xyz[gid], t, mask, 400)
    t[pt["n_inner"]:] += 100.0
    l2, g2, _ = O.loss_and_grad(flat, dims, pt["row_ptr"], pt["col"], nin[gid], xyz[gid], t, mask, 400)
    assert l1 == l2
    np.testing.assert_array_equal(g1, g2)


def test_param_layout_counts():
    assert O.param_count(64, 4, 6, 4) == 130500
    assert O.param_count(128, 15, 6, 4) == 1787780
    assert O.param_count(64, 4, 6, 4) == sum(int(np.prod(s)) for _, s, _, _ in synth.param_blocks(64, 4, 6, 4))


def test_multiscale_graph_matches_independent_construction():
    """Sec. III-C: edge set = kNN within each nested level plus links from
    every point new in level l to its 3 nearest points of level l-1,
    symmetrised; rebuilt here from scipy cKDTree queries and python sets."""
    from scipy.spatial import cKDTree
    sizes = [60, 240, 700]
    xyz, _ = synth.nested_levels(sizes, 17)
    rp, col, cp, cperm = O.multiscale_graph(xyz, sizes, k=6, k_cross=3)
    x = xyz.astype(np.float64)
    want = set()
    for lv, n_l in enumerate(sizes):
        _, nb = cKDTree(x[:n_l]).query(x[:n_l], 7)
        for i in range(n_l):
            for j in nb[i, 1:]:
                want |= {(i, int(j)), (int(j), i)}
        if lv:
            n0 = sizes[lv - 1]
            _, nb = cKDTree(x[:n0]).query(x[n0:n_l], 3)
            for t, i in enumerate(range(n0, n_l)):
                for j in nb[t]:
                    want |= {(i, int(j)), (int(j), i)}
    got = {(i, int(j)) for i in range(len(xyz)) for j in col[rp[i]:rp[i + 1]]}
    assert got == want
    assert np.all(np.diff(col[rp[0]:rp[1]]) > 0)
    # the CSC permutation lists every edge once, grouped by sender
    assert sorted(cperm.tolist()) == list(range(len(col)))
    recv = np.repeat(np.arange(len(xyz)), np.diff(rp))
    assert np.all(np.diff(col[cperm]) >= 0)
    assert np.array_equal(np.sort(recv[cperm][:cp[1]]), recv[cperm][:cp[1]])


def test_multiscale_single_level_is_knn_graph():
    xyz, _ = synth.nested_levels([400], 18)
    a = O.multiscale_graph(xyz, [400])
    b = O.symmetrise(O.knn(xyz, 6), 400)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_fourier_features_closed_form():
    """sin/cos of 2pi, 4pi, 8pi times each coordinate, sines first per frequency."""
    x = np.array([[0.0, 0.25, 0.125], [0.5, -0.25, 1.0]], np.float32)
    f = O.fourier_features(x, 3)
    assert f.shape == (2, 18)
    want0 = [0, 1, np.sin(np.pi / 4), 1, 0, np.cos(np.pi / 4),      # 2 pi
             0, 0, 1, 1, -1, 0,                                       # 4 pi
             0, 0, 0, 1, 1, -1]                                       # 8 pi
    np.testing.assert_allclose(f[0], want0, atol=1e-12)
    np.testing.assert_allclose(f[1, :6], [0, -1, 0, -1, 0, 1], atol=1e-12)
    assert O.fourier_features(x, 0).shape == (2, 0)
