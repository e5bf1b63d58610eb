"""FP64 CPU oracle for the X-MeshGraphNet message-passing path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg call it.  It shares no code with the CUDA library and does not import the
package.

It is a plain, slow, obviously-correct restatement of what the method
computes (arXiv 2411.17164):

* kNN graph construction (Sec. III-B "K-Nearest Neighbor Connectivity"):
  brute force over all pairs on the integer lattice ``q = rint(x * 2^21)``,
  squared distances exact in int64, ties broken by the smaller index, self
  excluded.  For clouds too large for brute force, ``knn_tree`` takes its
  candidates from a k-d tree (scipy) and applies the same exact rule.
* Symmetrised receiver-major CSR: the edge set of eq. (2)'s neighbourhoods
  ``N(i)``, made undirected by set union (no duplicates, no self loops).
* Partitioning (Sec. III-A "Graph Partitioning"): recursive coordinate
  bisection stands in for METIS; halo of depth equal to the number of
  message-passing layers, local ordering that keeps every receiver's
  summation order of the full graph.
* MeshGraphNet encode-process-decode, eqs. (1)-(4): message
  ``m_ij = phi_m(h_i, h_j, e_ij)``, sum aggregation ``m_i = sum_j m_ij``,
  node update ``h_i' = phi_u(h_i, m_i)``, L layers with distinct weights; each
  MLP is Linear-SiLU-Linear-LayerNorm, residuals on processor edge and node
  updates, decoder without LayerNorm.
* MSE loss over inner (non-halo) nodes only (Sec. III-D), global normaliser.
* Reverse-mode gradient written by hand (no autodiff library), and the
  partitioned training step whose summed partition gradients equal the
  full-graph gradient (Sec. III-A "Gradient Aggregation").

Every array is float64 except integer graph data.  numpy's matmul (a BLAS
call) is the only library primitive used for dense products; scipy's k-d
tree only proposes kNN candidates, which the exact rule then decides.
"""
from __future__ import annotations

import numpy as np

LATTICE_SCALE = 2.0 ** 21
LATTICE_LIMIT = 2 ** 24
LN_EPS = 1e-5
IN_EDGE = 4


# ===========================================================================
# Graph construction
# ===========================================================================
def quantize(xyz, scale: float = LATTICE_SCALE) -> np.ndarray:
    """Lattice coordinates q = rint(x * scale) (round half to even), int64.

    Raises ValueError if any |q| >= 2^24 (keeps squared distances exact)."""
    x = np.asarray(xyz, dtype=np.float32).astype(np.float64)
    q = np.rint(x * scale)
    if q.size and np.max(np.abs(q)) >= LATTICE_LIMIT:
        raise ValueError("coordinate outside the lattice range")
    return q.astype(np.int64)


def knn(xyz, k: int, scale: float = LATTICE_SCALE, rows=None, chunk: int = 64) -> np.ndarray:
    """k nearest other points of each point (Sec. III-B), by (d^2, index).

    ``rows`` restricts the query to a subset of points (each row is still
    searched against all N points).  Returns int32 [len(rows), k], nearest
    first."""
    q = quantize(xyz, scale)
    n = len(q)
    if k < 1 or n < k + 1:
        raise ValueError("need 1 <= k < N")
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    out = np.empty((len(rows), k), dtype=np.int32)
    big = np.iinfo(np.int64).max
    for s in range(0, len(rows), chunk):
        r = rows[s:s + chunk]
        d2 = np.zeros((len(r), n), dtype=np.int64)
        for a in range(3):
            d = q[r, a][:, None] - q[None, :, a]
            d2 += d * d
        d2[np.arange(len(r)), r] = big  # a point is not its own neighbour
        kth = np.partition(d2, k - 1, axis=1)[:, k - 1]
        for t in range(len(r)):
            cand = np.nonzero(d2[t] <= kth[t])[0]
            order = np.lexsort((cand, d2[t, cand]))  # primary d^2, secondary index
            out[s + t] = cand[order[:k]]
    return out


def knn_among(xyz, rows, n_ref: int, k: int, scale: float = LATTICE_SCALE) -> np.ndarray:
    """k nearest of the first ``n_ref`` points for each point in ``rows``
    (none of which is among them), by (d^2, index).  int32 [len(rows), k]."""
    q = quantize(xyz, scale)
    rows = np.asarray(rows, dtype=np.int64)
    if k < 1 or n_ref < k or (len(rows) and rows.min() < n_ref):
        raise ValueError("need k <= n_ref and query rows outside the reference prefix")
    out = np.empty((len(rows), k), dtype=np.int32)
    for t, i in enumerate(rows):
        d2 = ((q[:n_ref] - q[i]) ** 2).sum(axis=1)
        out[t] = np.lexsort((np.arange(n_ref), d2))[:k]
    return out


def knn_tree(xyz, k: int, scale: float = LATTICE_SCALE, n_ref: int | None = None, rows=None,
             chunk: int = 1 << 19) -> np.ndarray:
    """The result of ``knn`` (n_ref None: the k nearest other points of each
    row) or of ``knn_among`` (n_ref given: the k nearest of the first n_ref
    points, for query rows outside that prefix), for clouds too large for the
    brute-force search.

    A k-d tree (scipy cKDTree, a library search structure) over the lattice
    coordinates only proposes candidates; the choice is the rule of ``knn``:
    exact int64 squared distance, then the smaller index.  Lattice coordinates
    are integers below 2^24 in magnitude, so the tree's float64 squared
    distances are exact and it returns the m nearest points in exact order
    (up to ties).  Every point it leaves out is at least as far as the
    farthest candidate, so a row whose k-th choice is strictly nearer than
    that is complete; any other row (a tie that a lower-indexed, equally
    distant point outside the list could win) is asked again with twice the
    candidates, until it is complete or the list holds every reference point.
    Returns int32 [len(rows), k], nearest first."""
    from scipy.spatial import cKDTree
    q = quantize(xyz, scale)
    n = len(q)
    among = n_ref is not None
    if among:
        ref = q[:n_ref]
        rows = np.asarray(rows, dtype=np.int64)
        if k < 1 or n_ref < k or (len(rows) and rows.min() < n_ref):
            raise ValueError("need k <= n_ref and query rows outside the reference prefix")
    else:
        ref = q
        if k < 1 or n < k + 1:
            raise ValueError("need 1 <= k < N")
        rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    nr = len(ref)
    tree = cKDTree(ref.astype(np.float64))
    out = np.empty((len(rows), k), dtype=np.int32)
    big = np.iinfo(np.int64).max
    todo = np.arange(len(rows))
    m = k + (0 if among else 1) + 4
    while len(todo):
        mm = min(m, nr)
        again = []
        for s in range(0, len(todo), chunk):
            t = todo[s:s + chunk]
            r = rows[t]
            _, cand = tree.query(q[r].astype(np.float64), k=mm, workers=-1)
            cand = np.asarray(cand, dtype=np.int64).reshape(len(t), mm)
            d2 = ((ref[cand] - q[r][:, None, :]) ** 2).sum(axis=2)
            dmax = d2.max(axis=1)
            if not among:
                d2[cand == r[:, None]] = big  # a point is not its own neighbour
            order = np.lexsort((cand, d2), axis=1)  # primary d^2, secondary index
            kth = np.take_along_axis(d2, order[:, k - 1:k], axis=1)[:, 0]
            done = (kth < dmax) | (mm >= nr)
            out[t[done]] = np.take_along_axis(cand, order[:, :k], axis=1)[done]
            again.append(t[~done])
        todo = np.concatenate(again)
        m *= 2
    return out


def symmetrise(nbr: np.ndarray, n: int, csc: bool = True):
    """Undirected edge set of the kNN relation as receiver-major CSR.

    Edge (receiver i, sender j) exists iff j in kNN(i) or i in kNN(j).
    Returns row_ptr int64 [n+1], col int32 [E] (senders ascending within a
    row), csc_ptr int64 [n+1] and csc_perm int32 [E] (CSR positions of the
    edges listed sender-major, receivers ascending; both None if ``csc`` is
    false)."""
    nbr = np.asarray(nbr, dtype=np.int64)
    k = nbr.shape[1]
    return symmetrise_pairs(np.repeat(np.arange(n, dtype=np.int64), k), nbr.reshape(-1), n, csc)


def multiscale_graph(xyz, sizes, k: int = 6, k_cross: int = 3, scale: float = LATTICE_SCALE,
                     tree: bool = False):
    """Multi-scale graph (Sec. III-C): level l is the first sizes[l] points
    (each level contains the previous one); edges are the kNN relation within
    every level, plus a link from each point first present in level l >= 1 to
    its k_cross nearest points of level l-1; all symmetrised into one CSR (as
    ``symmetrise``).  ``tree`` takes the neighbours from ``knn_tree`` (same
    result) instead of the brute-force search."""
    sizes = [int(v) for v in sizes]
    if any(a >= b for a, b in zip(sizes, sizes[1:])) or sizes[-1] != len(xyz):
        raise ValueError("level sizes must increase and end at N")
    recv, send = [], []
    for lv, n_l in enumerate(sizes):
        nb = knn_tree(np.asarray(xyz)[:n_l], k, scale) if tree else knn(np.asarray(xyz)[:n_l], k, scale)
        recv.append(np.repeat(np.arange(n_l, dtype=np.int64), k))
        send.append(nb.reshape(-1).astype(np.int64))
        if lv > 0:
            rows = np.arange(sizes[lv - 1], n_l)
            nb = (knn_tree(xyz, k_cross, scale, n_ref=sizes[lv - 1], rows=rows) if tree
                  else knn_among(xyz, rows, sizes[lv - 1], k_cross, scale))
            recv.append(np.repeat(rows, k_cross))
            send.append(nb.reshape(-1).astype(np.int64))
    return symmetrise_pairs(np.concatenate(recv), np.concatenate(send), len(xyz))


def symmetrise_pairs(recv, send, n: int, csc: bool = True):
    """Receiver-major CSR of the undirected edge set {(i, j), (j, i)} over the
    given directed pairs, without duplicates or self loops (as ``symmetrise``)."""
    recv = np.asarray(recv, dtype=np.int64)
    send = np.asarray(send, dtype=np.int64)
    r = np.concatenate([recv, send])
    s = np.concatenate([send, recv])
    keep = r != s
    key = np.unique(r[keep] * n + s[keep])
    r, s = key // n, key % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=row_ptr[1:])
    if not csc:
        return row_ptr, s.astype(np.int32), None, None
    csc_perm = np.lexsort((r, s)).astype(np.int32)
    csc_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(s, minlength=n), out=csc_ptr[1:])
    return row_ptr, s.astype(np.int32), csc_ptr, csc_perm


def edge_receivers(row_ptr: np.ndarray) -> np.ndarray:
    n = len(row_ptr) - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))


def rcb(xyz, P: int, scale: float = LATTICE_SCALE) -> np.ndarray:
    """Recursive coordinate bisection into P parts (stand-in for METIS, Sec. III-A).

    A set of n points destined for P parts is split along the axis of largest
    lattice extent (first of x, y, z on ties); the first floor(n*floor(P/2)/P)
    points in (coordinate, index) order form the left set, which receives part
    ids [base, base+floor(P/2)); the rest recurse with the remaining ids."""
    q = quantize(xyz, scale)
    n = len(q)
    if P < 1 or P > n:
        raise ValueError("need 1 <= P <= N")
    part = np.empty(n, dtype=np.int32)

    def split(ids, parts, base):
        if parts == 1:
            part[ids] = base
            return
        sub = q[ids]
        ext = sub.max(axis=0) - sub.min(axis=0)
        axis = int(np.argmax(ext))
        order = np.lexsort((ids, sub[:, axis]))
        pl = parts // 2
        nl = (len(ids) * pl) // parts
        split(np.sort(ids[order[:nl]]), pl, base)
        split(np.sort(ids[order[nl:]]), parts - pl, base + pl)

    split(np.arange(n, dtype=np.int64), P, 0)
    return part


def halo_partition(row_ptr, col, part, P: int, depth: int):
    """Inner set plus ``depth``-hop halo of every part (Sec. III-A).

    Returns a list of dicts, one per part, with
      gid     int64 [n_p]   global ids: inner ascending, then halo by (hop, id)
      hop     int64 [n_p]   BFS distance from the inner set (0 = inner)
      n_inner int
      row_ptr int64 [n_p+1], col int64 [e_p]: induced subgraph, receiver-major
              in local order, senders in ascending *global* id within a row.
    """
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    part = np.asarray(part)
    n = len(row_ptr) - 1
    deg = np.diff(row_ptr)
    out = []
    for p in range(P):
        dist = np.full(n, -1, dtype=np.int64)
        inner = np.nonzero(part == p)[0]
        dist[inner] = 0
        frontier = inner
        for h in range(1, depth + 1):
            if len(frontier) == 0:
                break
            starts = np.repeat(row_ptr[frontier], deg[frontier])
            offs = np.arange(len(starts)) - np.repeat(np.cumsum(deg[frontier]) - deg[frontier], deg[frontier])
            nb = np.unique(col[starts + offs])
            new = nb[dist[nb] < 0]
            dist[new] = h
            frontier = new
        halo = np.nonzero(dist > 0)[0]
        halo = halo[np.lexsort((halo, dist[halo]))]
        gid = np.concatenate([inner, halo])
        local = np.full(n, -1, dtype=np.int64)
        local[gid] = np.arange(len(gid))
        lrow = [0]
        lcol = []
        for g in gid:
            nb = col[row_ptr[g]:row_ptr[g + 1]]
            nb = local[nb]
            nb = nb[nb >= 0]
            lcol.append(nb)
            lrow.append(lrow[-1] + len(nb))
        out.append(dict(gid=gid, hop=dist[gid], n_inner=len(inner),
                        row_ptr=np.asarray(lrow, dtype=np.int64),
                        col=np.concatenate(lcol) if lcol else np.zeros(0, np.int64)))
    return out


def bfs_hops(row_ptr, col, sources, limit: int) -> np.ndarray:
    """Hop distance (<= limit, else -1) from a source set; used for sampled parity."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    dist = np.full(n, -1, dtype=np.int64)
    src = np.unique(np.asarray(sources, dtype=np.int64))
    dist[src] = 0
    frontier = src
    for h in range(1, limit + 1):
        nb = np.unique(np.concatenate([col[row_ptr[v]:row_ptr[v + 1]] for v in frontier])) if len(frontier) else np.zeros(0, np.int64)
        new = nb[dist[nb] < 0]
        dist[new] = h
        frontier = new
    return dist


def induced_subgraph(row_ptr, col, gid):
    """Induced subgraph on the node list ``gid`` (local order = order of gid),
    senders kept in ascending global id within each row."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    local = np.full(n, -1, dtype=np.int64)
    local[np.asarray(gid)] = np.arange(len(gid))
    lrow = [0]
    lcol = []
    for g in gid:
        nb = local[col[row_ptr[g]:row_ptr[g + 1]]]
        nb = nb[nb >= 0]
        lcol.append(nb)
        lrow.append(lrow[-1] + len(nb))
    return np.asarray(lrow, dtype=np.int64), (np.concatenate(lcol) if lcol else np.zeros(0, np.int64))


# ===========================================================================
# Parameters
# ===========================================================================
def param_shapes(H: int, L: int, in_node: int, out: int):
    """Packed parameter order: node encoder, edge encoder, L x (edge MLP, node
    MLP), decoder.  Each MLP is W1 [in,H], b1 [H], W2 [H,out], b2 [out] and,
    where it ends in LayerNorm, gamma [out], beta [out]."""
    names = []

    def mlp(p, fin, fout, ln):
        names.extend([(p + "W1", (fin, H)), (p + "b1", (H,)), (p + "W2", (H, fout)), (p + "b2", (fout,))])
        if ln:
            names.extend([(p + "g", (fout,)), (p + "be", (fout,))])

    mlp("ne.", in_node, H, True)
    mlp("ee.", IN_EDGE, H, True)
    for l in range(L):
        mlp(f"e{l}.", 3 * H, H, True)
        mlp(f"n{l}.", 2 * H, H, True)
    mlp("d.", H, out, False)
    return names


def unpack(flat, H, L, in_node, out):
    flat = np.asarray(flat, dtype=np.float64)
    res, o = {}, 0
    for name, shape in param_shapes(H, L, in_node, out):
        sz = int(np.prod(shape))
        res[name] = flat[o:o + sz].reshape(shape)
        o += sz
    if o != len(flat):
        raise ValueError(f"parameter vector has {len(flat)} entries, layout needs {o}")
    return res


def pack(grads: dict, H, L, in_node, out) -> np.ndarray:
    return np.concatenate([np.asarray(grads[name], dtype=np.float64).reshape(-1)
                           for name, _ in param_shapes(H, L, in_node, out)])


def param_count(H, L, in_node, out) -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(H, L, in_node, out))


# ===========================================================================
# MLP pieces
# ===========================================================================
def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def layer_norm(v, g, be, eps=LN_EPS):
    """Per-row LayerNorm, biased variance (a per-element op: allowed by Sec. III-A)."""
    mu = v.mean(axis=1, keepdims=True)
    var = ((v - mu) ** 2).mean(axis=1, keepdims=True)
    rstd = 1.0 / np.sqrt(var + eps)
    xh = (v - mu) * rstd
    return xh * g + be, (xh, rstd)


def mlp_forward(x, p, pre, ln=True):
    z1 = x @ p[pre + "W1"] + p[pre + "b1"]
    a1 = silu(z1)
    z2 = a1 @ p[pre + "W2"] + p[pre + "b2"]
    if not ln:
        return z2, (x, z1, a1, None)
    y, lnc = layer_norm(z2, p[pre + "g"], p[pre + "be"])
    return y, (x, z1, a1, lnc)


def mlp_backward(dy, cache, p, pre, grads):
    x, z1, a1, lnc = cache
    if lnc is not None:
        xh, rstd = lnc
        g = p[pre + "g"]
        grads[pre + "g"] += (dy * xh).sum(axis=0)
        grads[pre + "be"] += dy.sum(axis=0)
        dxh = dy * g
        dz2 = rstd * (dxh - dxh.mean(axis=1, keepdims=True) - xh * (dxh * xh).mean(axis=1, keepdims=True))
    else:
        dz2 = dy
    grads[pre + "W2"] += a1.T @ dz2
    grads[pre + "b2"] += dz2.sum(axis=0)
    da1 = dz2 @ p[pre + "W2"].T
    dz1 = da1 * silu_grad(z1)
    grads[pre + "W1"] += x.T @ dz1
    grads[pre + "b1"] += dz1.sum(axis=0)
    return dz1 @ p[pre + "W1"].T


def segment_sum(vals, row_ptr):
    """sum over each CSR row, accumulated strictly in CSR order (eq. 2)."""
    n = len(row_ptr) - 1
    out = np.zeros((n, vals.shape[1]))
    deg = np.diff(row_ptr)
    start = row_ptr[:-1]
    for t in range(int(deg.max()) if n else 0):
        sel = np.nonzero(deg > t)[0]
        out[sel] += vals[start[sel] + t]
    return out


def scatter_sum_by(vals, index, n):
    """out[index[e]] += vals[e], accumulated in increasing e."""
    order = np.argsort(index, kind="stable")
    idx = index[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(idx, minlength=n), out=ptr[1:])
    return segment_sum(vals[order], ptr)


# ===========================================================================
# Model: encode - process - decode (eqs. 1-4)
# ===========================================================================
def fourier_features(xyz, F: int) -> np.ndarray:
    """Fourier features of the coordinates (Sec. IV-A, IV-D: frequencies
    2 pi, 4 pi, 8 pi for F = 3): for q < F, sin(2^(q+1) pi x_c) for the three
    coordinates, then cos of the same.  float64 [n, 6F]."""
    x = np.asarray(xyz, dtype=np.float32).astype(np.float64)
    out = []
    for q in range(F):
        a = (2.0 ** (q + 1)) * np.pi * x
        out += [np.sin(a), np.cos(a)]
    return np.concatenate(out, axis=1) if out else np.zeros((len(x), 0))


def edge_inputs(xyz, row_ptr, col):
    """(x_j - x_i, |x_j - x_i|) with j the sender, i the receiver (Sec. II-E)."""
    x = np.asarray(xyz, dtype=np.float32).astype(np.float64)
    recv = edge_receivers(row_ptr)
    send = np.asarray(col, dtype=np.int64)
    d = x[send] - x[recv]
    return np.concatenate([d, np.linalg.norm(d, axis=1, keepdims=True)], axis=1)


def forward(flat_params, dims, row_ptr, col, node_in, xyz, keep=False):
    """Encode-process-decode on one graph.

    dims = (H, L, in_node, out).  Returns y [n, out] and, if ``keep``, the
    cache needed by ``backward``."""
    H, L, in_node, out = dims
    p = unpack(flat_params, H, L, in_node, out)
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    recv = edge_receivers(row_ptr)
    h, c_ne = mlp_forward(np.asarray(node_in, np.float32).astype(np.float64), p, "ne.")
    e, c_ee = mlp_forward(edge_inputs(xyz, row_ptr, col), p, "ee.")
    caches = []
    for l in range(L):
        m, c_e = mlp_forward(np.concatenate([h[recv], h[col], e], axis=1), p, f"e{l}.")  # eq. 1
        e = e + m
        agg = segment_sum(m, row_ptr)                                                  # eq. 2
        u, c_n = mlp_forward(np.concatenate([h, agg], axis=1), p, f"n{l}.")              # eq. 3
        h = h + u
        caches.append((c_e, c_n))
    y, c_d = mlp_forward(h, p, "d.", ln=False)
    if not keep:
        return y
    return y, dict(p=p, dims=dims, recv=recv, col=col, row_ptr=row_ptr, c_ne=c_ne, c_ee=c_ee,
                   caches=caches, c_d=c_d, n=len(row_ptr) - 1)


def mse_loss(y, targets, mask, n_norm):
    """sum over masked (inner) nodes of squared error / (out * n_norm)."""
    t = np.asarray(targets, dtype=np.float32).astype(np.float64)
    w = np.asarray(mask, dtype=np.float64)[:, None]
    diff = (y - t) * w
    denom = y.shape[1] * float(n_norm)
    return float((diff * diff).sum() / denom), 2.0 * diff / denom


def backward(dy, cache):
    """Hand-written reverse mode through ``forward``; returns the flat gradient."""
    H, L, in_node, out = cache["dims"]
    p = cache["p"]
    grads = {k: np.zeros_like(v) for k, v in p.items()}
    recv, col, row_ptr, n = cache["recv"], cache["col"], cache["row_ptr"], cache["n"]
    dh = mlp_backward(dy, cache["c_d"], p, "d.", grads)
    de = np.zeros((len(col), H))
    for l in reversed(range(L)):
        c_e, c_n = cache["caches"][l]
        dx = mlp_backward(dh, c_n, p, f"n{l}.", grads)      # h' = h + phi_u([h, agg])
        dh = dh + dx[:, :H]
        dagg = dx[:, H:]
        dm = de + dagg[recv]                                # e' = e + m, agg_i = sum m_ij
        dx = mlp_backward(dm, c_e, p, f"e{l}.", grads)
        de = de + dx[:, 2 * H:]
        dh = dh + scatter_sum_by(dx[:, :H], recv, n) + scatter_sum_by(dx[:, H:2 * H], col, n)
    mlp_backward(de, cache["c_ee"], p, "ee.", grads)
    mlp_backward(dh, cache["c_ne"], p, "ne.", grads)
    return pack(grads, H, L, in_node, out)


def loss_and_grad(flat_params, dims, row_ptr, col, node_in, xyz, targets, mask=None, n_norm=None):
    """Full-graph training objective (Sec. IV-C MSE) and its parameter gradient."""
    n = len(row_ptr) - 1
    mask = np.ones(n) if mask is None else mask
    n_norm = n if n_norm is None else n_norm
    y, cache = forward(flat_params, dims, row_ptr, col, node_in, xyz, keep=True)
    loss, dy = mse_loss(y, targets, mask, n_norm)
    return loss, backward(dy, cache), y


# ===========================================================================
# Partitioned step (Sec. III-A, III-D)
# ===========================================================================
def partitioned_step(flat_params, dims, parts, node_in, xyz, targets, n_total, with_grad=True):
    """Run every halo partition independently; inner outputs assembled by
    global id (halo predictions discarded), loss over inner nodes only with
    the global normaliser, gradients summed over partitions in part order."""
    node_in = np.asarray(node_in)
    xyz = np.asarray(xyz)
    out = dims[3]
    y_full = np.zeros((n_total, out))
    loss = 0.0
    grad = None
    for pt in parts:
        gid = pt["gid"]
        mask = np.zeros(len(gid))
        mask[:pt["n_inner"]] = 1.0
        if with_grad:
            lp, gp, y = loss_and_grad(flat_params, dims, pt["row_ptr"], pt["col"], node_in[gid], xyz[gid],
                                      np.asarray(targets)[gid], mask, n_total)
            loss += lp
            grad = gp if grad is None else grad + gp
        else:
            y = forward(flat_params, dims, pt["row_ptr"], pt["col"], node_in[gid], xyz[gid])
        y_full[gid[:pt["n_inner"]]] = y[:pt["n_inner"]]
    return y_full, loss, grad
