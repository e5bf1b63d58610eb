"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module holds *no* arithmetic of the method (no kNN, no partitioning, no
message passing).  It only draws the workloads the paper's case study is shaped
like (Sec. IV-A/IV-C: uniform surface point clouds of a car body, 6 nearest
neighbours, smooth target fields, randomly initialised MLP weights) from fixed
seeds, so that both sides of every parity test consume identical arrays.

Every generator is a pure function of its arguments and a seed.  Point clouds
are float32 (the dtype the C-ABI takes).

Workload recipe (stated once here, repeated in the design notes):

* ``sphere_cloud(n, seed)``: ``n`` points uniform on the unit sphere (normal
  = position).
* ``car_body(n, seed, jitter)``: union of an ellipsoid (semi-axes 2.0, 0.9,
  0.6), a cabin box and a lower box, sampled uniformly by surface area; points
  falling strictly inside another primitive are rejected.  ``jitter`` scales
  each primitive dimension by a seeded factor in ``[1-jitter, 1+jitter]``.
  Points are emitted in Morton (Z-curve) order of their coordinates, the way a
  surface mesh file keeps neighbouring vertices close in memory.
* ``nested_levels(sizes, seed)``: one body cloud of ``sizes[-1]`` points whose
  prefixes of length ``sizes[l]`` are uniform subsets (Sec. III-C, each coarser
  cloud is a subset of the next finer one); Morton order is applied within
  each level increment so the prefix property holds.
* ``fourier_targets(xyz, seed, out)``: per output channel the sum of 8 modes
  ``a_m sin(2 pi f_m . x + phi_m)``, ``f_m ~ N(0, I)``, ``a_m ~ N(0, 1/8)``,
  ``phi_m ~ U[0, 2 pi)``.
* ``init_params(H, L, in_node, out, seed)``: flat float32 vector in the
  parameter layout of ``include/xmgn.h``; ``W ~ N(0, 1/fan_in)``,
  ``b ~ 0.1 N(0, 1/fan_in)``, ``gamma = 1``, ``beta = 0`` (or perturbed).
"""
from __future__ import annotations

import numpy as np

IN_EDGE = 4  # (x_j - x_i, |x_j - x_i|), Sec. II-E


# --------------------------------------------------------------------------
# point clouds
# --------------------------------------------------------------------------
def sphere_cloud(n: int, seed: int):
    """``n`` points uniform on the unit sphere; returns (xyz f32 [n,3], normals f32 [n,3])."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    xyz = v.astype(np.float32)
    return xyz, xyz.copy()


def _morton_order(xyz: np.ndarray) -> np.ndarray:
    lo = xyz.min(axis=0)
    span = np.maximum(xyz.max(axis=0) - lo, 1e-30)
    q = np.clip(((xyz - lo) / span * 1023.0).astype(np.int64), 0, 1023)
    code = np.zeros(len(xyz), np.int64)
    for b in range(10):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return np.argsort(code, kind="stable")


def _body_primitives(rng: np.random.Generator, jitter: float):
    s = 1.0 + jitter * (2.0 * rng.random(9) - 1.0) if jitter > 0 else np.ones(9)
    ell = ("ellipsoid", np.array([2.0 * s[0], 0.9 * s[1], 0.6 * s[2]]))
    cabin = ("box", np.array([-0.8 * s[3], -0.65 * s[4], 0.2]), np.array([0.7 * s[3], 0.65 * s[4], 0.2 + 0.7 * s[5]]))
    lower = ("box", np.array([-1.85 * s[6], -0.8 * s[7], -0.55 * s[8]]), np.array([1.85 * s[6], 0.8 * s[7], -0.1]))
    return [ell, cabin, lower]


def _area(prim) -> float:
    if prim[0] == "ellipsoid":
        a, b, c = prim[1]
        p = 1.6075  # Knud Thomsen's approximation (<= 1.1% error); only mixes primitives
        return 4.0 * np.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3.0) ** (1.0 / p)
    lo, hi = prim[1], prim[2]
    d = hi - lo
    return 2.0 * (d[0] * d[1] + d[0] * d[2] + d[1] * d[2])


def _sample_prim(rng, prim, m):
    if prim[0] == "ellipsoid":
        a, b, c = prim[1]
        out_p, out_n = [], []
        got = 0
        gmax = max(a * b, a * c, b * c)
        while got < m:
            u = rng.standard_normal((2 * m + 16, 3))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
            keep = rng.random(len(u)) < g / gmax
            u = u[keep]
            p = u * np.array([a, b, c])
            nrm = p / np.array([a * a, b * b, c * c])
            nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
            out_p.append(p)
            out_n.append(nrm)
            got += len(p)
        return np.concatenate(out_p)[:m], np.concatenate(out_n)[:m]
    lo, hi = prim[1], prim[2]
    d = hi - lo
    fa = np.array([d[1] * d[2], d[1] * d[2], d[0] * d[2], d[0] * d[2], d[0] * d[1], d[0] * d[1]])
    face = rng.choice(6, size=m, p=fa / fa.sum())
    p = lo + rng.random((m, 3)) * d
    nrm = np.zeros((m, 3))
    for f in range(6):
        ax, side = f // 2, f % 2
        sel = face == f
        p[sel, ax] = hi[ax] if side else lo[ax]
        nrm[sel, ax] = 1.0 if side else -1.0
    return p, nrm


def _inside(prim, p):
    if prim[0] == "ellipsoid":
        a, b, c = prim[1]
        return (p[:, 0] / a) ** 2 + (p[:, 1] / b) ** 2 + (p[:, 2] / c) ** 2 < 1.0 - 1e-9
    lo, hi = prim[1], prim[2]
    return np.all((p > lo + 1e-9) & (p < hi - 1e-9), axis=1)


def _raw_body(n: int, rng: np.random.Generator, jitter: float):
    prims = _body_primitives(rng, jitter)
    areas = np.array([_area(p) for p in prims])
    pts, nrms = [], []
    have = 0
    while have < n:
        m = int((n - have) * 1.6) + 64
        cnt = rng.multinomial(m, areas / areas.sum())
        for i, prim in enumerate(prims):
            if cnt[i] == 0:
                continue
            p, nr = _sample_prim(rng, prim, int(cnt[i]))
            ok = np.ones(len(p), bool)
            for j, other in enumerate(prims):
                if j != i:
                    ok &= ~_inside(other, p)
            pts.append(p[ok])
            nrms.append(nr[ok])
            have += int(ok.sum())
    p = np.concatenate(pts)
    nr = np.concatenate(nrms)
    perm = rng.permutation(len(p))[:n]  # uniform subset, random order
    return p[perm], nr[perm]


def car_body(n: int, seed: int, jitter: float = 0.0, morton: bool = True):
    """Car-like closed body surface cloud; returns (xyz f32 [n,3], unit normals f32 [n,3])."""
    rng = np.random.default_rng(seed)
    p, nr = _raw_body(n, rng, jitter)
    if morton:
        o = _morton_order(p)
        p, nr = p[o], nr[o]
    return p.astype(np.float32), nr.astype(np.float32)


def nested_levels(sizes, seed: int, jitter: float = 0.0):
    """Nested multi-resolution cloud: prefix ``[:sizes[l]]`` is level ``l``."""
    sizes = list(sizes)
    assert all(a < b for a, b in zip(sizes, sizes[1:]))
    rng = np.random.default_rng(seed)
    p, nr = _raw_body(sizes[-1], rng, jitter)
    order = []
    lo = 0
    for hi in sizes:
        seg = np.arange(lo, hi)
        order.append(seg[_morton_order(p[seg])])
        lo = hi
    o = np.concatenate(order)
    return p[o].astype(np.float32), nr[o].astype(np.float32)


def bfs_regions(row_ptr: np.ndarray, col: np.ndarray, n_regions: int, size_lo: float, size_hi: float,
                seed: int) -> np.ndarray:
    """Disjoint node regions grown breadth-first from seeded seed nodes.

    Region r has a log-uniform target size in [size_lo, size_hi]; it starts at
    a random unassigned node and takes unassigned nodes level by level of a
    breadth-first search, each level in ascending id, until the size is
    reached (or its component runs out).  Returns int32 [n]: region id, or -1
    for nodes outside every region.
    """
    rng = np.random.default_rng(seed)
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    part = np.full(n, -1, dtype=np.int32)
    sizes = np.round(np.exp(rng.uniform(np.log(size_lo), np.log(size_hi), n_regions))).astype(np.int64)
    deg = np.diff(row_ptr)
    for r in range(n_regions):
        free = np.nonzero(part < 0)[0]
        if len(free) == 0:
            break
        frontier = np.array([free[rng.integers(len(free))]], dtype=np.int64)
        part[frontier] = r
        taken = 1
        while taken < sizes[r] and len(frontier):
            starts = np.repeat(row_ptr[frontier], deg[frontier])
            offs = np.arange(len(starts)) - np.repeat(np.cumsum(deg[frontier]) - deg[frontier], deg[frontier])
            nb = np.unique(col[starts + offs])
            nb = nb[part[nb] < 0][: sizes[r] - taken]
            part[nb] = r
            taken += len(nb)
            frontier = nb
    return part


def node_inputs(xyz: np.ndarray, normals: np.ndarray) -> np.ndarray:
    """Six node input features: position and unit normal (Sec. IV-A)."""
    return np.concatenate([xyz, normals], axis=1).astype(np.float32)


def fourier_targets(xyz: np.ndarray, seed: int, out: int = 4, modes: int = 8) -> np.ndarray:
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((out, modes, 3))
    a = rng.standard_normal((out, modes)) * np.sqrt(1.0 / modes)
    phi = rng.random((out, modes)) * 2.0 * np.pi
    x = xyz.astype(np.float64)
    t = np.zeros((len(x), out))
    for c in range(out):
        for m in range(modes):
            t[:, c] += a[c, m] * np.sin(2.0 * np.pi * (x @ f[c, m]) + phi[c, m])
    return t.astype(np.float32)


# --------------------------------------------------------------------------
# parameters (layout documented in include/xmgn.h)
# --------------------------------------------------------------------------
def param_blocks(H: int, L: int, in_node: int, out: int):
    """List of (name, shape, kind, fan_in) in the packed order of the C-ABI."""
    blocks = []

    def mlp(prefix, fin, fout, ln):
        blocks.append((prefix + ".W1", (fin, H), "W", fin))
        blocks.append((prefix + ".b1", (H,), "b", fin))
        blocks.append((prefix + ".W2", (H, fout), "W", H))
        blocks.append((prefix + ".b2", (fout,), "b", H))
        if ln:
            blocks.append((prefix + ".gamma", (fout,), "g", 0))
            blocks.append((prefix + ".beta", (fout,), "be", 0))

    mlp("node_enc", in_node, H, True)
    mlp("edge_enc", IN_EDGE, H, True)
    for l in range(L):
        mlp(f"proc{l}.edge", 3 * H, H, True)
        mlp(f"proc{l}.node", 2 * H, H, True)
    mlp("dec", H, out, False)
    return blocks


def init_params(H: int, L: int, in_node: int, out: int, seed: int, perturb_ln: bool = False) -> np.ndarray:
    rng = np.random.default_rng(seed)
    chunks = []
    for _, shape, kind, fan_in in param_blocks(H, L, in_node, out):
        n = int(np.prod(shape))
        if kind == "W":
            v = rng.standard_normal(n) * np.sqrt(1.0 / fan_in)
        elif kind == "b":
            v = 0.1 * rng.standard_normal(n) * np.sqrt(1.0 / fan_in)
        elif kind == "g":
            v = 1.0 + 0.1 * rng.standard_normal(n) if perturb_ln else np.ones(n)
        else:
            v = 0.1 * rng.standard_normal(n) if perturb_ln else np.zeros(n)
        chunks.append(v)
    return np.concatenate(chunks).astype(np.float32)


def random_vector(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded N(0, scale^2) float32 vector (directions for derivative checks)."""
    return (np.random.default_rng(seed).standard_normal(n) * scale).astype(np.float32)
