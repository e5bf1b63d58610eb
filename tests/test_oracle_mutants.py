"""Planted mistakes in the oracle are caught by its pins.

Each case below is a plausible one-line error (a dropped term, a wrong sign
or index, a swapped operand, a wrong ordering rule) applied to a copy of the
oracle's source on the CPU; the copy is run through every pin of
tests/test_oracle.py, and at least one pin must fail.  The oracle itself is
never modified.
"""
import importlib.util
import inspect
import os
import types

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SRC = os.path.join(HERE, "..", "oracle", "xmgn_oracle.py")

# (name, text in the oracle, replacement)
MUTANTS = [
    # graph construction (Sec. III-B)
    ("lattice by truncation", "q = np.rint(x * scale)", "q = np.trunc(x * scale)"),
    ("kNN ties to the larger index", "order = np.lexsort((cand, d2[t, cand]))",
     "order = np.lexsort((-cand, d2[t, cand]))"),
    ("kNN keeps the point itself", "d2[np.arange(len(r)), r] = big", "d2[np.arange(len(r)), r] = 0"),
    ("no self-loop removal", "keep = r != s", "keep = r == r"),
    ("directed kNN relation, no union",
     "    r = np.concatenate([recv, send])\n    s = np.concatenate([send, recv])\n",
     "    r = recv.copy()\n    s = send.copy()\n"),
    ("cross-level links to one point only", "else knn_among(xyz, rows, sizes[lv - 1], k_cross, scale))",
     "else knn_among(xyz, rows, sizes[lv - 1], 1, scale))"),
    ("tree kNN never widens a tied candidate list", "done = (kth < dmax) | (mm >= nr)",
     "done = (kth <= dmax) | (mm >= nr)"),
    ("tree kNN keeps the point itself", "d2[cand == r[:, None]] = big", "d2[cand == r[:, None]] = 0"),
    ("tree kNN ties to the tree's order", "order = np.lexsort((cand, d2), axis=1)",
     "order = np.argsort(d2, axis=1, kind=\"stable\")"),
    # partitioning (Sec. III-A)
    ("RCB splits the shortest axis", "axis = int(np.argmax(ext))", "axis = int(np.argmin(ext))"),
    ("halo one hop short", "        for h in range(1, depth + 1):\n            if len(frontier) == 0:",
     "        for h in range(1, depth):\n            if len(frontier) == 0:"),
    ("RCB halves the points for any part count", "nl = (len(ids) * pl) // parts", "nl = len(ids) // 2"),
    ("halo BFS relabels visited nodes",
     "            new = nb[dist[nb] < 0]\n            dist[new] = h\n            frontier = new\n        halo = np.nonzero",
     "            new = nb[dist[nb] != 0]\n            dist[new] = h\n            frontier = new\n        halo = np.nonzero"),
    ("halo in id order, not (hop, id)", "halo = halo[np.lexsort((halo, dist[halo]))]", "halo = np.sort(halo)"),
    ("sampled neighbourhood one hop short", "    for h in range(1, limit + 1):", "    for h in range(1, limit):"),
    ("induced subgraph keeps the first sender only", "        nb = local[col[row_ptr[g]:row_ptr[g + 1]]]",
     "        nb = local[col[row_ptr[g]:row_ptr[g] + 1]]"),
    ("partition gradients not summed", "grad = gp if grad is None else grad + gp", "grad = gp"),
    # MLP pieces
    ("LayerNorm with unbiased variance", "var = ((v - mu) ** 2).mean(axis=1, keepdims=True)",
     "var = ((v - mu) ** 2).sum(axis=1, keepdims=True) / (v.shape[1] - 1)"),
    ("LayerNorm epsilon outside the root", "rstd = 1.0 / np.sqrt(var + eps)", "rstd = 1.0 / (np.sqrt(var) + eps)"),
    ("SiLU derivative is the sigmoid", "return s * (1.0 + z * (1.0 - s))", "return s"),
    ("LayerNorm backward without the mean term",
     "dxh - dxh.mean(axis=1, keepdims=True) - xh * (dxh * xh).mean(axis=1, keepdims=True)",
     "dxh - xh * (dxh * xh).mean(axis=1, keepdims=True)"),
    ("second weight gradient from the pre-activation", 'grads[pre + "W2"] += a1.T @ dz2',
     'grads[pre + "W2"] += z1.T @ dz2'),
    ("segmented sum skips each row's last entry", "for t in range(int(deg.max()) if n else 0):",
     "for t in range(int(deg.max()) - 1 if n else 0):"),
    ("first bias gradient dropped", 'grads[pre + "b1"] += dz1.sum(axis=0)', 'grads[pre + "b1"] += 0.0'),
    # model (eqs. 1-4) and loss
    ("edge inputs with receiver and sender swapped", "np.concatenate([h[recv], h[col], e], axis=1)",
     "np.concatenate([h[col], h[recv], e], axis=1)"),
    ("displacement sign", "d = x[send] - x[recv]", "d = x[recv] - x[send]"),
    ("edge residual dropped", "        e = e + m\n", "        e = m\n"),
    ("node residual dropped", "        h = h + u\n", "        h = u\n"),
    ("mean aggregation", "agg = segment_sum(m, row_ptr)",
     "agg = segment_sum(m, row_ptr) / np.maximum(np.diff(row_ptr), 1)[:, None]"),
    ("aggregation of updated edge states", "agg = segment_sum(m, row_ptr)", "agg = segment_sum(e, row_ptr)"),
    ("Fourier frequencies one octave low", "a = (2.0 ** (q + 1)) * np.pi * x", "a = (2.0 ** q) * np.pi * x"),
    ("loss normaliser without the output count", "denom = y.shape[1] * float(n_norm)", "denom = float(n_norm)"),
    ("halo rows in the loss", "diff = (y - t) * w", "diff = (y - t)"),
    # hand-written backward
    ("aggregation transpose dropped", "dm = de + dagg[recv]", "dm = de"),
    ("edge-state residual gradient dropped", "de = de + dx[:, 2 * H:]", "de = dx[:, 2 * H:]"),
    ("sender gradient sent to receivers", "scatter_sum_by(dx[:, H:2 * H], col, n)",
     "scatter_sum_by(dx[:, H:2 * H], recv, n)"),
    ("node residual gradient dropped", "dh = dh + dx[:, :H]", "dh = dx[:, :H]"),
]


def _source():
    with open(ORACLE_SRC) as f:
        return f.read()


def _mutant_module(old, new):
    src = _source()
    assert src.count(old) == 1, f"mutation site not unique or missing: {old!r}"
    mod = types.ModuleType("xmgn_oracle_mutant")
    mod.__file__ = ORACLE_SRC
    exec(compile(src.replace(old, new), "xmgn_oracle_mutant", "exec"), mod.__dict__)
    return mod


def _pins():
    """A private copy of the pin module, whose oracle handle can be swapped."""
    spec = importlib.util.spec_from_file_location("oracle_pins_under_mutation", os.path.join(HERE, "test_oracle.py"))
    pins = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(pins)
    return pins


def _calls(fn):
    """Argument sets of a pin (its parametrize marks, else none)."""
    marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    if not marks:
        return [()]
    names, values = marks[0].args[0], marks[0].args[1]
    assert "," not in names
    return [(v,) for v in values]


def _failing_pins(pins):
    failed = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_") or fn.__module__ != pins.__name__:
            continue
        for args in _calls(fn):
            try:
                fn(*args)
            except pytest.skip.Exception:
                pass
            except Exception:
                failed.append(name)
                break
    return failed


def test_pins_pass_on_the_oracle():
    pins = _pins()
    assert _failing_pins(pins) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, old, new):
    pins = _pins()
    pins.O = _mutant_module(old, new)
    failed = _failing_pins(pins)
    assert failed, f"no pin catches: {name}"
