"""Input generators (CPU): the breadth-first regions used for batched
partitions are disjoint, connected, of their drawn sizes, and reproducible."""
import numpy as np

from oracle import xmgn_oracle as O
from paper_2411_17164_gb300 import synth
from tests.helpers import case


def test_bfs_regions_disjoint_connected_sized():
    xyz, _ = case("body", 4000, 12)
    rp, col, _, _ = O.symmetrise(O.knn(xyz, 6), len(xyz))
    part = synth.bfs_regions(rp, col, 5, 50, 600, 3)
    rng = np.random.default_rng(3)
    want = np.round(np.exp(rng.uniform(np.log(50), np.log(600), 5))).astype(np.int64)
    np.testing.assert_array_equal(np.bincount(part[part >= 0], minlength=5), want)
    np.testing.assert_array_equal(part, synth.bfs_regions(rp, col, 5, 50, 600, 3))
    for r in range(5):  # each region is one connected piece of the graph
        members = np.nonzero(part == r)[0]
        seen = {int(members[0])}
        stack = [int(members[0])]
        while stack:
            u = stack.pop()
            for v in col[rp[u]:rp[u + 1]]:
                if part[v] == r and int(v) not in seen:
                    seen.add(int(v))
                    stack.append(int(v))
        assert len(seen) == len(members)
