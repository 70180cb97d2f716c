"""Writes the oracle's response of two groups of the four-layer 600x600 grid
(1.44M nodes, 256 groups) at their load nodes and 32 more, every output time, for the GPU parity
test of that grid.  Calls only the oracle (oracle/rmatex_ref.py): the FP64
SuperLU factors of C + gamma G and G take about ten minutes and 12 GB, too
long to repeat inside the GPU test suite.

    python tests/golden/make_mesh4x600x600_reference.py

Groups: the two with the fewest local transition spots (five, i.e. one
pulse template each).  Nodes: the load nodes of both groups (where their
response is largest), 16 drawn at random (seeded) and 16 on the central line
x = 300 of every layer, where the top separators of a nested-dissection
ordering of the mesh lie.  Stored: the node indices, the
group ids, the oracle's Krylov dimension per segment, and the load response
(without the constant pads' part) at those nodes for every output time.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gridgen  # noqa: E402
from oracle import rmatex_ref as R  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mesh4x600x600_2groups.npz")


def rows_for(p, groups):
    side = p.meta["nx"]
    plane = side * side
    rng = np.random.default_rng(1511045190)
    rand = rng.choice(p.n, 16, replace=False)
    line = [layer * plane + (side // 2) * side + y for layer in range(4)
            for y in (0, side // 4, side // 2, 3 * side // 4)]
    loads = p.src_node[np.isin(p.src_group, groups)]
    return np.unique(np.concatenate([loads, rand, line])).astype(np.int32)


def main():
    p = gridgen.config2()
    nb = np.array([len(R.local_transition_spots(p, k)) for k in range(p.n_groups)])
    groups = [int(g) for g in np.argsort(nb, kind="stable")[:2]]
    rows = rows_for(p, groups)
    fac = R.factorize(p)
    X, ms = [], []
    for g in groups:
        res = R.rmatex(p, fac=fac, groups=[g], nodes=rows, include_dc=False)
        X.append(res.X)
        ms.append(np.asarray(res.logs[0].m, np.int32))
    np.savez_compressed(OUT, rows=rows, groups=np.array(groups, np.int32), X=np.stack(X),
                        m=np.stack(ms))
    print(OUT, [x.shape for x in X], [list(m) for m in ms])


if __name__ == "__main__":
    main()
