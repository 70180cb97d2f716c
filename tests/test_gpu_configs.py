"""GPU parity on the uneven-group (config 2) and uneven-grid (config 4)
workloads: the same structure at sizes the oracle checks element by element,
and at full size the properties that hold at any size plus oracle parity on
sampled grids."""
import numpy as np
import pytest

import gridgen
from oracle import rmatex_ref as R

pytestmark = pytest.mark.gpu

TOL_V = 1e-9


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04519_gb300 import build
    build.build()
    from paper_1511_04519_gb300 import matex
    return matex


from tests.parity_util import check_adaptive, oracle_m  # noqa: E402,F401


def parity(M, p, rows=None, **kw):
    ref = R.rmatex(p, nodes=rows, fac=kw.pop("fac", None),
                   groups=None if kw.get("group_select", -1) < 0 else [kw["group_select"]],
                   include_dc=kw.get("include_dc", True))
    sim = M.Sim(p, rows=rows, **kw)
    X = sim.run().cpu().numpy()
    err = check_adaptive(p.meta.get("label", "case"), p, X, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, rows=rows, replay_m=m, **kw).run().cpu().numpy())
    return err, sim.stats


@pytest.mark.parametrize("seed", [0, 1])
def test_uneven_groups_four_layer_reduced(M, seed):
    # config-2 structure: 4 layers, per-layer R scaling, 0.02-ohm vias, groups
    # of 1..14 templates (4..43 breakpoints), all groups in one batched run
    p = gridgen.config2(seed=gridgen.SEED_BASE + 2 + 100 * seed, side=24, n_src=160,
                        n_groups=10, n_pads=12, max_tpl=14)
    err, stats = parity(M, p)
    assert err <= TOL_V * p.vdd
    assert stats.rounds >= 13 and stats.nonconv == 0


def test_uneven_grids_reduced(M):
    # config-4 structure: independent single-layer grids of different sizes
    for p in gridgen.config4(count=6, side_range=(12, 40)):
        err, _ = parity(M, p)
        assert err <= TOL_V * p.vdd


def test_uneven_grids_full_size_sampled(M):
    """Two grids of the 96 (side U[100,450]): the smallest and one more, full
    parity against the oracle on 31 sampled rows."""
    probs = gridgen.config4()
    order = np.argsort([p.n for p in probs])
    for idx in (order[0], order[len(order) // 4]):
        p = probs[idx]
        rows = np.sort(np.random.default_rng(int(idx)).choice(p.n, 31, replace=False)).astype(np.int32)
        err, stats = parity(M, p, rows=rows)
        assert err <= TOL_V * p.vdd
        assert stats.nonconv == 0


class _StoredOracle:
    """The oracle's result for one group as stored by the golden script."""

    def __init__(self, X, m):
        self.X = X
        self.logs = [type("Log", (), {"m": m})()]


def test_uneven_groups_full_size_against_stored_oracle(M):
    """The four-layer 600x600 grid (1.44M nodes; nnz(L) ~ 1.9e8, supernodes
    thousands of nodes wide): two groups against the oracle at their load
    nodes and 32 more (16 random, 16 on the central line of every layer, where
    the top separators lie), every output time, from tests/golden (written by
    the committed script beside it, which calls only the oracle); and the
    solves with both factors at 1, 8 and 64 right-hand sides against the
    sparse matrices."""
    import os
    import torch
    import scipy.sparse as sp
    ref = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                               "mesh4x600x600_2groups.npz"))
    p = gridgen.config2()
    rows = ref["rows"].astype(np.int32)
    for gi, g in enumerate(ref["groups"].tolist()):
        kw = dict(group_select=int(g), rows=rows, include_dc=False)
        sim = M.Sim(p, **kw)
        X = sim.run().cpu().numpy()
        stored = _StoredOracle(ref["X"][gi], ref["m"][gi])
        err = check_adaptive(f"mesh4x600x600_group{g}_32rows", p, X, sim.m_sequence(), stored,
                             lambda m: M.Sim(p, replay_m=m, **kw).run().cpu().numpy())
        assert err <= TOL_V * p.vdd
        assert np.abs(ref["X"][gi]).max() > 1e-4  # the group's loads move their own nodes
        if gi == 0:
            rng = np.random.default_rng(2)
            for which in (0, 1):
                A = sp.csr_matrix(sp.diags(p.c) + p.gamma * p.G()) if which == 0 else p.G()
                amax = abs(A).max()
                for ncols in (1, 8, 64):
                    b = rng.standard_normal((ncols, p.n))
                    x = sim.solve(which, torch.from_numpy(b).cuda()).cpu().numpy()
                    for q in range(ncols):
                        r = np.abs(A @ x[q] - b[q]).max()
                        assert r <= 1e-11 * max(np.abs(b[q]).max(), amax * np.abs(x[q]).max())
        sim.close()
        torch.cuda.empty_cache()


def test_uneven_groups_full_size_properties(M):
    """Config 2 at full size (1.44M nodes, 256 groups with 4..199 breakpoints):
    one batched run; every output finite, t = 0 equal to the DC state (Vdd),
    drops within (0, 0.5 V), no segment stopped unconverged; with every load
    removed the grid stays at Vdd."""
    import torch
    p = gridgen.config2()
    rows = np.sort(np.random.default_rng(0).choice(p.n, 64, replace=False)).astype(np.int32)
    sim = M.Sim(p, rows=rows)
    X = sim.run().cpu().numpy()
    assert np.isfinite(X).all()
    assert np.abs(X[0] - p.vdd).max() <= 1e-9
    drop = p.vdd - X
    assert drop.max() < 0.5 and drop.min() > -1e-6 and drop.max() > 1e-4
    assert sim.stats.nonconv == 0
    assert sim.stats.n_segments == sum(len(R.local_transition_spots(p, k)) - 1 for k in range(p.n_groups))
    sim.set_sources(np.zeros_like(p.pwl_v))
    X0 = sim.run().cpu().numpy()
    assert np.abs(X0 - p.vdd).max() <= 1e-12
    torch.cuda.empty_cache()
