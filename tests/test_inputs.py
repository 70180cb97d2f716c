"""The seeded synthetic inputs: each benchmark grid has the stated shape,
value ranges and source structure, and its G is the stamped conductance matrix
of an RC mesh with pads (symmetric, Kirchhoff row sums equal to the pad
conductances, positive definite)."""
import numpy as np
import pytest

import gridgen


def branch_values(p):
    """Off-diagonal conductances g of the branches (G holds -g there)."""
    G = p.G().tocoo()
    off = G.row != G.col
    return G.row[off], G.col[off], -G.data[off]


def check_stamped(p, r_pad=0.01):
    G = p.G()
    assert (G - G.T).nnz == 0                          # exactly symmetric
    assert np.all(np.diff(p.g_rowptr) > 0)
    # Kirchhoff: every branch adds +g to both diagonals and -g off them, so
    # G 1 is the pads' conductance to ground, and the pads inject Vdd / R_pad
    rs = G @ np.ones(p.n)
    pads = np.nonzero(p.dc_inject)[0]
    expect = np.zeros(p.n)
    expect[pads] = 1.0 / r_pad
    assert np.abs(rs - expect).max() <= 1e-12 * G.diagonal().max()
    assert np.allclose(p.dc_inject[pads], p.vdd / r_pad, rtol=0, atol=0)
    _, _, g = branch_values(p)
    assert np.all(g > 0)
    assert np.all(p.c > 0)


def check_sources(p, plane):
    assert p.pwl_off.shape[0] == p.n_src + 1 and np.all(np.diff(p.pwl_off) == 3)
    t = p.pwl_t.reshape(-1, 3)
    v = p.pwl_v.reshape(-1, 3)
    assert np.all(np.diff(t, axis=1) > 0)              # start < peak < end
    rise, fall = t[:, 1] - t[:, 0], t[:, 2] - t[:, 1]
    assert rise.min() >= 10e-12 and rise.max() <= 100e-12
    assert fall.min() >= 10e-12 and fall.max() <= 100e-12
    assert t[:, 0].min() >= 0.0 and t[:, 0].max() <= 8e-9
    assert np.all(v[:, 0] == 0) and np.all(v[:, 2] == 0)
    peak = -v[:, 1]                                    # loads draw current
    assert peak.min() >= 1e-3 and peak.max() <= 10e-3
    assert np.all(p.src_node < plane)                  # bottom layer
    assert np.unique(p.src_node).shape[0] == p.n_src
    assert p.src_group.min() == 0 and p.src_group.max() == p.n_groups - 1


def templates_per_group(p):
    t = p.pwl_t.reshape(-1, 3)
    return [np.unique(t[p.src_group == k], axis=0).shape[0] for k in range(p.n_groups)]


def test_config0_grid():
    p = gridgen.config0()
    assert p.n == 1024 and p.n_src == 64 and p.n_groups == 1
    assert (p.t_end, p.dt_out, p.gamma, p.tol, p.m_max) == (10e-9, 10e-12, 1e-11, 1e-7, 20)
    assert p.n_out == 1001
    assert p.g_col.shape[0] == 1024 + 2 * (2 * 32 * 31)   # diagonal + 4-neighbour branches
    assert np.count_nonzero(p.dc_inject) == 16
    check_stamped(p)
    check_sources(p, 1024)
    assert templates_per_group(p) == [64]              # every source its own template
    assert p.c.min() >= 1e-15 and p.c.max() <= 1e-13
    _, _, g = branch_values(p)
    assert g.min() >= 1.0 - 1e-12 and g.max() <= 10.0 + 1e-9   # R in [0.1, 1] ohm
    assert np.linalg.eigvalsh(p.G().toarray()).min() > 0


def test_config1_grid():
    p = gridgen.config1()
    plane = 300 * 300
    assert p.n == 2 * plane and p.n_src == 2000 and p.n_groups == 64
    vias = 75 * 75                                     # every 4th node in each direction
    assert p.g_col.shape[0] == p.n + 2 * (2 * 2 * 300 * 299 + vias)
    pads = np.nonzero(p.dc_inject)[0]
    assert pads.shape[0] == 400 and pads.min() >= plane   # top layer
    check_stamped(p)
    check_sources(p, plane)
    assert templates_per_group(p) == [1] * 64          # one pulse shape per group
    r, c, g = branch_values(p)
    via = (np.abs(r - c) == plane)
    assert np.count_nonzero(via) == 2 * vias and np.allclose(g[via], 1.0 / 0.05)
    assert g[~via].min() >= 2.0 - 1e-9 and g[~via].max() <= 20.0 + 1e-9   # R in [0.05, 0.5]


def test_config2_grid():
    p = gridgen.config2()
    plane = 600 * 600
    assert p.n == 4 * plane and p.n_src == 10000 and p.n_groups == 256
    check_stamped(p)
    check_sources(p, plane)
    d = np.asarray(templates_per_group(p))
    assert d.min() >= 1 and d.max() <= 66 and d.sum() <= 10000
    assert np.count_nonzero(p.dc_inject) == 2000
    r, c, g = branch_values(p)
    layer_r, layer_c = r // plane, c // plane
    via = layer_r != layer_c
    assert np.allclose(g[via], 1.0 / 0.02)
    for k, s in enumerate([1.0, 0.5, 0.25, 0.1]):      # per-layer resistance scale
        gk = g[~via & (layer_r == k)]
        assert gk.min() >= 1.0 / (0.5 * s) * (1 - 1e-12) and gk.max() <= 1.0 / (0.05 * s) * (1 + 1e-12)
    assert p.c.min() >= 1e-15 and p.c.max() <= 1e-12


def test_config3_observed_nodes():
    p, q = gridgen.config3(), gridgen.config1()
    assert p.observed.shape[0] == 256 and np.unique(p.observed).shape[0] == 256
    assert p.observed.max() < 300 * 300                # bottom layer
    for k in ("c", "g_val", "g_col", "pwl_t", "pwl_v", "src_node", "src_group"):
        assert np.array_equal(getattr(p, k), getattr(q, k)), k


def test_config4_grids():
    probs = gridgen.config4()
    assert len(probs) == 96
    for p in probs[:: 12]:
        side = p.meta["nx"]
        assert 100 <= side <= 450 and p.n == side * side
        assert 8 <= p.n_src <= 64 and 4 <= p.n_groups <= 16
        assert np.count_nonzero(p.dc_inject) == max(16, side * side * 16 // 1024)
        check_stamped(p)
        check_sources(p, p.n)


def test_inputs_are_seeded():
    a, b = gridgen.config0(), gridgen.config0()
    for k in ("c", "g_val", "pwl_t", "pwl_v", "src_node"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    c = gridgen.config0(seed=gridgen.SEED_BASE + 99)
    assert not np.array_equal(a.c, c.c)
