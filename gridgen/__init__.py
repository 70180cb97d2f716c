"""Seeded synthetic RC power-grid problems (inputs only).

This module builds the circuit that the integrator is run on: the MNA matrices
of Eq. 1 (C diagonal node capacitances, G branch + pad conductances), the pad
Norton injections, and piecewise-linear (triangular pulse) current loads
grouped into "bump" groups (Sec. 3.1, grouping of sources that share
t_delay/t_rise/t_fall/t_width).  It holds none of the integrator's arithmetic:
both the oracle and the CUDA library consume its output, and nothing here
solves, factors or exponentiates anything.

The workloads stand in for the IBM power-grid benchmarks of Sec. 4, which are
not available: meshes, value distributions and source counts follow the
benchmark configurations listed in ``CONFIGS``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

SEED_BASE = 1511045190


@dataclass
class Problem:
    """One RC grid with its loads; every array is in original node order."""

    n: int
    c: np.ndarray            # float64[n], node capacitance (F); C = diag(c)
    g_rowptr: np.ndarray     # int64[n+1], CSR of G (symmetric, SPD with pads)
    g_col: np.ndarray        # int32[nnz]
    g_val: np.ndarray        # float64[nnz] (S)
    dc_inject: np.ndarray    # float64[n], constant pad injection Vdd/R_pad (A)
    src_node: np.ndarray     # int32[n_src], node each load draws from
    pwl_off: np.ndarray      # int32[n_src+1], offsets into pwl_t / pwl_v
    pwl_t: np.ndarray        # float64, breakpoint times (s), increasing per source
    pwl_v: np.ndarray        # float64, injected current at the breakpoints (A); loads < 0
    src_group: np.ndarray    # int32[n_src], bump group of each source
    n_groups: int
    vdd: float = 1.0
    t_end: float = 10e-9
    dt_out: float = 10e-12
    gamma: float = 1e-11
    tol: float = 1e-7
    m_max: int = 20
    observed: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    meta: dict = field(default_factory=dict)

    @property
    def n_src(self) -> int:
        return int(self.src_node.shape[0])

    @property
    def n_out(self) -> int:
        """Number of output times t_o = o*dt_out, o = 0..N."""
        return int(round(self.t_end / self.dt_out)) + 1

    def G(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.g_val, self.g_col, self.g_rowptr), shape=(self.n, self.n))


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def _assemble(n, a, b, g, pad_nodes, r_pad, vdd):
    """Stamp branch conductances g between nodes a,b and pads to ground."""
    rows = np.concatenate([a, b, a, b, pad_nodes])
    cols = np.concatenate([a, b, b, a, pad_nodes])
    vals = np.concatenate([g, g, -g, -g, np.full(pad_nodes.shape[0], 1.0 / r_pad)])
    G = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    G.sum_duplicates()
    G.sort_indices()
    dc = np.zeros(n)
    dc[pad_nodes] = vdd / r_pad
    return G, dc


def mesh_branches(layers, nx, ny, rng, r_lo, r_hi, layer_r_scale, via_r, via_every):
    """4-neighbour branches per layer plus vias between adjacent layers."""
    plane = nx * ny
    idx = np.arange(plane).reshape(nx, ny)
    a_list, b_list, g_list = [], [], []
    for layer in range(layers):
        base = layer * plane
        h_a = idx[:, :-1].ravel() + base
        h_b = idx[:, 1:].ravel() + base
        v_a = idx[:-1, :].ravel() + base
        v_b = idx[1:, :].ravel() + base
        la = np.concatenate([h_a, v_a])
        lb = np.concatenate([h_b, v_b])
        r = rng.uniform(r_lo, r_hi, la.shape[0]) * layer_r_scale[layer]
        a_list.append(la)
        b_list.append(lb)
        g_list.append(1.0 / r)
    if layers > 1:
        ii, jj = np.meshgrid(np.arange(0, nx, via_every), np.arange(0, ny, via_every), indexing="ij")
        via_cells = idx[ii.ravel(), jj.ravel()]
        for layer in range(layers - 1):
            a_list.append(via_cells + layer * plane)
            b_list.append(via_cells + (layer + 1) * plane)
            g_list.append(np.full(via_cells.shape[0], 1.0 / via_r))
    return np.concatenate(a_list), np.concatenate(b_list), np.concatenate(g_list)


def _pulse_templates(rng, count, start_hi=8e-9, tr=(10e-12, 100e-12), tf=(10e-12, 100e-12)):
    start = rng.uniform(0.0, start_hi, count)
    rise = rng.uniform(tr[0], tr[1], count)
    fall = rng.uniform(tf[0], tf[1], count)
    return start, rise, fall


def _sources_from_templates(src_tpl, start, rise, fall, peak):
    """Triangular pulse per source: 0 at start, -peak at start+rise, 0 after the fall."""
    n_src = src_tpl.shape[0]
    t = np.empty((n_src, 3))
    t[:, 0] = start[src_tpl]
    t[:, 1] = start[src_tpl] + rise[src_tpl]
    t[:, 2] = t[:, 1] + fall[src_tpl]
    v = np.zeros((n_src, 3))
    v[:, 1] = -peak
    off = (np.arange(n_src + 1) * 3).astype(np.int32)
    return off, t.ravel().copy(), v.ravel().copy()


def make_mesh_problem(*, seed, layers, nx, ny, r_range, c_range, n_pads, n_src,
                      group_templates, layer_r_scale=None, via_r=0.05, via_every=4,
                      r_pad=0.01, vdd=1.0, peak_range=(1e-3, 10e-3), n_observed=0,
                      t_end=10e-9, dt_out=10e-12, gamma=1e-11, tol=1e-7, m_max=20,
                      start_hi=8e-9, label=""):
    """Layered RC mesh with pads on the top layer and pulse loads on the bottom.

    ``group_templates`` is a list giving, per group, how many distinct pulse
    templates (start, rise, fall) it owns.  Every template gets at least one
    source; remaining sources go to uniformly drawn templates.  Sources of a
    template share its breakpoints but each has its own peak.
    """
    rng = np.random.default_rng(seed)
    plane = nx * ny
    n = layers * plane
    if layer_r_scale is None:
        layer_r_scale = [1.0] * layers
    a, b, g = mesh_branches(layers, nx, ny, rng, r_range[0], r_range[1], layer_r_scale, via_r, via_every)
    c = _loguniform(rng, c_range[0], c_range[1], n)
    top = (layers - 1) * plane
    pad_nodes = np.sort(rng.choice(plane, size=n_pads, replace=False) + top).astype(np.int64)
    G, dc = _assemble(n, a, b, g, pad_nodes, r_pad, vdd)

    group_templates = np.asarray(group_templates, dtype=np.int64)
    n_tpl = int(group_templates.sum())
    if n_tpl > n_src:
        raise ValueError("more pulse templates than sources")
    tpl_group = np.repeat(np.arange(group_templates.shape[0]), group_templates).astype(np.int32)
    start, rise, fall = _pulse_templates(rng, n_tpl, start_hi=start_hi)
    extra = rng.integers(0, n_tpl, n_src - n_tpl) if n_src > n_tpl else np.zeros(0, np.int64)
    src_tpl = np.concatenate([np.arange(n_tpl), extra]).astype(np.int64)
    src_node = rng.choice(plane, size=n_src, replace=False).astype(np.int32)  # bottom layer
    peak = rng.uniform(peak_range[0], peak_range[1], n_src)
    pwl_off, pwl_t, pwl_v = _sources_from_templates(src_tpl, start, rise, fall, peak)
    observed = np.sort(rng.choice(plane, size=n_observed, replace=False)).astype(np.int32) if n_observed else np.zeros(0, np.int32)
    return Problem(
        n=n, c=c, g_rowptr=G.indptr.astype(np.int64), g_col=G.indices.astype(np.int32),
        g_val=G.data.astype(np.float64), dc_inject=dc, src_node=src_node, pwl_off=pwl_off,
        pwl_t=pwl_t, pwl_v=pwl_v, src_group=tpl_group[src_tpl].astype(np.int32),
        n_groups=int(group_templates.shape[0]), vdd=vdd, t_end=t_end, dt_out=dt_out,
        gamma=gamma, tol=tol, m_max=m_max, observed=observed,
        meta=dict(label=label, seed=seed, layers=layers, nx=nx, ny=ny, n_pads=n_pads,
                  pad_nodes=pad_nodes, n_templates=n_tpl))


# ---------------------------------------------------------------------------
# The benchmark configurations (R-MATEX workloads shaped like Sec. 4's grids)
# ---------------------------------------------------------------------------

def config0(seed=SEED_BASE + 0):
    """32x32 single-layer mesh, 16 pads, 64 pulse loads each with its own
    template, all in one group (plain R-MATEX, one column)."""
    return make_mesh_problem(seed=seed, layers=1, nx=32, ny=32, r_range=(0.1, 1.0),
                             c_range=(1e-15, 1e-13), n_pads=16, n_src=64,
                             group_templates=[64], label="mesh32x32_1layer_64src_1group")


def config1(seed=SEED_BASE + 1, n_observed=0):
    """Two-layer 300x300 mesh (180k nodes), vias 0.05 ohm every 4th node,
    400 pads, 2000 loads in 64 single-template groups."""
    return make_mesh_problem(seed=seed, layers=2, nx=300, ny=300, r_range=(0.05, 0.5),
                             c_range=(1e-15, 1e-13), n_pads=400, n_src=2000,
                             group_templates=[1] * 64, via_r=0.05, n_observed=n_observed,
                             label="mesh2x300x300_2000src_64groups")


def config2(seed=SEED_BASE + 2, side=600, n_src=10000, n_groups=256, n_pads=2000, max_tpl=66):
    """Four-layer 600x600 mesh (1.44M nodes), per-layer R x1/x0.5/x0.25/x0.1,
    vias 0.02 ohm, 2000 pads, 10000 loads in 256 groups of 1..66 templates
    (4..199 breakpoints per group).  Smaller sides/counts give the same
    structure at sizes the oracle can check."""
    rng = np.random.default_rng(seed + 1000)
    d = rng.integers(1, max_tpl + 1, n_groups)
    while d.sum() > n_src:
        d = np.maximum(1, d - 1)
    return make_mesh_problem(seed=seed, layers=4, nx=side, ny=side, r_range=(0.05, 0.5),
                             layer_r_scale=[1.0, 0.5, 0.25, 0.1], c_range=(1e-15, 1e-12),
                             n_pads=n_pads, n_src=n_src, group_templates=d, via_r=0.02,
                             label=f"mesh4x{side}x{side}_{n_src}src_{n_groups}groups")


def config3(seed=SEED_BASE + 1):
    """The config-1 grid with 256 observed bottom-layer nodes (adjoint workload)."""
    p = config1(seed=seed, n_observed=256)
    p.meta["label"] = "mesh2x300x300_adjoint_256obs"
    return p


def config4(seed=SEED_BASE + 4, count=96, side_range=(100, 450)):
    """96 independent single-layer meshes with side U[100,450], config-0 value
    distributions, 8-64 loads in 4-16 groups each."""
    rng = np.random.default_rng(seed)
    probs = []
    for gidx in range(count):
        side = int(rng.integers(side_range[0], side_range[1] + 1))
        n_src = int(rng.integers(8, 65))
        n_groups = int(rng.integers(4, min(16, n_src) + 1))
        n_tpl = int(rng.integers(n_groups, n_src + 1))
        per_group = np.ones(n_groups, np.int64)
        per_group += np.bincount(rng.integers(0, n_groups, n_tpl - n_groups), minlength=n_groups)
        n_pads = max(16, (side * side * 16) // 1024)
        probs.append(make_mesh_problem(seed=seed * 1000 + gidx, layers=1, nx=side, ny=side,
                                       r_range=(0.1, 1.0), c_range=(1e-15, 1e-13),
                                       n_pads=n_pads, n_src=n_src, group_templates=per_group,
                                       label=f"mesh{side}x{side}_grid{gidx}"))
    return probs


def small_mesh(seed, nx=8, ny=8, layers=1, n_src=6, group_templates=None, n_pads=3,
               c_range=(1e-15, 1e-13), r_range=(0.1, 1.0), t_end=1e-9, dt_out=10e-12,
               start_hi=None, **kw):
    """Tiny mesh for brute-force checks (<= a few hundred nodes)."""
    if group_templates is None:
        group_templates = [n_src]
    return make_mesh_problem(seed=seed, layers=layers, nx=nx, ny=ny, r_range=r_range,
                             c_range=c_range, n_pads=n_pads, n_src=n_src,
                             group_templates=group_templates, t_end=t_end, dt_out=dt_out,
                             start_hi=start_hi if start_hi is not None else 0.8 * t_end,
                             label=f"small{layers}x{nx}x{ny}", **kw)


def with_sources(p: Problem, src_node, pwl_off, pwl_t, pwl_v, src_group, n_groups) -> Problem:
    """Copy of ``p`` with a different set of loads (for invariant checks)."""
    q = Problem(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.src_node = np.asarray(src_node, np.int32)
    q.pwl_off = np.asarray(pwl_off, np.int32)
    q.pwl_t = np.asarray(pwl_t, np.float64)
    q.pwl_v = np.asarray(pwl_v, np.float64)
    q.src_group = np.asarray(src_group, np.int32)
    q.n_groups = int(n_groups)
    q.meta = dict(p.meta)
    return q


CONFIGS = {0: config0, 1: config1, 2: config2, 3: config3, 4: config4}
