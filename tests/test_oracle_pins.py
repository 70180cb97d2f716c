"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a closed form, a dense library routine on
a special case, a brute-force integrator, or an invariant of the linear ODE
(Eq. 1), chosen so that a plausible slip in the oracle (a sign in F or P, a
dropped A^{-2} b' term, a wrong H_m map, a transposed operand, a wrong
segment/output assignment) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import gridgen
from gridgen import Problem
from oracle import rmatex_ref as R


def one_node_problem(c=2e-13, g=5.0, vdd=1.0, pulses=((10e-12, 30e-12, 60e-12, -4e-3),),
                     t_end=100e-12, dt_out=1e-12, gamma=1e-11):
    """A single RC node tied to a pad (conductance g to Vdd) with triangular loads."""
    n_src = len(pulses)
    pwl_t = np.array([[a, b, cc] for (a, b, cc, _) in pulses]).ravel()
    pwl_v = np.array([[0.0, pk, 0.0] for (_, _, _, pk) in pulses]).ravel()
    return Problem(
        n=1, c=np.array([c]), g_rowptr=np.array([0, 1], np.int64), g_col=np.array([0], np.int32),
        g_val=np.array([g]), dc_inject=np.array([vdd * g]), src_node=np.zeros(n_src, np.int32),
        pwl_off=(np.arange(n_src + 1) * 3).astype(np.int32), pwl_t=pwl_t, pwl_v=pwl_v,
        src_group=np.zeros(n_src, np.int32), n_groups=1, vdd=vdd, t_end=t_end, dt_out=dt_out,
        gamma=gamma, tol=1e-7, m_max=20)


def one_node_closed_form(p, t_query):
    """x(t) for c x' = -g x + g Vdd + u(t), u piecewise linear: on a segment
    with u = u0 + s*tau the solution is x_p(tau) + (x0 - x_p(0)) exp(-g tau / c)
    with x_p(tau) = (g Vdd + u0 + s tau)/g - c s / g^2 (textbook, by hand)."""
    c, g, vdd = p.c[0], p.g_val[0], p.vdd
    knots = sorted(set([0.0, p.t_end] + [t for t in p.pwl_t if 0 < t < p.t_end]))

    def u(t):
        tot = 0.0
        for s in range(p.n_src):
            ts = p.pwl_t[3 * s:3 * s + 3]
            vs = p.pwl_v[3 * s:3 * s + 3]
            tot += float(np.interp(t, ts, vs))
        return tot

    x0 = (g * vdd + u(0.0)) / g
    vals = []
    for tq in t_query:
        x = x0
        t = 0.0
        for a, b in zip(knots[:-1], knots[1:]):
            if tq <= a:
                break
            end = min(b, tq)
            u0 = u(a)
            sl = (u(b) - u0) / (b - a)
            xp0 = (g * vdd + u0) / g - c * sl / g ** 2
            tau = end - a
            x = (g * vdd + u0 + sl * tau) / g - c * sl / g ** 2 + (x - xp0) * math.exp(-g * tau / c)
            t = end
        vals.append(x)
    return np.array(vals)


def test_single_rc_node_closed_form():
    p = one_node_problem()
    res = R.rmatex(p)
    t = R.output_times(p)
    ref = one_node_closed_form(p, t)
    err = np.abs(res.X[:, 0] - ref).max()
    assert err <= 1e-12 * p.vdd, err
    # one node: the shift-and-invert basis is exact at m = 1 and H = -g/c
    assert all(m in (0, 1) for m in res.logs[0].m)
    assert (p.vdd - ref).max() > 1e-4  # the load does something


def test_single_rc_node_two_overlapping_pulses_and_offset_grid():
    # breakpoints off the output grid and overlapping pulses in one group
    p = one_node_problem(pulses=((3.3e-12, 17.1e-12, 40.05e-12, -2e-3), (12.7e-12, 20e-12, 77.7e-12, -5e-3)),
                         c=7e-14, g=2.5, t_end=90e-12, dt_out=3e-12)
    res = R.rmatex(p)
    ref = one_node_closed_form(p, R.output_times(p))
    assert np.abs(res.X[:, 0] - ref).max() <= 1e-12


def test_single_node_rational_map_is_exact():
    # Htilde = c/(c + gamma g) gives H = (1 - 1/Htilde)/gamma = -g/c exactly (Eq. 9)
    c, g, gam = 3e-13, 4.0, 1e-11
    Ht = np.array([[c / (c + gam * g)]])
    assert abs(R.rational_H(Ht, gam)[0, 0] - (-g / c)) <= 1e-12 * g / c


def small_random_rc(seed, n=8, c_range=(1e-13, 1e-12)):
    """Dense-enough tiny RC: random spanning tree + extra branches, 2 pads."""
    rng = np.random.default_rng(seed)
    a, b = [], []
    for i in range(1, n):
        a.append(i)
        b.append(int(rng.integers(0, i)))
    for _ in range(n):
        i, j = rng.choice(n, 2, replace=False)
        a.append(int(i))
        b.append(int(j))
    g = rng.uniform(1.0, 10.0, len(a))
    pads = np.array([0, n - 1])
    G, dc = gridgen._assemble(n, np.array(a), np.array(b), g, pads, 0.05, 1.0)
    c = np.exp(rng.uniform(np.log(c_range[0]), np.log(c_range[1]), n))
    n_src = 4
    tpl = np.arange(n_src)
    start = rng.uniform(0, 60e-12, n_src)
    rise = rng.uniform(5e-12, 20e-12, n_src)
    fall = rng.uniform(5e-12, 20e-12, n_src)
    off, pt, pv = gridgen._sources_from_templates(tpl, start, rise, fall, rng.uniform(1e-3, 5e-3, n_src))
    return Problem(n=n, c=c, g_rowptr=G.indptr.astype(np.int64), g_col=G.indices.astype(np.int32),
                   g_val=G.data, dc_inject=dc, src_node=rng.integers(0, n, n_src).astype(np.int32),
                   pwl_off=off, pwl_t=pt, pwl_v=pv, src_group=np.array([0, 0, 1, 1], np.int32),
                   n_groups=2, t_end=120e-12, dt_out=2e-12, gamma=1e-11, tol=1e-15, m_max=20)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_happy_breakdown_equals_dense_augmented_exponential(seed):
    # with m_max >= n the Krylov space is the whole space: R-MATEX is exact
    p = small_random_rc(seed)
    res = R.rmatex(p)
    ref = R.dense_augmented(p, R.output_times(p))
    err = np.abs(res.X - ref).max()
    assert err <= 1e-11 * p.vdd, err
    assert (p.vdd - ref).max() > 1e-5


def test_krylov_truncation_within_tolerance_on_mesh():
    # <= 200 nodes: tol 1e-12 -> 1e-9 Vdd; tol 1e-7 -> error of order tol
    p = gridgen.small_mesh(3, nx=10, ny=10, layers=2, n_src=8, n_pads=4, t_end=0.3e-9,
                           dt_out=5e-12, c_range=(1e-14, 1e-12), group_templates=[4, 4])
    ref = R.dense_augmented(p, R.output_times(p))
    p.tol = 1e-12
    tight = R.rmatex(p)
    assert np.abs(tight.X - ref).max() <= 1e-9 * p.vdd
    p.tol = 1e-7
    loose = R.rmatex(p)
    e = np.abs(loose.X - ref).max()
    assert e <= 1e-5 * p.vdd and e > 0
    assert (p.vdd - ref).max() > 1e-4


def tr_grid_problem():
    """Tiny mesh whose breakpoints sit on the TR grid, mild stiffness."""
    p = gridgen.small_mesh(5, nx=5, ny=5, n_src=3, n_pads=2, t_end=60e-12, dt_out=5e-12,
                           c_range=(1e-12, 1e-11), r_range=(0.5, 1.0))
    p.pwl_t = np.array([5e-12, 15e-12, 30e-12, 10e-12, 20e-12, 45e-12, 0.0, 25e-12, 40e-12])
    p.tol = 1e-13
    return p


def test_trapezoidal_brute_force_converges_to_oracle():
    p = tr_grid_problem()
    res = R.rmatex(p)
    t_out = R.output_times(p)
    errs = []
    for h in (0.1e-12, 0.05e-12):
        ts, xs = R.trapezoidal(p, h)
        step = int(round(p.dt_out / h))
        errs.append(np.abs(xs[::step][: t_out.shape[0]] - res.X).max())
    # second order: halving h quarters the error
    assert 3.0 < errs[0] / errs[1] < 5.0, errs
    ts1, x1 = R.trapezoidal(p, 0.1e-12)
    ts2, x2 = R.trapezoidal(p, 0.05e-12)
    rich = (4 * x2[::100] - x1[::50]) / 3
    assert np.abs(rich[: t_out.shape[0]] - res.X).max() < 0.05 * errs[1]


def test_no_loads_gives_vdd_everywhere():
    p = gridgen.small_mesh(7, nx=8, ny=8, n_src=4)
    q = gridgen.with_sources(p, [], [0], [], [], [], 1)
    res = R.rmatex(q)
    assert np.abs(res.X - q.vdd).max() <= 1e-12 * q.vdd


def test_superposition_of_groups_equals_single_group():
    p = gridgen.small_mesh(8, nx=9, ny=9, n_src=9, group_templates=[3, 3, 3])
    p.tol = 1e-12
    split = R.rmatex(p)
    one = gridgen.with_sources(p, p.src_node, p.pwl_off, p.pwl_t, p.pwl_v,
                               np.zeros(p.n_src, np.int32), 1)
    one.tol = 1e-12
    joint = R.rmatex(one)
    assert np.abs(split.X - joint.X).max() <= 1e-9 * p.vdd
    assert len(split.logs) == 3 and len(joint.logs) == 1


def test_amplitude_linearity():
    p = gridgen.small_mesh(9, nx=8, ny=8, n_src=5)
    base = R.rmatex(p)
    replay = [log.m for log in base.logs]
    dbl = R.rmatex(p, replay_m=replay, amp_scale=np.full(p.n_src, 2.0))
    drop1 = p.vdd - base.X
    drop2 = p.vdd - dbl.X
    assert np.abs(drop2 - 2 * drop1).max() <= 1e-12 * p.vdd


def test_ramp_then_hold_reaches_dc_solution():
    p = gridgen.small_mesh(10, nx=7, ny=7, n_src=1, t_end=200e-12, dt_out=10e-12)
    # one source ramping to -5 mA over [10 ps, 30 ps] then holding
    q = gridgen.with_sources(p, [5], [0, 2], [10e-12, 30e-12], [0.0, -5e-3], [0], 1)
    res = R.rmatex(q)
    u = q.dc_inject.copy()
    u[5] += -5e-3
    dc = sp.linalg.spsolve(q.G().tocsc(), u)
    assert np.abs(res.X[-1] - dc).max() <= 1e-9 * q.vdd
    assert (q.vdd - dc).max() > 1e-4


def test_arnoldi_orthonormal_and_relation():
    p = gridgen.small_mesh(11, nx=10, ny=10, n_src=4, c_range=(1e-14, 1e-12))
    fac = R.factorize(p)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(p.n)
    b = R.arnoldi(fac, v, (5e-12,), 0.0, 8)
    V = b.V
    assert np.abs(V @ V.T - np.eye(b.m)).max() <= 1e-12
    # (C + gamma G)^{-1} C V_m = V_{m+1} Htilde  (Arnoldi relation, Sec. 3.3.2)
    lhs = np.stack([fac.solve_M(fac.c * V[i]) for i in range(b.m - 1)], axis=1)
    Vfull = V.T  # first m columns
    rhs = Vfull[:, : b.m] @ b.Ht[: b.m, : b.m - 1]
    assert np.abs(lhs - rhs).max() <= 1e-10 * np.abs(lhs).max()


def test_error_falls_as_step_grows_fig4_trend():
    # Fig. 4: with m fixed, |e^{hA}v - V_m e^{hH_m} e_1 ||v||| shrinks as h grows
    p = gridgen.small_mesh(12, nx=8, ny=8, n_src=2, c_range=(1e-14, 1e-12))
    fac = R.factorize(p)
    G = p.G().toarray()
    A = -G / p.c[:, None]
    v = np.random.default_rng(1).standard_normal(p.n)
    b = R.arnoldi(fac, v, (1e-12,), 0.0, 3, replay_m=3)
    errs = []
    for h in (0.5e-12, 5e-12, 50e-12):
        exact = sla.expm(h * A) @ v
        approx = b.V.T @ R.krylov_expv(b, h)
        errs.append(np.abs(exact - approx).max())
    assert errs[0] > errs[1] > errs[2], errs


def test_output_assignment_breakpoint_on_output_time():
    # an output that coincides with a breakpoint is produced by the segment that ends there
    lts = np.array([0.0, 20e-12, 50e-12])
    t = np.arange(6) * 10e-12
    segs = R.segment_outputs(lts, t)
    assert list(segs[0]) == [1, 2] and list(segs[1]) == [3, 4, 5]


def test_config0_statistics():
    p = gridgen.config0()
    res = R.rmatex(p)
    ms = [m for lg in res.logs for m in lg.m]
    assert len(ms) == len(R.local_transition_spots(p, 0)) - 1
    assert sum(lg.nonconv for lg in res.logs) == 0
    assert np.abs(res.x_dc - p.vdd).max() <= 1e-12
    assert 0 < (p.vdd - res.X).max() < 0.1


# ---------------------------------------------------------------------------
# The other two Krylov spaces of the circuit solver (Sec. 2.3 standard / MEXP,
# Sec. 3.3.1 inverted / I-MATEX), on the same skeleton
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["I", "S"])
def test_variant_single_rc_node_closed_form(variant):
    # one node: every Krylov space is the whole space at m = 1
    p = one_node_problem()
    res = R.rmatex(p, variant=variant)
    ref = one_node_closed_form(p, R.output_times(p))
    assert np.abs(res.X[:, 0] - ref).max() <= 1e-12 * p.vdd
    assert all(m in (0, 1) for m in res.logs[0].m)


@pytest.mark.parametrize("variant", ["I", "S"])
@pytest.mark.parametrize("seed", [0, 1])
def test_variant_happy_breakdown_equals_dense_augmented_exponential(variant, seed):
    p = small_random_rc(seed)
    res = R.rmatex(p, variant=variant)
    ref = R.dense_augmented(p, R.output_times(p))
    assert np.abs(res.X - ref).max() <= 1e-10 * p.vdd


def test_variant_maps_single_node():
    # Htilde of -A^{-1} = G^{-1} C is c/g, so H'^{-1} = -g/c; the standard
    # Hessenberg of A = -g/c is itself
    c, g = 3e-13, 4.0
    assert abs(R.krylov_H(np.array([[c / g]]), 1e-11, "I")[0, 0] - (-g / c)) <= 1e-12 * g / c
    assert R.krylov_H(np.array([[-g / c]]), 1e-11, "S")[0, 0] == -g / c


def test_variant_dimensions_follow_table1_trend():
    """Table 1: on a stiff RC mesh the standard space (MEXP) needs far larger
    bases than the inverted and rational ones for the same tolerance, and all
    three agree with the dense solution to about tol."""
    p = gridgen.small_mesh(31, nx=12, ny=12, layers=1, n_src=6, n_pads=4, t_end=0.3e-9,
                           dt_out=5e-12, c_range=(1e-15, 1e-12), group_templates=[6])
    p.m_max = 144
    ref = R.dense_augmented(p, R.output_times(p))
    stats = {}
    for v in ("R", "I", "S"):
        res = R.rmatex(p, variant=v)
        ms = [m for lg in res.logs for m in lg.m if m > 0]
        stats[v] = (np.mean(ms), max(ms), np.abs(res.X - ref).max())
    assert stats["S"][0] > 4 * stats["R"][0] and stats["S"][0] > 4 * stats["I"][0], stats
    for v in ("R", "I", "S"):
        assert stats[v][2] <= 1e-5 * p.vdd, stats
