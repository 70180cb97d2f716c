"""The oracle's ramp decomposition (Sec. 3.1 carried to single ramps) pinned
by what the mathematics fixes: the ramps add up to every source's PWL input
at any time in [0, T]; each ramp column has one segment that builds a basis,
starting from zero state; and the ramp-decomposed run equals the
group-decomposed run and the dense exact solution within the Krylov
tolerance (superposition of a linear system)."""
import numpy as np
import pytest

import gridgen
from oracle import rmatex_ref as R


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ramps_reproduce_every_input(seed):
    p = gridgen.small_mesh(seed, nx=9, ny=8, n_src=9, group_templates=[2, 3, 4], t_end=0.5e-9,
                           dt_out=5e-12)
    # one source that starts before 0 and one still rising at T: ramps at 0 and
    # a starting value, and a breakpoint past T that contributes nothing
    t = np.asarray(p.pwl_t, np.float64).copy()
    t[0:3] = [-20e-12, 30e-12, 60e-12]
    t[3:6] = [0.45e-9, 0.48e-9, 0.6e-9]
    p.pwl_t = t
    q = R.ramp_decomposition(p)
    T = R.sim_end(p)
    for x in np.linspace(0.0, T, 401):
        a = R.full_input_vector(p, x)
        b = R.full_input_vector(q, x)
        assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max() + 1e-18, x
    # a starting value group exists (source 0 is non-zero at t = 0)
    assert any(np.all(q.pwl_t[q.pwl_off[s]:q.pwl_off[s + 1]] == [0.0]) for s in range(q.n_src))


def test_each_ramp_column_has_one_basis_segment():
    p = gridgen.small_mesh(3, nx=10, ny=9, layers=2, n_src=8, group_templates=[2, 3, 3],
                           t_end=0.4e-9, dt_out=5e-12)
    q = R.ramp_decomposition(p)
    res = R.rmatex(q)
    for lg in res.logs:
        assert np.count_nonzero(lg.m) <= 1
    # every breakpoint inside (0, T) of a group becomes one column
    T = R.sim_end(p)
    expect = sum(len([x for x in R.local_transition_spots(p, k) if 0.0 < x < T])
                 for k in range(p.n_groups))
    assert q.n_groups == expect


def test_ramp_run_equals_group_run_and_dense_solution():
    p = gridgen.small_mesh(4, nx=12, ny=10, layers=2, n_src=10, group_templates=[2, 3, 1, 4],
                           t_end=0.4e-9, dt_out=5e-12)
    p.tol = 1e-12
    q = R.ramp_decomposition(p)
    Xg = R.rmatex(p).X
    Xr = R.rmatex(q).X
    assert np.abs(Xg - Xr).max() <= 1e-11 * p.vdd
    Xe = R.dense_augmented(p, R.output_times(p))
    assert np.abs(Xe - Xr).max() <= 1e-9 * p.vdd
