"""The single-column level kernels (one right-hand side: everything static
loaded before the previous level completes, one group of lanes per output
row or column) against sparse direct solves, against the batched level
kernels of the same factor, and in whole runs (R-MATEX with one group, the
trapezoidal baseline) against the batched path and the oracle.

Both kernels sum each row's products in their own order (the single-column
one over 2^k lanes by shuffles, the batched one over four lanes and column
chunks), so single solves agree to a few units in the last place of the
solution and whole runs to rounding carried through the Krylov steps.  Cases
span one-lane rows (narrow leaves packed 32 rows to a warp), 32-lane rows
with several trips (the 180k-node grid's 898-wide root and its ~1,200-row
separators), four-layer grids and the trapezoidal factor C + h/2 G.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
from oracle import rmatex_ref as R
from tests.parity_util import check_adaptive

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


def _check_solves(p, on, off, seed, reps=3):
    import torch
    rng = np.random.default_rng(seed)
    for which in (0, 1):
        A = sp.csr_matrix(sp.diags(p.c) + p.gamma * p.G()) if which == 0 else p.G()
        for _ in range(reps):
            b = torch.from_numpy(rng.standard_normal(p.n)).cuda()
            x = on.solve(which, b).cpu().numpy()
            xf = off.solve(which, b).cpu().numpy()
            bn = b.cpu().numpy()
            r = np.abs(A @ x - bn).max()
            assert r <= 1e-11 * max(np.abs(bn).max(), np.abs(A).max() * np.abs(x).max()), which
            assert np.abs(x - xf).max() <= 1e-12 * np.abs(xf).max(), which


@pytest.mark.parametrize("case", ["config0", "threelayer", "fourlayer"])
def test_single_column_solves_small_grids(M, case):
    if case == "config0":
        p = gridgen.config0()
    elif case == "threelayer":
        p = gridgen.small_mesh(3, nx=23, ny=17, layers=3, n_src=6)
    else:
        p = gridgen.config2(side=40, n_src=60, n_groups=4, n_pads=30, max_tpl=4)
    on = M.Sim(p, single_column="on", resident="off")
    off = M.Sim(p, single_column="off", resident="off")
    assert on.setup_stats()["single_column"] == 1
    assert off.setup_stats()["single_column"] == 0
    _check_solves(p, on, off, 51)


def test_single_column_solves_bench_grid(M):
    p = gridgen.config1()
    on = M.Sim(p, single_column="on", rows=np.arange(4, dtype=np.int32), include_dc=False)
    off = M.Sim(p, single_column="off", rows=np.arange(4, dtype=np.int32), include_dc=False)
    _check_solves(p, on, off, 52, reps=2)
    # the setup's tuner picks the single-column kernels on this grid by itself
    auto = M.Sim(p, rows=np.arange(4, dtype=np.int32), include_dc=False)
    assert auto.setup_stats()["single_column"] == 1
    t_auto = auto.time_solve(0, 1, reps=10)[0]
    t_off = off.time_solve(0, 1, reps=10)[0]
    assert t_auto < t_off, (t_auto, t_off)


def test_single_group_run_matches_batched_and_oracle(M):
    """One group: every Arnoldi solve and input solve has one column."""
    p = gridgen.small_mesh(7, nx=20, ny=18, layers=2, n_src=8, group_templates=[8],
                           t_end=0.5e-9, dt_out=5e-12)
    on = M.Sim(p, single_column="on", resident="off")
    Xa = on.run().cpu().numpy()
    Xb = on.run().cpu().numpy()  # graph replay
    assert on.stats.graph_replay == 1
    assert np.abs(Xb - Xa).max() <= 1e-12 * p.vdd
    off = M.Sim(p, single_column="off", resident="off", replay_m=on.m_sequence())
    Xo = off.run().cpu().numpy()
    assert np.abs(Xa - Xo).max() <= 1e-11 * p.vdd
    ref = R.rmatex(p)
    err = check_adaptive("single_column_run", p, Xa, on.m_sequence(), ref,
                         lambda m: M.Sim(p, single_column="on", resident="off",
                                         replay_m=m).run().cpu().numpy())
    assert err <= TOL_V * p.vdd


def test_trapezoidal_on_single_column_kernels(M):
    p = gridgen.small_mesh(21, nx=9, ny=8, layers=2, n_src=10, group_templates=[3, 3, 4],
                           t_end=0.4e-9, dt_out=10e-12)
    for sub in (1, 2):
        X, _ = M.Sim(p, single_column="on").tr_run(sub)
        Xo, _ = M.Sim(p, single_column="off").tr_run(sub)
        _, xs = R.trapezoidal(p, p.dt_out / sub)
        assert np.abs(X.cpu().numpy() - xs[::sub]).max() <= TOL_V * p.vdd
        assert np.abs(X.cpu().numpy() - Xo.cpu().numpy()).max() <= 1e-12 * p.vdd


def test_single_column_option_checked(M):
    p = gridgen.small_mesh(1, nx=9, ny=7, n_src=4)
    with pytest.raises(Exception):
        M.Sim(p, single_column=3)
