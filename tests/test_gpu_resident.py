"""Resident rounds: on small grids one CTA runs a column's whole segment
(input solutions of Eq. 5/6, the Arnoldi process of Alg. 1 with the residual
test of Sec. 3.3.3, the output coefficients, the next state), its triangular
substitutions level by level in shared memory.

Checked against the oracle (1e-9 Vdd, with the adaptive-m bookkeeping of
tests/parity_util.py), against the batched path of the same problem with the
same Krylov dimensions (rounding only: both sum the same products in another
order), and bit for bit against itself (no atomics: a run, its graph replay
and the host-buffer run are identical).  Cases: the one-group grid of 192
sequential segments, multi-group meshes, quiescent segments, m_max = 1,
replay, group selection with output rows and no DC part, a single node
against its closed form, the inverted Krylov space, ramp columns, one group
at a time, batches of grids, and the size limits.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
from oracle import rmatex_ref as R
from tests.parity_util import check_adaptive, oracle_m

pytestmark = pytest.mark.gpu

TOL_V = 1e-9
TOL_SAME = 1e-12  # resident vs batched rounds of one problem, same m (V)


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04519_gb300 import build
    build.build()
    from paper_1511_04519_gb300 import matex
    return matex


def resident_vs_oracle(M, p, case, ref=None, **kw):
    """Resident run against the oracle and against the batched path with the
    resident run's Krylov dimensions; returns (X, sim)."""
    if ref is None:
        ref = R.rmatex(p, groups=None if kw.get("group_select", -1) < 0 else [kw["group_select"]],
                       nodes=kw.get("rows"), include_dc=kw.get("include_dc", True))
    sim = M.Sim(p, resident="on", **kw)
    X = sim.run().cpu().numpy()
    assert sim.stats.resident == 1
    m = sim.m_sequence()
    err = check_adaptive(case, p, X, m, ref,
                         lambda mm: M.Sim(p, resident="on", replay_m=mm, **kw).run().cpu().numpy())
    assert err <= TOL_V * p.vdd, (case, err)
    off = M.Sim(p, resident="off", replay_m=m, **kw)
    Xo = off.run().cpu().numpy()
    assert off.stats.resident == 0
    assert np.abs(X - Xo).max() <= TOL_SAME * p.vdd, case
    # the counters the host derives after a resident run match the batched run's
    assert sim.stats.solve_columns == off.stats.solve_columns
    assert sim.stats.sum_m == off.stats.sum_m
    # the resident run solves every record's z' and w ahead of the rounds in
    # two sweeps, where the batched run takes two per round
    assert sim.stats.sweeps_G in (off.stats.sweeps_G, off.stats.sweeps_G - 2 * off.stats.rounds + 2)
    return X, sim


@pytest.mark.parametrize("case", ["small", "config0", "ragged3layer", "twolayer"])
def test_resident_solve_matches_sparse_direct(M, case):
    import torch
    if case == "small":
        p = gridgen.small_mesh(1, nx=9, ny=7, n_src=4)
    elif case == "config0":
        p = gridgen.config0()
    elif case == "ragged3layer":
        p = gridgen.small_mesh(3, nx=23, ny=17, layers=3, n_src=6)
    else:  # 32 x 32 x 2 = 2048 nodes
        p = gridgen.small_mesh(11, nx=32, ny=32, layers=2, n_src=8, group_templates=[2, 2])
    sim = M.Sim(p, resident="on")
    rng = np.random.default_rng(31)
    for which in (0, 1):
        A = sp.csr_matrix(sp.diags(p.c) + p.gamma * p.G()) if which == 0 else p.G()
        b = torch.from_numpy(rng.standard_normal((3, p.n))).cuda()
        x = torch.empty_like(b)
        M.matex_solve_resident(sim.ctx, which, 3, b.data_ptr(), x.data_ptr())
        x2 = torch.empty_like(b)
        M.matex_solve_resident(sim.ctx, which, 3, b.data_ptr(), x2.data_ptr())
        torch.cuda.synchronize()
        xb = sim.solve(which, b).cpu().numpy()
        xn, bn = x.cpu().numpy(), b.cpu().numpy()
        assert np.array_equal(xn, x2.cpu().numpy())  # no atomics: reproducible
        for q in range(3):
            r = np.abs(A @ xn[q] - bn[q]).max()
            assert r <= 1e-11 * max(np.abs(bn[q]).max(), np.abs(A).max() * np.abs(xn[q]).max()), (which, q)
            assert np.abs(xn[q] - xb[q]).max() <= 1e-12 * np.abs(xb[q]).max(), (which, q)
    sim.close()


def test_config0_resident_matches_oracle_and_is_chosen(M):
    p = gridgen.config0()
    X, sim = resident_vs_oracle(M, p, "resident_config0")
    assert X.shape == (1001, 1024)
    # the setup's timing picks the resident rounds for this grid by itself,
    # and the run launches two kernels per segment round
    auto = M.Sim(p)
    auto.run()
    assert auto.stats.resident == 1, auto.setup_stats()
    assert auto.stats.kernel_launches <= 2 * auto.stats.rounds + 64


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_small_meshes_resident(M, seed):
    p = gridgen.small_mesh(seed, nx=9 + seed, ny=7, layers=1 + seed % 2, n_src=6,
                           group_templates=[2, 3, 1], t_end=0.4e-9, dt_out=5e-12)
    resident_vs_oracle(M, p, f"resident_small_{seed}")


def test_multi_group_mesh_resident(M):
    p = gridgen.small_mesh(20, nx=30, ny=25, layers=2, n_src=40, group_templates=[2, 3, 1, 4] * 3,
                           t_end=0.6e-9, dt_out=5e-12)
    resident_vs_oracle(M, p, "resident_12groups")


def test_quiescent_segments_and_breakpoints_on_outputs(M):
    p = gridgen.small_mesh(6, nx=6, ny=6, n_src=3, t_end=100e-12, dt_out=10e-12)
    # one pulse entirely after T, one with breakpoints exactly on output times, one before 0
    q = gridgen.with_sources(p, [1, 2, 3], [0, 3, 6, 9],
                             [200e-12, 210e-12, 230e-12, 20e-12, 40e-12, 60e-12, -50e-12, -30e-12, -5e-12],
                             [0, -1e-3, 0, 0, -2e-3, 0, 0, -3e-3, 0], [0, 1, 1], 2)
    resident_vs_oracle(M, q, "resident_outside_window")


def test_m_max_one_and_replay(M):
    p = gridgen.small_mesh(9, nx=7, ny=7, n_src=4)
    p.m_max = 1
    ref = R.rmatex(p)
    X = M.Sim(p, resident="on").run().cpu().numpy()
    assert np.abs(X - ref.X).max() <= TOL_V
    # replaying the oracle's dimensions of a normal run
    p2 = gridgen.small_mesh(9, nx=7, ny=7, n_src=4)
    ref2 = R.rmatex(p2)
    sim = M.Sim(p2, resident="on", replay_m=oracle_m(ref2))
    X2 = sim.run().cpu().numpy()
    assert np.array_equal(sim.m_sequence(), oracle_m(ref2))
    assert np.abs(X2 - ref2.X).max() <= TOL_V * p2.vdd


def test_group_select_rows_and_no_dc(M):
    p = gridgen.small_mesh(7, nx=10, ny=10, n_src=6, group_templates=[3, 3])
    rows = np.array([0, 5, 17, 99, 42], np.int32)
    X, _ = resident_vs_oracle(M, p, "resident_group_select_rows", group_select=1, rows=rows,
                              include_dc=False)
    assert X.shape[1] == 5


def test_single_node_closed_form(M):
    from tests.test_oracle_pins import one_node_closed_form, one_node_problem
    p = one_node_problem()
    sim = M.Sim(p, resident="on")
    X = sim.run().cpu().numpy()
    assert sim.stats.resident == 1
    ref = one_node_closed_form(p, R.output_times(p))
    assert np.abs(X[:, 0] - ref).max() <= 1e-12


def test_inverted_space_resident(M):
    p = gridgen.small_mesh(21, nx=16, ny=12, layers=2, n_src=10, group_templates=[2, 3],
                           t_end=0.5e-9, dt_out=5e-12)
    ref = R.rmatex(p, variant="I")
    resident_vs_oracle(M, p, "resident_inverted", ref=ref, krylov="I")


def test_ramp_columns_resident(M):
    p = gridgen.small_mesh(22, nx=12, ny=12, layers=2, n_src=12, group_templates=[2, 2, 3],
                           t_end=0.5e-9, dt_out=5e-12)
    sim = M.Sim(p, resident="on", decompose="ramps")
    Xr = sim.run().cpu().numpy()
    assert sim.stats.resident == 1
    off = M.Sim(p, resident="off", decompose="ramps", replay_m=sim.m_sequence())
    assert np.abs(Xr - off.run().cpu().numpy()).max() <= TOL_SAME * p.vdd
    ref = R.rmatex(p)
    assert np.abs(Xr - ref.X).max() <= max(TOL_V * p.vdd, 10 * p.tol)


def test_one_group_at_a_time_matches_batched(M):
    p = gridgen.small_mesh(12, nx=25, ny=20, layers=2, n_src=30, group_templates=[3, 1, 4, 1, 5, 6],
                           t_end=0.4e-9)
    sim = M.Sim(p, resident="on")
    Xb = sim.run().cpu().numpy()
    mb = sim.m_sequence()
    sim.one_group_at_a_time(True)
    Xs = sim.run().cpu().numpy()
    assert np.array_equal(sim.m_sequence(), mb)
    assert np.abs(Xs - Xb).max() <= 1e-13


@pytest.mark.parametrize("case", ["config0", "12groups"])
def test_input_solves_ahead_equal_inline_bit_for_bit(M, case):
    """Every segment's z' and w solved ahead of the rounds (one launch) or by
    each round kernel (resident = 3, the path when they do not fit memory):
    the same code in the same order, so the same bits, new currents too."""
    if case == "config0":
        p = gridgen.config0()
    else:
        p = gridgen.small_mesh(20, nx=30, ny=25, layers=2, n_src=40,
                               group_templates=[2, 3, 1, 4] * 3, t_end=0.6e-9, dt_out=5e-12)
    ahead = M.Sim(p, resident="on")
    inline = M.Sim(p, resident="on_inline_inputs")
    Xa = ahead.run().cpu().numpy()
    Xi = inline.run().cpu().numpy()
    assert ahead.stats.resident == 1 and inline.stats.resident == 1
    assert np.array_equal(Xa, Xi)
    assert np.array_equal(ahead.m_sequence(), inline.m_sequence())
    # the ahead launch is one more kernel per run
    assert ahead.stats.kernel_launches == inline.stats.kernel_launches + 1
    amp = np.random.default_rng(5).uniform(0.5, 2.0, p.n_src)
    src_of = np.repeat(np.arange(p.n_src), np.diff(p.pwl_off))
    assert np.array_equal(ahead.run_host(p.pwl_v * amp[src_of]), inline.run_host(p.pwl_v * amp[src_of]))


def test_graph_replay_and_host_buffers_are_bit_identical(M):
    p = gridgen.small_mesh(10, nx=20, ny=18, layers=2, n_src=9, group_templates=[3, 3, 2])
    sim = M.Sim(p, resident="on")
    X1 = sim.run().cpu().numpy()
    assert sim.stats.graph_replay == 0
    X2 = sim.run().cpu().numpy()
    assert sim.stats.graph_replay == 1
    assert np.array_equal(X1, X2)
    assert np.array_equal(sim.run_host(), X1)
    plain = M.Sim(p, resident="on", graph=False)
    assert np.array_equal(plain.run().cpu().numpy(), X1)
    # new currents through the host path: the replayed graph follows them
    amp = np.random.default_rng(3).uniform(0.5, 2.0, p.n_src)
    src_of = np.repeat(np.arange(p.n_src), np.diff(p.pwl_off))
    X3 = sim.run_host(p.pwl_v * amp[src_of])
    ref = R.rmatex(p, amp_scale=amp)
    err = check_adaptive("resident_new_currents", p, X3, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, resident="on", replay_m=m).run_host(p.pwl_v * amp[src_of]))
    assert err <= TOL_V * p.vdd


def test_batch_of_resident_grids(M):
    probs = gridgen.config4(count=4, side_range=(12, 40))
    sims = [M.Sim(p, resident="on") for p in probs]
    single = [s.run().cpu().numpy() for s in sims]
    batch = M.Batch(sims)
    outs, ms = batch.run()
    assert np.all(ms > 0)
    for p, s, x, X in zip(probs, sims, outs, single):
        assert s.stats.resident == 1 and s.stats.graph_replay == 1
        assert np.array_equal(x.cpu().numpy(), X)
    batch.close()


def test_two_layer_grid_and_limits(M):
    p = gridgen.small_mesh(11, nx=32, ny=32, layers=2, n_src=8, group_templates=[2, 2],
                           t_end=0.3e-9)
    resident_vs_oracle(M, p, "resident_2048_nodes")
    big = gridgen.small_mesh(11, nx=65, ny=64, layers=2, n_src=8, group_templates=[2, 2],
                             t_end=0.3e-9)
    assert big.n > 8192
    with pytest.raises(M.MatexError) as ei:
        M.Sim(big, resident="on")
    assert ei.value.status == 1  # MATEX_ERR_ARG
    s = M.Sim(big)  # auto: the batched path
    s.run()
    assert s.stats.resident == 0
    import torch
    b = torch.zeros(big.n, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MatexError) as ei:
        M.matex_solve_resident(s.ctx, 0, 1, b.data_ptr(), b.data_ptr())
    assert ei.value.status == 7  # MATEX_ERR_STATE
