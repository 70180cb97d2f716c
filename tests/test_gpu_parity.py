"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar: max node-voltage error <= 1e-9 * Vdd.  When the
adaptive Krylov dimension picked on the GPU differs from the oracle's on some
segment (a residual within rounding of tol), the run is repeated in replay
mode with the oracle's m sequence and must meet the bar there.
"""
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


from tests.parity_util import check_adaptive, oracle_m  # noqa: E402


def compare_run(M, p, ref=None, fac=None, case=None, **kw):
    """Run GPU (adaptive, then replay if m differs) and compare with the
    oracle; the adaptive run's m mismatches and error are bounded and
    recorded (tests/parity_util.py).  The batched path unless resident= is
    given (the resident rounds have their own file)."""
    kw.setdefault("resident", "off")
    if ref is None:
        ref = R.rmatex(p, fac=fac, groups=None if kw.get("group_select", -1) < 0 else [kw["group_select"]],
                       include_dc=kw.get("include_dc", True))
    sim = M.Sim(p, **kw)
    X = sim.run().cpu().numpy()
    m_gpu = sim.m_sequence()
    m_ref = oracle_m(ref)

    def replay(m):
        sim2 = M.Sim(p, replay_m=m, **kw)
        Xr = sim2.run().cpu().numpy()
        assert np.array_equal(sim2.m_sequence(), m)
        return Xr

    err = check_adaptive(case or p.meta.get("label", "case"), p, X, m_gpu, ref, replay)
    return err, X, ref, m_gpu, m_ref, sim.stats


@pytest.mark.parametrize("width", [0, 16])
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("case", ["small", "config0", "ragged3layer"])
def test_solve_matches_sparse_direct(M, which, case, width):
    import torch
    import scipy.sparse as sp
    if case == "small":
        p = gridgen.small_mesh(1, nx=12, ny=9, layers=2, n_src=4)
    elif case == "config0":
        p = gridgen.config0()
    else:
        p = gridgen.small_mesh(2, nx=37, ny=23, layers=3, n_src=3)
    sim = M.Sim(p, max_width=width)
    rng = np.random.default_rng(3)
    for ncols in (1, 3, 8, 13):
        b = rng.standard_normal((ncols, p.n))
        x = sim.solve(which, torch.from_numpy(b).cuda()).cpu().numpy()
        A = sp.csr_matrix(sp.diags(p.c) + p.gamma * p.G()) if which == 0 else p.G()
        for q in range(ncols):
            assert np.abs(A @ x[q] - b[q]).max() <= 1e-12 * np.abs(b[q]).max()


@pytest.mark.parametrize("which", [0, 1])
def test_chunked_level_solves_on_the_bench_grid(M, which):
    """The 180k-node grid's top supernodes (up to 898 wide) are wide enough
    for the level launches to split their reductions over several CTAs at
    small column counts (and over fewer at large ones).  Level-by-level
    solves of 1 to 64 right-hand sides against the sparse matrix (residual)
    and against the same solves without chunks (the allocation-free entry
    point runs them unchunked)."""
    import torch
    import scipy.sparse as sp
    p = gridgen.config1()
    sim = M.Sim(p, solve_mode=1)
    A = sp.csr_matrix(sp.diags(p.c) + p.gamma * p.G()) if which == 0 else p.G()
    rng = np.random.default_rng(21)
    for ncols in (1, 2, 5, 16, 64):
        b = torch.from_numpy(rng.standard_normal((ncols, p.n))).cuda()
        x = sim.solve(which, b)
        xu = torch.empty_like(b)
        M.matex_solve_noalloc(sim.ctx, which, ncols, b.data_ptr(), xu.data_ptr())
        torch.cuda.synchronize()
        xn, bn, xun = x.cpu().numpy(), b.cpu().numpy(), xu.cpu().numpy()
        for q in range(ncols):
            # residual at the scale of backward-stable solves: eps |A| |x| with
            # |A| ~ 200 S here (1e-11 leaves room; a wrong chunk sum is O(1))
            r = np.abs(A @ xn[q] - bn[q]).max()
            assert r <= 1e-11 * max(np.abs(bn[q]).max(), np.abs(A).max() * np.abs(xn[q]).max()), (ncols, q)
            assert np.abs(xn[q] - xun[q]).max() <= 1e-12 * np.abs(xun[q]).max(), (ncols, q)
    sim.close()


def test_expm_matches_scipy(M):
    import torch
    import scipy.linalg as sla
    p = gridgen.small_mesh(1, nx=4, ny=4, n_src=1)
    sim = M.Sim(p)
    rng = np.random.default_rng(5)
    for m in (1, 2, 5, 13, 20):
        A = rng.standard_normal((6, m, m))
        A[0] = np.diag(-np.logspace(0, 6, m))                 # stiff, diagonal
        A[1] = np.triu(rng.standard_normal((m, m)), -1) - 3 * np.eye(m)  # Hessenberg
        h = np.array([1e-3, 0.5, 1.0, 2.0, 30.0, 1e-6])
        E = M.expm(sim, torch.from_numpy(A).cuda(), torch.from_numpy(h).cuda()).cpu().numpy()
        for b in range(6):
            ref = sla.expm(h[b] * A[b])
            assert np.abs(E[b] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (m, b)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_small_meshes_match_oracle(M, seed):
    p = gridgen.small_mesh(seed, nx=9 + seed, ny=7, layers=1 + seed % 2, n_src=6,
                           group_templates=[2, 3, 1], t_end=0.4e-9, dt_out=5e-12)
    err, *_ = compare_run(M, p)
    assert err <= TOL_V * p.vdd


def test_config0_matches_oracle(M):
    p = gridgen.config0()
    err, X, ref, m_gpu, m_ref, stats = compare_run(M, p)
    assert err <= TOL_V * p.vdd
    assert X.shape == (1001, 1024)
    assert stats.n_segments == len(m_ref)
    # the adaptive decisions agree on all but a handful of borderline segments
    assert np.mean(m_gpu == m_ref) >= 0.95


def test_single_node_closed_form(M):
    from tests.test_oracle_pins import one_node_closed_form, one_node_problem
    p = one_node_problem()
    X = M.Sim(p).run().cpu().numpy()
    ref = one_node_closed_form(p, R.output_times(p))
    assert np.abs(X[:, 0] - ref).max() <= 1e-12


def test_no_sources_is_vdd(M):
    p = gridgen.small_mesh(5, nx=8, ny=8, n_src=3)
    q = gridgen.with_sources(p, [], [0], [], [], [], 1)
    X = M.Sim(q).run().cpu().numpy()
    assert np.abs(X - q.vdd).max() <= 1e-12


def test_sources_outside_window_and_breakpoint_on_output(M):
    p = gridgen.small_mesh(6, nx=6, ny=6, n_src=3, t_end=100e-12, dt_out=10e-12)
    # one pulse entirely after T, one with breakpoints exactly on output times, one before 0
    q = gridgen.with_sources(p, [1, 2, 3], [0, 3, 6, 9],
                             [200e-12, 210e-12, 230e-12, 20e-12, 40e-12, 60e-12, -50e-12, -30e-12, -5e-12],
                             [0, -1e-3, 0, 0, -2e-3, 0, 0, -3e-3, 0], [0, 1, 1], 2)
    err, *_ = compare_run(M, q)
    assert err <= TOL_V * q.vdd


def test_group_select_rows_and_no_dc(M):
    p = gridgen.small_mesh(7, nx=10, ny=10, n_src=6, group_templates=[3, 3])
    rows = np.array([0, 5, 17, 99, 42], np.int32)
    ref = R.rmatex(p, groups=[1], nodes=rows, include_dc=False)
    sim = M.Sim(p, group_select=1, rows=rows, include_dc=False)
    X = sim.run().cpu().numpy()
    assert X.shape == (ref.X.shape[0], 5)
    err = check_adaptive("group_select_rows", p, X, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, group_select=1, rows=rows, include_dc=False,
                                         replay_m=m).run().cpu().numpy())
    assert err <= TOL_V * p.vdd


@pytest.mark.parametrize("col_block", [1, 2, 4, 8])
def test_column_blocks_agree(M, col_block):
    p = gridgen.small_mesh(8, nx=20, ny=20, layers=2, n_src=24, group_templates=[2] * 12,
                           t_end=0.3e-9)
    base = M.Sim(p, col_block=1, resident="off").run().cpu().numpy()
    X = M.Sim(p, col_block=col_block, resident="off").run().cpu().numpy()
    assert np.abs(X - base).max() <= 1e-13


def test_one_group_at_a_time_matches_batched(M):
    p = gridgen.small_mesh(12, nx=25, ny=20, layers=2, n_src=30, group_templates=[3, 1, 4, 1, 5, 6],
                           t_end=0.4e-9)
    sim = M.Sim(p, resident="off")
    Xb = sim.run().cpu().numpy()
    mb = sim.m_sequence()
    sim.one_group_at_a_time(True)
    Xs = sim.run().cpu().numpy()
    assert np.array_equal(sim.m_sequence(), mb)
    assert np.abs(Xs - Xb).max() <= 1e-13


@pytest.mark.parametrize("mode", [0, 1])
def test_persistent_and_level_solves_agree(M, mode):
    p = gridgen.small_mesh(13, nx=30, ny=30, layers=2, n_src=20, group_templates=[5] * 4, t_end=0.3e-9)
    ref = R.rmatex(p)
    sim = M.Sim(p, solve_mode=mode, replay_m=oracle_m(ref), resident="off")
    X = sim.run().cpu().numpy()
    assert np.abs(X - ref.X).max() <= TOL_V * p.vdd


def test_bounded_wait_reports_timeout_and_context_recovers(M):
    import time
    p = gridgen.small_mesh(14, nx=12, ny=12, n_src=4)
    sim = M.Sim(p, solve_mode=0, resident="off")  # the hook acts on the persistent solve
    good = sim.run().cpu().numpy()
    M.matex_debug_inject_wait(sim.ctx, True)
    t0 = time.time()
    with pytest.raises(M.MatexError) as ei:
        sim.run()
    assert ei.value.status == 4  # MATEX_ERR_TIMEOUT
    assert time.time() - t0 < 30
    M.matex_debug_inject_wait(sim.ctx, False)
    again = sim.run().cpu().numpy()
    assert np.array_equal(again, good)


def test_autotuner_measures_both_modes(M):
    p = gridgen.small_mesh(15, nx=30, ny=30, layers=2, n_src=20, group_templates=[2] * 10)
    sim = M.Sim(p)
    tab = sim.autotune()
    assert [t["ncols"] for t in tab][:4] == [1, 2, 4, 8]
    for t in tab:
        assert t["mode"] in (0, 1) and t["persistent_ms"] > 0 and t["level_ms"] > 0
        # level launches unless the persistent one is at least 10 % faster
        assert t["mode"] == (0 if t["persistent_ms"] < 0.9 * t["level_ms"] else 1)


def test_m_max_one_and_replay(M):
    p = gridgen.small_mesh(9, nx=7, ny=7, n_src=4)
    p.m_max = 1
    ref = R.rmatex(p)
    X = M.Sim(p).run().cpu().numpy()
    assert np.abs(X - ref.X).max() <= TOL_V


def test_host_buffers_end_to_end(M):
    p = gridgen.small_mesh(10, nx=9, ny=9, n_src=5)
    sim = M.Sim(p)
    Xd = sim.run().cpu().numpy()
    Xh = sim.run_host()
    assert np.array_equal(Xd, Xh)
    # new source currents through the host path, against the oracle run at
    # those currents (replaying the oracle's Krylov dimensions where the
    # adaptive choice differs on a borderline segment)
    amp = np.random.default_rng(10).uniform(0.5, 2.0, p.n_src)
    src_of = np.repeat(np.arange(p.n_src), np.diff(p.pwl_off))
    X2 = sim.run_host(p.pwl_v * amp[src_of])
    ref = R.rmatex(p, amp_scale=amp)
    err = check_adaptive("host_buffers_new_currents", p, X2, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, replay_m=m).run_host(p.pwl_v * amp[src_of]))
    assert err <= TOL_V * p.vdd
    # and back to the setup currents through the same call
    X1 = sim.run_host(p.pwl_v)
    assert np.abs(X1 - Xd).max() <= 1e-12 * p.vdd


@pytest.fixture(scope="module")
def cfg1():
    p = gridgen.config1()
    fac = R.factorize(p)
    return p, fac


@pytest.mark.parametrize("group", [0, 37, 63])
def test_config1_sampled_groups_match_oracle(M, cfg1, group):
    p, fac = cfg1
    err, *_ = compare_run(M, p, fac=fac, group_select=group, include_dc=False)
    assert err <= TOL_V * p.vdd


def test_full_run_is_superposition_of_groups(M):
    """The batched run (all groups as columns) equals x_dc plus the per-group
    runs; exercises column retirement and the in-kernel superposition."""
    p = gridgen.small_mesh(11, nx=40, ny=30, layers=2, n_src=40, group_templates=[1, 2, 3, 4] * 4,
                           t_end=0.5e-9)
    X = M.Sim(p).run().cpu().numpy()
    acc = M.Sim(gridgen.with_sources(p, [], [0], [], [], [], 1)).run().cpu().numpy()
    for g in range(p.n_groups):
        acc += M.Sim(p, group_select=g, include_dc=False).run().cpu().numpy()
    assert np.abs(X - acc).max() <= 1e-12


def test_config1_full_run_matches_oracle_on_sampled_rows(M, cfg1):
    """Full-size batched run (64 groups, 180k nodes), every output time, on 19
    sampled nodes against the whole oracle run on the same rows."""
    p, fac = cfg1
    rows = np.sort(np.random.default_rng(7).choice(p.n, 19, replace=False)).astype(np.int32)
    ref = R.rmatex(p, fac=fac, nodes=rows)
    sim = M.Sim(p, rows=rows)
    X = sim.run().cpu().numpy()
    err = check_adaptive("mesh2x300x300_64groups_19rows", p, X, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, rows=rows, replay_m=m).run().cpu().numpy())
    assert err <= TOL_V * p.vdd
    assert sim.stats.nonconv == 0
