"""CUDA-graph replay of a run and batches of independent grids in one graph.

A context records its run as a CUDA graph after a plain run and replays it
while the device's active-column counts equal the recorded ones; otherwise it
redoes the run plainly and records again.  Replays and plain runs differ only
in the order of the FP64 atomic additions of the triangular solves, so they
agree to rounding (1e-12 Vdd here), far inside the 1e-9 Vdd parity bound and
far below the ~tol difference a changed Krylov dimension would make.
"""
import numpy as np
import pytest

import gridgen
from oracle import rmatex_ref as R
from tests.parity_util import check_adaptive  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_V = 1e-9
TOL_SAME = 1e-12


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04519_gb300 import build
    build.build()
    from paper_1511_04519_gb300 import matex
    return matex


def uneven_groups(seed=0):
    # several rounds, groups of different segment counts, varying m per column
    return gridgen.config2(seed=gridgen.SEED_BASE + 2 + 100 * seed, side=24, n_src=160,
                           n_groups=10, n_pads=12, max_tpl=14)


def test_replay_matches_plain_run_and_oracle(M):
    p = uneven_groups()
    sim = M.Sim(p, resident="off")
    X1 = sim.run().cpu().numpy()
    s1 = sim.stats.as_dict()
    assert s1["graph_replay"] == 0 and s1["graph_capture_ms"] > 0
    X2 = sim.run().cpu().numpy()
    s2 = sim.stats.as_dict()
    assert s2["graph_replay"] == 1
    for k in ("sum_m", "max_m", "n_segments", "krylov_segments", "sweeps_M", "sweeps_G",
              "solve_columns", "rounds", "nonconv"):
        assert s1[k] == s2[k], k
    assert np.abs(X2 - X1).max() <= TOL_SAME * p.vdd
    plain = M.Sim(p, resident="off", graph=False)
    X3 = plain.run().cpu().numpy()
    assert plain.stats.graph_replay == 0
    assert np.abs(X3 - X1).max() <= TOL_SAME * p.vdd
    ref = R.rmatex(p)
    err = check_adaptive("uneven_groups_graph_replay", p, X2, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, resident="off", replay_m=m).run().cpu().numpy())
    assert err <= TOL_V * p.vdd
    # a third run replays again
    X4 = sim.run().cpu().numpy()
    assert sim.stats.graph_replay == 1 and np.abs(X4 - X1).max() <= TOL_SAME * p.vdd


def test_changed_counts_fall_back_and_record_again(M):
    """Scaling every current by 1e-4 shrinks the residuals, so columns retire
    after fewer Arnoldi steps: the replay's guard sees other counts, the run is
    redone plainly, and the next run replays the new recording."""
    p = uneven_groups(1)
    sim = M.Sim(p, resident="off")
    sim.run()
    sim.run()
    assert sim.stats.graph_replay == 1
    m_before = sim.m_sequence().copy()
    scaled = np.asarray(p.pwl_v) * 1e-4
    sim.set_sources(scaled)
    Xa = sim.run().cpu().numpy()
    assert sim.stats.graph_replay == 0
    assert not np.array_equal(sim.m_sequence(), m_before)
    q = uneven_groups(1)
    q.pwl_v = scaled
    fresh = M.Sim(q, resident="off", graph=False)
    Xf = fresh.run().cpu().numpy()
    assert np.array_equal(fresh.m_sequence(), sim.m_sequence())
    assert np.abs(Xa - Xf).max() <= TOL_SAME * p.vdd
    Xb = sim.run().cpu().numpy()
    assert sim.stats.graph_replay == 1
    assert np.abs(Xb - Xf).max() <= TOL_SAME * p.vdd


def test_replay_follows_new_capacitances_and_sources(M):
    """With the Krylov dimensions fixed (replay), new capacitances and new
    source values change only buffer contents: the graph keeps replaying and
    matches a fresh context built with those values."""
    p = uneven_groups()
    per_group = [list(lg.m) for lg in R.rmatex(p).logs]
    ms = np.concatenate([np.asarray(m, np.int32) for m in per_group])
    sim = M.Sim(p, resident="off", replay_m=ms)
    sim.run()
    c2 = np.asarray(p.c) * np.random.default_rng(3).uniform(0.8, 1.25, p.n)
    v2 = np.asarray(p.pwl_v) * 1.5
    sim.set_caps(c2)
    sim.set_sources(v2)
    X = sim.run().cpu().numpy()
    assert sim.stats.graph_replay == 1
    q = uneven_groups()
    q.c = c2
    q.pwl_v = v2
    Xf = M.Sim(q, resident="off", replay_m=ms, graph=False).run().cpu().numpy()
    assert np.abs(X - Xf).max() <= TOL_SAME * p.vdd
    assert np.abs(X - R.rmatex(q, replay_m=per_group).X).max() <= TOL_V * p.vdd


def test_sources_breaking_the_zero_pattern_are_rejected(M):
    """Segments with no injection yet are skipped at setup; currents that
    would make one of them non-zero are refused and change nothing."""
    p = gridgen.small_mesh(11, nx=8, ny=7, layers=1, n_src=6, group_templates=[2, 2, 2],
                           t_end=0.3e-9, dt_out=10e-12)
    sim = M.Sim(p, resident="off")
    X0 = sim.run().cpu().numpy()
    bad = np.asarray(p.pwl_v).copy()
    first = np.asarray(p.pwl_off)[:-1]
    bad[first] = -1e-3          # every source now injects from t = 0
    with pytest.raises(M.MatexError):
        sim.set_sources(bad)
    X1 = sim.run().cpu().numpy()
    assert np.abs(X1 - X0).max() <= TOL_SAME * p.vdd


def test_batch_of_uneven_grids_matches_individual_runs(M):
    probs = gridgen.config4(count=6, side_range=(12, 40))
    sims = [M.Sim(p, resident="off") for p in probs]
    single = [s.run().cpu().numpy() for s in sims]
    batch = M.Batch(sims)
    outs, ms = batch.run()
    assert len(outs) == len(probs) and np.all(ms > 0)
    for p, s, x, X in zip(probs, sims, outs, single):
        assert s.stats.graph_replay == 1
        assert np.abs(x.cpu().numpy() - X).max() <= TOL_SAME * p.vdd
    # the oracle on two of the grids
    for i in (0, len(probs) - 1):
        ref = R.rmatex(probs[i])
        err = check_adaptive(f"uneven_grids_batch_grid{i}", probs[i], outs[i].cpu().numpy(),
                             sims[i].m_sequence(), ref,
                             lambda m: M.Sim(probs[i], resident="off", replay_m=m).run().cpu().numpy())
        assert err <= TOL_V * probs[i].vdd
    # one grid's counts change: only that grid is redone plainly
    sims[2].set_sources(np.asarray(probs[2].pwl_v) * 1e-4)
    outs2, _ = batch.run()
    assert sims[2].stats.graph_replay == 0
    assert all(s.stats.graph_replay == 1 for k, s in enumerate(sims) if k != 2)
    q = gridgen.config4(count=6, side_range=(12, 40))[2]
    q.pwl_v = np.asarray(q.pwl_v) * 1e-4
    Xq = M.Sim(q, resident="off", graph=False).run().cpu().numpy()
    assert np.abs(outs2[2].cpu().numpy() - Xq).max() <= TOL_SAME * q.vdd
    for k in (0, 1, 3, 4, 5):
        assert np.abs(outs2[k].cpu().numpy() - single[k]).max() <= TOL_SAME * probs[k].vdd
    # the rebuilt batch replays every grid again
    outs3, _ = batch.run()
    assert all(s.stats.graph_replay == 1 for s in sims)
    assert np.abs(outs3[2].cpu().numpy() - Xq).max() <= TOL_SAME * q.vdd
    batch.close()


def test_contexts_of_different_sizes_coexist(M):
    """Kernel launch limits are process-wide: a small context set up after a
    large one must not lower what the large one launches with (both plain and
    replayed runs of the large one still work, and so does the batch)."""
    big_p = gridgen.config1()
    rows = np.arange(0, big_p.n, 997, dtype=np.int32)
    big = M.Sim(big_p, resident="off", rows=rows, group_select=5, graph=False)
    X0 = big.run().cpu().numpy()
    small = M.Sim(gridgen.small_mesh(2, nx=6, ny=5, layers=1, n_src=4, group_templates=[2, 2],
                                     t_end=0.2e-9, dt_out=10e-12))
    Xs = small.run().cpu().numpy()
    for solve_mode in (0, 1):
        again = M.Sim(big_p, resident="off", rows=rows, group_select=5, solve_mode=solve_mode)
        tiny = M.Sim(gridgen.small_mesh(3, nx=5, ny=5, layers=1, n_src=3, group_templates=[3],
                                        t_end=0.2e-9, dt_out=10e-12), solve_mode=solve_mode)
        for _ in range(2):
            X1 = again.run().cpu().numpy()
            assert np.abs(X1 - X0).max() <= TOL_SAME * big_p.vdd
        tiny.run()
        batch = M.Batch([again, small, tiny])
        outs, _ = batch.run()
        assert np.abs(outs[0].cpu().numpy() - X0).max() <= TOL_SAME * big_p.vdd
        assert np.abs(outs[1].cpu().numpy() - Xs).max() <= TOL_SAME * big_p.vdd
        batch.close()
