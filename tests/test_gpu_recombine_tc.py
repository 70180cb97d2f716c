"""The recombination's V y on the tensor cores (error-free 6-bit bf16 slices,
exact FP32 integer sums, FP64 result) against the FP64 FMA kernel and the
oracle.

Both paths compute the same sums of products; they differ by rounding, at
the level of an FP64 dot product (1e-15 relative to the largest term), far
below the 1e-9 Vdd parity bar.  Cases: node and output counts that are not
multiples of the 128 x 48 tiles; rounds of more than 448 basis vectors (two
exact-sum windows drained in turn); rounds of fewer than 16 basis vectors
(left to the FP64 kernel); and the bench grid against the oracle.
"""
import numpy as np
import pytest

import gridgen
from oracle import rmatex_ref as R
from tests.parity_util import check_adaptive

pytestmark = pytest.mark.gpu

TOL_V = 1e-9
TOL_SAME = 1e-13  # tensor-core vs FP64 recombination of the same run (V)


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04519_gb300 import build
    build.build()
    from paper_1511_04519_gb300 import matex
    return matex


def both_paths(M, p, **kw):
    a = M.Sim(p, resident="off", **kw)
    Xa = a.run().cpu().numpy()
    assert a.stats.tc_rounds > 0
    b = M.Sim(p, resident="off", recombine="fp64", replay_m=a.m_sequence(), **kw)
    Xb = b.run().cpu().numpy()
    assert b.stats.tc_rounds == 0
    return Xa, Xb, a


@pytest.mark.parametrize("seed", [0, 1])
def test_ragged_tiles_match_fp64_and_oracle(M, seed):
    # 37 x 29 x 2 = 2146 nodes (16 full tiles of 128 + 98), 201 outputs (4 tiles of 48 + 9)
    p = gridgen.small_mesh(40 + seed, nx=37, ny=29, layers=2, n_src=48,
                           group_templates=[2, 3, 1, 4, 2, 3, 1, 2, 3, 2] * 2, t_end=2e-9,
                           dt_out=10e-12)
    Xa, Xb, sim = both_paths(M, p)
    assert np.abs(Xa - Xb).max() <= TOL_SAME * p.vdd
    ref = R.rmatex(p)
    err = check_adaptive(f"tc_ragged_{seed}", p, Xa, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, resident="off", replay_m=m).run().cpu().numpy())
    assert err <= TOL_V * p.vdd


def test_more_than_one_exact_sum_window(M):
    """128 groups and a tolerance of 1e-11 V: rounds of several hundred basis
    vectors; more basis vectors in all than 448 per round, so some round
    exceeds 448 and drains its accumulators twice."""
    p = gridgen.small_mesh(44, nx=40, ny=40, layers=2, n_src=128, group_templates=[1] * 128,
                           t_end=0.5e-9, dt_out=5e-12, start_hi=0.05e-9)
    p.tol = 1e-11
    Xa, Xb, sim = both_paths(M, p)
    st = sim.stats
    assert st.sum_m > 448 * st.rounds, (st.sum_m, st.rounds)
    assert np.abs(Xa - Xb).max() <= TOL_SAME * p.vdd
    ref = R.rmatex(p)
    err = check_adaptive("tc_two_windows", p, Xa, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, resident="off", replay_m=m).run().cpu().numpy())
    assert err <= TOL_V * p.vdd


def test_small_rounds_and_one_group_at_a_time(M):
    """One group at a time: every round has a single column of a few basis
    vectors (below 16, the FP64 kernel's); batched, the tensor cores.  Both
    equal the FP64-only run."""
    p = gridgen.small_mesh(45, nx=20, ny=20, layers=1, n_src=12, group_templates=[2] * 6,
                           t_end=0.5e-9)
    sim = M.Sim(p, resident="off")
    Xb = sim.run().cpu().numpy()
    sim.one_group_at_a_time(True)
    Xs = sim.run().cpu().numpy()
    Xf = M.Sim(p, resident="off", recombine="fp64", replay_m=sim.m_sequence()).run().cpu().numpy()
    assert np.abs(Xb - Xf).max() <= TOL_SAME * p.vdd
    assert np.abs(Xs - Xf).max() <= TOL_SAME * p.vdd


def test_bench_grid_matches_fp64_recombination(M):
    """The 180k-node, 64-group grid as the benchmark runs it (graph replay),
    tensor-core recombination against the FP64 one on every node and output
    time."""
    import torch
    p = gridgen.config1()
    a = M.Sim(p, resident="off")
    Xa = a.run()
    a.run(Xa)
    # the long tails on the tensor cores; the rise and fall rounds (each column
    # holding a few outputs of a wide range) stay on the FP64 kernel
    assert a.stats.graph_replay == 1 and 1 <= a.stats.tc_rounds < a.stats.rounds
    b = M.Sim(p, resident="off", recombine="fp64", replay_m=a.m_sequence())
    Xb = b.run()
    diff = float((Xa - Xb).abs().max())
    assert diff <= TOL_SAME * p.vdd, diff
    del Xa, Xb
    torch.cuda.empty_cache()
