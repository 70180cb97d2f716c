"""The benchmark's whole-run work model (the terms of Eq. 11-12: solve
columns, the per-group chain of sweeps, the segment-aligned batched sweeps and
the recombination's V y flops), against counts taken segment by segment from
the oracle's own transition spots, output assignment and Krylov dimensions."""
import numpy as np
import pytest

import bench
import gridgen
from oracle import rmatex_ref as R


def brute_counts(p, logs):
    t_out = R.output_times(p)
    cols, chain, vy = 0, 0, 0.0
    per_round = {}
    for k, lg in enumerate(logs):
        lts = R.local_transition_spots(p, k)
        outs = R.segment_outputs(lts, t_out)
        assert len(outs) == len(lg.m)
        own = 0
        for j, m in enumerate(lg.m):
            if m > 0:
                own += m + 2
                per_round.setdefault(j, []).append(m)
                vy += 2.0 * p.n * len(outs[j]) * m
        cols += own
        chain = max(chain, own)
    batched = sum(max(v) + 2 for v in per_round.values())
    return cols, chain, batched, vy / 1e9


@pytest.mark.parametrize("seed,templates", [(51, [3, 2, 4]), (52, [1, 5])])
def test_work_model_matches_segment_counts(seed, templates):
    p = gridgen.small_mesh(seed, nx=7, ny=6, layers=1, n_src=sum(templates) + 2,
                           group_templates=templates, t_end=0.4e-9, dt_out=10e-12)
    res = R.rmatex(p)
    m_seq = np.concatenate([np.asarray(lg.m, np.int32) for lg in res.logs])
    wm = bench.work_model(p, m_seq)
    cols, chain, batched, vy = brute_counts(p, res.logs)
    assert wm["solve_columns"] == cols
    assert wm["critical_path_sweeps"] == chain
    assert wm["batched_sweeps"] == batched
    assert wm["recombine_vy_gflop"] == pytest.approx(vy, rel=1e-12)
    assert cols > 0 and chain <= cols and batched >= chain


def test_work_model_rejects_a_sequence_of_the_wrong_length():
    p = gridgen.small_mesh(53, nx=5, ny=5, layers=1, n_src=3, group_templates=[3])
    n_seg = len(R.local_transition_spots(p, 0)) - 1
    with pytest.raises(ValueError):
        bench.work_model(p, np.ones(n_seg + 1, np.int32))
