"""The wide supernodes' solve products on the tensor cores (error-free 6-bit
bf16 digit split, exact FP32 integer sums, FP64 result) against sparse
direct solves, against the FP64 level solves of the same factor, and, in a
whole run, against the FP64-solve run and the oracle.  On the bench grid the
whole runs differ by a few 1e-12 V (each solve's rounding carried through the
Krylov steps of 28 sweeps and 1,000 outputs), bounded here at 1e-11 Vdd.

Both paths sum the same products with different rounding: the split keeps
every digit down to 2^-54 of a row's and a column's largest entry, the order
of an FP64 dot product's rounding, so solutions agree to about 1e-13 relative
and whole runs to rounding, far below the 1e-9 Vdd parity bar.  Cases: the
bench grid (supernodes up to ~900 wide: several 448-term exact-sum windows,
ragged row tiles) at 1 to 64 right-hand sides, a three-layer grid with the
width threshold lowered to 32, and whole runs with graph replay.
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


@pytest.fixture(scope="module")
def cfg1():
    return gridgen.config1()


def _solves(M, p, sims, ncols_list, seed):
    import torch
    rng = np.random.default_rng(seed)
    on, off = sims
    for which in (0, 1):
        A = sp.csr_matrix(sp.diags(p.c) + p.gamma * p.G()) if which == 0 else p.G()
        for k in ncols_list:
            b = torch.from_numpy(rng.standard_normal((k, p.n))).cuda()
            x = on.solve(which, b).cpu().numpy()
            xf = off.solve(which, b).cpu().numpy()
            bn = b.cpu().numpy()
            for q in range(k):
                r = np.abs(A @ x[q] - bn[q]).max()
                assert r <= 1e-11 * max(np.abs(bn[q]).max(), np.abs(A).max() * np.abs(x[q]).max()), \
                    (which, k, q)
                assert np.abs(x[q] - xf[q]).max() <= 1e-12 * np.abs(xf[q]).max(), (which, k, q)


def test_bench_grid_solves_match_fp64_and_sparse_direct(M, cfg1):
    p = cfg1
    on = M.Sim(p, tc_solve="on", solve_mode=1, include_dc=False, rows=np.arange(4, dtype=np.int32))
    off = M.Sim(p, tc_solve="off", solve_mode=1, include_dc=False, rows=np.arange(4, dtype=np.int32))
    st = on.setup_stats()
    assert st["tc_solve_supernodes"] > 0 and st["tc_solve_min_cols"] == 1
    assert off.setup_stats()["tc_solve_supernodes"] == 0
    _solves(M, p, (on, off), (1, 5, 16, 64), 41)
    on.close()
    off.close()


def test_lower_width_threshold_on_three_layer_grid(M):
    p = gridgen.small_mesh(3, nx=40, ny=37, layers=3, n_src=12, group_templates=[3, 4, 5])
    on = M.Sim(p, tc_solve="on", tc_min_width=32, solve_mode=1, resident="off")
    off = M.Sim(p, tc_solve="off", solve_mode=1, resident="off")
    assert on.setup_stats()["tc_solve_supernodes"] > 0
    _solves(M, p, (on, off), (1, 3, 8, 33), 42)


def test_whole_run_matches_fp64_solves_and_oracle(M):
    p = gridgen.small_mesh(5, nx=40, ny=40, layers=2, n_src=40, group_templates=[2, 3, 1, 4] * 4,
                           t_end=0.6e-9, dt_out=5e-12)
    on = M.Sim(p, tc_solve="on", tc_min_width=32, solve_mode=1, resident="off")
    Xa = on.run().cpu().numpy()
    Xb = on.run().cpu().numpy()  # graph replay
    assert on.stats.graph_replay == 1
    assert on.setup_stats()["tc_solve_supernodes"] > 0
    off = M.Sim(p, tc_solve="off", solve_mode=1, resident="off", replay_m=on.m_sequence())
    Xf = off.run().cpu().numpy()
    assert np.abs(Xa - Xf).max() <= 1e-12 * p.vdd
    assert np.abs(Xb - Xa).max() <= 1e-12 * p.vdd
    ref = R.rmatex(p)
    err = check_adaptive("tc_solve_run", p, Xa, on.m_sequence(), ref,
                         lambda m: M.Sim(p, tc_solve="on", tc_min_width=32, solve_mode=1,
                                         resident="off", replay_m=m).run().cpu().numpy())
    assert err <= TOL_V * p.vdd


def test_bench_grid_run_matches_fp64_solves(M, cfg1):
    """The 180k-node, 64-group grid as the benchmark runs it, wide panels on
    the tensor cores against the FP64 solves with the same Krylov dimensions,
    at sampled rows of every output time."""
    import torch
    p = cfg1
    rows = np.sort(np.random.default_rng(7).choice(p.n, 40, replace=False)).astype(np.int32)
    on = M.Sim(p, tc_solve="on", rows=rows)
    Xa = on.run()
    on.run(Xa)
    assert on.stats.graph_replay == 1
    off = M.Sim(p, tc_solve="off", rows=rows, replay_m=on.m_sequence())
    Xf = off.run()
    # ~1e-13 relative per solve, carried through 28 sweeps and 1,000 outputs
    assert float((Xa - Xf).abs().max()) <= 1e-11 * p.vdd
    del Xa, Xf
    torch.cuda.empty_cache()
