"""Tail skipping (tail_eps > 0).  Past the last output of a segment where the
coefficient vector's norm ||y||_2 exceeds eps/2, a group's term of an output
(Eq. 6 with -P) is taken without V y, whose entries are at most ||y||_2 for an
orthonormal basis; it is left out entirely when the -P term's bound
max|z - w| + L max|z'| is below eps/2 as well.  Each output entry then stays
within eps x (number of groups) of the exact run, and the exact run is what
the oracle checks."""
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


def bound(p, eps):
    return p.n_groups * eps * (1.0 + 1e-9) + TOL_SAME * p.vdd


def uneven_groups():
    return gridgen.config2(seed=gridgen.SEED_BASE + 2, side=24, n_src=160, n_groups=10,
                           n_pads=12, max_tpl=14)


def test_zero_eps_is_the_exact_run(M):
    p = uneven_groups()
    X = M.Sim(p).run().cpu().numpy()
    X0 = M.Sim(p, tail_eps=0.0).run().cpu().numpy()
    assert np.abs(X0 - X).max() <= TOL_SAME * p.vdd


@pytest.mark.parametrize("eps_vdd", [1e-12, 1e-6, 1e-3])
def test_within_bound_of_exact_run(M, eps_vdd):
    p = uneven_groups()
    eps = eps_vdd * p.vdd
    exact = M.Sim(p)
    X = exact.run().cpu().numpy()
    sim = M.Sim(p, tail_eps=eps)
    Xt = sim.run().cpu().numpy()
    assert np.array_equal(sim.m_sequence(), exact.m_sequence())
    d = np.abs(Xt - X).max()
    assert d <= bound(p, eps), (d, bound(p, eps))
    if eps_vdd >= 1e-6:
        assert d > 0.0          # terms were left out
    # the recorded graph replays the same shortened run
    Xr = sim.run().cpu().numpy()
    assert sim.stats.graph_replay == 1
    assert np.abs(Xr - Xt).max() <= TOL_SAME * p.vdd


def test_small_eps_keeps_oracle_parity(M):
    p = uneven_groups()
    ref = R.rmatex(p)
    sim = M.Sim(p, tail_eps=1e-12 * p.vdd)
    X = sim.run().cpu().numpy()
    err = check_adaptive("uneven_groups_tail_eps_1e-12", p, X, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, tail_eps=1e-12 * p.vdd, replay_m=m).run().cpu().numpy())
    assert err <= TOL_V * p.vdd


def test_bench_grid_sampled_rows(M):
    """The 180k-node, 64-group grid as the benchmark runs it (all groups, one
    batched run), 29 sampled rows: within 64 eps of the exact run, and a
    looser eps still within its bound."""
    p = gridgen.config1()
    rows = np.sort(np.random.default_rng(11).choice(p.n, 29, replace=False)).astype(np.int32)
    X = M.Sim(p, rows=rows).run().cpu().numpy()
    for eps_vdd in (1e-12, 1e-7):
        eps = eps_vdd * p.vdd
        Xt = M.Sim(p, rows=rows, tail_eps=eps).run().cpu().numpy()
        assert np.abs(Xt - X).max() <= bound(p, eps)


def test_invalid_tail_eps_rejected(M):
    p = gridgen.small_mesh(42, nx=5, ny=5, layers=1, n_src=3, group_templates=[3])
    for bad in (-1e-9, float("nan"), float("inf")):
        with pytest.raises(M.MatexError):
            M.Sim(p, tail_eps=bad)
    with pytest.raises(M.MatexError):
        M.Sim(p, tail_eps=1e-9, tape=True)
