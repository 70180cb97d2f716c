"""Ramp decomposition on the GPU (opts.decompose = 1): every group's input
split into single ramps inside matex_setup, every ramp a column of one
batched round, against the oracle's own ramp decomposition of the same
problem (oracle/rmatex_ref.py: ramp_decomposition), and against the
group-decomposed GPU run within the Krylov tolerance."""
import numpy as np
import pytest

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


def ramp_parity(M, p, case, rows=None):
    ref = R.rmatex(R.ramp_decomposition(p), nodes=rows)
    sim = M.Sim(p, resident="off", decompose="ramps", rows=rows)
    X = sim.run().cpu().numpy()
    err = check_adaptive(case, p, X, sim.m_sequence(), ref,
                         lambda m: M.Sim(p, resident="off", decompose="ramps", rows=rows,
                                         replay_m=m).run().cpu().numpy())
    return err, sim


@pytest.mark.parametrize("seed", [0, 1])
def test_small_meshes_ramps_match_oracle(M, seed):
    p = gridgen.small_mesh(30 + seed, nx=11, ny=9, layers=2, n_src=10,
                           group_templates=[2, 3, 1, 4], t_end=0.5e-9, dt_out=5e-12)
    err, sim = ramp_parity(M, p, f"ramps_small_{seed}")
    assert err <= TOL_V * p.vdd
    # one round: every ramp's basis is built in the same batched sweep
    assert sim.stats.rounds <= 2


def test_uneven_groups_four_layer_reduced_ramps(M):
    """Config-2 structure at a size the oracle checks: 4 layers, 10 groups of
    1..14 templates; as ramps, 100+ independent columns instead of 13+
    sequential segment rounds."""
    p = gridgen.config2(seed=gridgen.SEED_BASE + 2, side=24, n_src=160, n_groups=10, n_pads=12,
                        max_tpl=14)
    err, sim = ramp_parity(M, p, "ramps_mesh4x24x24")
    assert err <= TOL_V * p.vdd
    seg = M.Sim(p, resident="off")
    seg.run()
    assert sim.stats.rounds < seg.stats.rounds


def test_ramps_equal_groups_at_tight_tolerance(M):
    """Both decompositions of the same transient converge to the same
    solution: with tol = 1e-12 V they agree within 1e-9 Vdd."""
    p = gridgen.small_mesh(33, nx=30, ny=30, layers=2, n_src=24, group_templates=[2] * 12,
                           t_end=0.6e-9, dt_out=5e-12)
    p.tol = 1e-12
    Xg = M.Sim(p, resident="off").run().cpu().numpy()
    Xr = M.Sim(p, resident="off", decompose="ramps").run().cpu().numpy()
    assert np.abs(Xg - Xr).max() <= TOL_V * p.vdd


def test_ramps_refuse_new_currents(M):
    p = gridgen.small_mesh(34, nx=8, ny=8, n_src=4, group_templates=[2, 2])
    sim = M.Sim(p, resident="off", decompose="ramps")
    sim.run()
    with pytest.raises(M.MatexError) as ei:
        sim.set_sources(np.asarray(p.pwl_v) * 2.0)
    assert ei.value.status == 7  # MATEX_ERR_STATE


def test_ramp_columns_in_batches_match_oracle(M):
    """100 single-template groups give 300 ramp columns, more than one batch
    of 256: the second batch reuses the first one's state and basis slots
    (ramps hand no state to later segments)."""
    p = gridgen.small_mesh(35, nx=20, ny=20, layers=2, n_src=100, group_templates=[1] * 100,
                           t_end=0.5e-9, dt_out=5e-12)
    rows = np.sort(np.random.default_rng(35).choice(p.n, 40, replace=False)).astype(np.int32)
    q = R.ramp_decomposition(p)
    assert q.n_groups > 256
    err, sim = ramp_parity(M, p, "ramps_two_batches", rows=rows)
    assert err <= TOL_V * p.vdd
    with pytest.raises(M.MatexError):
        sim.one_group_at_a_time(True)
