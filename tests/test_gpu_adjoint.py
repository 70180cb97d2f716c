"""GPU adjoint (matex_grad, IRDrop autograd) against the FP64 CPU adjoint and
central differences.

The GPU reverse differentiates the computation the GPU forward performed, with
its Krylov dimensions; the CPU adjoint is run with the same dimensions
(replay), so the two must agree to rounding.  Central differences use the same
replayed dimensions (the map is then smooth) and runs without the constant DC
part (x_dc = Vdd on these grids, and it does not depend on the parameters), so
that the loss sees the IR drop itself rather than a voltage near 1 V with
three fewer significant digits: amplitudes h = 1e-6 (relative); capacitances
Richardson-extrapolated with h = 4e-3 (a 1e-6 step moves the loss by about
1e-10 of itself, at the forward's rounding).
"""
import numpy as np
import pytest

import gridgen
from oracle import adjoint_ref as A
from oracle import rmatex_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04519_gb300 import build
    build.build()
    from paper_1511_04519_gb300 import autograd as AG
    from paper_1511_04519_gb300 import matex as M
    return torch, M, AG


def small_case(seed, layers=1, nx=8, ny=7):
    p = gridgen.small_mesh(seed, nx=nx, ny=ny, layers=layers, n_src=8, group_templates=[2, 3, 3],
                           t_end=0.3e-9, dt_out=10e-12, c_range=(1e-14, 1e-12))
    obs = np.sort(np.random.default_rng(seed).choice(p.n, 9, replace=False)).astype(np.int32)
    drop = p.vdd - R.rmatex(p, nodes=obs).X
    theta = float(np.quantile(drop, 0.6))
    return p, obs, theta


def gpu_loss_grad(env, p, obs, theta, sim=None, vdd=None):
    """Loss max(0, vdd - v - theta)^2 integrated over the rows; vdd = 0 with a
    Sim built without the DC part (then -v is the IR drop)."""
    torch, M, AG = env
    sim = sim or AG.make_sim(p, obs)
    c = torch.tensor(p.c, dtype=torch.float64, requires_grad=True)
    amp = torch.ones(p.n_src, dtype=torch.float64, requires_grad=True)
    X = AG.IRDrop.apply(c, amp, sim)
    L = AG.hinge_ir_drop_loss(X, p.vdd if vdd is None else vdd, theta, p.dt_out)
    L.backward()
    return L.item(), c.grad.cpu().numpy(), amp.grad.cpu().numpy(), sim


def richardson_derivative(f, x0, h):
    """dF/dx at x0 from central differences at h, h/2, h/4, extrapolated twice
    (Richardson): truncation O(h^6), so a step large enough to keep the
    loss's rounding noise (the order of the forward solves' FP64 atomic
    additions varies from run to run) far below the change it measures."""
    def D(k):
        return (f(x0 + k) - f(x0 - k)) / (2 * k)
    d1, d2, d4 = D(h), D(h / 2), D(h / 4)
    r1, r2 = (4 * d2 - d1) / 3, (4 * d4 - d2) / 3
    return (16 * r2 - r1) / 15


def per_group_m(p, sim):
    """The GPU's m sequence split per group (replay layout)."""
    m = sim.m_sequence()
    out, pos = [], 0
    for k in range(p.n_groups):
        nseg = len(R.local_transition_spots(p, k)) - 1
        out.append(list(m[pos:pos + nseg]))
        pos += nseg
    return out


@pytest.mark.parametrize("tape", ["full", "checkpoint"])
@pytest.mark.parametrize("seed,layers", [(3, 1), (4, 2), (5, 1)])
def test_gpu_adjoint_matches_cpu_adjoint(env, seed, layers, tape):
    torch, M, AG = env
    p, obs, theta = small_case(seed, layers=layers)
    L, dc, da, sim = gpu_loss_grad(env, p, obs, theta, sim=AG.make_sim(p, obs, tape=tape))
    ms = per_group_m(p, sim)
    Lr, cbar, abar, _ = A.loss_and_grad(p, obs, theta, replay_m=ms)
    assert L > 0 and abs(L - Lr) <= 1e-9 * Lr
    assert np.abs(dc - cbar).max() <= 1e-9 * np.abs(cbar).max()
    assert np.abs(da - abar).max() <= 1e-9 * np.abs(abar).max()


def test_gpu_adjoint_matches_central_differences(env):
    torch, M, AG = env
    p, obs, theta = small_case(6, layers=2, nx=9, ny=9)
    sim = AG.make_sim(p, obs, include_dc=False)
    L, dc, da, sim = gpu_loss_grad(env, p, obs, theta, sim=sim, vdd=0.0)
    ms = np.concatenate(per_group_m(p, sim)).astype(np.int32)
    fd_sim = M.Sim(p, rows=obs, replay_m=ms, include_dc=False)
    base = np.asarray(p.pwl_v, dtype=np.float64)
    src_of = np.repeat(np.arange(p.n_src), np.diff(p.pwl_off))

    def loss(c=None, amp=None):
        fd_sim.set_caps(p.c if c is None else c)
        fd_sim.set_sources(base * (np.ones(p.n_src) if amp is None else amp)[src_of])
        return float(AG.hinge_ir_drop_loss(fd_sim.run(), 0.0, theta, p.dt_out))

    rng = np.random.default_rng(0)
    for s in range(p.n_src):
        ap = np.ones(p.n_src); ap[s] += 1e-6
        am = np.ones(p.n_src); am[s] -= 1e-6
        fd = (loss(amp=ap) - loss(amp=am)) / 2e-6
        assert abs(da[s] - fd) <= 1e-6 * abs(fd), (s, da[s], fd)
    rel = []
    for i in rng.choice(p.n, 6, replace=False):
        def f(ci):
            cp = p.c.copy(); cp[i] = ci
            return loss(c=cp)
        fd = richardson_derivative(f, p.c[i], 2e-2 * p.c[i])
        rel.append(abs(dc[i] - fd) / abs(fd))
    assert max(rel) <= 1e-6, rel


def test_amplitude_gradient_away_from_unit_amplitudes(env):
    """IRDrop at amplitudes drawn from U[0.5, 2], one of them zero (its group
    keeps another non-zero source): the amplitude gradient is dL/d amp at that
    amp, against the CPU adjoint run at the same amplitudes (same Krylov
    dimensions) and against central differences."""
    torch, M, AG = env
    # 12 sources on 8 pulse templates: some template drives two sources.  The
    # source set to zero is one of those, so its group's input is still
    # non-zero on every segment where that source is (a group whose input is
    # all zero on a segment builds no basis there, and the run's derivative
    # then lacks the exponential term, as matex_grad states)
    p = gridgen.small_mesh(8, nx=8, ny=8, layers=2, n_src=12, group_templates=[2, 3, 3],
                           t_end=0.3e-9, dt_out=10e-12, c_range=(1e-14, 1e-12))
    obs = np.sort(np.random.default_rng(8).choice(p.n, 9, replace=False)).astype(np.int32)
    theta = float(np.quantile(p.vdd - R.rmatex(p, nodes=obs).X, 0.6))
    t3 = np.asarray(p.pwl_t).reshape(-1, 3)
    shared = [s for s in range(p.n_src)
              if any(q != s and np.array_equal(t3[q], t3[s]) and p.src_group[q] == p.src_group[s]
                     for q in range(p.n_src))]
    assert shared
    rng = np.random.default_rng(8)
    amp = rng.uniform(0.5, 2.0, p.n_src)
    zero = shared[0]
    amp[zero] = 0.0
    sim = AG.make_sim(p, obs, include_dc=False)
    c = torch.tensor(p.c, dtype=torch.float64, requires_grad=True)
    a = torch.tensor(amp, dtype=torch.float64, requires_grad=True)
    X = AG.IRDrop.apply(c, a, sim)
    L = AG.hinge_ir_drop_loss(X, 0.0, theta, p.dt_out)
    L.backward()
    da = a.grad.cpu().numpy()
    dc = c.grad.cpu().numpy()
    ms = per_group_m(p, sim)
    # CPU adjoint at the same amplitudes (the loss on the load response: no DC part)
    Xr, tapes, _, fac = A.forward_tape(p, obs, amp_scale=amp, replay_m=ms, include_dc=False)
    Lr, Gobs = A.hinge_loss(Xr, 0.0, theta, p.dt_out)
    assert abs(L.item() - Lr) <= 1e-9 * Lr
    cbar, abar = A.reverse(p, obs, fac, p.c, tapes, Gobs)
    assert np.abs(da - abar).max() <= 1e-9 * np.abs(abar).max()
    assert np.abs(dc - cbar).max() <= 1e-9 * np.abs(cbar).max()
    # the gradient is not the unit-amplitude one rescaled: at amp_s = 0 it is non-zero
    assert abs(da[zero]) > 1e-6 * np.abs(da).max()
    # central differences in amp with the same Krylov dimensions
    fd_sim = M.Sim(p, rows=obs, replay_m=np.concatenate(ms).astype(np.int32), include_dc=False)
    base = np.asarray(p.pwl_v, dtype=np.float64)
    src_of = np.repeat(np.arange(p.n_src), np.diff(p.pwl_off))

    def loss(av):
        fd_sim.set_sources(base * av[src_of])
        return float(AG.hinge_ir_drop_loss(fd_sim.run(), 0.0, theta, p.dt_out))

    for s in range(p.n_src):
        h = 1e-6 * max(amp[s], 1.0)
        ap = amp.copy(); ap[s] += h
        am = amp.copy(); am[s] -= h
        fd = (loss(ap) - loss(am)) / (2 * h)
        assert abs(da[s] - fd) <= 1e-6 * abs(fd), (s, amp[s], da[s], fd)


@pytest.mark.parametrize("window,block", [(1, 1), (2, 3), (3, 2), (0, 0)])
def test_checkpointed_adjoint_equals_full_tape(env, window, block):
    """Checkpoints every `window` segment rounds, segments recomputed `block`
    groups at a time (0: the sizes chosen at setup): the same gradients as
    the full tape, up to the order of the solves' FP64 atomic additions.
    Six groups of uneven breakpoint counts, so windows and blocks have
    ragged ends and groups that start or finish inside a window."""
    torch, M, AG = env
    p = gridgen.small_mesh(16, nx=12, ny=11, layers=2, n_src=14,
                           group_templates=[1, 3, 2, 4, 1, 3], t_end=0.4e-9, dt_out=10e-12,
                           c_range=(1e-14, 1e-12))
    obs = np.sort(np.random.default_rng(16).choice(p.n, 11, replace=False)).astype(np.int32)
    drop = p.vdd - R.rmatex(p, nodes=obs).X
    theta = float(np.quantile(drop, 0.6))
    full = AG.make_sim(p, obs, tape="full")
    L1, dc1, da1, _ = gpu_loss_grad(env, p, obs, theta, sim=full)
    ms = np.concatenate(per_group_m(p, full)).astype(np.int32)
    ck = AG.make_sim(p, obs, tape="checkpoint", tape_window=window, tape_block=block,
                     replay_m=ms)
    st = ck.setup_stats()
    assert st["tape_window"] >= 1 and st["tape_block"] >= 1 and st["tape_bytes"] > 0
    if window:
        assert (st["tape_window"], st["tape_block"]) == (window, block)
    L2, dc2, da2, _ = gpu_loss_grad(env, p, obs, theta, sim=ck)
    assert abs(L2 - L1) <= 1e-12 * L1
    assert np.abs(dc2 - dc1).max() <= 1e-10 * np.abs(dc1).max()
    assert np.abs(da2 - da1).max() <= 1e-10 * np.abs(da1).max()


def test_grad_requires_tape_and_a_run(env):
    torch, M, AG = env
    p, obs, theta = small_case(7)
    plain = M.Sim(p, rows=obs)
    plain.run()
    with pytest.raises(M.MatexError):
        plain.grad(torch.zeros((plain.n_times, plain.n_rows), dtype=torch.float64, device="cuda"))
    taped = AG.make_sim(p, obs)
    with pytest.raises(M.MatexError):
        taped.grad(torch.zeros((taped.n_times, taped.n_rows), dtype=torch.float64, device="cuda"))


@pytest.fixture(scope="module")
def cfg3(env):
    p = gridgen.config3()
    return p


def test_config3_adjoint_against_cpu_adjoint_and_differences(env, cfg3):
    """The config-1 grid with 256 observed nodes: GPU gradients with respect to
    all 180k capacitances and 2000 amplitudes; the amplitudes of two groups'
    sources against the CPU reverse of those groups (driven by the same output
    adjoint), and central differences on 16 capacitances and 16 amplitudes."""
    torch, M, AG = env
    p = cfg3
    obs = p.observed.astype(np.int32)
    sim = AG.make_sim(p, obs, include_dc=False, tape="checkpoint")
    X0 = sim.run().cpu().numpy()
    st = sim.setup_stats()
    # checkpoints per segment round, every group recomputed at once: x and z
    # of the 192 segments plus one round's tape, not the 12 GB full tape
    assert (st["tape_window"], st["tape_block"]) == (1, 64)
    assert st["tape_bytes"] < 6e9
    drop = -X0                      # x_dc = Vdd on this grid: the load response is the drop
    theta = float(np.quantile(drop, 0.9))
    assert (drop > theta).mean() >= 0.09
    L, dc, da, sim = gpu_loss_grad(env, p, obs, theta, sim=sim, vdd=0.0)
    assert L > 0 and np.isfinite(dc).all() and np.isfinite(da).all()
    ms = per_group_m(p, sim)
    # the full tape of the same run (same Krylov dimensions) gives the same gradients
    full = AG.make_sim(p, obs, include_dc=False, tape="full",
                       replay_m=np.concatenate(ms).astype(np.int32))
    Lf, dcf, daf, _ = gpu_loss_grad(env, p, obs, theta, sim=full, vdd=0.0)
    assert abs(Lf - L) <= 1e-12 * L
    assert np.abs(dcf - dc).max() <= 1e-10 * np.abs(dc).max()
    assert np.abs(daf - da).max() <= 1e-10 * np.abs(da).max()
    full.close()
    del full
    # CPU reverse of two groups, output adjoint from the GPU forward's rows
    Lr, G = A.hinge_loss(X0, 0.0, theta, p.dt_out)
    groups = [5, 41]
    _, tapes, _, fac = A.forward_tape(p, obs, replay_m={k: ms[k] for k in groups}, groups=groups)
    cbar, abar = A.reverse(p, obs, fac, p.c, tapes, G)
    sel = np.isin(p.src_group, groups)
    assert np.abs(da[sel] - abar[sel]).max() <= 1e-8 * np.abs(abar[sel]).max()
    # capacitances: the GPU reverse of a context holding only those two groups,
    # driven by the same output adjoint, against the CPU reverse of the groups
    off = np.concatenate([[0], np.cumsum(np.diff(p.pwl_off)[sel])]).astype(np.int32)
    keep = np.repeat(sel, np.diff(p.pwl_off))
    q = gridgen.with_sources(p, p.src_node[sel], off, np.asarray(p.pwl_t)[keep],
                             np.asarray(p.pwl_v)[keep],
                             np.searchsorted(groups, p.src_group[sel]), len(groups))
    sub = AG.make_sim(q, obs, include_dc=False,
                      replay_m=np.concatenate([ms[k] for k in groups]).astype(np.int32))
    sub.run()
    dc2, _ = sub.grad(torch.from_numpy(G).cuda())
    dc2 = dc2.cpu().numpy()
    assert np.abs(dc2 - cbar).max() <= 1e-8 * np.abs(cbar).max()
    # central differences with the GPU's m replayed
    msr = np.concatenate(ms).astype(np.int32)
    fd_sim = M.Sim(p, rows=obs, replay_m=msr, include_dc=False)
    base = np.asarray(p.pwl_v, dtype=np.float64)
    src_of = np.repeat(np.arange(p.n_src), np.diff(p.pwl_off))

    def loss(c=None, amp=None):
        if c is not None:
            fd_sim.set_caps(c)
        fd_sim.set_sources(base * (np.ones(p.n_src) if amp is None else amp)[src_of])
        return float(AG.hinge_ir_drop_loss(fd_sim.run(), 0.0, theta, p.dt_out))

    rng = np.random.default_rng(1)
    active = np.nonzero(np.abs(da) > 1e-3 * np.abs(da).max())[0]
    rel_a = []
    for s in rng.choice(active, 16, replace=False):
        ap = np.ones(p.n_src); ap[s] += 1e-6
        am = np.ones(p.n_src); am[s] -= 1e-6
        fd = (loss(amp=ap) - loss(amp=am)) / 2e-6
        rel_a.append(abs(da[s] - fd) / abs(fd))
    assert max(rel_a) <= 1e-6, rel_a
    bigc = np.argsort(-np.abs(dc))[:400]
    rel_c = []
    for i in rng.choice(bigc, 16, replace=False):
        def f(ci):
            cp = p.c.copy(); cp[i] = ci
            return loss(c=cp)
        fd = richardson_derivative(f, p.c[i], 2e-2 * p.c[i])
        rel_c.append(abs(dc[i] - fd) / abs(fd))
    assert max(rel_c) <= 1e-6, rel_c
