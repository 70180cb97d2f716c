"""Pins of the oracle's hand-written adjoint against brute-force central
differences of the oracle forward (Krylov dimensions replayed so the forward
map is smooth).

Step sizes: amplitude scales use h = 1e-6 (relative).  A capacitance moves
the loss by only ~1e-10 of itself per 1e-6 relative step, below the rounding
of the forward, so capacitances use Richardson-extrapolated central
differences (4 D(h/2) - D(h)) / 3 with h = 4e-3 relative; their noise floor is
about 1e-6 (relative), so the bar there is a median of 1e-6 and a maximum of
5e-6.  The tight pin for the capacitance path is the comparison with torch
autograd through a dense exact solution (Eq. 4 via the augmented matrix
exponential) on a grid small enough that the Krylov space is the whole space.
"""
import numpy as np
import pytest

import gridgen
from oracle import adjoint_ref as A
from oracle import rmatex_ref as R


def adjoint_problem(seed):
    p = gridgen.small_mesh(seed, nx=7, ny=6, layers=1 + seed % 2, n_src=6, group_templates=[2, 2, 2],
                           t_end=0.3e-9, dt_out=10e-12, c_range=(1e-14, 1e-12))
    obs = np.sort(np.random.default_rng(seed).choice(p.n, 6, replace=False))
    drop = p.vdd - R.rmatex(p, nodes=obs).X
    theta = float(np.quantile(drop, 0.6))
    return p, obs, theta


def fd_c(p, obs, theta, ms, i, rel):
    def D(h):
        cp = p.c.copy(); cp[i] += h
        cm = p.c.copy(); cm[i] -= h
        return (A.forward_loss(p, obs, theta, c=cp, replay_m=ms)[0]
                - A.forward_loss(p, obs, theta, c=cm, replay_m=ms)[0]) / (2 * h)
    h = rel * p.c[i]
    return (4 * D(h / 2) - D(h)) / 3


@pytest.mark.parametrize("seed", [3, 4])
def test_adjoint_matches_central_differences(seed):
    p, obs, theta = adjoint_problem(seed)
    L, cbar, abar, ms = A.loss_and_grad(p, obs, theta)
    assert L > 0
    drop = p.vdd - R.rmatex(p, nodes=obs).X
    assert (drop > theta).mean() >= 0.1  # the hinge is active: the check is not vacuous
    rng = np.random.default_rng(seed)
    rel = []
    for i in rng.choice(p.n, 5, replace=False):
        fd = fd_c(p, obs, theta, ms, i, 4e-3)
        rel.append(abs(cbar[i] - fd) / abs(fd))
    assert np.median(rel) <= 1e-6 and max(rel) <= 5e-6, rel
    for s in range(p.n_src):
        amp_p = np.ones(p.n_src); amp_p[s] += 1e-6
        amp_m = np.ones(p.n_src); amp_m[s] -= 1e-6
        fd = (A.forward_loss(p, obs, theta, amp_scale=amp_p, replay_m=ms)[0]
              - A.forward_loss(p, obs, theta, amp_scale=amp_m, replay_m=ms)[0]) / 2e-6
        assert abs(abar[s] - fd) <= 1e-6 * abs(fd), (s, abar[s], fd)


def test_adjoint_zero_when_hinge_inactive():
    p, obs, theta = adjoint_problem(3)
    L, cbar, abar, _ = A.loss_and_grad(p, obs, 1.0)  # threshold above every drop
    assert L == 0 and not cbar.any() and not abar.any()


def test_amplitude_gradient_homogeneity():
    # x - x_dc is linear in the amplitude scales, so for a common scale a the
    # drop d(a) = a d(1) and sum_s a_s dL/da_s = dL/da along the ray; checked
    # against the derivative of L(a) = sum w max(0, a d - theta)^2 in closed form.
    p, obs, theta = adjoint_problem(4)
    L, cbar, abar, ms = A.loss_and_grad(p, obs, theta)
    res = R.rmatex(p, nodes=obs, replay_m=ms)
    d = p.vdd - res.X
    w = A.trapezoid_weights(d.shape[0], p.dt_out)
    ray = float((w[:, None] * 2 * np.maximum(d - theta, 0) * d).sum())
    assert abs(abar.sum() - ray) <= 1e-9 * abs(ray)


def krylov_loss_torch(p, obs, theta, c, amp, ms):
    """The R-MATEX forward (Alg. 2 per group, Alg. 1 with X1 = C + gamma G,
    X2 = C, modified Gram-Schmidt, Eq. 9, Eq. 5/6 via G-solves) restated with
    dense torch ops and the Krylov dimensions ms held fixed, so that autograd
    differentiates exactly the computation the hand-written adjoint reverses."""
    import torch
    n = p.n
    G = torch.tensor(p.G().toarray())
    M = torch.diag(c) + p.gamma * G
    t_out = R.output_times(p)

    def u_vec(k, t):
        u = torch.zeros(n, dtype=torch.float64)
        vals = torch.tensor(A.source_values(p, t))
        for s in R.group_sources(p, k):
            u = u + torch.nn.functional.one_hot(torch.tensor(int(p.src_node[s])), n).double() * amp[s] * vals[s]
        return u

    X = [torch.linalg.solve(G, torch.tensor(p.dc_inject)) for _ in range(t_out.shape[0])]
    for k in range(p.n_groups):
        lts = R.local_transition_spots(p, k)
        outs = R.segment_outputs(lts, t_out)
        x = torch.linalg.solve(G, u_vec(k, lts[0]))
        X[0] = X[0] + x
        for j in range(lts.shape[0] - 1):
            l0, l1 = float(lts[j]), float(lts[j + 1])
            L = l1 - l0
            z = torch.linalg.solve(G, u_vec(k, l0))
            zp = torch.linalg.solve(G, (u_vec(k, l1) - u_vec(k, l0)) / L)
            w = torch.linalg.solve(G, c * zp)
            v = x + (-z + w)
            m = ms[k][j]
            hs = [float(t_out[q]) - l0 for q in outs[j]] + [L]
            if m == 0:
                ys = None
            else:
                beta = torch.linalg.norm(v)
                Q = [v / beta]
                Ht = torch.zeros(m + 1, m, dtype=torch.float64)
                for jj in range(m):
                    wv = torch.linalg.solve(M, c * Q[jj])
                    col = []
                    for i in range(jj + 1):
                        hij = wv @ Q[i]
                        col.append(hij)
                        wv = wv - hij * Q[i]
                    hn = torch.linalg.norm(wv)
                    Ht = Ht + torch.zeros_like(Ht).index_put((torch.arange(jj + 2), torch.full((jj + 2,), jj)),
                                                            torch.stack(col + [hn]))
                    Q.append(wv / hn)
                Hm = (torch.eye(m, dtype=torch.float64) - torch.linalg.inv(Ht[:m, :m])) / p.gamma
                Qm = torch.stack(Q[:m])
                ys = [Qm.T @ (beta * torch.linalg.matrix_exp(h * Hm)[:, 0]) for h in hs]
            for idx, q in enumerate(list(outs[j]) + [None]):
                val = z + hs[idx] * zp - w
                if ys is not None:
                    val = val + ys[idx]
                if q is None:
                    x = val
                else:
                    X[q] = X[q] + val
    Xs = torch.stack(X)[:, torch.tensor(obs)]
    wts = torch.tensor(A.trapezoid_weights(t_out.shape[0], p.dt_out))
    a = torch.clamp(p.vdd - Xs - theta, min=0.0)
    return (wts[:, None] * a * a).sum()


@pytest.mark.parametrize("seed", [3, 4])
def test_adjoint_matches_autograd_of_the_same_forward(seed):
    torch = pytest.importorskip("torch")
    p, obs, theta = adjoint_problem(seed)
    L, cbar, abar, ms = A.loss_and_grad(p, obs, theta)
    c = torch.tensor(p.c, requires_grad=True)
    amp = torch.ones(p.n_src, dtype=torch.float64, requires_grad=True)
    Lt = krylov_loss_torch(p, obs, theta, c, amp, ms)
    Lt.backward()
    assert abs(Lt.item() - L) <= 1e-10 * L
    assert np.abs(cbar - c.grad.numpy()).max() <= 1e-8 * np.abs(c.grad.numpy()).max()
    assert np.abs(abar - amp.grad.numpy()).max() <= 1e-8 * np.abs(amp.grad.numpy()).max()
