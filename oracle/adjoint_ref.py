"""Hand-written discrete adjoint of the oracle's R-MATEX forward (test
infrastructure only; see oracle/__init__.py).

Loss (integrated IR-drop hinge over observed nodes, trapezoid over the output
times t_o = o * dt_out):

    L = sum_{i in obs} sum_o w_o max(0, Vdd - x_i(t_o) - theta)^2,
    w_o = dt_out (interior), dt_out / 2 (first and last output).

Parameters: the node capacitances c (C = diag(c)) and one amplitude scale per
source (its PWL currents are multiplied by it).

The reverse pass differentiates, step by step in reverse order, exactly the
computation of ``rmatex_ref.run_group`` with the Krylov dimensions held fixed
(the ones the forward chose, or replayed ones):

  segment inputs   z = G^{-1} u0, z' = G^{-1} s, w = G^{-1} (c * z')   (Eq. 5/6)
  start vector     v = x - z + w, beta = ||v||, q_0 = v / beta
  Arnoldi (Alg. 1) a_k = (C + gamma G)^{-1} (c * q_k), h_k = Q_k^T a_k,
                   r_k = a_k - Q_k h_k, q_{k+1} = r_k / ||r_k||
                   (the modified Gram-Schmidt of the forward equals this
                   projection up to rounding)
  rational map     H = (I - Htilde^{-1}) / gamma                      (Eq. 9)
  outputs          x(t_o) = Q^T y_o + z + h_o z' - w, y_o = beta e^{h_o H} e_1
  hand-off         x(l_{j+1}) = Q^T y_L + z + L z' - w

The exponential is reversed through its Frechet derivative:
<Ybar, d e^{X}> = <L(X^T, Ybar), dX> (scipy.linalg.expm_frechet computes L).
(C + gamma G) and G are symmetric, so every reverse solve uses the same
factorisations as the forward.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import rmatex_ref as R


def trapezoid_weights(n_out, dt):
    w = np.full(n_out, dt)
    w[0] = w[-1] = dt / 2.0
    return w


def hinge_loss(Xobs, vdd, theta, dt):
    """L and dL/dX for X restricted to the observed nodes ((N+1) x n_obs)."""
    w = trapezoid_weights(Xobs.shape[0], dt)
    a = np.maximum(vdd - Xobs - theta, 0.0)
    L = float((w[:, None] * a * a).sum())
    G = -2.0 * w[:, None] * a
    return L, G


def source_values(p, t):
    """Unscaled PWL value of every source at time t (its d(B u)/d amp_s)."""
    out = np.zeros(p.n_src)
    for s in range(p.n_src):
        ts = p.pwl_t[p.pwl_off[s]:p.pwl_off[s + 1]]
        vs = p.pwl_v[p.pwl_off[s]:p.pwl_off[s + 1]]
        out[s] = np.interp(t, ts, vs)
    return out


def forward_loss(p, obs, theta, c=None, amp_scale=None, replay_m=None):
    """Oracle forward restricted to the observed rows, and its loss."""
    pc = p
    if c is not None:
        pc = _with_c(p, c)
    res = R.rmatex(pc, nodes=obs, replay_m=replay_m, amp_scale=amp_scale)
    L, G = hinge_loss(res.X, p.vdd, theta, p.dt_out)
    return L, res


def _with_c(p, c):
    import copy
    q = copy.copy(p)
    q.c = np.asarray(c, dtype=np.float64)
    return q


def forward_tape(p, obs, c=None, amp_scale=None, replay_m=None, groups=None, include_dc=True):
    """Oracle forward (all nodes per group) keeping each segment's data; returns
    (X at the observed rows, tapes, m per group, factors, x_dc)."""
    c = p.c if c is None else np.asarray(c, dtype=np.float64)
    amp = np.ones(p.n_src) if amp_scale is None else np.asarray(amp_scale, dtype=np.float64)
    pc = _with_c(p, c)
    fac = R.factorize(pc, c)
    t_out = R.output_times(p)
    obs = np.asarray(obs)
    x_dc = fac.solve_G(p.dc_inject)
    X = np.zeros((t_out.shape[0], obs.shape[0]))
    if include_dc:
        X += x_dc[obs][None, :]
    tapes, ms = {}, {}
    for k in (range(p.n_groups) if groups is None else groups):
        keep = []
        rm = None if replay_m is None else replay_m[k]
        Xg = np.zeros((t_out.shape[0], p.n))
        log = R.run_group(pc, fac, k, Xg, t_out, replay_m=rm, amp_scale=amp, keep=keep)
        X += Xg[:, obs]
        tapes[k] = (log.lts, keep)
        ms[k] = list(log.m)
    return X, tapes, ms, fac


def reverse(p, obs, fac, c, tapes, Gobs):
    """Hand-written reverse of the taped groups for output adjoints Gobs
    ((N+1) x n_obs, dL/dX at the observed rows); returns (cbar, abar) summed
    over the taped groups."""
    c = np.asarray(c, dtype=np.float64)
    t_out = R.output_times(p)
    obs = np.asarray(obs)
    cbar = np.zeros(p.n)
    abar = np.zeros(p.n_src)
    gam = p.gamma
    for k, (lts, keep) in tapes.items():
        src = R.group_sources(p, k)
        outs = R.segment_outputs(lts, t_out)
        xbar_next = np.zeros(p.n)
        for seg in reversed(keep):
            j, l0, Lseg = seg["j"], seg["l0"], seg["L"]
            z, zp, w, basis = seg["z"], seg["zp"], seg["w"], seg["basis"]
            o_idx = outs[j]
            hs = t_out[o_idx] - l0
            xb_out = np.zeros((o_idx.shape[0], p.n))
            xb_out[:, obs] = Gobs[o_idx]
            zbar = xb_out.sum(axis=0) + xbar_next
            zpbar = (hs[:, None] * xb_out).sum(axis=0) + Lseg * xbar_next
            wbar = -zbar.copy()
            xbar = np.zeros(p.n)
            if basis is not None:
                Q, m, beta, H, Ht = basis.V, basis.m, basis.beta, basis.H, basis.Ht
                e1 = np.zeros(m)
                e1[0] = 1.0
                Qbar = np.zeros((m, p.n))
                Hbar = np.zeros((m, m))
                betabar = 0.0
                for h, xb in list(zip(hs, xb_out)) + [(Lseg, xbar_next)]:
                    E = sla.expm(h * H)
                    y = beta * E[:, 0]
                    ybar = Q @ xb
                    Qbar += np.outer(y, xb)
                    betabar += ybar @ E[:, 0]
                    Hbar += h * sla.expm_frechet((h * H).T, np.outer(ybar, beta * e1),
                                                 compute_expm=False)
                Htinv = np.linalg.inv(Ht[:m, :m])
                Htbar = Htinv.T @ Hbar @ Htinv.T / gam
                qbar = Qbar
                for kk in reversed(range(m)):
                    a_k = fac.solve_M(c * Q[kk])
                    h_k = Ht[:kk + 1, kk]
                    if kk < m - 1:
                        q1 = Q[kk + 1]
                        rbar = (qbar[kk + 1] - q1 * (q1 @ qbar[kk + 1])) / Ht[kk + 1, kk] \
                            + q1 * Htbar[kk + 1, kk]
                    else:
                        rbar = np.zeros(p.n)
                    hbar = Htbar[:kk + 1, kk] - Q[:kk + 1] @ rbar
                    a_bar = rbar + Q[:kk + 1].T @ hbar
                    qbar[:kk + 1] += -np.outer(h_k, rbar) + np.outer(hbar, a_k)
                    u = fac.solve_M(a_bar)
                    qbar[kk] += c * u
                    cbar += u * (Q[kk] - a_k)
                q0 = Q[0]
                vbar = (qbar[0] - q0 * (q0 @ qbar[0])) / beta + q0 * betabar
                xbar += vbar
                zbar -= vbar
                wbar += vbar
            # w = G^{-1}(c * z'), z' = G^{-1}(u1 - u0)/L, z = G^{-1} u0
            pw = fac.solve_G(wbar)
            zpbar += c * pw
            cbar += pw * zp
            sbar = fac.solve_G(zpbar)
            u0bar = fac.solve_G(zbar) - sbar / Lseg
            u1bar = sbar / Lseg
            v0 = source_values(p, l0)
            v1 = source_values(p, l0 + Lseg)
            for s in src:
                nd = p.src_node[s]
                abar[s] += v0[s] * u0bar[nd] + v1[s] * u1bar[nd]
            xbar_next = xbar
        # initial state x(0) = G^{-1} B u(0), also output 0
        xb0 = xbar_next.copy()
        xb0[obs] += Gobs[0]
        u_bar = fac.solve_G(xb0)
        v0 = source_values(p, lts[0])
        for s in src:
            abar[s] += v0[s] * u_bar[p.src_node[s]]
    return cbar, abar


def loss_and_grad(p, obs, theta, c=None, amp_scale=None, replay_m=None):
    """Returns (L, dL/dc [n], dL/damp_scale [n_src], m sequence per group)."""
    c = p.c if c is None else np.asarray(c, dtype=np.float64)
    X, tapes, ms, fac = forward_tape(p, obs, c=c, amp_scale=amp_scale, replay_m=replay_m)
    L, Gobs = hinge_loss(X, p.vdd, theta, p.dt_out)
    cbar, abar = reverse(p, obs, fac, c, tapes, Gobs)
    return L, cbar, abar, [ms[k] for k in range(p.n_groups)]
