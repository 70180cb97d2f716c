"""Plain FP64 CPU R-MATEX (test infrastructure only; see oracle/__init__.py).

Slow and direct on purpose: SuperLU (scipy.sparse.linalg.splu) for the
factorisations, modified Gram-Schmidt exactly as Alg. 1 writes it, and
scipy.linalg.expm for every small exponential.  Nothing is blocked, fused or
reordered beyond what the paper's algorithms state.

Problem (Eq. 1):   C x' = -G x + B u(t)   with C = diag(c), G SPD.
ODE form (Eq. 3):  A = -C^{-1} G, b(t) = C^{-1} B u(t); A is never formed.
Exact PWL step (Eq. 5/6):  x(t+h) = e^{hA}(x(t) + F) - P(t+h) with
    F = A^{-1} b(t) + A^{-2} b',   P(t+h) = A^{-1} b(t+h) + A^{-2} b'.
Because A^{-1} b = -G^{-1} B u and A^{-2} b' = G^{-1} C G^{-1} B s
(s = du/dt on the segment), with z = G^{-1}Bu(l), z' = G^{-1}Bs, w = G^{-1}Cz':
    F = -z + w,   -P(l+h) = z + h z' - w.
Nothing here needs C^{-1}, matching the regularisation-free property of
Sec. 3.3.3.

Rational (shift-and-invert) Krylov, Sec. 3.3.2: Arnoldi on
(I - gamma A)^{-1} = (C + gamma G)^{-1} C gives V_m, Htilde_m and
    e^{hA} v ~= ||v|| V_m e^{h H_m} e_1,   H_m = (I - Htilde_m^{-1}) / gamma  (Eq. 9)
with the empirical residual of Sec. 3.3.3
    r_m(h) = ||v|| * |htilde_{m+1,m} e_m^T e^{h H_m} e_1|.

Readings where the paper is silent:
  * residual checked at h_c = first output offset in the segment and at the
    segment length; both must be below tol (the basis is reused for every
    step inside the segment, Alg. 2, and Fig. 4 says error falls with h);
  * happy breakdown when htilde_{j+1,j} <= 1e-13 * htilde_{1,1};
  * m = m_max accepted without convergence (counted);
  * each group starts from G^{-1} B_k u_k(0); the pads form their own
    constant part x_dc = G^{-1} b_pad, added once;
  * simulation end = N * dt_out with N = round(t_end / dt_out).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BREAKDOWN_REL = 1e-13
QUIESCENT_BETA = 1e-300


# ---------------------------------------------------------------------------
# Input handling: transition spots, LTS per group, PWL evaluation (Sec. 2.2, 3.1)
# ---------------------------------------------------------------------------

def output_times(p):
    """t_o = o * dt_out for o = 0..N (FP64, the same product on every side)."""
    N = int(round(p.t_end / p.dt_out))
    return np.arange(N + 1, dtype=np.float64) * p.dt_out


def sim_end(p):
    N = int(round(p.t_end / p.dt_out))
    return N * p.dt_out


def group_sources(p, k):
    return np.nonzero(p.src_group == k)[0]


def local_transition_spots(p, k):
    """LTS of group k (Sec. 3.1 definition): the union of its sources'
    breakpoints inside (0, T), plus the interval ends 0 and T."""
    T = sim_end(p)
    pts = [0.0, T]
    for s in group_sources(p, k):
        ts = p.pwl_t[p.pwl_off[s]:p.pwl_off[s + 1]]
        pts.extend(float(t) for t in ts if 0.0 < t < T)
    return np.unique(np.asarray(pts, dtype=np.float64))


def input_vector(p, k, t, amp_scale=None):
    """B_k u_k(t): each source's PWL value (held constant outside its
    breakpoints) injected at its node.  amp_scale multiplies per source."""
    u = np.zeros(p.n)
    for s in group_sources(p, k):
        ts = p.pwl_t[p.pwl_off[s]:p.pwl_off[s + 1]]
        vs = p.pwl_v[p.pwl_off[s]:p.pwl_off[s + 1]]
        a = 1.0 if amp_scale is None else amp_scale[s]
        u[p.src_node[s]] += a * np.interp(t, ts, vs)
    return u


def full_input_vector(p, t, amp_scale=None):
    """b_pad + sum over all groups of B_k u_k(t) (the whole right-hand side)."""
    u = p.dc_inject.copy()
    for k in range(p.n_groups):
        u += input_vector(p, k, t, amp_scale)
    return u


def _slope_right(ts, vs, x):
    """Slope of a PWL waveform just right of x (0 before its first and from
    its last breakpoint on: the value is held there)."""
    if x < ts[0] or x >= ts[-1]:
        return 0.0
    j = int(np.searchsorted(ts, x, side="right")) - 1
    return (vs[j + 1] - vs[j]) / (ts[j + 1] - ts[j])


def _slope_left(ts, vs, x):
    """Slope of a PWL waveform just left of x."""
    if x <= ts[0] or x > ts[-1]:
        return 0.0
    j = int(np.searchsorted(ts, x, side="left")) - 1
    return (vs[j + 1] - vs[j]) / (ts[j + 1] - ts[j])


def ramp_decomposition(p):
    """The decomposition of Sec. 3.1 carried down to single ramps.

    On [0, T] a source's PWL input equals its value at t = 0 plus, for each of
    its breakpoints tau in (0, T), the ramp ds * max(0, t - tau), ds the change
    of slope at tau (slope right of tau minus slope left of it), plus a ramp at
    tau = 0 with the slope right of 0.  Every (group, tau) pair becomes a group
    of its own whose sources are those ramps (one per source of the group
    whose slope changes at tau), so its only local transition spot inside
    (0, T) is tau; a group whose sources start from non-zero values gets one
    more group holding those constant values.  By superposition the groups'
    responses sum to the original problem's.  A ramp starts from zero at tau
    with x(tau) = 0, so its Krylov basis starts from w = G^{-1} C G^{-1} B ds,
    which does not depend on any earlier state: all ramps are independent.

    Group order: by original group, then its constant part, then ramps by
    tau; sources of a new group in the original order.  Each ramp source's
    PWL has the points (tau, 0) and (T, ds (T - tau))."""
    import copy
    T = sim_end(p)
    entries = {}  # (k, kind, tau) -> list of (source, points)
    for s in range(p.n_src):
        o0, o1 = int(p.pwl_off[s]), int(p.pwl_off[s + 1])
        ts = np.asarray(p.pwl_t[o0:o1], np.float64)
        vs = np.asarray(p.pwl_v[o0:o1], np.float64)
        k = int(p.src_group[s])
        u0 = float(np.interp(0.0, ts, vs))
        if u0 != 0.0:
            entries.setdefault((k, 0, 0.0), []).append((s, [(0.0, u0)]))
        s0 = _slope_right(ts, vs, 0.0)
        if s0 != 0.0:
            entries.setdefault((k, 1, 0.0), []).append((s, [(0.0, 0.0), (T, s0 * T)]))
        for tau in ts:
            tau = float(tau)
            if not (0.0 < tau < T):
                continue
            ds = _slope_right(ts, vs, tau) - _slope_left(ts, vs, tau)
            if ds != 0.0:
                entries.setdefault((k, 1, tau), []).append((s, [(tau, 0.0), (T, ds * (T - tau))]))
    node, off, tt, vv, grp = [], [0], [], [], []
    for g, key in enumerate(sorted(entries)):
        for s, pts in entries[key]:
            node.append(int(p.src_node[s]))
            grp.append(g)
            for t, v in pts:
                tt.append(t)
                vv.append(v)
            off.append(len(tt))
    q = copy.copy(p)
    q.src_node = np.asarray(node, np.int32)
    q.pwl_off = np.asarray(off, np.int32)
    q.pwl_t = np.asarray(tt, np.float64)
    q.pwl_v = np.asarray(vv, np.float64)
    q.src_group = np.asarray(grp, np.int32)
    q.n_groups = len(entries)
    return q


def segment_outputs(lts, t_out):
    """For each segment [l_j, l_{j+1}] the output indices o with
    l_j < t_o <= l_{j+1} (an output on a breakpoint belongs to the segment
    that ends there)."""
    res = []
    for j in range(lts.shape[0] - 1):
        sel = np.nonzero((t_out > lts[j]) & (t_out <= lts[j + 1]))[0]
        res.append(sel)
    return res


# ---------------------------------------------------------------------------
# Factorisations (the one-time serial part of Alg. 2: X1 factored once)
# ---------------------------------------------------------------------------

@dataclass
class Factors:
    G: sp.csc_matrix
    c: np.ndarray
    gamma: float
    lu_M: object = None   # X1 = C + gamma G for R-MATEX (Sec. 3.3.2)
    lu_G: object = None   # G, for F and P (Eq. 6) and the DC solution

    def solve_M(self, b):
        return self.lu_M.solve(b)

    def solve_G(self, b):
        return self.lu_G.solve(b)

    def op(self, variant, v):
        """The Arnoldi operator of each Krylov variant (the solve step of
        Alg. 1, X1^{-1} X2 v):
          'R' rational (Sec. 3.3.2):  X1 = C + gamma G, X2 = C: (C + gamma G)^{-1} C v
          'I' inverted (Sec. 3.3.1):  X1 = G, X2 = C:            G^{-1} C v  (= -A^{-1} v)
          'S' standard (Sec. 2.3, MEXP):                          -C^{-1} G v (= A v)"""
        if variant == "R":
            return self.solve_M(self.c * v)
        if variant == "I":
            return self.solve_G(self.c * v)
        if variant == "S":
            return -(self.G @ v) / self.c
        raise ValueError(variant)


def factorize(p, c=None):
    """SuperLU factors of X1 = C + gamma G and of G.  Both are symmetric, so the
    column ordering is the minimum degree ordering of A^T + A (SuperLU's
    choice for a symmetric nonzero structure) rather than its default COLAMD,
    which orders for an unsymmetric LU and triples the fill on these grids;
    the solves are the same linear solves either way."""
    c = p.c if c is None else c
    G = p.G().tocsc()
    M = (sp.diags(c) + p.gamma * G).tocsc()
    return Factors(G=G, c=c, gamma=p.gamma, lu_M=spla.splu(M, permc_spec="MMD_AT_PLUS_A"),
                   lu_G=spla.splu(G, permc_spec="MMD_AT_PLUS_A"))


# ---------------------------------------------------------------------------
# Alg. 1 (the Arnoldi process of the circuit solver) with X1 = C + gamma G, X2 = C  (Sec. 3.3.2)
# ---------------------------------------------------------------------------

@dataclass
class Basis:
    beta: float
    V: np.ndarray          # (m, n) orthonormal rows v_1..v_m
    Ht: np.ndarray         # (m+1, m) Hessenberg of the shift-and-invert Arnoldi
    m: int
    H: np.ndarray          # (m, m) = (I - Ht_m^{-1}) / gamma   (Eq. 9)
    converged: bool
    breakdown: bool
    residuals: list = field(default_factory=list)


def rational_H(Ht_m, gamma):
    """H_m = (I - Htilde_m^{-1}) / gamma (Eq. 9)."""
    m = Ht_m.shape[0]
    return (np.eye(m) - np.linalg.inv(Ht_m)) / gamma


def krylov_H(Ht_m, gamma, variant="R"):
    """The matrix whose exponential stands for e^{hA} on the Krylov space:
    rational  (I - Htilde^{-1}) / gamma (Eq. 9);
    inverted  H'^{-1}, where the Arnoldi of -A^{-1} gives Htilde = -H' (Sec. 3.3.1);
    standard  the Arnoldi Hessenberg of A itself (Sec. 2.3)."""
    if variant == "R":
        return rational_H(Ht_m, gamma)
    if variant == "I":
        return -np.linalg.inv(Ht_m)
    if variant == "S":
        return Ht_m.copy()
    raise ValueError(variant)


def residual(beta, h_next, H, h):
    """Empirical posterior error of Sec. 3.3.3:
    ||v|| |htilde_{m+1,m} e_m^T e^{hH_m} e_1|."""
    e = sla.expm(h * H)
    return beta * abs(h_next) * abs(e[-1, 0])


def residual_scale(variant, gamma):
    """The empirical residual of Sec. 3.3.3 uses h_{m+1,m} of the variant's own
    Arnoldi: dimensionless for the rational operator, in seconds for the
    inverted one, in 1/s for A itself.  So that one tolerance in volts serves
    all three, h_{m+1,m} is scaled by the shift: the rational operator acts
    on a stiff mode like the inverted one divided by gamma, and like A^{-1}
    divided by -gamma."""
    return {"R": 1.0, "I": 1.0 / gamma, "S": gamma}[variant]


def arnoldi(fac, v, h_checks, tol, m_max, replay_m=None, variant="R"):
    """Alg. 1 for the operator of ``variant`` (default the shift-and-invert
    w = (C+gamma G)^{-1} C v_j), with modified Gram-Schmidt as written.  Stops
    at the first j whose residual at every h in ``h_checks`` is below tol, at
    a happy breakdown, at m_max, or exactly at ``replay_m`` when given."""
    beta = float(np.linalg.norm(v))
    n = v.shape[0]
    V = np.zeros((m_max + 1, n))
    Ht = np.zeros((m_max + 1, m_max))
    V[0] = v / beta
    res_log = []
    m = m_max
    converged = False
    breakdown = False
    limit = m_max if replay_m is None else replay_m
    for j in range(limit):
        w = fac.op(variant, V[j])                # R, I: a forward/backward substitution pair
        for i in range(j + 1):                   # modified Gram-Schmidt
            Ht[i, j] = w @ V[i]
            w = w - Ht[i, j] * V[i]
        Ht[j + 1, j] = np.linalg.norm(w)
        m = j + 1
        if Ht[j + 1, j] <= BREAKDOWN_REL * abs(Ht[0, 0]):   # |.|: h_11 < 0 for 'S'
            breakdown = True
            converged = True
            break
        V[j + 1] = w / Ht[j + 1, j]
        if replay_m is not None:
            continue
        H = krylov_H(Ht[:m, :m], fac.gamma, variant)
        hs = residual_scale(variant, fac.gamma) * Ht[m, m - 1]
        rs = [residual(beta, hs, H, h) for h in h_checks]
        res_log.append(max(rs))
        if max(rs) < tol:
            converged = True
            break
    H = krylov_H(Ht[:m, :m], fac.gamma, variant)
    return Basis(beta=beta, V=V[:m].copy(), Ht=Ht[:m + 1, :m].copy(), m=m, H=H,
                 converged=converged, breakdown=breakdown, residuals=res_log)


def krylov_expv(basis, h):
    """||v|| e^{h H_m} e_1, the coefficient vector of Eq. 9."""
    return basis.beta * sla.expm(h * basis.H)[:, 0]


# ---------------------------------------------------------------------------
# Alg. 2 (circuit solver) for one group, with superposition over groups
# ---------------------------------------------------------------------------

@dataclass
class GroupLog:
    lts: np.ndarray
    m: list = field(default_factory=list)       # m per segment (0 = quiescent)
    nonconv: int = 0
    breakdowns: int = 0


def run_group(p, fac, k, X, t_out, nodes=None, replay_m=None, amp_scale=None, keep=None,
              variant="R"):
    """Simulate group k (Alg. 2) and add its response at the output times
    into X (rows = output index, columns = ``nodes`` or all nodes)."""
    lts = local_transition_spots(p, k)
    outs = segment_outputs(lts, t_out)
    log = GroupLog(lts=lts)
    sel = slice(None) if nodes is None else nodes
    # the local initial solution of Alg. 2: the group's own DC state at t = 0.
    x = fac.solve_G(input_vector(p, k, lts[0], amp_scale))
    X[0] += x[sel]
    for j in range(lts.shape[0] - 1):
        l0, l1 = lts[j], lts[j + 1]
        L = l1 - l0
        u0 = input_vector(p, k, l0, amp_scale)
        u1 = input_vector(p, k, l1, amp_scale)
        s = (u1 - u0) / L                          # slope of B_k u_k on the segment
        z = fac.solve_G(u0)                        # -A^{-1} b(l_j)
        zp = fac.solve_G(s)                        # -A^{-1} b'
        w = fac.solve_G(fac.c * zp)                # A^{-2} b'
        v = x + (-z + w)                           # x(t) + F(t,h), Eq. 6
        o_idx = outs[j]
        hs = t_out[o_idx] - l0
        if np.linalg.norm(v) <= QUIESCENT_BETA:
            basis = None
            log.m.append(0)
        else:
            h_first = hs[0] if hs.shape[0] else L
            rm = None if replay_m is None else replay_m[j]
            basis = arnoldi(fac, v, (min(h_first, L), L), p.tol, p.m_max, replay_m=rm,
                            variant=variant)
            log.m.append(basis.m)
            log.nonconv += int(not basis.converged)
            log.breakdowns += int(basis.breakdown)
        if keep is not None:
            keep.append(dict(j=j, l0=l0, L=L, z=z, zp=zp, w=w, v=v, basis=basis))
        # snapshots inside (l_j, l_{j+1}]: reuse the basis, only e^{h_a H_m} changes
        if o_idx.shape[0]:
            P = z[sel][None, :] + hs[:, None] * zp[sel][None, :] - w[sel][None, :]
            if basis is not None:
                Y = np.stack([krylov_expv(basis, h) for h in hs], axis=1)   # (m, n_o)
                P = P + (basis.V[:, sel].T @ Y).T
            X[o_idx] += P
        # state at the next LTS point
        x_next = z + L * zp - w
        if basis is not None:
            x_next = x_next + basis.V.T @ krylov_expv(basis, L)
        x = x_next
    return log


@dataclass
class RunResult:
    X: np.ndarray                      # (N+1, n_nodes): node voltages at t_o
    logs: list
    x_dc: np.ndarray


def rmatex(p, groups=None, nodes=None, replay_m=None, fac=None, amp_scale=None,
           include_dc=True, variant="R"):
    """R-MATEX over every group (or the listed ones) with superposition:
    X[o] = x_dc + sum_k x_k(t_o).  ``replay_m[k][j]`` forces m per segment.
    ``variant`` 'I' or 'S' runs the same circuit solver with the inverted
    (I-MATEX) or standard (MEXP) Krylov space instead of the rational one."""
    fac = factorize(p) if fac is None else fac
    t_out = output_times(p)
    ncols = p.n if nodes is None else len(nodes)
    X = np.zeros((t_out.shape[0], ncols))
    x_dc = fac.solve_G(p.dc_inject)
    if include_dc:
        X += (x_dc if nodes is None else x_dc[nodes])[None, :]
    logs = []
    for k in (range(p.n_groups) if groups is None else groups):
        rm = None if replay_m is None else replay_m[k]
        logs.append(run_group(p, fac, k, X, t_out, nodes=nodes, replay_m=rm, amp_scale=amp_scale,
                              variant=variant))
    return RunResult(X=X, logs=logs, x_dc=x_dc)


# ---------------------------------------------------------------------------
# Independent references used to pin the oracle
# ---------------------------------------------------------------------------

def trapezoidal(p, h, t_stop=None, amp_scale=None):
    """Fixed-step TR (Eq. 2) on the whole system from the DC state; returns
    the states at every multiple of h up to t_stop (inclusive)."""
    t_stop = sim_end(p) if t_stop is None else t_stop
    G = p.G().tocsc()
    C = sp.diags(p.c)
    lhs = spla.splu((C / h + G / 2).tocsc())
    rhs_mat = (C / h - G / 2).tocsr()
    nsteps = int(round(t_stop / h))
    x = spla.splu(G).solve(full_input_vector(p, 0.0, amp_scale))
    xs = [x]
    b_prev = full_input_vector(p, 0.0, amp_scale)
    for i in range(1, nsteps + 1):
        b_next = full_input_vector(p, i * h, amp_scale)
        x = lhs.solve(rhs_mat @ x + 0.5 * (b_prev + b_next))
        xs.append(x)
        b_prev = b_next
    return np.arange(nsteps + 1) * h, np.array(xs)


def all_transition_spots(p):
    """GTS: the union of every group's LTS."""
    pts = [local_transition_spots(p, k) for k in range(p.n_groups)]
    return np.unique(np.concatenate(pts)) if pts else np.array([0.0, sim_end(p)])


def dense_augmented(p, t_query, amp_scale=None):
    """Exact solution of Eq. 1 with PWL input via Eq. 4, integrated on each
    GTS segment with the augmented matrix exponential (Van Loan 1978):
    d/dtau [x; a; c] = [[A, b', b0], [0, 0, 1], [0, 0, 0]] [x; a; c],
    a(0) = 0, c = 1, so x' = A x + b0 + b' tau.  Uses A = -C^{-1}G densely;
    only for small n.  Independent of the A^{-1} algebra of Eq. 5/6."""
    n = p.n
    G = p.G().toarray()
    Cinv = 1.0 / p.c
    A = -Cinv[:, None] * G
    gts = all_transition_spots(p)
    x = np.linalg.solve(G, full_input_vector(p, 0.0, amp_scale))
    out = {}
    t_query = np.asarray(t_query, dtype=np.float64)
    for j in range(gts.shape[0] - 1):
        l0, l1 = gts[j], gts[j + 1]
        b0 = Cinv * full_input_vector(p, l0, amp_scale)
        bs = Cinv * (full_input_vector(p, l1, amp_scale) - full_input_vector(p, l0, amp_scale)) / (l1 - l0)
        Aug = np.zeros((n + 2, n + 2))
        Aug[:n, :n] = A
        Aug[:n, n] = bs
        Aug[:n, n + 1] = b0
        Aug[n, n + 1] = 1.0
        z0 = np.concatenate([x, [0.0, 1.0]])
        for q in np.nonzero((t_query > l0) & (t_query <= l1))[0]:
            out[int(q)] = (sla.expm((t_query[q] - l0) * Aug) @ z0)[:n]
        x = (sla.expm((l1 - l0) * Aug) @ z0)[:n]
    res = np.zeros((t_query.shape[0], n))
    x0 = np.linalg.solve(G, full_input_vector(p, 0.0, amp_scale))
    for q in range(t_query.shape[0]):
        res[q] = out.get(q, x0)
    return res
