"""GPU-vs-oracle comparison shared by the GPU parity tests, with the
bookkeeping of the adaptive Krylov dimension.

The oracle and the GPU evaluate the residual of Sec. 3.3.3 with different
rounding, so a segment whose residual lies within rounding of tol can stop at
a different m.  Such a segment changes the result by about tol (1e-7 V), not
1e-9: the parity bar is then applied to a rerun in replay mode with the
oracle's m sequence.  So that a GPU residual bug cannot hide behind the
replay, every comparison also bounds the adaptive run itself:

* at most max(2, 5 %) of the Krylov segments may pick another m;
* the adaptive run stays within max(1e-9 Vdd, 10 tol) of the oracle.

Each comparison appends a record (mismatch count, adaptive-mode error, replay
error) to REPORT; with MATEX_TEST_REPORT set, the session writes REPORT there
as JSON.
"""
import numpy as np

TOL_V = 1e-9
REPORT = []


def oracle_m(res):
    """The oracle's Krylov dimension per (group, segment), in replay layout."""
    if not res.logs:
        return np.zeros(0, np.int32)
    return np.concatenate([np.asarray(lg.m, np.int32) for lg in res.logs])


def mismatch_bound(n_krylov):
    return max(2, int(0.05 * n_krylov))


def check_adaptive(case, p, X_adaptive, m_gpu, ref, replay_run):
    """Bound the adaptive run, rerun in replay mode where m differs, record
    both, and return the error to hold against 1e-9 Vdd.  replay_run(m) must
    return the GPU result for the given m sequence."""
    m_ref = oracle_m(ref)
    m_gpu = np.asarray(m_gpu)
    n_kry = int(np.count_nonzero(m_ref))
    mism = int(np.count_nonzero(m_gpu != m_ref)) if m_gpu.shape == m_ref.shape else len(m_ref)
    err_a = float(np.abs(np.asarray(X_adaptive) - ref.X).max())
    err = err_a
    if mism:
        err = float(np.abs(np.asarray(replay_run(m_ref)) - ref.X).max())
    REPORT.append({"case": case, "n": int(p.n), "segments": int(len(m_ref)),
                   "krylov_segments": n_kry, "m_mismatch": mism, "adaptive_err_v": err_a,
                   "replay_err_v": err if mism else None})
    assert mism <= mismatch_bound(n_kry), (case, mism, n_kry)
    assert err_a <= max(TOL_V * p.vdd, 10.0 * p.tol), (case, err_a)
    return err
