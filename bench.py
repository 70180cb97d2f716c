"""Benchmark of batched R-MATEX on one GB300 (or N replicas under torchrun).

Workload: the two-layer 300x300 RC mesh (180,000 nodes, vias every 4th node,
400 pads), 2,000 triangular-pulse loads in 64 bump groups, 10 ns simulated,
output every 10 ps (1,001 output times), gamma = 1e-11 s, m <= 20, tol 1e-7.
One step = one complete batched R-MATEX transient of that grid (every group,
every segment, every output), inputs resident on the device.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead
(rank 0 only), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("node-steps/sec (nodes × output steps × groups) FP64, batched vs one-group "
          "launches; SpTRSV HBM GB/s")
UNIT = "node-steps/s"
WORKLOAD = "rmatex_mesh2x300x300_180k_nodes_2000src_64groups_10ns_10ps"
TAIL_EPS = 1e-12  # per group, in units of Vdd: 64 groups stay 64x inside the 1e-9 Vdd bound


def work_model(p, m_seq):
    """Whole-run work model (the terms of Eq. 11-12) from the Krylov
    dimension of every (group, segment) of a run, groups in order and
    segments in time order (segments that built no basis have m = 0):

    * solve_columns: sum over Krylov segments of (m + 2) (m shift-and-invert
      solves, plus the G-solves of z' and w);
    * critical_path_sweeps: the longest per-group chain, max_k sum (m + 2):
      what one compute node per group would run in sequence;
    * batched_sweeps: the segment-aligned rounds run here, sum over rounds
      of (largest m in the round + 2);
    * recombine_vy_gflop: 2 n sum over segments of nout * m, the V y part of
      the recombination (an output t_o belongs to the segment with
      l_j < t_o <= l_{j+1})."""
    import numpy as np
    n_steps = int(round(p.t_end / p.dt_out))
    T = n_steps * p.dt_out
    t_out = np.arange(n_steps + 1, dtype=np.float64) * p.dt_out
    m_seq = np.asarray(m_seq)
    pos = cols = chain = 0
    round_max = {}
    vy = 0.0
    for k in range(p.n_groups):
        pts = {0.0, T}
        for s in np.nonzero(p.src_group == k)[0]:
            pts.update(float(t) for t in p.pwl_t[p.pwl_off[s]:p.pwl_off[s + 1]] if 0.0 < t < T)
        lts = sorted(pts)
        ms = m_seq[pos:pos + len(lts) - 1]
        pos += len(lts) - 1
        own = 0
        for j, m in enumerate(int(v) for v in ms):
            if m <= 0:
                continue
            own += m + 2
            round_max[j] = max(round_max.get(j, 0), m)
            nout = int(np.count_nonzero((t_out > lts[j]) & (t_out <= lts[j + 1])))
            vy += 2.0 * p.n * nout * m
        cols += own
        chain = max(chain, own)
    if pos != m_seq.shape[0]:
        raise ValueError(f"m sequence has {m_seq.shape[0]} entries, the schedule {pos}")
    return {"solve_columns": cols, "critical_path_sweeps": chain,
            "batched_sweeps": sum(m + 2 for m in round_max.values()),
            "recombine_vy_gflop": vy / 1e9}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = 6800.0, "fallback"
    try:
        with open(path) as f:
            d = json.load(f)
        hbm, src = float(d["hbm_gbs"]), "measured"
    except Exception:
        pass
    # FP64 peak from the unit counts and clocks: 152 SMs x 2070 MHz x 2 FP64 FMA
    # per SM per clock (= 4 flop), i.e. the 1.25 TFLOP/s FP64 rate of GB300.
    fp64 = 152 * 2070e6 * 4 / 1e12
    return hbm, src, fp64


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


_POOL = {}


def _oracle_group(g):
    """One group of the workload through the oracle, in a pool worker (the
    problem and its factors are inherited from the parent at fork)."""
    from oracle import rmatex_ref as R
    t0 = time.perf_counter()
    R.rmatex(_POOL["p"], fac=_POOL["fac"], groups=[int(g)])
    return time.perf_counter() - t0


def oracle_pool(workers):
    """The bench grid factorised once by the oracle, then a pool of `workers`
    processes forked from this process (which never touches the GPU), one
    BLAS thread each; returns (problem, pool)."""
    import multiprocessing as mp

    import gridgen
    from oracle import rmatex_ref as R
    p = gridgen.config1()
    _POOL["p"] = p
    _POOL["fac"] = R.factorize(p)
    return p, mp.get_context("fork").Pool(workers)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_oracle_sample(workers: int) -> dict:
    """The oracle as it stands on `workers` groups of the workload, one group
    per worker process running at once (factorisation excluded)."""
    p, pool = oracle_pool(workers)
    groups = list(range(min(workers, p.n_groups)))
    t0 = time.perf_counter()
    per = pool.map(_oracle_group, groups, chunksize=1)
    dt = time.perf_counter() - t0
    pool.close()
    pool.join()
    units = p.n * (p.n_out - 1) * len(groups)
    return {"value": units / dt, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{len(groups)} of 64 groups of the same grid, all 180,000 nodes, "
                      f"1,000 output steps, one group per worker process on {workers} host "
                      f"cores at once; factorisation excluded; {dt:.1f} s wall, "
                      f"{sum(per):.1f} s of CPU work"}


def run_cpu_sample(workers: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-oracle-sample",
                          str(workers)], env=env, stdout=subprocess.PIPE, text=True,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def measured_traffic():
    """DRAM bytes per batched solve call from the committed ncu summary of the
    bench step, valid only while the solve kernels' source is the one the
    counters were taken on (else None, with the reason)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "traffic_solve_mesh2x300x300.md")
    csrc = os.path.join(ROOT, "paper_1511_04519_gb300", "csrc")
    try:
        text = open(path).read()
        h = hashlib.sha256()
        for f in ("k_sptrsv.cu", "k_sptrsv_k1.cu"):
            h.update(open(os.path.join(csrc, f), "rb").read())
        sha = h.hexdigest()[:16]
    except OSError as exc:
        return None, f"no summary: {exc}"
    m_b = re.search(r"traffic_per_solve_call_bytes:\s*([0-9.eE+]+)", text)
    m_s = re.search(r"solve_kernels_sha256_16:\s*([0-9a-f]+)", text)
    if not m_b or not m_s:
        return None, "summary without the traffic line"
    if m_s.group(1) != sha:
        return None, "the solve kernels changed since the counters were taken"
    return float(m_b.group(1)), f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {path}"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, pg, device):
    """x (a time) as the job's clock sees it: the largest over the ranks of the
    process group module pg (None: one process, x itself)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job rate: every one of `world` ranks processed units_per_rank
    in `seconds` (the slowest rank's time)."""
    return world * units_per_rank / seconds


def workload_config(p, world):
    """The `config` of both arms' JSON lines."""
    return {"workload": WORKLOAD, "nodes": p.n, "groups": p.n_groups,
            "output_steps": p.n_out - 1, "sources": p.n_src,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "working set (factors, bases, 1.44 GB of outputs) > 129 MB L2"}


def reference_arm(args):
    """The oracle as it stands on the host's cores: each step runs one group
    per core at once (a forked pool; this process never touches the GPU),
    cycling through the 64 groups."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    workers = host_cores()
    p, pool = oracle_pool(workers)
    times, cpu_s = [], 0.0
    g0 = 0
    for i in range(args.warmup + args.steps):
        groups = [(g0 + k) % p.n_groups for k in range(min(workers, p.n_groups))]
        g0 += len(groups)
        t0 = time.perf_counter()
        per = pool.map(_oracle_group, groups, chunksize=1)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            cpu_s += sum(per)
    pool.close()
    pool.join()
    step_s = sum(times) / len(times)
    per_step = min(workers, p.n_groups)
    value = p.n * (p.n_out - 1) * per_step / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(p, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"each step: {per_step} of the 64 groups of the same "
                                       f"grid through the FP64 oracle (SuperLU, MGS, scipy "
                                       f"expm), all nodes and outputs, one group per worker "
                                       f"process on {workers} host cores at once; "
                                       f"factorisation excluded; {cpu_s:.1f} s of CPU work "
                                       f"over the timed steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def ncu_case(what: str) -> int:
    """The bench grid restricted to groups 0-7 (32 for "levels"; a few GB on the
    device, solve panels still larger than L2): one warm call, then the
    profiled call.  "solve": matex_solve of 16 columns with the persistent
    kernel; "levels": 64 columns with one launch per tree level; "run": one
    full matex_run; "ksweep": bare solve pairs of 1, 4 and 64 columns on the
    whole grid; "small": one run of the 1,024-node single-group grid;
    "tcsolve": one 64-column solve pair of the whole grid with the wide panels
    on the tensor cores."""
    import numpy as np
    import torch

    import gridgen
    from paper_1511_04519_gb300 import build as B
    B.build()
    from paper_1511_04519_gb300 import matex as M
    p = gridgen.config1()
    groups = 32 if what == "levels" else 8
    sel = p.src_group < groups
    off = np.concatenate([[0], np.cumsum(np.diff(p.pwl_off)[sel])]).astype(np.int32)
    q = gridgen.with_sources(p, p.src_node[sel], off, p.pwl_t.reshape(-1, 3)[sel].ravel(),
                             p.pwl_v.reshape(-1, 3)[sel].ravel(), p.src_group[sel], groups)
    if what == "tcsolve":
        # the whole bench grid, wide panels forced onto the tensor cores: one
        # 64-column solve pair of C + gamma G after a warm one
        sim = M.Sim(p, tc_solve="on", solve_mode=1, include_dc=False,
                    rows=np.arange(4, dtype=np.int32))
        sim.time_solve(0, 64, reps=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        sim.time_solve(0, 64, reps=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_case": what, "max_memory_gb": torch.cuda.max_memory_allocated() / 1e9}))
        return 0
    if what == "k1":
        # the whole bench grid, one right-hand side on the single-column level
        # kernels: one solve pair of C + gamma G after a warm one
        sim = M.Sim(p, single_column="on", include_dc=False, rows=np.arange(4, dtype=np.int32))
        sim.time_solve(0, 1, reps=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        sim.time_solve(0, 1, reps=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_case": what, "max_memory_gb": torch.cuda.max_memory_allocated() / 1e9}))
        return 0
    if what == "small":
        # the single-group 1,024-node grid as set up by default (resident
        # rounds): one warm run, then one run inside the profiler range
        sim = M.Sim(gridgen.config0(), graph=False)
        x = sim.run()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        sim.run(x)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_case": what, "resident": sim.stats.resident}))
        return 0
    if what == "ksweep":
        # the whole bench grid, level-by-level launches: one bare solve pair of
        # 1, 4 and 64 right-hand sides (each after its own warm-up call)
        sim = M.Sim(p, solve_mode=1)
        for k in (1, 4, 64):
            sim.time_solve(0, k, reps=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for k in (1, 4, 64):
            sim.time_solve(0, k, reps=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_case": what, "max_memory_gb": torch.cuda.max_memory_allocated() / 1e9}))
        return 0
    sim = M.Sim(q, solve_mode={"solve": 0, "levels": 1}.get(what, 2))
    if what in ("solve", "levels"):
        k = 16 if what == "solve" else 64
        b = torch.randn(k, p.n, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        M.matex_solve(sim.ctx, 0, k, b.data_ptr(), x.data_ptr())
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        M.matex_solve(sim.ctx, 0, k, b.data_ptr(), x.data_ptr())
    else:
        out = sim.run()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        sim.run(out)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"ncu_case": what, "max_memory_gb": torch.cuda.max_memory_allocated() / 1e9}))
    return 0


def batch_grids(args, M, stream):
    """The uneven-grid workload: independent single-layer meshes (side
    U[100, 450], 4-16 groups each) run as one CUDA graph launch, one branch per
    grid.  Each grid outputs 64 sampled nodes (its internal output buffer
    still holds every node)."""
    import numpy as np
    import torch

    import gridgen
    probs = gridgen.config4()[: args.grids]
    t0 = time.perf_counter()
    sims = []
    for p in probs:
        rows = np.sort(np.random.default_rng(p.n).choice(p.n, 64, replace=False)).astype(np.int32)
        sims.append(M.Sim(p, rows=rows, stream=stream))
    setup_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = M.Batch(sims)          # a plain, recorded run of every grid
    record_s = time.perf_counter() - t0
    outs = [torch.empty((s.n_times, s.n_rows), dtype=torch.float64, device="cuda") for s in sims]
    for _ in range(args.warmup):
        batch.run(outs)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    grid_ms = []
    for _ in range(args.steps):
        _, gm = batch.run(outs)
        grid_ms.append(gm)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    gm = np.mean(np.array(grid_ms), axis=0)
    replayed = sum(int(s.stats.graph_replay) for s in sims)
    units = sum(p.n * (p.n_out - 1) * p.n_groups for p in probs)
    # the same grids one after another (each its own graph replay)
    ev0.record(stream)
    for s, o in zip(sims, outs):
        s.run(o)
    ev1.record(stream)
    torch.cuda.synchronize()
    seq_ms = ev0.elapsed_time(ev1)
    res = {"workload": f"{len(probs)}_single_layer_meshes_side_100_450",
           "nodes": int(sum(p.n for p in probs)), "groups": int(sum(p.n_groups for p in probs)),
           "value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "grids_replayed": replayed, "sequential_ms": seq_ms,
           "concurrency_speedup": seq_ms / ms,
           "grid_ms": {"min": float(gm.min()), "median": float(np.median(gm)), "max": float(gm.max())},
           "setup_s": setup_s, "record_s": record_s}
    batch.close()
    del sims
    torch.cuda.empty_cache()
    return res


def small_grid(M, stream, steps):
    """The single-group 1,024-node grid (192 sequential segments): a recorded
    run, then `steps` timed graph replays, as set up by default (the setup
    picks resident rounds here) and on the batched path (resident off)."""
    import torch

    import gridgen
    p = gridgen.config0()
    res = {"workload": "grid32x32_1group", "nodes": p.n, "groups": p.n_groups}
    for name, mode in (("default", "auto"), ("batched_path", "off")):
        t0 = time.perf_counter()
        sim = M.Sim(p, stream=stream, resident=mode)
        setup_s = time.perf_counter() - t0
        x = sim.run()
        sim.run(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            sim.run(x)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = sim.stats.as_dict()
        res[name] = {"ms": ms, "value": p.n * (p.n_out - 1) * p.n_groups / (ms / 1e3), "unit": UNIT,
                     "resident": st["resident"], "kernel_launches": st["kernel_launches"],
                     "rounds": st["rounds"], "sum_m": st["sum_m"], "setup_s": setup_s,
                     "graph_replay": st["graph_replay"]}
        del sim, x
    res["resident_speedup"] = res["batched_path"]["ms"] / res["default"]["ms"]
    return res


def other_configs(M, stream, ramps_large=False):
    """One recorded run, then one timed graph replay, of the four-layer
    1.44M-node grid with 256 uneven groups (64 sampled output rows), and with
    ramps_large the same grid decomposed into ramps (25,600 columns in
    batches of 256)."""
    import numpy as np
    import torch

    import gridgen
    res = {}
    cases = [("mesh4x600x600_256groups", gridgen.config2(), 64, "groups")]
    if ramps_large:
        cases.append(("mesh4x600x600_256groups_ramps", gridgen.config2(), 64, "ramps"))
    for name, p, nrows, dec in cases:
        rows = None
        if nrows:
            rows = np.sort(np.random.default_rng(0).choice(p.n, nrows, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        sim = M.Sim(p, rows=rows, stream=stream, decompose=dec)
        setup_s = time.perf_counter() - t0
        x = sim.run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(x)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = sim.stats.as_dict()
        sst = sim.setup_stats()
        # one more run launch by launch, CUDA events around every kernel class
        sim.profile(on=True)
        sim.run(x)
        torch.cuda.synchronize()
        prof = sim.profile(on=False)
        res[name + "_profile_ms"] = {k: v["ms"] for k, v in prof.items()}
        res[name + "_tc_solve"] = {"supernodes": sst["tc_solve_supernodes"],
                                   "min_cols": sst["tc_solve_min_cols"]}
        res[name] = {"nodes": p.n, "groups": p.n_groups, "ms": ms,
                     "value": p.n * (p.n_out - 1) * p.n_groups / (ms / 1e3), "unit": UNIT,
                     "setup_s": setup_s, "graph_replay": st["graph_replay"],
                     "rounds": st["rounds"], "solve_columns": st["solve_columns"],
                     "nonconv": st["nonconv"], "nnz_L": st["nnz_L"],
                     "nnz_L_exact": st["nnz_L_exact"], "tc_rounds": st["tc_rounds"],
                     "decompose": dec, "sum_m": st["sum_m"]}
        del sim, x
        torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-oracle-sample", type=int, default=0)
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="oracle worker processes for cpu_baseline (0: every host core)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serial", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-tr", action="store_true")
    ap.add_argument("--no-ramps", action="store_true",
                    help="skip the ramp-decomposition run of the bench grid")
    ap.add_argument("--no-tail", action="store_true",
                    help="skip the separately reported tail-skipping run (tail_eps > 0)")
    ap.add_argument("--other-configs", action="store_true",
                    help="also time one graph-replayed run of the 1.44M-node 256-group grid "
                         "(about four minutes with its setup and recorded run)")
    ap.add_argument("--ramps-large", action="store_true",
                    help="with --other-configs, also the 1.44M-node grid as ramps")
    ap.add_argument("--variants", action="store_true",
                    help="also run the inverted (I-MATEX) and standard (MEXP) Krylov spaces "
                         "on the bench grid (Table 1's comparison)")
    ap.add_argument("--grids", type=int, default=96,
                    help="run that many of the 96 uneven single-layer grids as one batch graph "
                         "launch and report their aggregate rate (0: skip)")
    ap.add_argument("--profile-step", action="store_true",
                    help="warm up, run one step inside cudaProfilerStart/Stop, print its stats")
    ap.add_argument("--ncu-case", choices=["solve", "levels", "run", "ksweep", "small", "tcsolve", "k1"], default=None,
                    help="reduced case for full ncu captures: the same grid with 8 groups; "
                         "one warm call, then one call inside cudaProfilerStart/Stop")
    args = ap.parse_args()
    if args.cpu_oracle_sample:
        print(json.dumps(cpu_oracle_sample(args.cpu_oracle_sample)))
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    if args.ncu_case:
        return ncu_case(args.ncu_case)
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch

    import gridgen
    from paper_1511_04519_gb300 import build as B
    B.build()
    from paper_1511_04519_gb300 import matex as M

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    # replicas: every rank simulates its own independently seeded grid
    p = gridgen.config1(seed=gridgen.SEED_BASE + 1 + 1000 * rank)
    stream = torch.cuda.current_stream()
    sim = M.Sim(p, stream=stream)
    setup = sim.setup_stats()
    tuning = sim.autotune()
    level_blocks = sim.level_blocks()
    out = torch.empty((sim.n_times, sim.n_rows), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        sim.run(out)
    torch.cuda.synchronize()
    if args.profile_step:
        torch.cuda.profiler.start()
        sim.run(out)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": sim.stats.as_dict()}))
        return 0
    hbm_peak, hbm_src, fp64_nominal = _peaks()
    # FP64 peak measured on this device by the library's FMA probe
    fp64_peak, fp64_probe_ms = M.measure_fp64_peak(5)

    clk = ClockSampler(local)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        sim.run(out)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = clk.stop()
    launches_per_step = sim.stats.kernel_launches
    stats = sim.stats.as_dict()
    ms = max_over_ranks(ms, pg, "cuda")
    units = p.n * (p.n_out - 1) * p.n_groups
    value = job_rate(units, world, ms / 1e3)

    # profiled steps (CUDA events around every kernel class on the run's stream)
    sim.profile(on=True)
    ev0.record(stream)
    for _ in range(args.steps):
        sim.run(out)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_prof = ev0.elapsed_time(ev1) / args.steps
    prof = sim.profile(on=False)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    per_launch_ms = d["ms"] / max(1, d["units"])
    ridge = fp64_peak * 1e12 / (hbm_peak * 1e9)
    intensity = d["flops"] / d["bytes"] if d["bytes"] else float("inf")
    if intensity > ridge:
        roof = {"bound": "alu", "achieved": d["flops"] / (d["ms"] / 1e3) / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s"}
        roof["peak_source"] = ("FP64 measured: matex_measure_fp64_peak (independent FMA chains "
                               f"on every SM, best of 5, {fp64_probe_ms:.2f} ms); unit-count figure "
                               f"152 SM x 2070 MHz x 4 flop/clk = {fp64_nominal:.3f}")
    else:
        roof = {"bound": "hbm", "achieved": d["bytes"] / (d["ms"] / 1e3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "peak_source": f"{hbm_src} copy bandwidth"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = dom
    roof["per_launch_ms"] = per_launch_ms
    roof["algorithmic_per_launch"] = (d["flops"] if roof["unit"] == "TFLOP/s" else d["bytes"]) / max(
        1, d["units"])
    roof["algorithmic_bytes_per_launch"] = d["bytes"] / max(1, d["units"])
    traffic, traffic_src = measured_traffic() if dom == "solve" else (None, "not the solve class")
    roof["traffic"] = traffic
    roof["traffic_source"] = traffic_src
    s = prof["solve"]
    sptrsv = {"achieved_gbs": s["bytes"] / (s["ms"] / 1e3) / 1e9 if s["ms"] else None,
              "achieved_tflops": s["flops"] / (s["ms"] / 1e3) / 1e12 if s["ms"] else None,
              "frac_hbm": (s["bytes"] / (s["ms"] / 1e3) / 1e9) / hbm_peak if s["ms"] else None,
              "frac_fp64": (s["flops"] / (s["ms"] / 1e3) / 1e12) / fp64_peak if s["ms"] else None,
              "work_from": "exact fill of L (nnz_L_exact), not the amalgamated panels"}
    # The solve pair alone, per column count: where bytes dominate (one or two
    # right-hand sides) its roofline is HBM, above that the FP64 pipe.
    nnz = float(setup["nnz_L_exact"])
    by_k = []
    for K in (1, 2, 4, 8, 16, 32, 64):
        try:
            best, mean = sim.time_solve(0, K, reps=20)
        except M.MatexError:   # wider than the context's column buffer
            break
        byt = 2.0 * (12.0 * nnz + 4.0 * (p.n + 1)) + 8.0 * p.n + 32.0 * p.n * K
        fl = (4.0 * nnz + 2.0 * p.n) * K
        by_k.append({"ncols": K, "ms": best, "mean_ms": mean,
                     "gbs": byt / (best / 1e3) / 1e9, "frac_hbm": byt / (best / 1e3) / 1e9 / hbm_peak,
                     "tflops": fl / (best / 1e3) / 1e12,
                     "frac_fp64": fl / (best / 1e3) / 1e12 / fp64_peak})
    sptrsv["by_ncols"] = by_k
    sptrsv["k1"] = dict(by_k[0], algorithmic_bytes=2.0 * (12.0 * nnz + 4.0 * (p.n + 1)) + 40.0 * p.n,
                        single_column_kernels=int(setup.get("single_column", 0)),
                        note="one right-hand side: the column count where the solve's bytes "
                             "dominate (0.2 flop/byte), so its roofline is HBM")

    # one group at a time: the same kernels, one column per launch
    serial = None
    if not args.no_serial:
        sim.one_group_at_a_time(True)
        sim.run(out)
        torch.cuda.synchronize()
        ev0.record(stream)
        sim.run(out)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_serial = ev0.elapsed_time(ev1)
        sim.one_group_at_a_time(False)
        serial = {"value": units / (ms_serial / 1e3), "ms_per_step": ms_serial,
                  "batched_speedup": ms_serial / ms}

    # end to end through the host-buffer C-ABI call: pinned H2D of the source
    # currents, the run, and the D2H of every node voltage at every output time
    pin_v = torch.from_numpy(np.asarray(p.pwl_v, np.float64)).pin_memory().numpy()
    pin_out = torch.empty((sim.n_times, sim.n_rows), dtype=torch.float64).pin_memory().numpy()
    sim.run_host(pin_v, pin_out)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.run_host(pin_v, pin_out)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(e2e_s, pg, "cuda")
    e2e = {"value": job_rate(units, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(pin_v.nbytes),
           "d2h_bytes_per_step": int(pin_out.nbytes), "ms_per_step": e2e_s * 1e3}

    # the paper's comparison method on the same solves: fixed-step trapezoidal
    # integration with h = 10 ps (the output step), all sources at once
    trap = None
    if not args.no_tr:
        sim.run(out)
        xr = out.clone()
        t0 = time.perf_counter()
        xt, _ = sim.tr_run(1)                       # factor of C + h/2 G, recorded loop
        first_s = time.perf_counter() - t0
        tr_ms = min(sim.tr_run(1, xt)[1] for _ in range(2))
        trap = {"h_ps": p.dt_out * 1e12, "steps": p.n_out - 1, "ms": tr_ms,
                "rmatex_speedup": tr_ms / ms, "first_call_s": first_s,
                "max_abs_diff_vs_rmatex_v": float((xt - xr).abs().max())}
        del xt, xr

    # the work model beside the measured counts and times (auxiliary: a
    # failure here is reported in the line, never fatal)
    try:
        wm = work_model(p, sim.m_sequence())
        rec_s = prof["recombine"]["ms"] / args.steps / 1e3
        wm["measured"] = {"solve_columns": stats["solve_columns"],
                          "sweeps": stats["sweeps_M"] + stats["sweeps_G"],
                          "solve_ms": prof["solve"]["ms"] / args.steps,
                          "recombine_ms": rec_s * 1e3,
                          "recombine_vy_tflops": wm["recombine_vy_gflop"] / 1e3 / rec_s
                          if rec_s > 0 else None}
        wm["note"] = ("measured solve columns and sweeps also count the one G-solve of the "
                      "pads' DC state")
    except Exception as exc:  # noqa: BLE001
        wm = {"error": f"{type(exc).__name__}: {exc}"}

    # tail skipping (opt-in, changes the work): a group's term of an output
    # loses V y once ||y||_2 stays below eps/2, and vanishes when its -P term
    # is below eps/2 too; every entry stays within n_groups * eps of the exact run
    tail = None
    if not args.no_tail:
        sim.run(out)
        xr = out.clone()
        eps = TAIL_EPS * p.vdd
        st_ = M.Sim(p, stream=stream, tail_eps=eps)
        xt = torch.empty_like(out)
        for _ in range(args.warmup):
            st_.run(xt)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            st_.run(xt)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_t = ev0.elapsed_time(ev1) / args.steps
        st_.profile(on=True)
        st_.run(xt)
        torch.cuda.synchronize()
        pt = st_.profile(on=False)
        tail = {"tail_eps_v": eps, "ms_per_step": ms_t, "value": world * units / (ms_t / 1e3),
                "unit": UNIT, "speedup_vs_exact": ms / ms_t,
                "recombine_ms": pt["recombine"]["ms"], "exact_recombine_ms": prof["recombine"]["ms"]
                / args.steps, "max_abs_diff_vs_exact_v": float((xt - xr).abs().max()),
                "bound_v": p.n_groups * eps}
        del st_, xt, xr

    # Table 1's comparison on the bench grid: the same circuit solver with the
    # rational, inverted and standard Krylov spaces (m_max = 20)
    variants = None
    if args.variants:
        sim.run(out)
        xr = out.clone()
        variants = {}
        for name, key in (("rational", "R"), ("inverted", "I"), ("standard", "S")):
            sv = M.Sim(p, stream=stream, krylov=key)
            xv = sv.run()
            sv.run(xv)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sv.run(xv)
            e1.record(stream)
            torch.cuda.synchronize()
            st = sv.stats.as_dict()
            ms_v = [int(m) for m in sv.m_sequence() if m > 0]
            variants[name] = {"ms": e0.elapsed_time(e1), "m_avg": sum(ms_v) / max(1, len(ms_v)),
                              "m_peak": max(ms_v) if ms_v else 0, "nonconv": st["nonconv"],
                              "solve_columns": st["solve_columns"],
                              "max_abs_diff_vs_rational_v": float((xv - xr).abs().max())}
            del sv, xv
        torch.cuda.empty_cache()

    # the paper's source decomposition carried to single ramps (opts.decompose
    # = 1): every ramp's basis in one batched round, no segment chain; same
    # superposed outputs (to the Krylov tolerance), timed like the headline
    ramps = None
    if not args.no_ramps:
        sim.run(out)
        xr = out.clone()
        sr = M.Sim(p, stream=stream, decompose="ramps")
        xq = torch.empty_like(out)
        for _ in range(args.warmup):
            sr.run(xq)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            sr.run(xq)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_r = ev0.elapsed_time(ev1) / args.steps
        st_r = sr.stats.as_dict()
        ramps = {"ms_per_step": ms_r, "value": world * units / (ms_r / 1e3), "unit": UNIT,
                 "speedup_vs_groups": ms / ms_r, "columns": int(sr.n_segments),
                 "rounds": st_r["rounds"], "solve_columns": st_r["solve_columns"],
                 "sum_m": st_r["sum_m"], "graph_replay": st_r["graph_replay"],
                 "max_abs_diff_vs_groups_v": float((xq - xr).abs().max()),
                 "note": "both decompositions meet tol = 1e-7 V per Krylov segment"}
        del sr, xq, xr
        torch.cuda.empty_cache()

    # adjoint: the same grid with 256 observed nodes, IR-drop hinge loss; cost
    # of matex_grad relative to the forward run that keeps what it needs:
    # checkpoints of x and z per segment round (segments recomputed in the
    # reverse sweep), and the full tape of every basis for comparison
    adjoint = None
    if not args.no_adjoint:
        from paper_1511_04519_gb300 import autograd as AG
        del sim
        torch.cuda.empty_cache()
        p3 = gridgen.config3(seed=gridgen.SEED_BASE + 1 + 1000 * rank)
        obs = p3.observed.astype(np.int32)
        adjoint = {"workload": "mesh2x300x300_256_observed_nodes_hinge_loss",
                   "params": {"caps": p3.n, "amplitudes": p3.n_src}}
        for mode in ("checkpoint", "full"):
            sim3 = AG.make_sim(p3, obs, include_dc=False, stream=stream, tape=mode)
            X3 = sim3.run()
            theta = float(torch.quantile((-X3).flatten(), 0.9))
            Xr = X3.detach().clone().requires_grad_(True)
            AG.hinge_ir_drop_loss(Xr, 0.0, theta, p3.dt_out).backward()
            xbar = Xr.grad.detach()
            f_ms, g_ms = [], []
            for it in range(args.warmup + args.steps):
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                sim3.run(X3)
                e1.record(stream)
                sim3.grad(xbar)
                e2.record(stream)
                torch.cuda.synchronize()
                if it >= args.warmup:
                    f_ms.append(e0.elapsed_time(e1))
                    g_ms.append(e1.elapsed_time(e2))
            fm, gm = sum(f_ms) / len(f_ms), sum(g_ms) / len(g_ms)
            st3 = sim3.setup_stats()
            adjoint[mode] = {"forward_ms": fm, "grad_ms": gm, "grad_over_forward": gm / fm,
                             "tape_bytes": st3["tape_bytes"], "tape_window": st3["tape_window"],
                             "tape_block": st3["tape_block"]}
            del sim3, X3, Xr, xbar
            torch.cuda.empty_cache()

    smallg = small_grid(M, stream, args.steps)
    grids = batch_grids(args, M, stream) if args.grids else None
    others = other_configs(M, stream, args.ramps_large) if args.other_configs else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = run_cpu_sample(args.cpu_workers or host_cores())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(p, world),
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "sptrsv": sptrsv, "one_group_at_a_time": serial,
            "cpu_baseline": cpu, "adjoint": adjoint, "trapezoidal": trap,
            "krylov_variants": variants, "tail_skip": tail, "ramp_decomposition": ramps,
            "work_model": wm,
            "profile_ms_per_step": ms_prof,
            "profile": {k: {kk: v[kk] / args.steps for kk in ("ms", "launches", "flops", "bytes")}
                        for k, v in prof.items()},
            "run_stats": {k: stats[k] for k in ("n_segments", "krylov_segments", "sum_m", "max_m",
                                                 "nonconv", "sweeps_M", "sweeps_G", "solve_columns",
                                                 "rounds", "kernel_launches", "graph_replay",
                                                 "graph_capture_ms")},
            "small_grid": smallg, "batch_grids": grids, "other_configs": others,
            "autotune": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in t.items()}
                         for t in tuning],
            "autotune_level_blocks": [{k: (round(v, 4) if isinstance(v, float) else v)
                                       for k, v in t.items()} for t in level_blocks],
            "setup_ms": {"order": setup["setup_order_ms"], "factor": setup["setup_factor_ms"],
                         "upload": setup["setup_upload_ms"], "nnz_L": setup["nnz_L"],
                         "supernodes": setup["n_supernodes"], "levels": setup["n_levels"]},
        }
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
