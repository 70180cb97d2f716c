"""The allocation-free solve entry point against the ordinary one.

matex_solve_noalloc serves callers that may not call cudaMalloc (code inside
another library's allocator or memory-pool callback, or in a process whose
device memory belongs to a pool it must not grow).  It runs the same
triangular solves with the context's factors, in the launch mode the context
uses for each column count, but takes its scratch from a static device array.
This file is collected last on purpose, so that a failure here does not hide
the results of the other GPU tests.
"""
import numpy as np
import pytest

import gridgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04519_gb300 import build
    build.build()
    from paper_1511_04519_gb300 import matex
    return matex


@pytest.mark.parametrize("case", ["config0", "mesh2x120x120"])
@pytest.mark.parametrize("which", [0, 1])
def test_noalloc_solve_matches_matex_solve_twice(M, case, which):
    import torch
    if case == "config0":
        p = gridgen.config0()
    else:
        p = gridgen.small_mesh(3, nx=120, ny=120, layers=2, n_src=12, group_templates=[3] * 4)
    sim = M.Sim(p)
    rng = np.random.default_rng(11)
    for ncols in (1, 5, 13):
        b = torch.from_numpy(rng.standard_normal((ncols, p.n))).cuda()
        ref = torch.empty_like(b)
        M.matex_solve(sim.ctx, which, ncols, b.data_ptr(), ref.data_ptr())
        scale = float(ref.abs().max())
        for _ in range(2):  # two calls in a row share (and reuse) the static scratch
            x = torch.full_like(b, float("nan"))
            M.matex_solve_noalloc(sim.ctx, which, ncols, b.data_ptr(), x.data_ptr())
            torch.cuda.synchronize()
            assert torch.isfinite(x).all()
            assert float((x - ref).abs().max()) <= 1e-12 * scale
    sim.close()


@pytest.mark.parametrize("which", [0, 1])
def test_noalloc_chunked_columns_on_a_large_grid(M, which):
    """125,000 nodes: the static scratch holds the two column buffers for at
    most 4 right-hand sides at a time, so 13 and 16 columns run as several
    chunks (the chunk-size reduction, the per-chunk counter resets and the
    ragged last chunk), each against matex_solve."""
    import torch
    p = gridgen.small_mesh(5, nx=250, ny=250, layers=2, n_src=12, group_templates=[3] * 4,
                           n_pads=40)
    sim = M.Sim(p)
    rng = np.random.default_rng(12)
    for ncols in (13, 16):
        b = torch.from_numpy(rng.standard_normal((ncols, p.n))).cuda()
        ref = torch.empty_like(b)
        M.matex_solve(sim.ctx, which, ncols, b.data_ptr(), ref.data_ptr())
        for _ in range(2):
            x = torch.full_like(b, float("nan"))
            M.matex_solve_noalloc(sim.ctx, which, ncols, b.data_ptr(), x.data_ptr())
            torch.cuda.synchronize()
            assert torch.isfinite(x).all()
            for q in range(ncols):
                scale = float(ref[q].abs().max())
                assert float((x[q] - ref[q]).abs().max()) <= 1e-12 * scale, (ncols, q)
    sim.close()


def test_noalloc_rejects_a_factor_above_its_limit(M):
    """920,000 nodes (a two-node-wide ladder, cheap to factor) exceed the
    static scratch's 917,504-node limit: a clear MATEX_ERR_ARG, nothing run."""
    import torch
    p = gridgen.small_mesh(6, nx=460000, ny=2, n_src=4, n_pads=3)
    assert p.n > 917504
    sim = M.Sim(p)
    b = torch.ones((1, p.n), dtype=torch.float64, device="cuda")
    x = torch.full_like(b, -7.0)
    with pytest.raises(M.MatexError) as ei:
        M.matex_solve_noalloc(sim.ctx, 0, 1, b.data_ptr(), x.data_ptr())
    assert ei.value.status == 1  # MATEX_ERR_ARG
    assert "917504" in str(ei.value)
    torch.cuda.synchronize()
    assert bool((x == -7.0).all())
    sim.close()


_LAZY_CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import gridgen
from paper_1511_04519_gb300 import matex as M
p = gridgen.config0()
sim = M.Sim(p)
g = torch.Generator(device="cuda").manual_seed(0)
b = torch.randn((5, p.n), dtype=torch.float64, device="cuda", generator=g)
x = torch.empty_like(b)
ref = torch.empty_like(b)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
M.matex_solve_noalloc(sim.ctx, 0, 5, b.data_ptr(), x.data_ptr())
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
M.matex_solve(sim.ctx, 0, 5, b.data_ptr(), ref.data_ptr())
torch.cuda.synchronize()
print(json.dumps({"free0": free0, "free1": free1,
                  "err": float((x - ref).abs().max()), "scale": float(ref.abs().max())}))
"""


def test_noalloc_first_call_allocates_nothing_with_lazy_module_loading(M):
    """In a fresh process with lazy module loading, the first allocation-free
    solve after setup leaves the device's free memory unchanged: setup has
    already loaded the module of the static array and every solve kernel."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    out = subprocess.run([sys.executable, "-c", _LAZY_CHILD, root], env=env, check=True,
                         stdout=subprocess.PIPE, text=True, timeout=600)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["free1"] == r["free0"], r
    assert r["err"] <= 1e-12 * r["scale"], r
