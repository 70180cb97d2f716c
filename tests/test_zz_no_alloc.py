"""The allocation-free solve entry point against the ordinary one.

matex_solve_noalloc serves callers that may not call cudaMalloc (code inside
another library's allocator or memory-pool callback, or in a process whose
device memory belongs to a pool it must not grow).  It runs the same
persistent triangular solves with the context's factors but takes its scratch
from a static device array.  This file is collected last on purpose, so that a
failure here does not hide the results of the other GPU tests.
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
