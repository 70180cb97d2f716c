"""CPU-side checks of the C ABI library: it builds, loads, exports every
symbol the header declares, rejects bad inputs before touching the GPU, and
its host setup (ordering + supernodal L D L^T) solves correctly."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import gridgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1511_04519_gb300 import build
    path = build.build()
    return C.CDLL(path)


def header_functions():
    src = open(os.path.join(ROOT, "include", "matex.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(matex_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def _P(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def host_factor_solve(lib, p, dshift, alpha, b, max_width=128):
    f = lib.matex_host_factor_solve
    f.restype = C.c_int
    x = np.zeros_like(b)
    info = np.zeros(5, np.int64)
    st = f(C.c_int64(p.n), _P(p.g_rowptr, C.c_int64), _P(p.g_col, C.c_int32),
           _P(p.g_val, C.c_double), _P(dshift, C.c_double), C.c_double(alpha),
           C.c_int32(max_width), C.c_int32(b.shape[0]), _P(b, C.c_double), _P(x, C.c_double),
           _P(info, C.c_int64))
    return st, x, info


@pytest.mark.parametrize("case", ["config0", "ragged3layer", "fourlayer", "mesh2x200x200"])
@pytest.mark.parametrize("width", [1, 16, 0])
def test_single_column_plan_covers_every_row_once(lib, case, width):
    """The single-column kernels' plan, walked lane by lane as the kernels
    walk it: every panel row (forward) and supernode column (backward) is
    taken by exactly one group of lanes of its own level and group size."""
    if case == "config0":
        p = gridgen.config0()
    elif case == "ragged3layer":
        p = gridgen.small_mesh(3, nx=23, ny=17, layers=3, n_src=6)
    elif case == "fourlayer":
        p = gridgen.config2(side=60, n_src=60, n_groups=4, n_pads=40, max_tpl=4)
    else:
        p = gridgen.small_mesh(4, nx=200, ny=200, layers=2, n_src=8)
    f = lib.matex_host_single_column_plan
    f.restype = C.c_int
    info = np.zeros(6, np.int64)
    st = f(C.c_int64(p.n), _P(p.g_rowptr, C.c_int64), _P(p.g_col, C.c_int32),
           _P(p.g_val, C.c_double), C.c_int32(width), _P(info, C.c_int64))
    assert st == 0, info
    levels, fw, bw, rows, cols, errors = info
    assert errors == 0 and levels >= 1 and fw >= 1 and bw >= 1
    assert cols == p.n            # every node is one column of one supernode
    assert rows >= p.n            # diagonal rows plus the rows below them
    if width == 1:
        assert rows - p.n > 0     # no amalgamation: the off-diagonal rows of L


@pytest.mark.parametrize("case", ["small2layer", "config0", "ragged"])
@pytest.mark.parametrize("width", [1, 7, 128])
def test_host_factorisation_solves(lib, case, width):
    if case == "small2layer":
        p = gridgen.small_mesh(1, nx=12, ny=9, layers=2, n_src=4)
    elif case == "config0":
        p = gridgen.config0()
    else:
        p = gridgen.small_mesh(2, nx=17, ny=5, layers=3, n_src=3)
    rng = np.random.default_rng(1)
    b = np.ascontiguousarray(rng.standard_normal((3, p.n)))
    for ds, al in ((None, 1.0), (p.c, p.gamma)):
        st, x, info = host_factor_solve(lib, p, ds, al, b, max_width=width)
        assert st == 0
        A = sp.csr_matrix((sp.diags(ds) if ds is not None else 0) + al * p.G())
        for q in range(3):
            assert np.abs(A @ x[q] - b[q]).max() <= 1e-12 * np.abs(b[q]).max()
        assert info[3] <= width
        # fill is modest: nested dissection on a mesh
        assert info[0] <= 40 * p.n
        # the dense panels hold the exact fill plus amalgamation's explicit
        # zeros; unit-width supernodes (no amalgamation) hold the fill alone
        assert info[4] <= info[0]
        if width == 1:
            assert info[4] == info[0]


def test_host_factorisation_rejects_indefinite(lib):
    p = gridgen.small_mesh(3, nx=4, ny=4, n_src=1)
    bad = gridgen.with_sources(p, p.src_node, p.pwl_off, p.pwl_t, p.pwl_v, p.src_group, 1)
    bad.g_val = -bad.g_val
    b = np.ones((1, p.n))
    st, _, _ = host_factor_solve(lib, bad, None, 1.0, b)
    assert st == 2  # MATEX_ERR_NOT_SPD


def _setup_status(lib, p, opts=None, **kw):
    f = lib.matex_setup
    f.restype = C.c_int
    ctx = C.c_void_p()
    a = dict(c=p.c, g_rowptr=p.g_rowptr, g_col=p.g_col, g_val=p.g_val, pwl_t=p.pwl_t,
             pwl_v=p.pwl_v, src_node=p.src_node, src_group=p.src_group, pwl_off=p.pwl_off)
    a.update(kw)
    arrs = {k: np.ascontiguousarray(v) for k, v in a.items()}
    st = f(C.byref(ctx), C.c_int64(p.n), _P(arrs["c"], C.c_double), _P(arrs["g_rowptr"], C.c_int64),
           _P(arrs["g_col"], C.c_int32), _P(arrs["g_val"], C.c_double),
           _P(p.dc_inject, C.c_double), C.c_int32(p.n_src), _P(arrs["src_node"], C.c_int32),
           _P(arrs["pwl_off"], C.c_int32), _P(arrs["pwl_t"], C.c_double),
           _P(arrs["pwl_v"], C.c_double), _P(arrs["src_group"], C.c_int32),
           C.c_int32(p.n_groups), C.c_double(p.gamma), C.c_double(p.tol), C.c_int32(p.m_max),
           C.c_double(p.t_end), C.c_double(p.dt_out), opts, None)
    lib.matex_last_error.restype = C.c_char_p
    return st, lib.matex_last_error(None).decode()


@pytest.mark.parametrize("mutation", ["negative_cap", "asymmetric", "bad_node", "bad_group",
                                      "unsorted_pwl", "bad_col"])
def test_setup_rejects_bad_inputs_before_gpu(lib, mutation):
    p = gridgen.small_mesh(4, nx=5, ny=5, n_src=3)
    kw = {}
    if mutation == "negative_cap":
        c = p.c.copy(); c[3] = -1.0; kw["c"] = c
    elif mutation == "asymmetric":
        v = p.g_val.copy(); v[1] *= 2.0; kw["g_val"] = v
    elif mutation == "bad_node":
        s = p.src_node.copy(); s[0] = p.n; kw["src_node"] = s
    elif mutation == "bad_group":
        s = p.src_group.copy(); s[0] = 5; kw["src_group"] = s
    elif mutation == "unsorted_pwl":
        t = p.pwl_t.copy(); t[1] = t[0]; kw["pwl_t"] = t
    elif mutation == "bad_col":
        cidx = p.g_col.copy(); cidx[0] = -3; kw["g_col"] = cidx
    st, msg = _setup_status(lib, p, **kw)
    assert st == 1, (st, msg)
    assert msg


@pytest.mark.parametrize("field,value", [("tail_eps", -1e-9), ("tail_eps", float("nan")),
                                         ("tail_eps", float("inf")), ("krylov", 3),
                                         ("solve_mode", 5), ("tape_tail", 1e-9),
                                         ("tape_krylov", 1), ("decompose", 2),
                                         ("decompose_tape", 1), ("recombine", 2),
                                         ("tape", 3), ("tape_window", -1), ("resident", 4),
                                         ("resident_krylov", 2), ("resident_tail", 1e-9),
                                         ("tc_solve", 3), ("tc_min_width", 16),
                                         ("single_column", 3)])
def test_setup_rejects_bad_options_before_gpu(lib, field, value):
    """Option checks run on the host before any device work: the status is
    MATEX_ERR_ARG with a message, on a machine without a GPU as well."""
    from paper_1511_04519_gb300 import matex as M
    p = gridgen.small_mesh(4, nx=5, ny=5, n_src=3)
    o = M.matex_default_opts()
    if field == "tape_tail":
        o.tape, o.tail_eps = 1, value
    elif field == "tape_krylov":
        o.tape, o.krylov = 1, value
    elif field == "decompose_tape":
        o.tape, o.decompose = 1, value
    elif field == "resident_krylov":
        o.resident, o.krylov = 2, value
    elif field == "resident_tail":
        o.resident, o.tail_eps = 2, value
    else:
        setattr(o, field, value)
    st, msg = _setup_status(lib, p, opts=C.byref(o))
    assert st == 1, (st, msg)
    assert msg


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib
    import paper_1511_04519_gb300.matex as M
    monkeypatch.setattr(M, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        M._load()
    importlib.reload(M)


def test_default_options_layout():
    """The binding's option and statistics structs line up with the header's
    (matex_default_opts fills every field; a shifted field shows up here)."""
    from paper_1511_04519_gb300 import build
    build.build()
    from paper_1511_04519_gb300 import matex as M
    o = M.matex_default_opts()
    assert (o.col_block, o.group_select, o.include_dc, o.n_rows, o.max_width, o.strict,
            o.solve_mode, o.tape, o.krylov, o.graph, o.tail_eps) == (0, -1, 1, 0, 1024, 0, 2, 0,
                                                                     0, 1, 0.0)
    # the library writes exactly sizeof(matex_opts) bytes: a sentinel-filled
    # buffer keeps every byte past the binding's struct
    size = C.sizeof(M.MatexOpts)
    buf = (C.c_ubyte * (size + 64))(*([0xA5] * (size + 64)))
    M._lib.matex_default_opts(C.cast(buf, C.POINTER(M.MatexOpts)))
    assert bytes(buf[size:]) == b"\xa5" * 64
    assert M.MatexOpts.from_buffer(buf).tail_eps == 0.0
    assert C.sizeof(M.MatexStats) == 3 * 8 + 8 + 4 * 12 + 8 + 4 * 4 + 8 + 8 + 4 * 2 + 8 + 8 + 8 + 8
    assert (o.tape_window, o.tape_block, o.recombine, o.decompose, o.resident, o.tc_solve,
            o.tc_min_width, o.single_column) == (0, 0, 0, 0, 0, 0, 0, 0)
