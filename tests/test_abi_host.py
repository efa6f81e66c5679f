"""Host-side checks that need no GPU: the C ABI library loads and exports every
entry point the header declares, arguments are validated before any device work,
and the near / multipole-to-local lists cover every source exactly once."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1610_04398_gb300 import api
from paper_1610_04398_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return api.load()


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pp_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    syms = _declared_symbols()
    assert "pp_plan_create" in syms and "pp_surface_traction" in syms
    for s in syms:
        assert hasattr(lib, s), f"libpp.so does not export {s}"


def test_error_strings(lib):
    for st in range(7):
        assert lib.pp_error_string(st)
    assert b"unknown" in lib.pp_error_string(99)


def test_plan_create_rejects_bad_arguments_without_touching_the_device(lib):
    h = ctypes.c_void_p()
    opt = api._Options()
    lib.pp_options_default(ctypes.byref(opt))
    bad = [
        (api._Grid(100, 0, 0), 0.01, 20, 0.5),   # n not a power of two
        (api._Grid(4, 0, 0), 0.25, 20, 0.5),     # n < 8
        (api._Grid(64, 0, 0), -1.0, 20, 0.5),    # h <= 0
        (api._Grid(64, 0, 0), 0.01, 1, 0.5),     # order < 2
        (api._Grid(64, 0, 0), 0.01, 41, 0.5),    # order > 40
        (api._Grid(64, 0, 0), 0.01, 20, 0.1),    # theta too small for the tree-code lists
        (api._Grid(64, 0, 0), 0.01, 20, 1.0),    # theta >= 1 never separates neighbours
    ]
    for g, hh, p, th in bad:
        assert lib.pp_plan_create(ctypes.byref(h), g, hh, p, th, ctypes.byref(opt)) == api.PP_ERR_ARG
    opt.precision = 7
    assert lib.pp_plan_create(ctypes.byref(h), api._Grid(64, 0, 0), 1 / 64, 20, 0.5,
                              ctypes.byref(opt)) == api.PP_ERR_ARG
    lib.pp_options_default(ctypes.byref(opt))
    assert opt.theta_surface == 0.0
    for bad_ts in (0.1, 0.99, -0.5):  # the surface tree-code's acceptance parameter
        opt.theta_surface = bad_ts
        assert lib.pp_plan_create(ctypes.byref(h), api._Grid(64, 0, 0), 1 / 64, 20, 0.5,
                                  ctypes.byref(opt)) == api.PP_ERR_ARG
    lib.pp_options_default(ctypes.byref(opt))
    opt.uinf_x = opt.uinf_y = 0.0
    assert lib.pp_plan_create(ctypes.byref(h), api._Grid(64, 0, 0), 1 / 64, 20, 0.5,
                              ctypes.byref(opt)) == api.PP_ERR_ARG
    assert lib.pp_rhs(None, None, None, None, None, None, 0.0, None) == api.PP_ERR_ARG
    assert lib.pp_pressure_solve(None, None) == api.PP_ERR_ARG
    assert lib.pp_pressure_solve_fft(None, None) == api.PP_ERR_ARG
    assert lib.pp_atree_solve(None, 20, None, None, None) == api.PP_ERR_ARG
    assert lib.pp_plan_destroy(None) == api.PP_OK
    pipe = ctypes.c_void_p()
    assert lib.pp_pipeline_create(None, 1.0, 0, None, 0.0, ctypes.byref(pipe)) == api.PP_ERR_ARG
    assert lib.pp_pipeline_create(None, 1.0, 0, None, 0.0, None) == api.PP_ERR_ARG
    assert lib.pp_pipeline_submit(None, None, None, None, None, None, None, None, None, None) == api.PP_ERR_ARG
    assert lib.pp_pipeline_wait(None) == api.PP_ERR_ARG
    assert lib.pp_pipeline_destroy(None) == api.PP_OK
    assert lib.pp_penal_force(None, None, None, None, None, None, 1.0, None) == api.PP_ERR_ARG


@pytest.mark.parametrize("theta,n_near,n_m2l", [(0.5, 25, 75), (0.6, 21, 63), (0.4, 37, 111)])
def test_list_sizes(lib, theta, n_near, n_m2l):
    """theta^2 |d|^2 <= 2 is near (ties near): 5x5 at 0.5, 5x5 minus corners at 0.6, ..."""
    assert len(api.pp_near_offsets(theta)) == n_near
    for c in range(4):
        assert len(api.pp_m2l_offsets(theta, c)) == n_m2l


@pytest.mark.parametrize("theta", [0.4, 0.5, 0.6, 0.75, 0.3])
def test_near_and_m2l_lists_cover_every_source_leaf_exactly_once(lib, theta):
    """For every target leaf, the near list plus the M2L lists of its ancestors at
    levels 2..L account for every source leaf exactly once (a uniform 32 x 32 tree)."""
    L = 5
    nl = 1 << L
    near = api.pp_near_offsets(theta)
    il = [api.pp_m2l_offsets(theta, c) for c in range(4)]
    ty, tx = np.divmod(np.arange(nl * nl), nl)
    count = np.zeros((nl * nl, nl * nl), np.int32)   # [target leaf, source leaf]
    sy, sx = np.divmod(np.arange(nl * nl), nl)
    for dx, dy in near:
        ok = (tx + dx >= 0) & (tx + dx < nl) & (ty + dy >= 0) & (ty + dy < nl)
        count[np.nonzero(ok)[0], ((ty + dy) * nl + tx + dx)[ok]] += 1
    for lev in range(2, L + 1):
        sh = L - lev
        bx, by = tx >> sh, ty >> sh
        par = (bx & 1) + 2 * (by & 1)
        side = 1 << lev
        sbx, sby = sx >> sh, sy >> sh
        for c in range(4):
            sel = par == c
            for dx, dy in il[c]:
                ok = sel & (bx + dx >= 0) & (bx + dx < side) & (by + dy >= 0) & (by + dy < side)
                rows = np.nonzero(ok)[0]
                if len(rows) == 0:
                    continue
                match = (sbx[None, :] == (bx[rows] + dx)[:, None]) & (sby[None, :] == (by[rows] + dy)[:, None])
                count[rows] += match.astype(np.int32)
    assert count.min() == 1 and count.max() == 1


def test_m2l_offsets_are_well_separated_and_near_offsets_are_not(lib):
    for theta in (0.4, 0.5, 0.6):
        for dx, dy in api.pp_near_offsets(theta):
            assert theta * theta * (dx * dx + dy * dy) <= 2.0
        for c in range(4):
            for dx, dy in api.pp_m2l_offsets(theta, c):
                assert theta * theta * (dx * dx + dy * dy) > 2.0


@pytest.mark.parametrize("theta", [0.4, 0.5, 0.6, 0.75, 0.3])
def test_interaction_entries_with_parent_sources_cover_every_leaf_exactly_once(lib, theta):
    """The lists the kernels use (same-level and parent-level sources) plus the near list
    account for every source leaf exactly once, and a parent-level entry is used only
    when all four of its children are separated from the target."""
    L = 5
    nl = 1 << L
    near = api.pp_near_offsets(theta)
    ent = [api.pp_m2l_entries(theta, c) for c in range(4)]
    for c in range(4):
        covered = set()
        for dx, dy, kind in ent[c]:
            if kind == 0:
                covered.add((dx, dy))
            else:
                for cp in range(4):
                    t = (2 * dx + (cp & 1) - (c & 1), 2 * dy + (cp >> 1) - (c >> 1))
                    assert theta * theta * (t[0] ** 2 + t[1] ** 2) > 2.0
                    covered.add(t)
        assert covered == set(map(tuple, api.pp_m2l_offsets(theta, c)))
    ty, tx = np.divmod(np.arange(nl * nl), nl)
    sy, sx = np.divmod(np.arange(nl * nl), nl)
    count = np.zeros((nl * nl, nl * nl), np.int32)
    for dx, dy in near:
        ok = (tx + dx >= 0) & (tx + dx < nl) & (ty + dy >= 0) & (ty + dy < nl)
        count[np.nonzero(ok)[0], ((ty + dy) * nl + tx + dx)[ok]] += 1
    for lev in range(2, L + 1):
        sh = L - lev
        bx, by = tx >> sh, ty >> sh
        par = (bx & 1) + 2 * (by & 1)
        side = 1 << lev
        for c in range(4):
            sel = par == c
            for dx, dy, kind in ent[c]:
                if kind == 0:
                    tbx, tby, ssh, sd = bx + dx, by + dy, sh, side
                else:
                    tbx, tby, ssh, sd = (bx >> 1) + dx, (by >> 1) + dy, sh + 1, side // 2
                ok = sel & (tbx >= 0) & (tbx < sd) & (tby >= 0) & (tby < sd)
                rows = np.nonzero(ok)[0]
                if len(rows) == 0:
                    continue
                match = (((sx >> ssh)[None, :] == tbx[rows][:, None]) &
                         ((sy >> ssh)[None, :] == tby[rows][:, None]))
                count[rows] += match.astype(np.int32)
    assert count.min() == 1 and count.max() == 1



def _m2l_tc_shape(theta):
    """Operator count, list stride and halo margin of the tensor-core translations, from the
    acceptance test restated: children of the parent's near boxes that are separated from the
    box, or their parent when all four are and the unequal-size test passes."""
    near = lambda dx, dy: theta * theta * (dx * dx + dy * dy) <= 2.0
    ops, stride, margin = set(), 0, 0
    for c in range(4):
        cx, cy = c & 1, c >> 1
        ent = []
        for Dx, Dy in api.pp_near_offsets(theta):
            kids = [(2 * Dx + (q & 1) - cx, 2 * Dy + (q >> 1) - cy) for q in range(4)]
            ox, oy = 2 * Dx + 0.5 - cx, 2 * Dy + 0.5 - cy
            if all(not near(*k) for k in kids) and theta * theta * (ox * ox + oy * oy) > 4.5:
                ent.append((int(Dx), int(Dy), 1))
            else:
                ent += [(kx, ky, 0) for kx, ky in kids if not near(kx, ky)]
        stride = max(stride, len(ent))
        for dx, dy, kind in ent:
            ops.add((2 * dx, 2 * dy, 1) if kind == 0 else (4 * dx + 1 - 2 * cx, 4 * dy + 1 - 2 * cy, 2))
            sx, sy = ((cx + dx) // 2, (cy + dy) // 2) if kind == 0 else (dx, dy)
            margin = max(margin, abs(sx), abs(sy))
    return len(ops), stride, margin

def test_plan_bytes_host_query(lib):
    """pp_plan_bytes (host only): argument errors, the surface scratch's growth rule, and
    the array the tensor-core near field adds (per near offset a 64 x 64 kernel matrix in
    two FP16 parts)."""
    out = ctypes.c_int64()
    opt = api._Options()
    lib.pp_options_default(ctypes.byref(opt))
    assert lib.pp_plan_bytes(100, 20, 0.5, ctypes.byref(opt), 0, ctypes.byref(out)) == api.PP_ERR_ARG
    assert lib.pp_plan_bytes(64, 1, 0.5, ctypes.byref(opt), 0, ctypes.byref(out)) == api.PP_ERR_ARG
    assert lib.pp_plan_bytes(64, 20, 0.1, ctypes.byref(opt), 0, ctypes.byref(out)) == api.PP_ERR_ARG
    assert lib.pp_plan_bytes(64, 20, 0.5, ctypes.byref(opt), -1, ctypes.byref(out)) == api.PP_ERR_ARG
    assert lib.pp_plan_bytes(64, 20, 0.5, ctypes.byref(opt), 0, None) == api.PP_ERR_ARG
    n = 1024
    base = api.plan_bytes(n, 12, 0.75, precision="mixed", tile=16)
    # a new plan's scratch holds 4096 points; 5000 grow it to 8192 (twice), 20000 to 20000:
    # 8 bytes per point plus 4 doubles per 64-point block
    sb = lambda cap: 8 * cap + 32 * ((cap + 63) // 64)
    assert api.plan_bytes(n, 12, 0.75, precision="mixed", tile=16, npts=4096) == base
    assert api.plan_bytes(n, 12, 0.75, precision="mixed", tile=16, npts=5000) - base == sb(8192) - sb(4096)
    assert api.plan_bytes(n, 12, 0.75, precision="mixed", tile=16, npts=20000) - base == sb(20000) - sb(4096)
    n_near = len(api.pp_near_offsets(0.75))
    tc = api.plan_bytes(n, 12, 0.75, precision="mixed", tile=128)
    assert tc - base == 2 * 2 * 64 * 64 * n_near
    # the tensor-core translations add every operator as two 32 x 32 FP16 matrices (4 KB) and
    # a 16-byte window entry per list slot and child position
    n_ops, stride, margin = _m2l_tc_shape(0.75)
    assert margin == 1
    assert api.plan_bytes(n, 12, 0.75, precision="mixed", tile=16, m2l_tensor=True) - base == \
        n_ops * 4096 + 4 * stride * 16
    n_ops6, stride6, margin6 = _m2l_tc_shape(0.6)
    assert margin6 == 2
    assert api.plan_bytes(n, 12, 0.6, precision="mixed", tile=16, m2l_tensor=True) - \
        api.plan_bytes(n, 12, 0.6, precision="mixed", tile=16) == n_ops6 * 4096 + 4 * stride6 * 16
    assert _m2l_tc_shape(0.4)[2] == 3  # a halo margin of 3: the FP32-core translations only
    assert api.plan_bytes(n, 12, 0.4, precision="mixed", tile=16, m2l_tensor=True) == \
        api.plan_bytes(n, 12, 0.4, precision="mixed", tile=16)
    assert api.plan_bytes(n, 20, 0.75, precision="mixed", tile=16, m2l_tensor=True) == \
        api.plan_bytes(n, 20, 0.75, precision="mixed", tile=16)  # order 20: FP32 cores only
    # FP64 holds the grid-sized and expansion arrays in 8 bytes instead of 4; mixed plans add
    # the box monopoles as float pairs (8 bytes a box) and the downward side buffers of
    # levels 2..L-4 (13 coefficients and one double a box), and FP64 plans neither (the FP64
    # constant tables add the rest)
    L = int(np.log2(n // 8))
    nbox = (4 ** (L + 1) - 1) // 3
    na = (4 ** (L - 3) - 1) // 3
    d = api.plan_bytes(n, 12, 0.75, precision="fp64") - base
    mixed_only = 8 * nbox + na * (13 * 8 + 8)
    assert 0 <= d - (4 * n * n + 2 * nbox * 13 * 8 - mixed_only) < 256 * 1024
