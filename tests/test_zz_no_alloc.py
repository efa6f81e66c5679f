"""The allocation-free traction entry point against the plan-based one.

pp_surface_forces_noalloc serves callers that cannot allocate device memory (a
host flow solver that owns the whole device, or a loop that cannot afford the
synchronisation of cudaMalloc).  It must give the same tractions and forces as
pp_surface_traction for the same surface pressure, call after call, although its
scratch is one fixed device array shared by every call; and, on its own, the
oracle's tractions and forces (Sec. 2.3) for that pressure.  This file is collected
last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1610_04398_gb300 import api, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()
    return api.load()


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _plan_reference(snap, precision, npts):
    plan = api.Plan(snap.n, snap.h, 20, 0.5, precision=precision, lift=snap.lift, uinf=snap.uinf)
    dt = plan.dtype
    f = [_dev(a, dt) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    plan.rhs(*f, snap.lam)
    pts = _dev(snap.points[:npts], torch.float64)
    nrm = _dev(snap.normals[:npts], torch.float64)
    per = torch.empty(npts * 5, dtype=torch.float64, device="cuda")
    F = plan.surface_traction(f[0], f[1], pts, nrm, snap.nu, per_point=per)
    torch.cuda.synchronize()
    plan.destroy()
    return f[0], f[1], pts, nrm, per.view(npts, 5), F


def _call(lib, prec, snap, u, v, pts, nrm, P, per, forces_ptr):
    st = lib.pp_surface_forces_noalloc(
        prec, api._Grid(snap.n, snap.x0, snap.y0), snap.h, ctypes.c_void_p(u.data_ptr()),
        ctypes.c_void_p(v.data_ptr()), int(pts.shape[0]), ctypes.c_void_p(pts.data_ptr()),
        ctypes.c_void_p(nrm.data_ptr()), None, ctypes.c_void_p(P.data_ptr()), 1.0, snap.nu, snap.lift,
        api.PP_NEAREST, snap.uinf[0], snap.uinf[1], ctypes.c_void_p(per.data_ptr()), forces_ptr,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == api.PP_OK, api.error_string(st)


@pytest.mark.parametrize("precision,prec,tol", [("fp64", api.PP_FP64, 1e-12), ("mixed", api.PP_MIXED, 1e-5)])
def test_noalloc_matches_plan_traction_two_calls_in_a_row(lib, precision, prec, tol):
    snap = synth.cylinder_flow(128, seed=2000)
    for npts in (2048, 333):  # a second shape reuses the same scratch with fewer blocks
        u, v, pts, nrm, per_ref, F_ref = _plan_reference(snap, precision, npts)
        P = per_ref[:, 0].contiguous()
        scale_t = torch.max(torch.abs(per_ref[:, 1:])).item()
        scale_f = max(np.hypot(F_ref[4], F_ref[5]), np.max(np.abs(F_ref[:4])))
        for call in range(2):
            per = torch.full((npts, 5), float("nan"), dtype=torch.float64, device="cuda")
            if call == 0:
                F = np.zeros(6)
                _call(lib, prec, snap, u, v, pts, nrm, P, per, ctypes.c_void_p(F.ctypes.data))
            else:
                Fd = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
                _call(lib, prec, snap, u, v, pts, nrm, P, per, ctypes.c_void_p(Fd.data_ptr()))
                torch.cuda.synchronize()
                F = Fd.cpu().numpy()
            torch.cuda.synchronize()
            assert torch.max(torch.abs(per - per_ref)).item() <= tol * scale_t
            assert np.max(np.abs(F - F_ref)) <= tol * scale_f, (F, F_ref)
        # the oracle's tractions for the same pressure, from the velocity the kernels read
        # (rounded to FP32 on mixed plans): FP64 arithmetic on both sides
        dt = np.float64 if precision == "fp64" else np.float32
        uo, vo = (np.asarray(a, dt).astype(np.float64) for a in (snap.u, snap.v))
        per_o, F_o = oracle.traction(uo, vo, snap.h, snap.points[:npts], snap.normals[:npts],
                                     P.cpu().numpy(), snap.nu, lift=snap.lift, uinf=snap.uinf)
        got = per.cpu().numpy()
        assert np.max(np.abs(got - per_o)) <= 1e-12 * np.max(np.abs(per_o))
        assert np.max(np.abs(F - F_o)) <= 1e-12 * max(np.hypot(F_o[4], F_o[5]), np.max(np.abs(F_o[:4])))


def test_noalloc_rejects_more_points_than_its_scratch_holds(lib):
    one = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = lib.pp_surface_forces_noalloc(
        api.PP_FP64, api._Grid(64, 0.0, 0.0), 1 / 64, ctypes.c_void_p(one.data_ptr()),
        ctypes.c_void_p(one.data_ptr()), api.PP_NOALLOC_MAX_POINTS + 1, ctypes.c_void_p(one.data_ptr()),
        ctypes.c_void_p(one.data_ptr()), None, ctypes.c_void_p(one.data_ptr()), 1.0, 1e-4, -1.0,
        api.PP_NEAREST, 1.0, 0.0, None, None, None)
    assert st == api.PP_ERR_ARG
