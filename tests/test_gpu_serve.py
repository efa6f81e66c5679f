"""Continuous-batching server: each result is the same alone and in the mix (the mix
overlaps requests of different grid sizes on the device), plus host-side failure
handling: invalid request, over-budget request, cancellation, wait timeout."""
import ctypes

import numpy as np
import pytest

from paper_1610_04398_gb300 import api, synth
from gpu_cases import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()


class Item:
    def __init__(self, snap):
        self.snap = snap
        self.f = [to_dev(a, torch.float32) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
        self.pts = to_dev(snap.points, torch.float64)
        self.nrm = to_dev(snap.normals, torch.float64)

    def outputs(self):
        s = self.snap
        return (torch.full((s.n * s.n,), float("nan"), dtype=torch.float32, device="cuda"),
                torch.full((len(s.points) * 5,), float("nan"), dtype=torch.float64, device="cuda"),
                torch.full((6,), float("nan"), dtype=torch.float64, device="cuda"))

    def submit(self, srv, outs):
        s = self.snap
        P, per, F = outs
        return srv.submit(s.n, s.h, *self.f, s.lam, nu=s.nu, lift=s.lift, uinf=s.uinf, points=self.pts,
                          normals=self.nrm, p_out=P, per_point=per, forces=F)


def _snaps():
    out = []
    for k, n in enumerate((128, 64, 256, 128, 64, 256, 128)):
        if k % 2:
            out.append(synth.swimmer_snapshot(n, phase=0.1 * k, seed=4100 + k, n_surface=256 + 64 * k))
        else:
            out.append(synth.cylinder_flow(n, seed=5000 + k, n_surface=300 + 50 * k))
    return out


@pytest.mark.parametrize("tile,theta", [(16, 0.6), (128, 0.75)])
def test_results_alone_equal_results_in_the_mix(tile, theta):
    """Tile 128 mixes tensor-core plans (n >= 128) with FP32-core plans (n = 64)."""
    items = [Item(s) for s in _snaps()]
    srv = api.Server(budget_bytes=1 << 30, slots=4, tile=tile, theta=theta)
    alone = []
    for it in items:  # one request in flight at a time
        outs = it.outputs()
        rid = it.submit(srv, outs)
        assert srv.wait(rid, 60.0) == api.PP_OK
        alone.append([o.cpu().numpy() for o in outs])
    # the mix: all requests (twice over) in flight together, sizes interleaved
    mixed = []
    ids = []
    for rep in range(2):
        for it in items:
            outs = it.outputs()
            ids.append(it.submit(srv, outs))
            mixed.append(outs)
    for rid in ids:
        assert srv.wait(rid, 120.0) == api.PP_OK
    st = srv.stats()
    assert st["completed"] == 3 * len(items) and st["failed"] == 0
    assert st["plans_resident"] >= 3  # trees of the three grid sizes stay on the device
    for k, outs in enumerate(mixed):
        ref = alone[k % len(items)]
        for got, want in zip(outs, ref):
            assert np.array_equal(got.cpu().numpy(), want)
    srv.destroy()


def test_server_rejects_and_times_out_on_the_host():
    it = Item(synth.cylinder_flow(64, seed=5100, n_surface=64))
    srv = api.Server(budget_bytes=64 << 20, slots=1)
    # invalid request: grid side not a power of two (rejected by the C ABI)
    odd = torch.zeros(100 * 100, dtype=torch.float32, device="cuda")
    with pytest.raises(api.PPError) as e:
        srv.submit(100, 0.01, odd, odd, odd, odd, odd, 1.0)
    assert e.value.status == api.PP_ERR_ARG
    # a plan that alone exceeds the budget is refused at submission
    big = torch.zeros(4096 * 4096, dtype=torch.float32, device="cuda")
    with pytest.raises(api.PPError) as e:
        srv.submit(4096, 1 / 4096, big, big, big, big, big, 1.0)
    assert e.value.status == api.PP_ERR_BUDGET
    # one slot: a long request, then a second one queued behind it that we cancel,
    # and a third one waited for with a zero timeout while the first still runs
    n = 2048
    fld = torch.rand(n * n, dtype=torch.float32, device="cuda")
    srv2 = api.Server(budget_bytes=2 << 30, slots=1)
    r1 = srv2.submit(n, 1 / n, fld, fld, fld, fld, fld, 1e4, p_out=torch.empty_like(fld))
    r2 = it.submit(srv2, it.outputs())
    r3 = it.submit(srv2, it.outputs())
    srv2.cancel(r2)
    assert srv2.query(r2)[0] == api.PP_SERVER_CANCELLED
    assert srv2.wait(r2, 1.0) == api.PP_ERR_STATE
    st3 = srv2.wait(r3, 0.0)
    assert st3 in (api.PP_ERR_TIMEOUT, api.PP_OK)
    assert srv2.wait(r1, 60.0) == api.PP_OK
    assert srv2.wait(r3, 60.0) == api.PP_OK
    status, err, (t_sub, t_start, t_done) = srv2.query(r3)
    assert status == api.PP_SERVER_DONE and t_sub <= t_start <= t_done
    srv2.destroy()
    srv.destroy()


@pytest.mark.parametrize("n,precision,tile,theta", [(64, "mixed", 16, 0.6), (256, "mixed", 128, 0.75),
                                                    (512, "fp64", 16, 0.5), (1024, "mixed", 128, 0.6)])
def test_plan_bytes_is_the_plan_workspace(n, precision, tile, theta):
    """pp_plan_bytes (host arithmetic) equals what pp_plan_create allocated, and again after
    a surface call grows the plan's surface scratch."""
    plan = api.Plan(n, 1.0 / n, 12, theta, precision=precision, tile=tile)
    assert plan.info().workspace_bytes == api.plan_bytes(n, 12, theta, precision=precision, tile=tile)
    npts = 5000
    z = torch.zeros(n * n, dtype=plan.dtype, device="cuda")
    ang = torch.linspace(0, 2 * np.pi, npts + 1, dtype=torch.float64, device="cuda")[:-1]
    nrm = torch.stack([torch.cos(ang), torch.sin(ang)], 1).contiguous()
    pts = (0.5 + 0.2 * nrm).contiguous()
    plan.rhs(z, z, z, z, z, 1.0)
    plan.surface_traction(z, z, pts, nrm, 1e-4)
    assert plan.info().workspace_bytes == api.plan_bytes(n, 12, theta, precision=precision, tile=tile, npts=npts)
    plan.destroy()


def test_budget_holds_for_tensor_core_plans_and_growing_surfaces():
    """Admission reserves what a request adds (a new plan with its tensor-core arrays, or a
    resident plan's surface scratch grown for more points) before it starts, so the plans
    never hold more than the budget: the budget here fits one plan of the largest size at
    a time, so requests of other sizes evict it or wait for it."""
    kw = dict(precision="mixed", tile=128)
    # room for the largest plan and the smallest beside it, not for the middle one too
    budget = api.plan_bytes(256, 12, 0.75, npts=10300, **kw) + api.plan_bytes(64, 12, 0.75, npts=10300, **kw) \
        + (64 << 10)
    assert budget < api.plan_bytes(256, 12, 0.75, **kw) + api.plan_bytes(128, 12, 0.75, **kw)
    sizes = (64, 128, 256)
    items = []
    for k, n in enumerate(sizes * 2):
        npts = 300 + 4000 * (k // 3) + 1200 * k   # later requests bring more points
        items.append(Item(synth.cylinder_flow(n, seed=5200 + k, n_surface=npts)))
    srv = api.Server(budget_bytes=budget, slots=2, tile=128, theta=0.75)
    ids = [it.submit(srv, it.outputs()) for it in items for _ in range(2)]
    peak = 0
    while True:
        st = srv.stats()
        peak = max(peak, st["bytes_held"])
        if st["completed"] + st["failed"] == len(ids):
            break
    for rid in ids:
        assert srv.wait(rid, 120.0) == api.PP_OK
    st = srv.stats()
    assert peak <= budget and st["bytes_held"] <= budget, (peak, st, budget)
    assert st["plans_evicted"] >= 1 and st["failed"] == 0
    # a request whose forces are host memory is refused at submission (the dispatcher
    # would otherwise copy and synchronise while it holds the server lock)
    it = items[0]
    s = it.snap
    host_forces = np.zeros(6)
    r = api.Request()
    r.grid = api._Grid(s.n, 0.0, 0.0)
    r.h = s.h
    r.u, r.v, r.chi, r.us_x, r.us_y = [ctypes.c_void_p(t.data_ptr()) for t in it.f]
    r.lam, r.nu, r.rho, r.lift, r.interp = s.lam, s.nu, 1.0, -1.0, api.PP_NEAREST
    r.uinf_x, r.uinf_y = 1.0, 0.0
    r.npts = len(s.points)
    r.points, r.normals = ctypes.c_void_p(it.pts.data_ptr()), ctypes.c_void_p(it.nrm.data_ptr())
    r.forces = ctypes.c_void_p(host_forces.ctypes.data)
    rid = ctypes.c_int64()
    assert srv._lib.pp_server_submit(srv._h, ctypes.byref(r), ctypes.byref(rid)) == api.PP_ERR_ARG
    srv.destroy()
