"""Snapshots streamed from host memory through pp_pipeline (two device slots, copies
overlapping the solve) give bitwise the same pressure and forces as each snapshot
solved alone from device memory (same kernels, deterministic reductions), however
many snapshots are in flight."""
import numpy as np
import pytest

from paper_1610_04398_gb300 import api, synth
from gpu_cases import run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()


def _host(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()


@pytest.mark.parametrize("precision,tile", [("mixed", 128), ("mixed", 16), ("fp64", 16)])
def test_pipeline_matches_single_solves(precision, tile):
    n = 256
    snaps = [synth.swimmer_snapshot(n, phase=0.11 * (k + 1), seed=4100 + k, n_surface=512) for k in range(5)]
    s0 = snaps[0]
    plan = api.Plan(n, s0.h, 20, 0.5, x0=s0.x0, y0=s0.y0, precision=precision, lift=s0.lift, uinf=s0.uinf,
                    tile=tile)
    dt = plan.dtype
    pipe = api.Pipeline(plan, s0.lam, npts=len(s0.points), nu=s0.nu)
    ins = [[_host(a, dt) for a in (s.u, s.v, s.chi, s.usx, s.usy)] for s in snaps]
    pts = [_host(s.points, torch.float64) for s in snaps]
    nrm = [_host(s.normals, torch.float64) for s in snaps]
    P = [torch.empty(n * n, dtype=dt).pin_memory() for _ in snaps]
    F = [torch.empty(6, dtype=torch.float64).pin_memory() for _ in snaps]
    for rep in range(2):  # the second round reuses both slots again
        for k in range(len(snaps)):
            pipe.submit(*ins[k], pts[k], nrm[k], P[k], F[k])
        pipe.wait()
        for k, s in enumerate(snaps):
            d = run_gpu(s, precision, tile=tile)
            assert np.array_equal(P[k].double().numpy().reshape(n, n), d["P"]), (rep, k)
            assert np.array_equal(F[k].numpy(), d["forces"]), (rep, k)
    pipe.destroy()
    plan.destroy()


def test_pipeline_without_surface_points():
    n = 128
    s = synth.cylinder_flow(n, seed=2010, n_surface=128)
    plan = api.Plan(n, s.h, 20, 0.5, precision="mixed", lift=s.lift, uinf=s.uinf)
    pipe = api.Pipeline(plan, s.lam, npts=0)
    ins = [_host(a, torch.float32) for a in (s.u, s.v, s.chi, s.usx, s.usy)]
    P = torch.empty(n * n, dtype=torch.float32).pin_memory()
    for _ in range(3):
        pipe.submit(*ins, p_out=P)
    pipe.wait()
    d = run_gpu(s, "mixed")
    assert np.array_equal(P.double().numpy().reshape(n, n), d["P"])
    pipe.destroy()
    plan.destroy()
