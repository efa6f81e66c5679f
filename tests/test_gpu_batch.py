"""Batched snapshots of uneven grids in one graph launch give the same results as
each snapshot solved alone (bitwise: same kernels, deterministic reductions)."""
import numpy as np
import pytest

from paper_1610_04398_gb300 import api, synth
from gpu_cases import run_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()


def _item(snap):
    plan = api.Plan(snap.n, snap.h, 20, 0.5, precision="mixed", lift=snap.lift, uinf=snap.uinf)
    f = [to_dev(a, torch.float32) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    pts = to_dev(snap.points, torch.float64)
    nrm = to_dev(snap.normals, torch.float64)
    P = torch.empty(snap.n * snap.n, dtype=torch.float32, device="cuda")
    per = torch.empty(len(snap.points) * 5, dtype=torch.float64, device="cuda")
    F = torch.empty(6, dtype=torch.float64, device="cuda")
    g = plan.capture_step(*f, snap.lam, p_out=P, points=pts, normals=nrm, nu=snap.nu, per_point=per, forces=F)
    return dict(plan=plan, graph=g, bufs=(f, pts, nrm), P=P, per=per, F=F)


def test_batch_of_uneven_swimmers_matches_single_solves():
    snaps = []
    for k, n in enumerate((64, 256, 128, 256, 64, 128)):
        snaps.append(synth.swimmer_snapshot(n, phase=0.13 * (k + 1), seed=4000 + k, n_surface=512))
    items = [_item(s) for s in snaps]
    batch = api.Batch([it["graph"] for it in items])
    for rep in range(2):
        batch.launch()
        torch.cuda.synchronize()
        for s, it in zip(snaps, items):
            d = run_gpu(s, "mixed")
            assert np.array_equal(it["P"].double().cpu().numpy().reshape(s.n, s.n), d["P"])
            assert np.array_equal(it["per"].cpu().numpy().reshape(-1, 5), d["per_point"])
            assert np.array_equal(it["F"].cpu().numpy(), d["forces"])
    batch.destroy()
