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


def test_swimmer_batch_full_size_against_oracle():
    """The swimmer batch workload at its full size: 64 snapshots, grid side and phase drawn
    from seed 4000 + k over {256, 512, 1024, 2048}, 4096 surface points each (lift 0:
    deforming body), mixed path at the setting bench.py uses for it (the autotuner over the
    batch's swimmers of grids up to 512^2 and the 1024^2 cylinder, surface acceptance
    included), all solved by one graph launch.  Every snapshot's pressure, tractions
    and forces equal (bitwise) its own step graph launched alone; against the oracle, each
    snapshot on 32 sampled cells (corners included) and 128 sampled surface points, and one
    snapshot of every grid size on all 4096 surface points with its drag and lift.  Bounds
    1e-4 on relative L2 and on the worst point (max|dP| / max|P|)."""
    import oracle
    from gpu_cases import force_err, rel_l2, worst_cell
    oracle.build()
    synth.set_device("cuda")
    try:
        snaps = synth.swimmer_batch(64)
    finally:
        synth.set_device(None)
    assert sorted(set(s.n for s in snaps)) == [256, 512, 1024, 2048]
    from paper_1610_04398_gb300 import autotune
    reps = autotune.batch_representatives(snaps) + [synth.cylinder_flow(1024, seed=2000)]
    best = autotune.autotune(reps, steps=2)["best"]
    assert best["ok"], best
    print(f"swimmer batch setting: p = {best['order']}, theta = {best['theta']}, tile {best['tile']}, "
          f"surface theta {best['theta_surface']}")
    items = []
    for s in snaps:
        plan = api.Plan(s.n, s.h, best["order"], best["theta"], precision="mixed", lift=s.lift, uinf=s.uinf,
                        tile=best["tile"], theta_surface=best["theta_surface"])
        f = [to_dev(a, torch.float32) for a in (s.u, s.v, s.chi, s.usx, s.usy)]
        pts, nrm = to_dev(s.points, torch.float64), to_dev(s.normals, torch.float64)
        P = torch.full((s.n * s.n,), float("nan"), dtype=torch.float32, device="cuda")
        per = torch.full((len(s.points) * 5,), float("nan"), dtype=torch.float64, device="cuda")
        F = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        g = plan.capture_step(*f, s.lam, p_out=P, points=pts, normals=nrm, nu=s.nu, per_point=per, forces=F)
        items.append(dict(plan=plan, graph=g, bufs=(f, pts, nrm), P=P, per=per, F=F))
    batch = api.Batch([it["graph"] for it in items])
    batch.launch()
    torch.cuda.synchronize()
    got = [(it["P"].double().cpu().numpy(), it["per"].cpu().numpy().reshape(-1, 5), it["F"].cpu().numpy())
           for it in items]
    for it in items:  # each graph alone, one after another
        it["graph"].launch()
    torch.cuda.synchronize()
    for (P, per, F), it in zip(got, items):
        assert np.array_equal(P, it["P"].double().cpu().numpy())
        assert np.array_equal(per, it["per"].cpu().numpy().reshape(-1, 5))
        assert np.array_equal(F, it["F"].cpu().numpy())
    rng = np.random.default_rng(77)
    full_done = set()
    worst = {}
    for k, (s, (P, per, F)) in enumerate(zip(snaps, got)):
        n = s.n
        q = oracle.source_weights(oracle.rhs(s.u, s.v, s.chi, s.usx, s.usy, h=s.h, lam=s.lam), s.h)
        cells = np.unique(np.concatenate([rng.choice(n * n, 28, replace=False), [0, n - 1, n * (n - 1), n * n - 1]]))
        X, Y = synth.cell_centres(n, s.h)
        Pc = oracle.green_sum_grid(q, s.h, X.ravel()[cells], Y.ravel()[cells])
        full = n not in full_done
        sel = np.arange(len(s.points)) if full else rng.choice(len(s.points), 128, replace=False)
        Ps = oracle.green_sum_grid(q, s.h, s.points[sel, 0], s.points[sel, 1])
        e = (rel_l2(P.ravel()[cells], Pc), worst_cell(P.ravel()[cells], Pc),
             rel_l2(per[sel, 0], Ps), worst_cell(per[sel, 0], Ps))
        worst[k] = e
        assert max(e) < 1e-4, (k, n, e)
        if full:
            full_done.add(n)
            _, Fr = oracle.traction(s.u, s.v, s.h, s.points, s.normals, Ps, s.nu, lift=s.lift, uinf=s.uinf)
            ed, el = force_err(F, Fr)
            assert ed < 1e-4 and el < 1e-4, (k, n, ed, el)
    print("swimmer batch: worst errors over 64 snapshots (cells L2, cells worst, surface L2, surface worst):",
          [float("%.2e" % max(e[i] for e in worst.values())) for i in range(4)])
    batch.destroy()
    for it in items:
        it["graph"].destroy()
        it["plan"].destroy()


def test_batch_refuses_two_graphs_of_one_plan():
    """The branches of a batch run at once and a plan's workspace holds one solve, so two
    step graphs captured on one plan cannot share a batch."""
    s = synth.swimmer_snapshot(64, phase=0.2, seed=4100, n_surface=128)
    it = _item(s)
    f, pts, nrm = it["bufs"]
    P2 = torch.empty(s.n * s.n, dtype=torch.float32, device="cuda")
    g2 = it["plan"].capture_step(*f, s.lam, p_out=P2, points=pts, normals=nrm, nu=s.nu)
    with pytest.raises(api.PPError) as ei:
        api.Batch([it["graph"], g2])
    assert ei.value.status == api.PP_ERR_ARG
