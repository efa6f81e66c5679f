"""The adaptive-grid pressure solve (pp_atree_solve, FP64) against the oracle's direct sum over
cells of several sizes (oracle.green_sum_var).

Tolerance: the FP64 path's bar, relative l2 <= 1e-6 at p = 20, theta = 0.5 (the truncation
error there is ~theta^(p+1) of the far field, far below it); the error must also fall by
orders of magnitude from p = 8 to p = 20."""
import numpy as np
import pytest

import oracle
from paper_1610_04398_gb300 import api, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()
    oracle.build()


def _case(lv, ix, iy, seed=3):
    xs, ys, hs = synth.block_cells(lv, ix, iy, cells=8)
    q = (np.random.default_rng(seed).normal(size=xs.size) + 0.5) * hs ** 2
    return xs, ys, hs, q


def _solve(lv, ix, iy, q, theta, order):
    P = api.adaptive_solve(lv, ix, iy, torch.from_numpy(q).cuda(), theta=theta, order=order)
    torch.cuda.synchronize()
    return P.cpu().numpy()


@pytest.mark.parametrize("theta", [0.5, 0.75])
def test_adaptive_solve_matches_direct_sum_on_every_cell(theta):
    lv, ix, iy = synth.adaptive_blocks(2, 5, centre=(0.45, 0.5), radius=0.15, band=1.0)
    xs, ys, hs, q = _case(lv, ix, iy)
    ref = oracle.green_sum_var(xs, ys, q, hs, xs, ys)
    e20 = np.linalg.norm(_solve(lv, ix, iy, q, theta, 20) - ref) / np.linalg.norm(ref)
    e8 = np.linalg.norm(_solve(lv, ix, iy, q, theta, 8) - ref) / np.linalg.norm(ref)
    print(f"theta {theta}: rel l2 p=8 {e8:.3e}  p=20 {e20:.3e}")
    assert e20 < 1e-6
    assert e20 < e8 / 100


def test_adaptive_solve_deep_layout_sampled_and_repeatable():
    """Levels 3..8 refined towards a small body (the finest cells 1/2048 of the domain),
    sampled cells against the oracle; two calls give the same bits."""
    lv, ix, iy = synth.adaptive_blocks(3, 8, centre=(0.3, 0.5), radius=0.05, band=1.0)
    assert lv.max() == 8 and lv.min() <= 4
    xs, ys, hs, q = _case(lv, ix, iy, seed=9)
    P1 = _solve(lv, ix, iy, q, 0.5, 20)
    P2 = _solve(lv, ix, iy, q, 0.5, 20)
    assert np.array_equal(P1, P2)
    rng = np.random.default_rng(1)
    cells = np.unique(np.concatenate([rng.choice(xs.size, 384, replace=False), [0, xs.size - 1]]))
    ref = oracle.green_sum_var(xs, ys, q, hs, xs[cells], ys[cells])
    assert np.linalg.norm(P1[cells] - ref) / np.linalg.norm(ref) < 1e-6


def test_adaptive_tree_reused_across_solves_and_orders():
    """A kept tree gives the same bits as one-shot solves, for two sources and for an order
    raised after a lower one (the expansions are reallocated)."""
    lv, ix, iy = synth.adaptive_blocks(2, 6, centre=(0.5, 0.45), radius=0.1, band=1.0)
    _, _, _, q1 = _case(lv, ix, iy, seed=4)
    _, _, _, q2 = _case(lv, ix, iy, seed=5)
    t = api.AdaptiveTree(lv, ix, iy, 0.6)
    try:
        got = []
        for q, order in ((q1, 12), (q2, 12), (q1, 20)):
            got.append(t.solve(torch.from_numpy(q).cuda(), order).cpu().numpy())
        for (q, order), g in zip(((q1, 12), (q2, 12), (q1, 20)), got):
            assert np.array_equal(g, _solve(lv, ix, iy, q, 0.6, order))
    finally:
        t.destroy()


def test_adaptive_solve_single_leaf_and_errors():
    lv, ix, iy = np.array([0]), np.array([0]), np.array([0])
    xs, ys, hs, q = _case(lv, ix, iy)
    ref = oracle.green_sum_var(xs, ys, q, hs, xs, ys)
    assert np.max(np.abs(_solve(lv, ix, iy, q, 0.5, 12) - ref)) < 1e-13 * np.max(np.abs(ref))
    for bad in (1, 31):
        with pytest.raises(api.PPError) as ei:
            _solve(lv, ix, iy, q, 0.5, bad)
        assert ei.value.status == api.PP_ERR_ARG


def test_adaptive_surface_treecode_matches_direct_sum():
    """pp_atree_surface_pressure: the tree-code over the adaptive tree at off-grid points (a
    circle around the body through the refined blocks, points inside the finest cells, and two
    points outside the domain where the root itself is accepted), against the oracle's direct
    sum over cells of several sizes; FP64 bar 1e-6 at p = 20, theta = 0.5, the error falling
    with the order, and a stricter theta more accurate."""
    lv, ix, iy = synth.adaptive_blocks(3, 7, centre=(0.3, 0.5), radius=0.05, band=2.0)
    xs, ys, hs, q = _case(lv, ix, iy, seed=5)
    t = np.linspace(0, 2 * np.pi, 700, endpoint=False)
    pts = np.concatenate([np.stack([0.3 + 0.053 * np.cos(t), 0.5 + 0.053 * np.sin(t)], 1),
                          np.stack([0.3 + 0.05 * np.cos(t[:50]) + 1e-5, 0.5 + 0.05 * np.sin(t[:50])], 1),
                          [[1.6, 0.5], [-0.4, -0.3]]])
    ref = oracle.green_sum_var(xs, ys, q, hs, pts[:, 0], pts[:, 1])
    tree = api.AdaptiveTree(lv, ix, iy, 0.5)
    qd = torch.from_numpy(q).cuda()
    pd = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    with pytest.raises(api.PPError) as e:
        tree.surface_pressure(qd, pd, 0.5)  # the multipoles come from a solve
    assert e.value.status == api.PP_ERR_STATE
    errs = {}
    for order, th in ((8, 0.5), (20, 0.5), (20, 0.3)):
        tree.solve(qd, order)
        P = tree.surface_pressure(qd, pd, th).cpu().numpy()
        errs[(order, th)] = np.linalg.norm(P - ref) / np.linalg.norm(ref)
        w = np.max(np.abs(P - ref)) / np.max(np.abs(ref))
        print(f"adaptive surface tree-code p={order} theta={th}: rel l2 {errs[(order, th)]:.2e} worst {w:.2e}")
    assert errs[(20, 0.5)] < 1e-6
    assert errs[(20, 0.5)] < 1e-2 * errs[(8, 0.5)]
    assert errs[(20, 0.3)] <= errs[(20, 0.5)]
    P1 = tree.surface_pressure(qd, pd, 0.5).cpu().numpy()
    P2 = tree.surface_pressure(qd, pd, 0.5).cpu().numpy()
    assert np.array_equal(P1, P2)
    tree.destroy()


def _solve_mixed(t, q, order):
    P = t.solve_mixed(torch.from_numpy(q).float().cuda(), order)
    torch.cuda.synchronize()
    return P.double().cpu().numpy()


@pytest.mark.parametrize("theta", [0.5, 0.75])
def test_adaptive_mixed_solve_matches_fp64_solve_and_direct_sum(theta):
    """pp_atree_solve_mixed (FP32 expansions and near field, FP64 monopoles and constants)
    against the FP64 solve at the same order (the mixed arithmetic alone) and against the
    oracle's direct sum (mixed arithmetic plus truncation), on every cell: relative l2 and the
    worst cell against the largest |P|, within 1e-5 at p = 12 and p = 20 (the FP32 level of
    the uniform-grid mixed path).  Two calls give the same bits."""
    lv, ix, iy = synth.adaptive_blocks(2, 5, centre=(0.45, 0.5), radius=0.15, band=1.0)
    xs, ys, hs, q = _case(lv, ix, iy)
    ref = oracle.green_sum_var(xs, ys, q, hs, xs, ys)
    t = api.AdaptiveTree(lv, ix, iy, theta)
    try:
        for order in (12, 20):
            pm = _solve_mixed(t, q, order)
            assert np.array_equal(pm, _solve_mixed(t, q, order))
            p64 = t.solve(torch.from_numpy(q).cuda(), order).cpu().numpy()
            e_arith = np.linalg.norm(pm - p64) / np.linalg.norm(p64)
            w_arith = np.max(np.abs(pm - p64)) / np.max(np.abs(p64))
            e_ref = np.linalg.norm(pm - ref) / np.linalg.norm(ref)
            print(f"theta {theta} p {order}: vs FP64 {e_arith:.2e} (worst {w_arith:.2e}), vs direct {e_ref:.2e}")
            assert e_arith < 1e-5 and w_arith < 1e-5
            if order == 20:
                assert e_ref < 1e-5
    finally:
        t.destroy()


def test_adaptive_mixed_solve_deep_layout_sampled():
    """Levels 3..8 (cells of 1/2048 next to the body and 1/64 far away), sampled cells against
    the oracle within 1e-5; the surface tree-code refuses to run on the stale FP64 multipoles
    a mixed solve leaves, and runs again after an FP64 solve."""
    lv, ix, iy = synth.adaptive_blocks(3, 8, centre=(0.3, 0.5), radius=0.05, band=1.0)
    xs, ys, hs, q = _case(lv, ix, iy, seed=9)
    t = api.AdaptiveTree(lv, ix, iy, 0.5)
    try:
        pm = _solve_mixed(t, q, 20)
        rng = np.random.default_rng(1)
        cells = np.unique(np.concatenate([rng.choice(xs.size, 384, replace=False), [0, xs.size - 1]]))
        ref = oracle.green_sum_var(xs, ys, q, hs, xs[cells], ys[cells])
        assert np.linalg.norm(pm[cells] - ref) / np.linalg.norm(ref) < 1e-5
        pts = torch.tensor([[0.3, 0.57], [0.37, 0.5]], dtype=torch.float64, device="cuda")
        qd = torch.from_numpy(q).cuda()
        with pytest.raises(api.PPError) as ei:
            t.surface_pressure(qd, pts, 0.5)
        assert ei.value.status == api.PP_ERR_STATE
        t.solve(qd, 20)
        t.surface_pressure(qd, pts, 0.5)
    finally:
        t.destroy()
