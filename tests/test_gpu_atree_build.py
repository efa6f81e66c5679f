"""The adaptive quadtree and its interaction lists built on the GPU (pp_atree_create_device:
Morton keys, radix sort, tiling check, level-by-level box scans, breadth-first dual-tree
walk) against the host build: the same boxes in the same order and the same sorted lists,
for layouts refined towards a body (shuffled leaf order), uniform layouts, a single leaf and
a larger layout; the brute-force coverage checks of tests/test_atree_host.py on a device
tree; invalid layouts (gap, overlap, duplicate, out of range) refused; a solve on a device
tree equal bitwise to one on the host tree (Appendix A.2's hierarchical grouping)."""
import time

import numpy as np
import pytest

from paper_1610_04398_gb300 import api, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("level", "ix", "iy", "parent", "first_child", "leaf", "m2l", "p2p", "max_level")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()


def _same(lv, ix, iy, theta):
    t0 = time.perf_counter()
    h = api.adaptive_tree(lv, ix, iy, theta)
    t1 = time.perf_counter()
    d = api.adaptive_tree(lv, ix, iy, theta, device=True)
    t2 = time.perf_counter()
    for k in KEYS:
        assert np.array_equal(np.asarray(h[k]), np.asarray(d[k])), k
    return d, t1 - t0, t2 - t1


def _layouts():
    out = [synth.adaptive_blocks(2, 5), synth.adaptive_blocks(3, 7, band=2.0),
           synth.adaptive_blocks(1, 6, seed=3, p_extra=0.3)]
    for L in (0, 1, 3):  # uniform, the single leaf included
        ix, iy = np.meshgrid(np.arange(1 << L), np.arange(1 << L))
        out.append((np.full(4 ** L, L, np.int32), ix.ravel().astype(np.int32), iy.ravel().astype(np.int32)))
    return out


@pytest.mark.parametrize("theta", [0.5, 0.75])
def test_device_tree_equals_host_tree(theta):
    rng = np.random.default_rng(7)
    for lv, ix, iy in _layouts():
        perm = rng.permutation(len(lv))  # the build may not depend on the leaf order given
        _same(lv[perm], ix[perm], iy[perm], theta)


def test_device_tree_passes_the_coverage_checks():
    import test_atree_host as host_checks
    lv, ix, iy = synth.adaptive_blocks(2, 6, seed=5, p_extra=0.2)
    for theta in (0.5, 0.75):
        d = api.adaptive_tree(lv, ix, iy, theta, device=True)
        host_checks._check_lists(d, len(lv), theta)


def test_large_layout_and_build_times():
    lv, ix, iy = synth.adaptive_blocks(4, 11, centre=(0.3, 0.5), radius=0.05, band=2.0)
    d, t_host, t_dev = _same(lv, ix, iy, 0.5)
    print(f"{len(lv)} leaves, {len(d['level'])} boxes, {len(d['m2l'])} + {len(d['p2p'])} pairs: "
          f"host build {t_host * 1e3:.1f} ms, device build {t_dev * 1e3:.1f} ms (first call)")
    t0 = time.perf_counter()
    api.adaptive_tree(lv, ix, iy, 0.5, device=True)
    print(f"device build again {1e3 * (time.perf_counter() - t0):.1f} ms")


def test_invalid_layouts_are_refused():
    lv, ix, iy = synth.adaptive_blocks(2, 4)
    bad = [
        (lv[1:], ix[1:], iy[1:]),                                               # a gap
        (np.append(lv, lv[0] - 1), np.append(ix, ix[0] // 2), np.append(iy, iy[0] // 2)),  # overlap
        (np.append(lv, lv[3]), np.append(ix, ix[3]), np.append(iy, iy[3])),     # duplicate
        (np.where(np.arange(len(lv)) == 2, 25, lv), ix, iy),                     # level out of range
        (lv, np.where(np.arange(len(lv)) == 2, 1 << 20, ix), iy),                # index out of range
    ]
    for b in bad:
        with pytest.raises(api.PPError) as e:
            api.adaptive_tree(*b, 0.5, device=True)
        assert e.value.status == api.PP_ERR_ARG
        with pytest.raises(api.PPError):
            api.adaptive_tree(*b, 0.5)


def test_solve_on_device_tree_equals_host_tree():
    lv, ix, iy = synth.adaptive_blocks(3, 7, band=2.0)
    xs, ys, hs = synth.block_cells(lv, ix, iy, cells=8)
    q = torch.from_numpy((np.random.default_rng(11).normal(size=xs.size) + 0.5) * hs ** 2).cuda()
    th = api.AdaptiveTree(lv, ix, iy, 0.5)
    td = api.AdaptiveTree(lv, ix, iy, 0.5, device=True)
    Ph = th.solve(q, 16)
    Pd = td.solve(q, 16)
    torch.cuda.synchronize()
    assert torch.equal(Ph, Pd)
    th.destroy()
    td.destroy()
