"""The adaptive quadtree and its dual-tree interaction lists (pp_atree_*), host only.

Checked against what the lists must satisfy, by brute force over all (target leaf, source
leaf) pairs: every pair covered exactly once (one near-field pair or one multipole-to-local
pair of ancestors); every multipole-to-local pair passes the acceptance test r_A + r_B <
theta d and its parent pair (the pair the walk split to reach it) does not; every near-field
pair fails it; on a uniform tree the near-field pairs are the uniform near list."""
import math

import numpy as np
import pytest

from paper_1610_04398_gb300 import api, synth


@pytest.fixture(scope="module")
def lib():
    try:
        return api.load()
    except RuntimeError as e:
        pytest.skip(str(e))


def _geom(t, b):
    s = 1.0 / (1 << int(t["level"][b]))
    return (t["ix"][b] + 0.5) * s, (t["iy"][b] + 0.5) * s, s


def _separated(t, a, b, theta):
    """The acceptance test written from its definition (r = half-diagonal; ties not separated)."""
    xa, ya, sa = _geom(t, a)
    xb, yb, sb = _geom(t, b)
    r = (sa + sb) * math.sqrt(2.0) / 2.0
    d = math.hypot(xa - xb, ya - yb)
    return r < theta * d * (1 - 1e-12)


def _leaf_sets(t):
    """For every box, the set of leaf indices below it (itself if a leaf)."""
    nb = len(t["level"])
    below = [None] * nb
    for b in range(nb - 1, -1, -1):  # children come after their parent
        if t["leaf"][b] >= 0:
            below[b] = [int(t["leaf"][b])]
        else:
            fc = int(t["first_child"][b])
            below[b] = below[fc] + below[fc + 1] + below[fc + 2] + below[fc + 3]
    return below


def _check_lists(t, nleaf, theta):
    below = _leaf_sets(t)
    cover = np.zeros((nleaf, nleaf), np.int32)
    for a, b in t["p2p"]:
        cover[a, b] += 1
    for a, b in t["m2l"]:
        cover[np.ix_(below[a], below[b])] += 1
    assert np.all(cover == 1), "every leaf pair exactly once"
    leaf_box = {int(t["leaf"][b]): b for b in range(len(t["level"])) if t["leaf"][b] >= 0}
    for a, b in t["p2p"]:
        ba, bb = leaf_box[a], leaf_box[b]
        assert ba == bb or not _separated(t, ba, bb, theta * (1 - 1e-9))  # a tie is not separated
    for a, b in t["m2l"]:
        assert _separated(t, a, b, theta), (a, b)
        # the split that produced (a, b) replaced a or b by a child: that parent pair failed
        pa, pb = int(t["parent"][a]), int(t["parent"][b])
        parents = [p for p in ((pa, b), (a, pb)) if p[0] >= 0 and p[1] >= 0]
        assert any(not _separated(t, x, y, theta * (1 - 1e-9)) for x, y in parents)


def test_single_leaf_domain(lib):
    t = api.adaptive_tree([0], [0], [0], 0.5)
    assert len(t["level"]) == 1 and t["leaf"][0] == 0 and t["first_child"][0] == -1
    assert t["m2l"].shape == (0, 2) and t["p2p"].tolist() == [[0, 0]]


@pytest.mark.parametrize("theta", [0.4, 0.5, 0.6, 0.75])
def test_uniform_tree_matches_uniform_lists(lib, theta):
    L = 4
    n = 1 << L
    iy, ix = np.divmod(np.arange(n * n), n)
    t = api.adaptive_tree(np.full(n * n, L), ix, iy, theta)
    assert len(t["level"]) == (4 ** (L + 1) - 1) // 3 and t["max_level"] == L
    near = {tuple(d) for d in api.pp_near_offsets(theta)}
    want = sorted((a, b) for a in range(n * n) for b in range(n * n)
                  if (ix[b] - ix[a], iy[b] - iy[a]) in near)
    assert [tuple(p) for p in t["p2p"]] == want
    _check_lists(t, n * n, theta)


@pytest.mark.parametrize("theta,seed", [(0.5, 1), (0.6, 2), (0.75, 3), (0.4, 4)])
def test_adaptive_trees_cover_every_pair_once(lib, theta, seed):
    lv, ix, iy = synth.adaptive_blocks(1, 6, centre=(0.3 + 0.05 * seed, 0.5), radius=0.1, band=1.0,
                                       seed=seed, p_extra=0.05)
    assert np.isclose(np.sum(4.0 ** (-lv.astype(np.float64))), 1.0)
    t = api.adaptive_tree(lv, ix, iy, theta)
    assert t["max_level"] == lv.max()
    # leaf indices refer to the caller's order
    for b in range(len(t["level"])):
        k = int(t["leaf"][b])
        if k >= 0:
            assert (t["level"][b], t["ix"][b], t["iy"][b]) == (lv[k], ix[k], iy[k])
    _check_lists(t, len(lv), theta)


def test_unbalanced_layout_is_accepted(lib):
    """Nothing requires 2:1 balance: one level-1 quadrant next to level-6 blocks."""
    leaves = [(1, 1, 0), (1, 0, 1), (1, 1, 1)]
    # refine quadrant (1, 0, 0) down to level 6 along its top-right corner only
    def refine(l, i, j):
        if l == 6:
            return [(l, i, j)]
        out = []
        for c in range(4):
            a, b = 2 * i + (c & 1), 2 * j + (c >> 1)
            if c == 3:
                out += refine(l + 1, a, b)
            else:
                out.append((l + 1, a, b))
        return out
    leaves += refine(1, 0, 0)
    lv, ix, iy = (np.array(v) for v in zip(*leaves))
    t = api.adaptive_tree(lv, ix, iy, 0.5)
    _check_lists(t, len(lv), 0.5)


def test_invalid_layouts(lib):
    ok = ([1, 1, 1, 1], [0, 1, 0, 1], [0, 0, 1, 1])
    api.adaptive_tree(*ok, 0.5)
    bad = [
        ([1, 1, 1], [0, 1, 0], [0, 0, 1]),                    # a gap
        ([1, 1, 1, 1, 1], [0, 1, 0, 1, 1], [0, 0, 1, 1, 1]),  # a duplicate
        ([1, 1, 1, 1, 2], [0, 1, 0, 1, 0], [0, 0, 1, 1, 0]),  # a leaf inside another leaf
        ([0, 1], [0, 0], [0, 0]),                              # the root and a child
        ([1, 1, 1, 1], [0, 2, 0, 1], [0, 0, 1, 1]),            # an index out of range
        ([21], [0], [0]),                                      # a level out of range
    ]
    for lv, ix, iy in bad:
        with pytest.raises(api.PPError) as ei:
            api.adaptive_tree(lv, ix, iy, 0.5)
        assert ei.value.status == api.PP_ERR_ARG
    with pytest.raises(api.PPError):
        api.adaptive_tree(*ok, 0.2)  # theta out of range


def test_tree_queries_and_solve_reject_bad_arguments_on_the_host(lib):
    """NULL handles, and pp_atree_solve's argument checks (done before any CUDA call)."""
    import ctypes
    sizes = (ctypes.c_int64 * 4)()
    assert lib.pp_atree_sizes(None, sizes) == api.PP_ERR_ARG
    assert lib.pp_atree_boxes(None, None, None, None, None, None, None) == api.PP_ERR_ARG
    assert lib.pp_atree_lists(None, None, None) == api.PP_ERR_ARG
    assert lib.pp_atree_destroy(None) == api.PP_OK
    assert lib.pp_atree_create(1, None, None, None, 0.5, None) == api.PP_ERR_ARG
    ip = ctypes.POINTER(ctypes.c_int)
    one = np.zeros(1, np.int32)
    h = ctypes.c_void_p()
    assert lib.pp_atree_create(1, one.ctypes.data_as(ip), one.ctypes.data_as(ip), one.ctypes.data_as(ip), 0.5,
                               ctypes.byref(h)) == api.PP_OK
    try:
        assert lib.pp_atree_sizes(h, None) == api.PP_ERR_ARG
        assert lib.pp_atree_sizes(h, sizes) == api.PP_OK and list(sizes) == [1, 0, 1, 0]
        fake = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
        assert lib.pp_atree_solve(h, 20, None, fake, None) == api.PP_ERR_ARG
        assert lib.pp_atree_solve(h, 20, fake, None, None) == api.PP_ERR_ARG
        for bad in (1, 31, -3):
            assert lib.pp_atree_solve(h, bad, fake, fake, None) == api.PP_ERR_ARG
    finally:
        lib.pp_atree_destroy(h)
