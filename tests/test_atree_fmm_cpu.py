"""An FMM assembled on the CPU from the adaptive tree's interaction lists (pp_atree_*) and the
oracle's expansion steps (Appendix A.2 and their standard local shifts) reproduces the direct
sum over cells of several sizes (oracle.green_sum_var) to within the truncation error, and the
error falls as the order grows.  This checks the lists as an FMM uses them: multipole-to-local
pairs between boxes of different levels, local shifts down the adaptive tree, and near-field
pairs between leaves of different sizes.

Tolerance: a pair accepted by r_A + r_B < theta d contributes with a truncation error below
~ theta^(p+1) of its size (the series in (r/d)); summed over the lists the relative l2 error
of the field is allowed 10 theta^(p+1)."""
import math

import numpy as np
import pytest

import oracle
from paper_1610_04398_gb300 import api, synth


@pytest.fixture(scope="module")
def lib():
    try:
        return api.load()
    except RuntimeError as e:
        pytest.skip(str(e))


def _fmm(t, lv, ix, iy, q, cells, p):
    nb = len(t["level"])
    side = 1.0 / (1 << t["level"].astype(np.int64))
    zc = (t["ix"] + 0.5) * side + 1j * (t["iy"] + 0.5) * side
    xs, ys, hs = synth.block_cells(lv, ix, iy, cells=cells)
    zs = xs + 1j * ys
    per = cells * cells
    leaf_cells = lambda k: slice(k * per, (k + 1) * per)  # noqa: E731
    # upward: leaves by P2M, internal boxes from their children (children follow parents)
    S = np.zeros(nb)
    alpha = np.zeros((nb, p), np.complex128)
    for b in range(nb - 1, -1, -1):
        k = int(t["leaf"][b])
        if k >= 0:
            S[b], alpha[b] = oracle.p2m(q[leaf_cells(k)], zs[leaf_cells(k)], zc[b], p)
        else:
            fc = int(t["first_child"][b])
            for c in range(fc, fc + 4):
                s_c, beta = oracle.m2m(S[c], alpha[c], zc[c], zc[b])
                S[b] += s_c
                alpha[b] += beta
    # multipole-to-local over the pair list, then local shifts down the tree
    loc = np.zeros((nb, p + 1), np.complex128)
    for a, b in t["m2l"]:
        loc[a] += oracle.m2l(S[b], alpha[b], zc[b], zc[a])
    for b in range(nb):
        par = int(t["parent"][b])
        if par >= 0:
            loc[b] += oracle.l2l(loc[par], zc[par], zc[b])
    # leaves: local expansion at their cells plus the near-field pairs, direct
    P = np.zeros(zs.size)
    for b in range(nb):
        k = int(t["leaf"][b])
        if k >= 0:
            P[leaf_cells(k)] += oracle.l2p(loc[b], zc[b], zs[leaf_cells(k)])
    for a, b in t["p2p"]:
        sa, sb = leaf_cells(int(a)), leaf_cells(int(b))
        P[sa] += oracle.green_sum_var(xs[sb], ys[sb], q[sb], hs[sb], xs[sa], ys[sa])
    return P, xs, ys, hs


@pytest.mark.parametrize("theta", [0.5, 0.6])
def test_fmm_from_the_lists_matches_the_direct_sum(lib, theta):
    lv, ix, iy = synth.adaptive_blocks(2, 5, centre=(0.45, 0.5), radius=0.15, band=1.0)
    assert len(np.unique(lv)) >= 3
    cells = 4
    xs, ys, hs = synth.block_cells(lv, ix, iy, cells=cells)
    rng = np.random.default_rng(3)
    q = (rng.normal(size=xs.size) + 0.5) * hs ** 2
    ref = oracle.green_sum_var(xs, ys, q, hs, xs, ys)
    t = api.adaptive_tree(lv, ix, iy, theta)
    assert len(t["m2l"]) > 0 and len(np.unique(t["level"][t["m2l"][:, 0]] - t["level"][t["m2l"][:, 1]])) > 1
    errs = {}
    for p in (6, 12):
        P, _, _, _ = _fmm(t, lv, ix, iy, q, cells, p)
        errs[p] = np.linalg.norm(P - ref) / np.linalg.norm(ref)
        assert errs[p] < 10 * theta ** (p + 1), (p, errs[p])
    assert errs[12] < errs[6] / 20


@pytest.mark.parametrize("theta", [0.5, 0.6])
def test_treecode_over_the_adaptive_tree_matches_the_direct_sum_at_surface_points(lib, theta):
    """Surface pressure by the tree-code of Appendix A.2 over the adaptive tree: a box is
    accepted for a point target when r_box < theta d (its multipole, Eq. pressTruncated), a
    leaf that is not accepted is summed directly; points on a circle through the refined
    region (off the cell centres)."""
    lv, ix, iy = synth.adaptive_blocks(2, 6, centre=(0.5, 0.5), radius=0.2, band=1.0)
    cells = 4
    xs, ys, hs = synth.block_cells(lv, ix, iy, cells=cells)
    q = (np.random.default_rng(8).normal(size=xs.size) + 0.3) * hs ** 2
    ang = np.linspace(0.0, 2 * math.pi, 97, endpoint=False)
    px, py = 0.5 + 0.2 * np.cos(ang), 0.5 + 0.2 * np.sin(ang)
    ref = oracle.green_sum_var(xs, ys, q, hs, px, py)
    t = api.adaptive_tree(lv, ix, iy, theta)
    nb = len(t["level"])
    side = 1.0 / (1 << t["level"].astype(np.int64))
    zc = (t["ix"] + 0.5) * side + 1j * (t["iy"] + 0.5) * side
    per = cells * cells
    p = 12
    S = np.zeros(nb)
    alpha = np.zeros((nb, p), np.complex128)
    zs = xs + 1j * ys
    for b in range(nb - 1, -1, -1):
        k = int(t["leaf"][b])
        if k >= 0:
            sl = slice(k * per, (k + 1) * per)
            S[b], alpha[b] = oracle.p2m(q[sl], zs[sl], zc[b], p)
        else:
            fc = int(t["first_child"][b])
            for c in range(fc, fc + 4):
                s_c, beta = oracle.m2m(S[c], alpha[c], zc[c], zc[b])
                S[b] += s_c
                alpha[b] += beta
    P = np.zeros(px.size)
    accepted = 0
    for i in range(px.size):
        z = px[i] + 1j * py[i]
        stack = [0]
        while stack:
            b = stack.pop()
            r = side[b] * math.sqrt(2.0) / 2.0
            if r < theta * abs(z - zc[b]):
                P[i] += oracle.m2p(S[b], alpha[b], zc[b], z)
                accepted += 1
            elif t["leaf"][b] >= 0:
                k = int(t["leaf"][b])
                sl = slice(k * per, (k + 1) * per)
                P[i] += oracle.green_sum_var(xs[sl], ys[sl], q[sl], hs[sl], [px[i]], [py[i]])[0]
            else:
                fc = int(t["first_child"][b])
                stack.extend(range(fc, fc + 4))
    assert accepted > 10 * px.size
    err = np.linalg.norm(P - ref) / np.linalg.norm(ref)
    assert err < 10 * theta ** (p + 1), err
