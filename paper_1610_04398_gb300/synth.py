"""Seeded synthetic flow snapshots shaped like the paper's workloads.

This module only *generates inputs*: velocity fields u, v, the penalisation mask
chi and the body velocity u_s on an N x N cell-centred grid, and ordered surface
polygons with outward normals.  It contains none of the method's arithmetic (no
Poisson source, no Green's sum, no traction) so that both the CUDA path and the
CPU oracle can be fed from it without sharing any of the method's code.

Workloads (all fields are float64, row-major ``[j, i]`` with j the y index):

* Lamb-Oseen vortex (Sec. 2.2 pressure Poisson equation test case):
  u_theta = Gamma / (2 pi r) (1 - exp(-r^2 / sigma^2)), no body.
* Rigid cylinder of Sec. 3.1 (impulsively started cylinder geometry): potential
  flow past a circle plus a seeded wake of Gaussian vortex blobs, chi from the
  signed distance smoothed over two cells (Sec. 2.1 smoothed Heaviside).
* Self-propelled swimmer of Sec. 3.3: zebrafish half-width profile (Eq. fishWidth)
  on a travelling-wave midline, deformation velocity inside the body and a blob
  wake outside.

Seeds use numpy's PCG64 so every snapshot is reproducible from (workload, seed).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Snapshot",
    "cell_centres",
    "smoothed_heaviside",
    "lamb_oseen",
    "circle_surface",
    "cylinder_flow",
    "fish_half_width",
    "swimmer_snapshot",
    "random_grid_sizes",
    "swimmer_batch",
]


@dataclass
class Snapshot:
    """One synthetic flow snapshot on an n x n cell-centred grid.

    ``points``/``normals`` describe a closed polygon ordered counter-clockwise
    with outward unit normals; ``lift`` is the recommended traction sample
    offset along the normal (2h for rigid bodies, 0 for deforming ones).
    """

    n: int
    h: float
    x0: float
    y0: float
    u: np.ndarray
    v: np.ndarray
    chi: np.ndarray
    usx: np.ndarray
    usy: np.ndarray
    lam: float
    nu: float
    points: np.ndarray
    normals: np.ndarray
    lift: float
    uinf: tuple = (1.0, 0.0)
    meta: dict = field(default_factory=dict)


def cell_centres(n: int, h: float, x0: float = 0.0, y0: float = 0.0):
    """Cell-centre coordinates X[j, i] = x0 + (i + 1/2) h, Y[j, i] = y0 + (j + 1/2) h."""
    c = (np.arange(n, dtype=np.float64) + 0.5) * h
    X, Y = np.meshgrid(x0 + c, y0 + c)
    return X, Y


def smoothed_heaviside(d: np.ndarray, eps: float) -> np.ndarray:
    """Smoothed step of half-width eps on the signed distance d (positive inside).

    H = 0 for d < -eps, 1 for d > eps and 1/2 (1 + d/eps + sin(pi d/eps)/pi)
    in between, so chi rises from 0 to 1 over two cells when eps = h.
    """
    d = np.asarray(d, dtype=np.float64)
    t = np.clip(d / eps, -1.0, 1.0)
    return 0.5 * (1.0 + t + np.sin(np.pi * t) / np.pi)


_DEVICE = None


def set_device(device):
    """Evaluate the blob velocity sums with torch on ``device`` (e.g. "cuda") instead of
    numpy; None restores numpy.  Same formula in FP64, only faster for large grids."""
    global _DEVICE
    _DEVICE = device


def _blob_velocity(X, Y, xb, yb, gam, sigma, u, v):
    """Add the velocity of Gaussian vortex blobs (in place).

    Each blob induces u_theta = gam / (2 pi r) (1 - exp(-r^2 / sigma^2)).
    """
    if _DEVICE is not None:
        import torch
        Xt = torch.from_numpy(np.ascontiguousarray(X)).to(_DEVICE)
        Yt = torch.from_numpy(np.ascontiguousarray(Y)).to(_DEVICE)
        ut = torch.zeros_like(Xt)
        vt = torch.zeros_like(Xt)
        for xc, yc, g in zip(xb, yb, gam):
            dx = Xt - float(xc)
            dy = Yt - float(yc)
            r2 = dx * dx + dy * dy
            k = torch.where(r2 > 0, -torch.expm1(-r2 / (sigma * sigma)) / torch.where(r2 > 0, r2, 1.0),
                            torch.full_like(r2, 1.0 / (sigma * sigma)))
            k = k * (float(g) / (2.0 * np.pi))
            ut -= dy * k
            vt += dx * k
        u += ut.cpu().numpy()
        v += vt.cpu().numpy()
        return
    for xc, yc, g in zip(xb, yb, gam):
        dx = X - xc
        dy = Y - yc
        r2 = dx * dx + dy * dy
        with np.errstate(divide="ignore", invalid="ignore"):
            k = -np.expm1(-r2 / (sigma * sigma)) / r2
        k = np.where(r2 > 0.0, k, 1.0 / (sigma * sigma))
        k *= g / (2.0 * np.pi)
        u -= dy * k
        v += dx * k


def lamb_oseen(n: int = 128, gamma: float = 1.0, sigma: float = 0.05,
               centre=(0.5, 0.5), n_circle: int = 256, r_circle: float = 0.15) -> Snapshot:
    """Lamb-Oseen vortex on [0,1]^2 (no body, chi = 0).

    Surface targets: ``n_circle`` points equally spaced in angle on a circle of
    radius ``r_circle`` around the vortex centre.
    """
    h = 1.0 / n
    X, Y = cell_centres(n, h)
    u = np.zeros((n, n))
    v = np.zeros((n, n))
    _blob_velocity(X, Y, [centre[0]], [centre[1]], [gamma], sigma, u, v)
    zero = np.zeros((n, n))
    pts, nrm = circle_surface(n_circle, centre, r_circle)
    return Snapshot(n=n, h=h, x0=0.0, y0=0.0, u=u, v=v, chi=zero.copy(), usx=zero.copy(),
                    usy=zero.copy(), lam=0.0, nu=0.0, points=pts, normals=nrm, lift=0.0,
                    meta=dict(kind="lamb_oseen", gamma=gamma, sigma=sigma, centre=centre))


def circle_surface(npts: int, centre, radius: float):
    """Counter-clockwise circle polygon with outward unit normals."""
    th = 2.0 * np.pi * np.arange(npts, dtype=np.float64) / npts
    nrm = np.stack([np.cos(th), np.sin(th)], axis=1)
    pts = np.asarray(centre, dtype=np.float64)[None, :] + radius * nrm
    return pts, nrm


def cylinder_flow(n: int = 1024, diameter: float = 0.1, centre=(0.3, 0.5), U: float = 1.0,
                  n_blobs: int = 64, blob_std: float = 0.1, lam: float = 1e4, nu: float = 1e-4,
                  n_surface: int = 2048, seed: int = 2000, with_potential: bool = True) -> Snapshot:
    """Rigid cylinder in a unit square: potential flow + seeded blob wake.

    * chi = H_h(R - r): smoothed over two cells.
    * u = (1 - chi) (u_potential + u_blobs), u_s = 0 (rigid, at rest).
    * 64 blobs of core 2h with strengths ~ N(0, blob_std^2), centres uniform
      in [xc + D, min(xc + 6D, 0.95)] x [yc - D, yc + D].
    * ``n_surface`` points equally spaced in angle on r = R; lift = 2h.
    """
    h = 1.0 / n
    R = 0.5 * diameter
    X, Y = cell_centres(n, h)
    dx = X - centre[0]
    dy = Y - centre[1]
    r = np.hypot(dx, dy)
    chi = smoothed_heaviside(R - r, h)
    u = np.zeros((n, n))
    v = np.zeros((n, n))
    if with_potential:
        # complex velocity W = u - i v = U (1 - R^2 / z^2) outside the circle
        fluid = r > 0.5 * R
        z = (dx + 1j * dy)[fluid]
        W = U * (1.0 - R * R / (z * z))
        u[fluid] = W.real
        v[fluid] = -W.imag
    rng = np.random.Generator(np.random.PCG64(seed))
    xb = rng.uniform(centre[0] + diameter, min(centre[0] + 6 * diameter, 0.95), n_blobs)
    yb = rng.uniform(centre[1] - diameter, centre[1] + diameter, n_blobs)
    gam = rng.normal(0.0, blob_std, n_blobs)
    _blob_velocity(X, Y, xb, yb, gam, 2.0 * h, u, v)
    u *= 1.0 - chi
    v *= 1.0 - chi
    zero = np.zeros((n, n))
    pts, nrm = circle_surface(n_surface, centre, R)
    return Snapshot(n=n, h=h, x0=0.0, y0=0.0, u=u, v=v, chi=chi, usx=zero.copy(),
                    usy=zero.copy(), lam=lam, nu=nu, points=pts, normals=nrm, lift=2.0 * h,
                    uinf=(U, 0.0), meta=dict(kind="cylinder", seed=seed, R=R, centre=centre))


def fish_half_width(s: np.ndarray, L: float) -> np.ndarray:
    """Zebrafish half-width profile w(s) of Eq. fishWidth (w_h = s_b = 0.04L,
    s_t = 0.95L, w_t = 0.01L)."""
    s = np.asarray(s, dtype=np.float64)
    wh = sb = 0.04 * L
    st = 0.95 * L
    wt = 0.01 * L
    head = np.sqrt(np.clip(2.0 * wh * s - s * s, 0.0, None))
    mid = wh - (wh - wt) * (s - sb) / (st - sb)
    tail = wt * (L - s) / (L - st)
    return np.where(s < sb, head, np.where(s < st, mid, tail))


def _midline(s: np.ndarray, L: float, phase: float, head=(0.4, 0.5)):
    """Travelling-wave midline (Sec. 3.3): y(s,t) = A(s) sin(2 pi (s/L - t/T)),
    A(s) = 0.125 L (0.03125 + s/L) / 1.03125; x(s) from inextensibility,
    integrated by the trapezoid rule from the head."""
    A = 0.125 * L * (0.03125 + s / L) / 1.03125
    arg = 2.0 * np.pi * (s / L - phase)
    y = A * np.sin(arg)
    dA = 0.125 / 1.03125
    dy = dA * np.sin(arg) + A * (2.0 * np.pi / L) * np.cos(arg)
    dxds = np.sqrt(np.clip(1.0 - dy * dy, 0.0, None))
    x = np.concatenate([[0.0], np.cumsum(0.5 * (dxds[1:] + dxds[:-1]) * np.diff(s))])
    return head[0] + x, head[1] + y


def swimmer_snapshot(n: int, phase: float, L: float = 0.2, n_surface: int = 4096,
                     n_blobs: int = 64, blob_std: float = 0.1, lam: float = 1e4,
                     nu: float = 1e-4, seed: int = 4000, n_mid: int = 2049) -> Snapshot:
    """Anguilliform swimmer at phase t/T on an n x n grid over [0,1]^2.

    * Midline from the head at (0.4, 0.5) towards +x; surface = midline +/- w(s)
      along the midline normal, n_surface/2 points per side at s = (i+1/2)L/(n/2),
      ordered counter-clockwise (right side head->tail, left side tail->head),
      outward normals from the polygon's central-difference tangents.
    * chi = H_h(w(s*) - |x - X(s*)|) with s* the nearest midline sample;
      u_s = time derivative of the midline position at s* (centred difference).
    * u = chi u_s + (1 - chi) u_wake, wake = blobs in [x_tail + 0.05, min(x_tail + 0.35, 0.95)]
      x [0.4, 0.6] with core 2h and strengths ~ N(0, blob_std^2).
    """
    h = 1.0 / n
    sm = np.linspace(0.0, L, n_mid)
    mx, my = _midline(sm, L, phase)
    dt = 1e-5
    mxp, myp = _midline(sm, L, phase + dt)
    mxm, mym = _midline(sm, L, phase - dt)
    vx = (mxp - mxm) / (2 * dt)
    vy = (myp - mym) / (2 * dt)
    w = fish_half_width(sm, L)

    X, Y = cell_centres(n, h)
    chi = np.zeros((n, n))
    usx = np.zeros((n, n))
    usy = np.zeros((n, n))
    pad = 0.02 * L + 2 * h
    i0 = max(int((mx.min() - pad) / h), 0)
    i1 = min(int((mx.max() + pad) / h) + 1, n)
    j0 = max(int((my.min() - 0.04 * L - pad) / h), 0)
    j1 = min(int((my.max() + 0.04 * L + pad) / h) + 1, n)
    Xb = X[j0:j1, i0:i1].ravel()
    Yb = Y[j0:j1, i0:i1].ravel()
    best = np.full(Xb.shape, np.inf)
    arg = np.zeros(Xb.shape, dtype=np.int64)
    for k0 in range(0, n_mid, 256):
        ddx = Xb[:, None] - mx[None, k0:k0 + 256]
        ddy = Yb[:, None] - my[None, k0:k0 + 256]
        d2 = ddx * ddx + ddy * ddy
        a = d2.argmin(axis=1)
        m = d2[np.arange(d2.shape[0]), a]
        upd = m < best
        best[upd] = m[upd]
        arg[upd] = a[upd] + k0
    sd = w[arg] - np.sqrt(best)
    shape = (j1 - j0, i1 - i0)
    chi[j0:j1, i0:i1] = smoothed_heaviside(sd, h).reshape(shape)
    usx[j0:j1, i0:i1] = vx[arg].reshape(shape)
    usy[j0:j1, i0:i1] = vy[arg].reshape(shape)

    rng = np.random.Generator(np.random.PCG64(seed))
    xt = mx[-1]
    xb = rng.uniform(xt + 0.05, min(xt + 0.35, 0.95), n_blobs)
    yb = rng.uniform(0.4, 0.6, n_blobs)
    gam = rng.normal(0.0, blob_std, n_blobs)
    uw = np.zeros((n, n))
    vw = np.zeros((n, n))
    _blob_velocity(X, Y, xb, yb, gam, 2.0 * h, uw, vw)
    u = chi * usx + (1.0 - chi) * uw
    v = chi * usy + (1.0 - chi) * vw

    half = n_surface // 2
    ss = (np.arange(half) + 0.5) * L / half
    px, py = _midline(ss, L, phase)
    # midline tangent and left normal by centred differences on a fine copy
    e = 1e-6 * L
    pxp, pyp = _midline(np.concatenate([[0.0], ss + e]), L, phase)
    pxm, pym = _midline(np.concatenate([[0.0], ss - e]), L, phase)
    tx = (pxp[1:] - pxm[1:]) / (2 * e)
    ty = (pyp[1:] - pym[1:]) / (2 * e)
    tn = np.hypot(tx, ty)
    nx, ny = -ty / tn, tx / tn
    ws = fish_half_width(ss, L)
    right = np.stack([px - ws * nx, py - ws * ny], axis=1)
    left = np.stack([px + ws * nx, py + ws * ny], axis=1)[::-1]
    pts = np.concatenate([right, left], axis=0)
    tan = np.roll(pts, -1, axis=0) - np.roll(pts, 1, axis=0)
    nrm = np.stack([tan[:, 1], -tan[:, 0]], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return Snapshot(n=n, h=h, x0=0.0, y0=0.0, u=u, v=v, chi=chi, usx=usx, usy=usy, lam=lam,
                    nu=nu, points=pts, normals=nrm, lift=0.0, uinf=(-1.0, 0.0),
                    meta=dict(kind="swimmer", phase=phase, seed=seed, L=L))


def random_grid_sizes(seed: int, choices=(256, 512, 1024, 2048)):
    """Grid side and phase for one swimmer snapshot, drawn from ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.choice(np.asarray(choices)))
    phase = float(rng.uniform(0.0, 1.0))
    return n, phase


def swimmer_batch(count: int = 64, seed0: int = 4000, n_surface: int = 4096,
                  choices=(256, 512, 1024, 2048)):
    """The swimmer batch workload: snapshot k has its grid side and phase drawn from seed
    seed0 + k (``random_grid_sizes``) and its wake from the same seed."""
    out = []
    for k in range(count):
        n, phase = random_grid_sizes(seed0 + k, choices)
        out.append(swimmer_snapshot(n, phase, seed=seed0 + k, n_surface=n_surface))
    return out


# ------------------------------------------------------------------ adaptive block layouts
def adaptive_blocks(min_level: int = 2, max_level: int = 6, centre=(0.3, 0.5), radius: float = 0.05,
                    band: float = 1.5, seed: int = None, p_extra: float = 0.0):
    """Leaf blocks (level, ix, iy) tiling the unit square, refined towards a circle the way a
    multiresolution grid refines towards a body: a block of side s at level l < max_level is
    split when its centre lies within band * s of the circle (plus, with a seed, a random
    fraction p_extra of the other blocks), then the layout is 2:1 balanced (blocks that touch,
    edges or corners, differ by at most one level).  Returns three int32 arrays."""
    rng = np.random.default_rng(seed) if seed is not None else None
    cx, cy = centre
    leaves = {(min_level, i, j) for i in range(1 << min_level) for j in range(1 << min_level)}

    def wants(l, i, j):
        if l >= max_level:
            return False
        s = 1.0 / (1 << l)
        d = abs(math.hypot((i + 0.5) * s - cx, (j + 0.5) * s - cy) - radius)
        if d < band * s:
            return True
        return rng is not None and rng.random() < p_extra

    def split(l, i, j):
        return [(l + 1, 2 * i + a, 2 * j + b) for b in (0, 1) for a in (0, 1)]

    changed = True
    while changed:
        changed = False
        for leaf in sorted(leaves):
            if wants(*leaf):
                leaves.remove(leaf)
                leaves.update(split(*leaf))
                changed = True
    # 2:1 balance: a leaf touching a leaf two or more levels finer is split
    changed = True
    while changed:
        changed = False
        finest = {}
        for (l, i, j) in leaves:
            finest[(l, i, j)] = l
        for (l, i, j) in sorted(leaves):
            s = 1 << l
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    ni, nj = i + di, j + dj
                    if (di, dj) == (0, 0) or not (0 <= ni < s and 0 <= nj < s):
                        continue
                    # any leaf inside the neighbour block at level >= l + 2 touches this one
                    if _deepest_inside(leaves, l, ni, nj) >= l + 2:
                        leaves.discard((l, i, j))
                        leaves.update(split(l, i, j))
                        changed = True
                        break
                else:
                    continue
                break
            if changed:
                break
    arr = np.array(sorted(leaves), dtype=np.int32)
    return arr[:, 0].copy(), arr[:, 1].copy(), arr[:, 2].copy()


def _deepest_inside(leaves, l, i, j, limit: int = 24):
    """Deepest level of the leaves inside block (l, i, j) (l itself if it is a leaf, -1 if a
    coarser leaf covers it)."""
    if (l, i, j) in leaves:
        return l
    for k in range(1, l + 1):  # covered by a coarser leaf
        if (l - k, i >> k, j >> k) in leaves:
            return -1
    best = -1
    stack = [(l, i, j)]
    while stack:
        a, b, c = stack.pop()
        if (a, b, c) in leaves:
            best = max(best, a)
        elif a < limit:
            stack.extend([(a + 1, 2 * b + x, 2 * c + y) for y in (0, 1) for x in (0, 1)])
    return best


def block_cells(level, ix, iy, cells: int = 8):
    """Cell centres and sides of the leaf blocks, cells x cells cells per block (row-major
    within a block, blocks in the given order): (x, y, h) arrays."""
    xs, ys, hs = [], [], []
    c = (np.arange(cells) + 0.5) / cells
    for l, i, j in zip(level, ix, iy):
        s = 1.0 / (1 << int(l))
        X, Y = np.meshgrid((i + c) * s, (j + c) * s)
        xs.append(X.ravel())
        ys.append(Y.ravel())
        hs.append(np.full(cells * cells, s / cells))
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(hs)
