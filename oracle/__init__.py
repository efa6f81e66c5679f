"""CPU oracle for the pressure / surface-force path — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (the CUDA library and its Python
binding) never calls it, and this package imports nothing from the product.

Everything here is plain FP64 (numpy, plus one small C file for the direct
Green's sum), written from the paper's equations:

* ``rhs``            — source of the pressure-Poisson equation, Eq. PoissonFinal
                       (Sec. 2.2), with second-order central differences.
* ``green_sum``      — the discrete free-space Green's sum, Eq. greenSum / green2D
                       (Appendix A.1), evaluated directly, O(sources x targets);
                       ``green_sum_var`` the same over cells of different sizes (the
                       paper's multiresolution grids), each source clamped at its own rho_h.
* ``traction``       — pointwise surface tractions and their closed-surface
                       integrals, Eqs. Fpress, FpressNet, CdP, Fvisc, FviscNet (Sec. 2.3).
* ``p2m``/``m2p``/``m2m`` — the multipole expansion of Appendix A.2
                       (Eqs. pressTruncated, alphaK, expandedShift, expandedBeta).
* ``penal_force``    — the penalisation force, the volume integral of the Brinkman term,
                       Eq. dragPenal (Sec. 3.1), and its drag/lift components.
* ``body_moments``, ``acceleration_sf``, ``acceleration_penal`` — the deforming body's
                       acceleration from the surface forces and from its centre-of-mass
                       velocity, Eqs. aSF and aPenal (Sec. 3.3).
* ``m2l``/``l2l``/``l2p`` — local expansions of the same log series (the paper only
                       cites Greengard & Rokhlin for the O(N) method; these are the
                       standard shifts of that series, written out in the same notation).

Readings of the paper that this oracle takes (stated once here, repeated at
each function):

* c1  Eq. pressTruncated drops the 1/(2 pi) on the series term that Eq. expanded1
      carries; the potential is P = (1/2pi) [S log|w| - Re sum_k alpha_k w^-k].
* c2  Eq. expandedBeta prints  -S z0^k / k ; in the paper's own convention the shift
      is exact only with  +S z0^k / k  (pinned by M2M(P2M(children)) == P2M(parent)).
* c4  the self term: |x - x'| is clamped below at rho_h = h exp(c0), c0 = pi/4 - 3/2
      - log(2)/2, the exact mean of log r over a square cell of side h; on a grid of
      mixed cell sizes each source cell uses its own h (reading c24).
* c6  derivatives: central differences inside, one-sided second order on the edge
      rows and columns; the penalty divergence differences the product chi (u_s - u).
* c11 "nearest-neighbour interpolation" of grad u on the lifted surface: the
      gradient at the cell containing the lifted point (floor), clamped to
      [1, N-2]; bilinear interpolation of the cell-centred gradient as an option.
* c12 tractions are integrated on the original surface with its normals and dS.
* c13 dS defaults to trapezoid weights on the closed, ordered polygon.
* c14 lift = F . (z x U_hat) = F . (-U_y, U_x)/|U|.
* c15 mu = rho nu.
* c22 Eq. dragPenal integrates lambda chi u for a static body (u_s = 0); for a moving
      body the integrand is the penalisation term itself, lambda chi (u - u_s), which
      reduces to the printed form when u_s = 0.  On the uniform grid dV = h^2.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "C0",
    "rho_h",
    "rhs",
    "source_weights",
    "green_sum",
    "green_sum_grid",
    "green_sum_var",
    "default_dS",
    "traction",
    "p2m",
    "m2p",
    "m2m",
    "m2l",
    "l2l",
    "l2p",
    "max_threads",
]

#: c0 = pi/4 - 3/2 - log(2)/2: mean of log r over the unit square centred on 0.
C0 = math.pi / 4.0 - 1.5 - 0.5 * math.log(2.0)

_HERE = os.path.dirname(os.path.abspath(__file__))
_LOCK = threading.Lock()
_LIB = None


def rho_h(h: float) -> float:
    """Clamp radius of the discrete Green's function (reading c4)."""
    return h * math.exp(C0)


def _lib():
    """Load (building with gcc if needed) the C part of the oracle."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        src = os.path.join(_HERE, "green_sum.c")
        so = os.path.join(_HERE, "_green_sum.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            build()
        lib = ctypes.CDLL(so)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_green_sum.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int64, dp, dp,
                                         ctypes.c_double, ctypes.c_int, dp]
        lib.oracle_green_sum.restype = None
        lib.oracle_green_sum_var.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int64, dp, dp,
                                             ctypes.c_int, dp]
        lib.oracle_green_sum_var.restype = None
        lib.oracle_max_threads.argtypes = [ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _LIB = lib
        return lib


def build() -> str:
    """Compile ``green_sum.c`` into ``_green_sum.so`` with gcc + OpenMP."""
    src = os.path.join(_HERE, "green_sum.c")
    so = os.path.join(_HERE, "_green_sum.so")
    tmp = so + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, so)
    return so


def max_threads(nthreads: int = 0) -> int:
    """Threads the oracle's OpenMP loop uses (``nthreads`` <= 0: the default)."""
    return int(_lib().oracle_max_threads(int(nthreads)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------- RHS
def _d_dx(g: np.ndarray, h: float) -> np.ndarray:
    """d/dx along axis 1 (i): central inside, one-sided 2nd order at i = 0, N-1 (c6)."""
    out = np.empty_like(g)
    out[:, 1:-1] = (g[:, 2:] - g[:, :-2]) / (2.0 * h)
    out[:, 0] = (-3.0 * g[:, 0] + 4.0 * g[:, 1] - g[:, 2]) / (2.0 * h)
    out[:, -1] = (3.0 * g[:, -1] - 4.0 * g[:, -2] + g[:, -3]) / (2.0 * h)
    return out


def _d_dy(g: np.ndarray, h: float) -> np.ndarray:
    """d/dy along axis 0 (j), same stencils as ``_d_dx``."""
    return _d_dx(g.T, h).T


def rhs(u, v, chi, usx, usy, h: float, rho: float = 1.0, lam: float = 0.0) -> np.ndarray:
    """Source f of the pressure-Poisson equation, Eq. PoissonFinal (Sec. 2.2):

        lap P = -rho (grad u^T : grad u) + rho lambda div(chi (u_s - u)),

    with grad u^T : grad u = u_{j,i} u_{i,j} = u_x^2 + 2 u_y v_x + v_y^2 (the index form
    the paper gives after Eq. PoissonDerive).  Derivatives per reading c6.
    Fields are row-major [j, i]; returns f with the same layout, FP64.
    """
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    chi = np.asarray(chi, np.float64)
    usx = np.asarray(usx, np.float64)
    usy = np.asarray(usy, np.float64)
    ux, uy = _d_dx(u, h), _d_dy(u, h)
    vx, vy = _d_dx(v, h), _d_dy(v, h)
    colon = ux * ux + 2.0 * uy * vx + vy * vy
    pen = _d_dx(chi * (usx - u), h) + _d_dy(chi * (usy - v), h)
    return -rho * colon + rho * lam * pen


def source_weights(f: np.ndarray, h: float) -> np.ndarray:
    """q = f h^2: the weights of Eq. greenSum on a uniform grid (cell area h^2)."""
    return np.asarray(f, np.float64) * (h * h)


# ------------------------------------------------------------------- Green's sum
def green_sum(xs, ys, q, xt, yt, rho_clamp: float, nthreads: int = 0) -> np.ndarray:
    """Direct FP64 evaluation of Eq. greenSum at arbitrary targets:

        P(x_t) = (1/2pi) sum_s q_s log max(|x_t - x_s|, rho_clamp).
    """
    xs = np.ascontiguousarray(xs, np.float64).ravel()
    ys = np.ascontiguousarray(ys, np.float64).ravel()
    q = np.ascontiguousarray(q, np.float64).ravel()
    xt = np.ascontiguousarray(xt, np.float64).ravel()
    yt = np.ascontiguousarray(yt, np.float64).ravel()
    P = np.empty(xt.shape[0], np.float64)
    _lib().oracle_green_sum(xs.shape[0], _ptr(xs), _ptr(ys), _ptr(q), xt.shape[0], _ptr(xt),
                            _ptr(yt), float(rho_clamp), int(nthreads), _ptr(P))
    return P


def green_sum_grid(q_grid, h: float, xt, yt, x0: float = 0.0, y0: float = 0.0,
                   nthreads: int = 0) -> np.ndarray:
    """Eq. greenSum with all cells of an n x n cell-centred grid as sources
    (x_i = x0 + (i + 1/2) h, weights q[j, i] already multiplied by h^2)."""
    n = q_grid.shape[0]
    c = (np.arange(n, dtype=np.float64) + 0.5) * h
    X, Y = np.meshgrid(x0 + c, y0 + c)
    return green_sum(X, Y, q_grid, xt, yt, rho_h(h), nthreads)


def green_sum_var(xs, ys, q, hs, xt, yt, nthreads: int = 0) -> np.ndarray:
    """Eq. greenSum over sources of different cell sizes hs (a multiresolution grid; weights
    q already multiplied by each cell's area): every source clamped at its own rho_h(h_s),
    the extension of reading c4 that keeps each cell's self term its own mean of log r.

        P(x_t) = (1/2pi) sum_s q_s log max(|x_t - x_s|, rho_h(h_s)).
    """
    xs, ys, q, hs, xt, yt = (np.ascontiguousarray(a, np.float64).ravel() for a in (xs, ys, q, hs, xt, yt))
    rho = hs * math.exp(C0)
    P = np.empty(xt.shape[0], np.float64)
    _lib().oracle_green_sum_var(xs.shape[0], _ptr(xs), _ptr(ys), _ptr(q), _ptr(rho), xt.shape[0], _ptr(xt),
                                _ptr(yt), int(nthreads), _ptr(P))
    return P


# ---------------------------------------------------------------------- traction
def default_dS(points) -> np.ndarray:
    """Trapezoid weights on a closed ordered polygon (reading c13):
    dS_i = (|x_{i+1} - x_i| + |x_i - x_{i-1}|) / 2, indices cyclic."""
    p = np.asarray(points, np.float64)
    seg = np.linalg.norm(np.roll(p, -1, axis=0) - p, axis=1)
    return 0.5 * (seg + np.roll(seg, 1))


def _cell_gradient(u, v, h, i, j):
    """Central-difference grad u at cells (i, j) (interior cells only)."""
    ux = (u[j, i + 1] - u[j, i - 1]) / (2.0 * h)
    uy = (u[j + 1, i] - u[j - 1, i]) / (2.0 * h)
    vx = (v[j, i + 1] - v[j, i - 1]) / (2.0 * h)
    vy = (v[j + 1, i] - v[j - 1, i]) / (2.0 * h)
    return ux, uy, vx, vy


def traction(u, v, h: float, points, normals, P_points, nu: float, rho: float = 1.0,
             lift: float = None, dS=None, uinf=(1.0, 0.0), x0: float = 0.0, y0: float = 0.0,
             interp: str = "nearest"):
    """Pointwise tractions and integrated forces on a closed surface (Sec. 2.3).

    * Pressure part, Eq. Fpress:  t_P = -P n, with P at the original surface point.
    * Viscous part, Eq. Fvisc:    t_nu = 2 mu D . n, D = (grad u + grad u^T)/2, mu = rho nu (c15),
      grad u taken on the lifted point y = x + lift n (Sec. 2.3.2; lift = 2h default
      for rigid bodies, 0 for deforming ones), at the nearest cell (c11).
    * Eqs. FpressNet / FviscNet: F = sum (t_P + t_nu) dS on the original surface (c12, c13).
    * Eq. CdP: drag = F . U/|U|;  lift force = F . (-U_y, U_x)/|U| (c14).

    Returns (per_point[n, 5] = P, tPx, tPy, tnux, tnuy;  forces[6] = FPx, FPy, Fnux, Fnuy,
    drag, lift) in FP64.
    """
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    n = u.shape[0]
    pts = np.asarray(points, np.float64)
    nrm = np.asarray(normals, np.float64)
    P = np.asarray(P_points, np.float64)
    if lift is None:
        lift = 2.0 * h
    if dS is None:
        dS = default_dS(pts)
    dS = np.asarray(dS, np.float64)
    y = pts + lift * nrm
    if interp == "nearest":
        i = np.clip(np.floor((y[:, 0] - x0) / h).astype(np.int64), 1, n - 2)
        j = np.clip(np.floor((y[:, 1] - y0) / h).astype(np.int64), 1, n - 2)
        ux, uy, vx, vy = _cell_gradient(u, v, h, i, j)
    elif interp == "bilinear":
        # bilinear weights between the four surrounding cell centres
        fx = (y[:, 0] - x0) / h - 0.5
        fy = (y[:, 1] - y0) / h - 0.5
        i0 = np.clip(np.floor(fx).astype(np.int64), 1, n - 3)
        j0 = np.clip(np.floor(fy).astype(np.int64), 1, n - 3)
        ax = np.clip(fx - i0, 0.0, 1.0)
        ay = np.clip(fy - j0, 0.0, 1.0)
        g = [np.zeros(len(pts)) for _ in range(4)]
        for di, dj, wgt in ((0, 0, (1 - ax) * (1 - ay)), (1, 0, ax * (1 - ay)),
                            (0, 1, (1 - ax) * ay), (1, 1, ax * ay)):
            comp = _cell_gradient(u, v, h, i0 + di, j0 + dj)
            for c in range(4):
                g[c] += wgt * comp[c]
        ux, uy, vx, vy = g
    else:
        raise ValueError(f"unknown interpolation {interp!r}")
    mu = rho * nu
    dxy = 0.5 * (uy + vx)
    tnx = 2.0 * mu * (ux * nrm[:, 0] + dxy * nrm[:, 1])
    tny = 2.0 * mu * (dxy * nrm[:, 0] + vy * nrm[:, 1])
    tPx = -P * nrm[:, 0]
    tPy = -P * nrm[:, 1]
    per = np.stack([P, tPx, tPy, tnx, tny], axis=1)
    FP = np.array([np.sum(tPx * dS), np.sum(tPy * dS)])
    Fn = np.array([np.sum(tnx * dS), np.sum(tny * dS)])
    U = np.asarray(uinf, np.float64)
    Uh = U / np.linalg.norm(U)
    F = FP + Fn
    drag = F @ Uh
    liftf = F @ np.array([-Uh[1], Uh[0]])
    return per, np.array([FP[0], FP[1], Fn[0], Fn[1], drag, liftf])


# -------------------------------------------------------------- expansions (A.2)
def _binom(n: int, k: int) -> float:
    return float(math.comb(n, k)) if 0 <= k <= n else 0.0


def p2m(q, z_src, z_c, p: int):
    """Multipole coefficients about z_c, Eq. alphaK with z' replaced by z' - z_c:
    S = sum q,  alpha_k = sum q (z' - z_c)^k / k,  k = 1..p."""
    q = np.asarray(q, np.float64).ravel()
    w = np.asarray(z_src, np.complex128).ravel() - z_c
    S = float(q.sum())
    alpha = np.array([np.sum(q * w ** k) / k for k in range(1, p + 1)], np.complex128)
    return S, alpha


def m2p(S: float, alpha, z_c, z):
    """Eq. pressTruncated about z_c (group form of Sec. A.2, reading c1):
    P(z) = (1/2pi) [S log|z - z_c| - Re sum_k alpha_k (z - z_c)^-k]."""
    w = np.asarray(z, np.complex128) - z_c
    ser = np.zeros_like(w)
    for k, a in enumerate(alpha, start=1):
        ser = ser + a / w ** k
    return (S * np.log(np.abs(w)) - ser.real) / (2.0 * math.pi)


def m2m(S: float, alpha, z_c, z_p):
    """Shift a child expansion about z_c to the parent centre z_p, Eq. expandedBeta
    with the sign of the S term read as + (reading c2):
    beta_k = S z0^k / k + sum_{l=1..k} alpha_l z0^(k-l) C(k-1, l-1),  z0 = z_c - z_p."""
    p = len(alpha)
    z0 = complex(z_c - z_p)
    beta = np.zeros(p, np.complex128)
    for k in range(1, p + 1):
        acc = S * z0 ** k / k
        for l in range(1, k + 1):
            acc += alpha[l - 1] * z0 ** (k - l) * _binom(k - 1, l - 1)
        beta[k - 1] = acc
    return S, beta


def m2l(S: float, alpha, z_c, z_L):
    """Local (Taylor) coefficients b_0..b_p about z_L of the group potential
    2 pi P = S log|z - z_c| - Re sum alpha_k (z - z_c)^-k, for |z - z_L| small.

    With a_0 = S, a_k = -alpha_k and t = z_c - z_L (Greengard & Rokhlin's shift of the
    series of Eq. logExpansion; real part taken at evaluation, so log|t| is used):
      b_0 = a_0 log|t| + sum_k a_k (-1)^k t^-k
      b_l = -a_0 / (l t^l) + t^-l sum_k a_k (-1)^k t^-k C(l+k-1, k-1)
    Returns b (p+1 complex) with 2 pi P(z) ~ Re sum_l b_l (z - z_L)^l.
    """
    p = len(alpha)
    t = complex(z_c - z_L)
    a = np.concatenate([[S], -np.asarray(alpha, np.complex128)])
    b = np.zeros(p + 1, np.complex128)
    b[0] = a[0] * math.log(abs(t)) + sum(a[k] * (-1) ** k / t ** k for k in range(1, p + 1))
    for l in range(1, p + 1):
        acc = -a[0] / (l * t ** l)
        for k in range(1, p + 1):
            acc += a[k] * (-1) ** k / t ** (k + l) * _binom(l + k - 1, k - 1)
        b[l] = acc
    return b


def l2l(b, z_L, z_new):
    """Re-centre a local expansion: c_l = sum_{k>=l} b_k C(k, l) (z_new - z_L)^(k-l)."""
    p = len(b) - 1
    d = complex(z_new - z_L)
    c = np.zeros(p + 1, np.complex128)
    for l in range(p + 1):
        c[l] = sum(b[k] * _binom(k, l) * d ** (k - l) for k in range(l, p + 1))
    return c


def l2p(b, z_L, z):
    """Evaluate a local expansion: P(z) = (1/2pi) Re sum_l b_l (z - z_L)^l."""
    w = np.asarray(z, np.complex128) - z_L
    acc = np.zeros_like(w)
    for l, bl in enumerate(b):
        acc = acc + bl * w ** l
    return acc.real / (2.0 * math.pi)


# ----------------------------------------------------------------------------------
# Penalisation force, Eq. dragPenal (Sec. 3.1), reading c22
# ----------------------------------------------------------------------------------
def penal_force(u, v, chi, usx, usy, h: float, lam: float, uinf=(1.0, 0.0)) -> np.ndarray:
    """F_penal = sum over cells of lambda chi (u - u_s) h^2 (Eq. dragPenal with dV = h^2 and
    the moving-body integrand of reading c22), summed in FP64.  Returns
    [Fx, Fy, drag, lift] with drag = F . U_hat and lift = F . (-U_hat_y, U_hat_x) (c14)."""
    c = np.asarray(chi, np.float64)
    fx = float(np.sum(c * (np.asarray(u, np.float64) - np.asarray(usx, np.float64)))) * lam * h * h
    fy = float(np.sum(c * (np.asarray(v, np.float64) - np.asarray(usy, np.float64)))) * lam * h * h
    U = np.asarray(uinf, np.float64)
    Uh = U / np.linalg.norm(U)
    F = np.array([fx, fy])
    return np.array([fx, fy, F @ Uh, F @ np.array([-Uh[1], Uh[0]])])


# ----------------------------------------------------------------------------------
# Acceleration of a deforming body, Eqs. aPenal and aSF (Sec. 3.3), reading c25
# ----------------------------------------------------------------------------------
def body_moments(u, v, chi, h: float, rho: float = 1.0) -> np.ndarray:
    """Mass and centre-of-mass velocity of the body marked by chi (reading c25: the body's
    density is the fluid's, its volume the sum of chi h^2): M = rho sum chi h^2,
    u_CM = sum chi u h^2 / sum chi h^2 (the same for v), summed in FP64.
    Returns [M, u_CM_x, u_CM_y]."""
    c = np.asarray(chi, np.float64)
    vol = float(np.sum(c)) * h * h
    ux = float(np.sum(c * np.asarray(u, np.float64))) * h * h / vol
    uy = float(np.sum(c * np.asarray(v, np.float64))) * h * h / vol
    return np.array([rho * vol, ux, uy])


def acceleration_sf(forces, mass: float) -> np.ndarray:
    """Eq. aSF: a_SF = (F_P + F_nu) / M, with forces = [FPx, FPy, Fnux, Fnuy, ...]."""
    F = np.asarray(forces, np.float64)
    return np.array([F[0] + F[2], F[1] + F[3]]) / mass


def acceleration_penal(u_cm_prev, u_cm_next, dt: float) -> np.ndarray:
    """Eq. aPenal: the second-order centred difference of the centre-of-mass velocity,
    a^n = (u_CM^(n+1) - u_CM^(n-1)) / (2 dt)."""
    return (np.asarray(u_cm_next, np.float64) - np.asarray(u_cm_prev, np.float64)) / (2.0 * dt)
