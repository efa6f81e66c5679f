"""Pins of the CPU oracle against facts it does not compute itself.

Each test ties one oracle function to something fixed by the paper or by the
mathematics: closed-form flows, exact behaviour of the stencils on polynomials,
invariants of the expansions, and brute force at high precision on tiny inputs.
Together they are chosen so that a dropped term, a wrong sign, a wrong factor
(1/2pi, 2mu, h^2) or a transposed index in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special
import sympy as sp

import oracle
from paper_1610_04398_gb300 import synth


# --------------------------------------------------------------- self term (c4)
def test_c0_is_mean_of_log_r_over_a_unit_cell():
    """rho_h = h exp(c0) makes log(rho_h) the exact cell mean of log r (reading c4)."""
    val, err = scipy.integrate.dblquad(lambda y, x: 0.5 * math.log(x * x + y * y),
                                       0.0, 0.5, 0.0, 0.5, epsabs=1e-13, epsrel=1e-13)
    mean = val / 0.25  # symmetric quarter of [-1/2, 1/2]^2
    assert abs(mean - oracle.C0) < 1e-9
    h = 0.37
    assert abs(math.log(oracle.rho_h(h)) - (math.log(h) + mean)) < 1e-9


# --------------------------------------------------------- Green's sum (greenSum)
def test_green_sum_matches_high_precision_brute_force():
    """Tiny grid, random weights, targets on and off the grid (mpmath, 40 digits)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(7)
    n, h = 5, 0.2
    q = rng.normal(size=(n, n))
    xt = np.array([0.1, 0.3, 0.55, 0.9001, 0.25])
    yt = np.array([0.1, 0.5, 0.42, 0.11, 0.7])
    got = oracle.green_sum_grid(q, h, xt, yt)
    rh = mpmath.mpf(h) * mpmath.e ** (mpmath.pi / 4 - mpmath.mpf(3) / 2 - mpmath.log(2) / 2)
    for t in range(len(xt)):
        acc = mpmath.mpf(0)
        for j in range(n):
            for i in range(n):
                dx = mpmath.mpf(xt[t]) - (i + mpmath.mpf(1) / 2) * mpmath.mpf(h)
                dy = mpmath.mpf(yt[t]) - (j + mpmath.mpf(1) / 2) * mpmath.mpf(h)
                r = mpmath.sqrt(dx * dx + dy * dy)
                acc += mpmath.mpf(q[j, i]) * mpmath.log(max(r, rh))
        ref = float(acc / (2 * mpmath.pi))
        assert abs(got[t] - ref) < 1e-13 * max(1.0, abs(ref))


def test_green_sum_on_the_grid_equals_zero_padded_fft_convolution():
    """At the cell centres the sum of Eq. greenSum is a linear convolution of the weights with
    the table (1/2pi) log max(h |(dx, dy)|, rho_h), |dx|, |dy| < n: the zero-padded FFT
    convolution of Hockney (the Fourier-based solver Appendix A.1 names), here scipy's."""
    import scipy.signal
    rng = np.random.default_rng(11)
    for n, h in ((24, 1.0 / 24), (17, 0.03)):
        q = rng.normal(size=(n, n))
        X, Y = synth.cell_centres(n, h)
        got = oracle.green_sum_grid(q, h, X.ravel(), Y.ravel()).reshape(n, n)
        d = np.arange(-(n - 1), n)
        DX, DY = np.meshgrid(d, d)
        K = np.log(np.maximum(h * np.hypot(DX, DY), oracle.rho_h(h))) / (2 * math.pi)
        ref = scipy.signal.fftconvolve(q, K, mode="full")[n - 1:2 * n - 1, n - 1:2 * n - 1]
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
        # the orientation matters: the transposed weights give another field
        assert np.max(np.abs(got - ref.T)) > 1e-3 * np.max(np.abs(ref))


def _mixed_cells():
    """Two level-1 blocks of 2 x 2 cells and four level-2 blocks of 2 x 2 cells (cells of side
    1/4 and 1/8) tiling the unit square: (x, y, h) of every cell centre."""
    from paper_1610_04398_gb300 import synth
    lv = np.array([1, 1, 1, 2, 2, 2, 2])
    ix = np.array([1, 0, 1, 0, 1, 0, 1])
    iy = np.array([0, 1, 1, 0, 0, 1, 1])
    return synth.block_cells(lv, ix, iy, cells=2)


def test_green_sum_var_matches_high_precision_brute_force():
    """Cells of two sizes, targets at cell centres (own-cell clamp active) and off-grid
    (mpmath, 40 digits)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    xs, ys, hs = _mixed_cells()
    assert np.isclose(np.sum(hs ** 2), 1.0)
    rng = np.random.default_rng(5)
    q = rng.normal(size=xs.size) * hs ** 2
    xt = np.concatenate([xs[[0, 5, 9, 17]], [0.123, 0.61]])
    yt = np.concatenate([ys[[0, 5, 9, 17]], [0.377, 0.05]])
    got = oracle.green_sum_var(xs, ys, q, hs, xt, yt)
    c0 = mpmath.pi / 4 - mpmath.mpf(3) / 2 - mpmath.log(2) / 2
    for t in range(len(xt)):
        acc = mpmath.mpf(0)
        for s in range(xs.size):
            r = mpmath.sqrt((mpmath.mpf(xt[t]) - mpmath.mpf(xs[s])) ** 2 + (mpmath.mpf(yt[t]) - mpmath.mpf(ys[s])) ** 2)
            acc += mpmath.mpf(q[s]) * mpmath.log(max(r, mpmath.mpf(hs[s]) * mpmath.e ** c0))
        ref = float(acc / (2 * mpmath.pi))
        assert abs(got[t] - ref) < 1e-14 * max(1.0, abs(ref))


def test_green_sum_var_with_one_cell_size_is_the_grid_sum():
    n, h = 16, 1.0 / 16
    rng = np.random.default_rng(6)
    q = rng.normal(size=(n, n)) * h * h
    X, Y = synth.cell_centres(n, h)
    xt, yt = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50)
    a = oracle.green_sum_grid(q, h, np.concatenate([X.ravel(), xt]), np.concatenate([Y.ravel(), yt]))
    b = oracle.green_sum_var(X, Y, q, np.full(n * n, h), np.concatenate([X.ravel(), xt]),
                             np.concatenate([Y.ravel(), yt]))
    assert np.max(np.abs(a - b)) <= 1e-15 * np.max(np.abs(a))


def test_green_sum_var_refined_block_matches_coarse_block_far_away():
    """A block of side s as one cell of weight Q, or refined into 4^k cells of weight Q/4^k:
    the monopole agrees and the dipole and quadrupole moments of the refined square vanish by
    symmetry, so far away the two potentials differ by less than ~ Q s^2 / d^2 and fall off at
    least as fast as d^-2 (a misplaced refined cell would leave a dipole error ~ Q s / d)."""
    s, Q = 0.1, 1.0
    d = np.array([1.0, 2.0, 4.0, 8.0])
    xt, yt = 0.05 + d * 0.6, 0.05 + d * 0.8
    coarse = oracle.green_sum_var([0.05], [0.05], [Q], [s], xt, yt)
    for k in (1, 2, 3):
        m = 1 << k
        c = (np.arange(m) + 0.5) * s / m
        X, Y = np.meshgrid(c, c)
        fine = oracle.green_sum_var(X, Y, np.full(m * m, Q / (m * m)), np.full(m * m, s / m), xt, yt)
        diff = np.abs(fine - coarse)
        assert np.all(diff < 0.05 * Q * s ** 2 / d ** 2)
        assert diff[-1] < diff[0] / 30  # second-order decay: (8/1)^2 = 64


def _gaussian_error(n, S=0.7, sigma=0.05):
    h = 1.0 / n
    X, Y = synth.cell_centres(n, h)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2
    q = S / (math.pi * sigma ** 2) * np.exp(-r2 / sigma ** 2) * h * h
    rng = np.random.default_rng(3)
    xt = 0.5 + rng.uniform(-0.3, 0.3, 300)
    yt = 0.5 + rng.uniform(-0.3, 0.3, 300)
    P = oracle.green_sum(X, Y, q, xt, yt, oracle.rho_h(h))
    r = np.hypot(xt - 0.5, yt - 0.5)
    exact = S / (2 * math.pi) * (np.log(r) + 0.5 * scipy.special.exp1(r * r / sigma ** 2))
    return np.max(np.abs(P - exact)) / np.max(np.abs(exact))


def test_green_sum_gaussian_source_closed_form_second_order():
    """Gaussian source of total S: P = (S/2pi)[log r + E1(r^2/sigma^2)/2] (no gauge);
    the midpoint-rule sum converges at second order in h."""
    e64 = _gaussian_error(64)
    e128 = _gaussian_error(128)
    assert e128 < 2e-3
    assert 3.0 < e64 / e128 < 5.5


# ------------------------------------------------------------- RHS (PoissonFinal)
def _poly_fields(n, h):
    x, y = sp.symbols("x y")
    u = 0.3 + 1.1 * x - 0.7 * y + 0.9 * x * x - 1.3 * x * y + 0.4 * y * y
    v = -0.2 + 0.5 * x + 0.8 * y - 0.6 * x * x + 0.35 * x * y - 1.2 * y * y
    chi = 0.25 + 0.5 * x - 0.3 * y
    usx = 0.1 - 0.4 * x + 0.2 * y + u  # so that usx - u is linear
    usy = -0.3 + 0.6 * x - 0.1 * y + v
    X, Y = synth.cell_centres(n, h)
    ev = lambda e: np.asarray(sp.lambdify((x, y), e, "numpy")(X, Y), np.float64) * np.ones_like(X)
    return (x, y), (u, v, chi, usx, usy), [ev(e) for e in (u, v, chi, usx, usy)]


def test_rhs_exact_on_quadratic_fields():
    """Second-order differences are exact on quadratics, edges included, so the
    discrete source must equal the symbolic one: -rho tr(J J) + rho lam div(chi(u_s-u)),
    J the velocity Jacobian (tr(J J) = u_{j,i} u_{i,j}, the colon product)."""
    n, h, rho, lam = 12, 0.1, 1.3, 7.0
    (x, y), (u, v, chi, usx, usy), arrs = _poly_fields(n, h)
    J = sp.Matrix([[sp.diff(u, x), sp.diff(u, y)], [sp.diff(v, x), sp.diff(v, y)]])
    colon = (J * J).trace()
    div = sp.diff(chi * (usx - u), x) + sp.diff(chi * (usy - v), y)
    fsym = -rho * colon + rho * lam * div
    X, Y = synth.cell_centres(n, h)
    want = sp.lambdify((x, y), fsym, "numpy")(X, Y) * np.ones_like(X)
    got = oracle.rhs(*arrs, h=h, rho=rho, lam=lam)
    assert np.max(np.abs(got - want)) < 1e-10 * np.max(np.abs(want))


def test_rhs_matches_laplacian_of_bernoulli_pressure():
    """Steady potential flow W = z^2 (u = x^2 - y^2, v = -2xy): Bernoulli gives
    P = -rho |u|^2 / 2 + const, so the source must be lap P = -8 rho (x^2 + y^2)."""
    n, h, rho = 16, 1.0 / 16, 0.8
    X, Y = synth.cell_centres(n, h)
    u = X * X - Y * Y
    v = -2 * X * Y
    z = np.zeros_like(X)
    x, y = sp.symbols("x y")
    Pb = -rho * ((x * x - y * y) ** 2 + (2 * x * y) ** 2) / 2
    lap = sp.lambdify((x, y), sp.diff(Pb, x, 2) + sp.diff(Pb, y, 2), "numpy")(X, Y)
    got = oracle.rhs(u, v, z, z, z, h=h, rho=rho, lam=5.0)
    assert np.allclose(got, lap, rtol=1e-12, atol=1e-12)


def test_rhs_penalty_sign_from_hydrostatic_balance():
    """Fluid at rest inside a body moving with chi u_s = (x, y): Eq. penalNS gives
    grad P = rho lam chi u_s, so P = rho lam (x^2+y^2)/2 and lap P = +2 rho lam."""
    n, h, rho, lam = 10, 0.1, 1.7, 300.0
    X, Y = synth.cell_centres(n, h)
    z = np.zeros_like(X)
    got = oracle.rhs(z, z, np.ones_like(X), X, Y, h=h, rho=rho, lam=lam)
    assert np.allclose(got, 2 * rho * lam, rtol=1e-12)


# --------------------------------------------------- Lamb-Oseen chain (RHS + sum)
def lamb_oseen_pressure(r, gamma=1.0, sigma=0.05, rho=1.0):
    """Closed-form Lamb-Oseen pressure (P -> 0 at infinity), x = r^2/sigma^2:
    P = -rho G^2/(8 pi^2 sigma^2) [(1-e^-x)^2/x + 2 E1(x) - 2 E1(2x)]."""
    x = np.maximum(np.asarray(r, np.float64) ** 2 / sigma ** 2, 1e-300)
    br = (-np.expm1(-x)) ** 2 / x + 2 * scipy.special.exp1(x) - 2 * scipy.special.exp1(2 * x)
    return -rho * gamma ** 2 / (8 * math.pi ** 2 * sigma ** 2) * br


def test_lamb_oseen_closed_form_satisfies_radial_balance():
    """The closed form used as a pin obeys dP/dr = rho u_theta^2 / r and P(0) = -rho G^2 ln2/(4 pi^2 s^2)."""
    g, s = 1.0, 0.05
    r = np.linspace(0.005, 0.4, 200)
    d = 1e-6
    dP = (lamb_oseen_pressure(r + d) - lamb_oseen_pressure(r - d)) / (2 * d)
    ut = g / (2 * math.pi * r) * (-np.expm1(-(r / s) ** 2))
    assert np.allclose(dP, ut * ut / r, rtol=1e-6)
    assert abs(lamb_oseen_pressure(1e-9) + g * g * math.log(2) / (4 * math.pi ** 2 * s * s)) < 1e-6


def _lamb_oseen_error(n):
    snap = synth.lamb_oseen(n)
    h = snap.h
    f = oracle.rhs(snap.u, snap.v, snap.chi, snap.usx, snap.usy, h=h)
    q = oracle.source_weights(f, h)
    X, Y = synth.cell_centres(n, h)
    r = np.hypot(X - 0.5, Y - 0.5)
    sel = r < 0.3
    xt = np.concatenate([X[sel], snap.points[:, 0]])
    yt = np.concatenate([Y[sel], snap.points[:, 1]])
    P = oracle.green_sum_grid(q, h, xt, yt)
    ex = lamb_oseen_pressure(np.hypot(xt - 0.5, yt - 0.5))
    # gauge (reading c7): the truncated domain adds a near-constant harmonic field
    dP = (P - P.mean()) - (ex - ex.mean())
    return np.sqrt(np.mean(dP ** 2)) / np.sqrt(np.mean((ex - ex.mean()) ** 2))


def test_lamb_oseen_chain_second_order():
    """RHS + Green's sum reproduce the Lamb-Oseen pressure, converging at O(h^2)."""
    e64 = _lamb_oseen_error(64)
    e128 = _lamb_oseen_error(128)
    assert e128 < 1.5e-2  # 1.0e-2 measured at 128^2, 3.9x smaller than at 64^2
    assert 3.0 < e64 / e128 < 5.5


# ------------------------------------------------------------ traction (Sec. 2.3)
def _potential_cylinder(n, U=1.0, R=0.05, gam=0.0, centre=(0.5, 0.5)):
    h = 1.0 / n
    X, Y = synth.cell_centres(n, h)
    zc = (X - centre[0]) + 1j * (Y - centre[1])
    zc = np.where(np.abs(zc) < 0.5 * R, 0.5 * R, zc)
    W = U * (1 - R * R / zc ** 2) - 1j * gam / (2 * math.pi * zc)
    return h, W.real, -W.imag


def test_traction_circulating_cylinder_kutta_joukowski():
    """Potential flow U past a cylinder with circulation G: Bernoulli surface pressure
    gives F_P = (0, -rho U G) (Kutta-Joukowski), and a constant P integrates to zero."""
    n, U, R, G, rho = 256, 1.0, 0.05, 0.2, 1.3
    h, u, v = _potential_cylinder(n, U, R, G)
    pts, nrm = synth.circle_surface(2048, (0.5, 0.5), R)
    th = np.arctan2(nrm[:, 1], nrm[:, 0])
    ut = -2 * U * np.sin(th) + G / (2 * math.pi * R)
    P = -0.5 * rho * ut ** 2
    per, F = oracle.traction(u, v, h, pts, nrm, P, nu=0.0, rho=rho)
    assert abs(F[0]) < 1e-9
    assert abs(F[1] - (-rho * U * G)) < 1e-6 * rho * U * G
    assert abs(F[5] - (-rho * U * G)) < 1e-6 * rho * U * G  # lift = F . (z x U_hat)
    assert abs(F[4] - F[0]) < 1e-12                             # drag along U = +x
    np.testing.assert_allclose(per[:, 1:3], -P[:, None] * nrm, rtol=0, atol=1e-14)
    _, F0 = oracle.traction(u, v, h, pts, nrm, np.full(len(pts), 3.7), nu=0.0, rho=rho)
    assert abs(F0[0]) < 1e-10 and abs(F0[1]) < 1e-10
    assert np.allclose((oracle.default_dS(pts)[:, None] * nrm).sum(0), 0.0, atol=1e-14)


def test_traction_viscous_part_matches_analytic_strain_at_nearest_cell():
    """t_nu = 2 rho nu D.n with D from the analytic velocity gradient at the centre of
    the cell containing the lifted point (x + 2h n): pins the lift, the cell choice,
    the symmetric part and the factor 2 mu (O(h^2) central-difference error only)."""
    n, U, R, G, rho, nu = 512, 1.0, 0.05, 0.15, 1.1, 2e-3
    h, u, v = _potential_cylinder(n, U, R, G)
    pts, nrm = synth.circle_surface(333, (0.5, 0.5), R)
    per, F = oracle.traction(u, v, h, pts, nrm, np.zeros(len(pts)), nu=nu, rho=rho)
    x, y = sp.symbols("x y", real=True)
    z = (x - 0.5) + sp.I * (y - 0.5)
    W = U * (1 - R * R / z ** 2) - sp.I * G / (2 * sp.pi * z)
    us, vs = sp.re(sp.expand_complex(W)), -sp.im(sp.expand_complex(W))
    grads = [sp.lambdify((x, y), sp.diff(a, b), "numpy") for a in (us, vs) for b in (x, y)]
    fu, fv = sp.lambdify((x, y), us, "numpy"), sp.lambdify((x, y), vs, "numpy")
    yl = pts + 2 * h * nrm
    ci = np.floor(yl[:, 0] / h).astype(int)
    cj = np.floor(yl[:, 1] / h).astype(int)
    xc, yc = (ci + 0.5) * h, (cj + 0.5) * h
    mu = rho * nu

    def t_nu(ux, uy, vx, vy):
        return (2 * mu * (ux * nrm[:, 0] + 0.5 * (uy + vx) * nrm[:, 1]),
                2 * mu * (0.5 * (uy + vx) * nrm[:, 0] + vy * nrm[:, 1]))

    # exact analytic gradient at the chosen cell centre: O(h^2) apart
    tx, ty = t_nu(*[g(xc, yc) for g in grads])
    scale = np.max(np.hypot(tx, ty))
    assert np.max(np.abs(per[:, 3] - tx)) < 5e-3 * scale
    assert np.max(np.abs(per[:, 4] - ty)) < 5e-3 * scale
    # the same cell's centred differences of the analytic field: equal to rounding
    cd = lambda f, dx, dy: (f(xc + dx, yc + dy) - f(xc - dx, yc - dy)) / (2 * h)
    tx2, ty2 = t_nu(cd(fu, h, 0), cd(fu, 0, h), cd(fv, h, 0), cd(fv, 0, h))
    assert np.max(np.abs(per[:, 3] - tx2)) < 1e-9 * scale
    assert np.max(np.abs(per[:, 4] - ty2)) < 1e-9 * scale


def test_traction_bilinear_reduces_to_nearest_on_linear_gradient_field():
    """On a quadratic velocity field grad u is linear, so bilinear interpolation of the
    cell gradients is exact at any point (checks the interpolation weights)."""
    n, h = 32, 1.0 / 32
    X, Y = synth.cell_centres(n, h)
    u = 0.5 * X * X + 0.3 * X * Y
    v = -0.2 * Y * Y + 0.7 * X * Y
    pts = np.array([[0.41, 0.37], [0.5, 0.52], [0.33, 0.61]])
    nrm = np.array([[1.0, 0.0], [0.0, 1.0], [0.6, 0.8]])
    per, _ = oracle.traction(u, v, h, pts, nrm, np.zeros(3), nu=0.5, rho=2.0, lift=0.0,
                             interp="bilinear")
    px, py = pts[:, 0], pts[:, 1]
    ux, uy = px + 0.3 * py, 0.3 * px
    vx, vy = 0.7 * py, -0.4 * py + 0.7 * px
    mu = 1.0
    tx = 2 * mu * (ux * nrm[:, 0] + 0.5 * (uy + vx) * nrm[:, 1])
    ty = 2 * mu * (0.5 * (uy + vx) * nrm[:, 0] + vy * nrm[:, 1])
    assert np.allclose(per[:, 3], tx, atol=1e-12) and np.allclose(per[:, 4], ty, atol=1e-12)


# ------------------------------------------------------------ expansions (A.2)
def _cluster(rng, m, zc, rad):
    z = zc + rad * (rng.uniform(-1, 1, m) + 1j * rng.uniform(-1, 1, m)) / math.sqrt(2)
    return rng.normal(size=m), z


def test_p2m_m2p_far_field_within_truncation_bound():
    """Eq. pressTruncated about the group centre converges like (r/d)^(p+1)."""
    rng = np.random.default_rng(11)
    q, z = _cluster(rng, 40, 0.3 + 0.2j, 0.05)
    zt = np.array([0.3 + 0.2j + 0.2 * np.exp(1j * a) for a in np.linspace(0, 6, 17)])
    direct = oracle.green_sum(z.real, z.imag, q, zt.real, zt.imag, 0.0)
    A = np.abs(q).sum()
    for p in (4, 8, 16, 24):
        S, al = oracle.p2m(q, z, 0.3 + 0.2j, p)
        approx = oracle.m2p(S, al, 0.3 + 0.2j, zt)
        a = 0.05 / 0.2
        bound = A / (2 * math.pi) * a ** (p + 1) / ((p + 1) * (1 - a))
        assert np.max(np.abs(approx - direct)) <= bound * 1.0001 + 1e-15
    # far away the expansion is dominated by (S / 2 pi) log|z|
    far = 1e10 + 0j
    assert abs(oracle.m2p(S, al, 0.3 + 0.2j, np.array([far]))[0]
               - S / (2 * math.pi) * math.log(abs(far - (0.3 + 0.2j)))) < 1e-9


def test_m2m_of_children_equals_p2m_of_parent():
    """Exactness of the shift (reading c2: +S z0^k/k). The printed sign fails this."""
    rng = np.random.default_rng(5)
    p = 20
    zp = 0.5 + 0.5j
    total_S, total = 0.0, np.zeros(p, np.complex128)
    qs, zs = [], []
    for zc in (0.45 + 0.45j, 0.55 + 0.45j, 0.45 + 0.55j, 0.55 + 0.55j):
        q, z = _cluster(rng, 9, zc, 0.05)
        S, al = oracle.p2m(q, z, zc, p)
        S2, be = oracle.m2m(S, al, zc, zp)
        total_S += S2
        total += be
        qs.append(q)
        zs.append(z)
    Sd, ad = oracle.p2m(np.concatenate(qs), np.concatenate(zs), zp, p)
    assert abs(total_S - Sd) < 1e-13
    assert np.max(np.abs(total - ad)) < 1e-13 * max(1.0, np.max(np.abs(ad)))


def test_m2l_l2p_matches_direct_sum_of_well_separated_cluster():
    rng = np.random.default_rng(9)
    q, z = _cluster(rng, 30, 0.8 + 0.3j, 0.05)
    zL = 0.5 + 0.3j
    zt = zL + 0.05 * (rng.uniform(-1, 1, 25) + 1j * rng.uniform(-1, 1, 25)) / math.sqrt(2)
    direct = oracle.green_sum(z.real, z.imag, q, zt.real, zt.imag, 0.0)
    errs = []
    for p in (8, 16, 30):
        S, al = oracle.p2m(q, z, 0.8 + 0.3j, p)
        b = oracle.m2l(S, al, 0.8 + 0.3j, zL)
        errs.append(np.max(np.abs(oracle.l2p(b, zL, zt) - direct)))
    A = np.abs(q).sum() / (2 * math.pi)
    assert errs[-1] < 1e-12 * A
    assert errs[0] > errs[1] > errs[2] or errs[1] < 1e-13 * A


def test_l2l_is_exact_recentering():
    rng = np.random.default_rng(2)
    b = rng.normal(size=13) + 1j * rng.normal(size=13)
    zL, zn = 0.2 + 0.1j, 0.23 + 0.08j
    c = oracle.l2l(b, zL, zn)
    zt = zn + 0.02 * (rng.normal(size=10) + 1j * rng.normal(size=10))
    assert np.allclose(oracle.l2p(c, zn, zt), oracle.l2p(b, zL, zt), rtol=1e-13, atol=1e-13)


def test_printed_m2m_sign_is_not_exact():
    """Reading c2: with the sign printed in Eq. expandedBeta (-S z0^k/k) the shifted
    expansion no longer matches the parent's own expansion."""
    rng = np.random.default_rng(5)
    p, zc, zp = 12, 0.45 + 0.45j, 0.5 + 0.5j
    q, z = _cluster(rng, 9, zc, 0.05)
    S, al = oracle.p2m(q, z, zc, p)
    _, be = oracle.m2m(S, al, zc, zp)
    k = np.arange(1, p + 1)
    printed = be - 2 * S * (zc - zp) ** k / k
    _, ad = oracle.p2m(q, z, zp, p)
    assert np.max(np.abs(be - ad)) < 1e-14
    assert np.max(np.abs(printed - ad)) > 1e-4 * abs(S)


# ---------------------------------------------------------------- penalisation force
@pytest.mark.parametrize("n", [256, 512])
def test_penal_force_of_uniform_flow_is_lambda_U_times_body_area(n):
    """Eq. dragPenal with u = U uniform and u_s = 0: F = lambda U int chi dV, and the
    smoothed indicator of the disk integrates to pi R^2 up to O((h/R)^2): pins the h^2
    cell weight, the lambda factor and the direction of the force."""
    snap = synth.cylinder_flow(n, seed=2000, n_surface=64)
    R, U, lam = 0.05, 0.7, 37.0
    u = np.full((n, n), U)
    z = np.zeros((n, n))
    F = oracle.penal_force(u, z, snap.chi, z, z, snap.h, lam)
    area = math.pi * R * R
    assert abs(F[0] / (lam * U * area) - 1.0) < 5.0 * (snap.h / R) ** 2
    assert F[1] == 0.0
    assert F[2] == F[0] and F[3] == 0.0  # drag along U_hat = (1, 0), no lift


def test_penal_force_vanishes_when_the_fluid_moves_with_the_body_and_is_linear():
    rng = np.random.default_rng(7)
    n, h = 64, 1.0 / 64
    chi = rng.uniform(0, 1, (n, n))
    u, v = rng.normal(size=(n, n)), rng.normal(size=(n, n))
    assert np.allclose(oracle.penal_force(u, v, chi, u, v, h, 5.0), 0.0, atol=0.0)
    a = oracle.penal_force(u, v, chi, 0 * u, 0 * v, h, 1.0)
    b = oracle.penal_force(u, v, chi, 0.5 * u, 0.5 * v, h, 2.0)  # lambda x 2, (u - u_s) x 1/2
    assert np.allclose(a, b, rtol=1e-13, atol=0.0)


def test_penal_force_drag_and_lift_follow_the_free_stream_direction():
    """drag = F . U_hat, lift = F . (-U_hat_y, U_hat_x) (reading c14): with U along +y a
    force along +x is pure negative lift, with U along +x it is pure drag."""
    n, h = 16, 1.0 / 16
    one, z = np.ones((n, n)), np.zeros((n, n))
    Fy_up = oracle.penal_force(one, z, one, z, z, h, 1.0, uinf=(0.0, 3.0))
    assert Fy_up[2] == 0.0 and Fy_up[3] == -Fy_up[0]
    Fx = oracle.penal_force(one, z, one, z, z, h, 1.0, uinf=(2.0, 0.0))
    assert Fx[2] == Fx[0] and Fx[3] == 0.0


# ---------------------------------------------------- Eqs. aPenal and aSF (Sec. 3.3)
@pytest.mark.parametrize("n", [128, 256])
def test_body_moments_of_a_disk_in_uniform_motion(n):
    """A smoothed disk moving with a uniform velocity: u_CM is that velocity exactly (any chi),
    and M = rho pi R^2 up to the smoothing's O((h/R)^2)."""
    snap = synth.cylinder_flow(n, diameter=0.3, centre=(0.5, 0.5), seed=1)
    U = np.full((n, n), 0.7)
    V = np.full((n, n), -0.2)
    M, ux, uy = oracle.body_moments(U, V, snap.chi, snap.h, rho=2.0)
    assert abs(ux - 0.7) < 1e-14 and abs(uy + 0.2) < 1e-14
    assert abs(M / (2.0 * math.pi * 0.15 ** 2) - 1.0) < 4 * (snap.h / 0.15) ** 2


def test_body_moments_of_a_rigid_rotation_about_the_centre_of_mass():
    """Solid-body rotation about the disk's centre: the centre of mass does not move."""
    n = 256
    snap = synth.cylinder_flow(n, diameter=0.3, centre=(0.5, 0.5), seed=1)
    X, Y = synth.cell_centres(n, snap.h)
    _, ux, uy = oracle.body_moments(-(Y - 0.5), X - 0.5, snap.chi, snap.h)
    assert abs(ux) < 1e-13 and abs(uy) < 1e-13


def test_accelerations_of_a_uniformly_accelerated_body():
    """Eq. aSF with F = M a gives a; Eq. aPenal on u_CM(t) = u0 + a t (and on a quadratic,
    where the centred difference is still exact) gives a."""
    a = np.array([0.3, -1.2])
    M = 2.5
    F = np.array([0.4 * M * a[0], 0.4 * M * a[1], 0.6 * M * a[0], 0.6 * M * a[1], 9.0, 9.0])
    assert np.allclose(oracle.acceleration_sf(F, M), a, rtol=1e-15, atol=0)
    dt, t = 0.01, 0.37
    u = lambda s: np.array([1.0, 0.5]) + a * s + np.array([0.2, -0.1]) * s * s  # noqa: E731
    got = oracle.acceleration_penal(u(t - dt), u(t + dt), dt)
    assert np.allclose(got, a + 2 * np.array([0.2, -0.1]) * t, rtol=1e-12, atol=1e-12)
