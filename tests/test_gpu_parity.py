"""CUDA path vs the CPU oracle, element by element, on the same seeded inputs.

Tolerances (relative L2 of pressure over the compared set, and the same bound on the
worst cell, max|dP| / max|P|; force errors relative to the reference force magnitude):
  FP64 path  p = 20, theta = 0.5: pressure <= 1e-6;  RHS <= 1e-12 (same arithmetic)
  mixed path p = 20, theta = 0.5: pressure <= 1e-4, drag and lift <= 1e-4
"""
import math

import numpy as np
import pytest

import oracle
from paper_1610_04398_gb300 import api, synth
from gpu_cases import force_err, rel_l2, run_gpu, run_oracle, to_dev, worst_cell

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_P = {"fp64": 1e-6, "mixed": 1e-4}
TOL_F = {"fp64": 1e-6, "mixed": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()
    oracle.build()


def _check_full(snap, precision, order=20, theta=0.5, tol=None, **kw):
    g = run_gpu(snap, precision, order, theta, **kw)
    kw.pop("tile", None)
    r = run_oracle(snap, interp=kw.get("interp", "nearest"), lift=kw.get("lift"), dS=kw.get("dS"))
    tol = TOL_P[precision] if tol is None else tol
    e_f = np.max(np.abs(g["f"] - r["f"])) / np.max(np.abs(r["f"]))
    e_p = rel_l2(g["P"].ravel(), r["P_cells"])
    e_s = rel_l2(g["per_point"][:, 0], r["P_surf"])
    w_p = worst_cell(g["P"].ravel(), r["P_cells"])
    w_s = worst_cell(g["per_point"][:, 0], r["P_surf"])
    assert e_f < (1e-12 if precision == "fp64" else 1e-5), e_f
    assert e_p < tol and w_p < tol, (e_p, w_p, tol)
    assert e_s < tol and w_s < tol, (e_s, w_s, tol)
    return g, r


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cylinder_128_full_grid(precision):
    snap = synth.cylinder_flow(128, seed=2000)
    g, r = _check_full(snap, precision)
    ed, el = force_err(g["forces"], r["forces"])
    assert ed < TOL_F[precision] and el < TOL_F[precision], (ed, el)
    # pointwise tractions follow from the same P and velocity gradient
    scale = np.max(np.abs(r["per_point"][:, 1:3]))
    assert np.max(np.abs(g["per_point"][:, 1:3] - r["per_point"][:, 1:3])) < 10 * TOL_P[precision] * scale
    vs = np.max(np.abs(r["per_point"][:, 3:5]))
    tolv = 1e-12 if precision == "fp64" else 1e-5
    assert np.max(np.abs(g["per_point"][:, 3:5] - r["per_point"][:, 3:5])) <= tolv * vs + 1e-300


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_swimmer_256_full_grid(precision):
    snap = synth.swimmer_snapshot(256, phase=0.3, seed=4001, n_surface=1024)
    _check_full(snap, precision)


def test_lamb_oseen_128_fp64_and_closed_form():
    snap = synth.lamb_oseen(128)
    g, r = _check_full(snap, "fp64")
    # the GPU pressure also reproduces the closed form at the oracle's accuracy (2nd order)
    X, Y = synth.cell_centres(128, snap.h)
    rr = np.hypot(X - 0.5, Y - 0.5)
    sel = rr < 0.3
    x = np.maximum(rr[sel] ** 2 / 0.05 ** 2, 1e-300)
    import scipy.special as sps
    ex = -1.0 / (8 * math.pi ** 2 * 0.05 ** 2) * ((-np.expm1(-x)) ** 2 / x + 2 * sps.exp1(x) - 2 * sps.exp1(2 * x))
    Pg = g["P"][sel]
    assert rel_l2(Pg - Pg.mean(), ex - ex.mean()) < 1.5e-2


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_small_grids_and_tree_depths(n):
    """n = 8: one leaf (near field only); 16: no M2L level; 32: first M2L level."""
    snap = synth.cylinder_flow(n, diameter=0.3, centre=(0.5, 0.5), n_surface=37, seed=7)
    _check_full(snap, "fp64")
    _check_full(snap, "mixed")


@pytest.mark.parametrize("theta", [0.4, 0.6, 0.75])
def test_other_theta(theta):
    snap = synth.cylinder_flow(128, seed=2001, n_surface=333)
    _check_full(snap, "fp64", theta=theta, tol=2e-6)


@pytest.mark.parametrize("order,tol", [(12, 1e-4), (16, 2e-5)])
def test_lower_order_mixed(order, tol):
    snap = synth.cylinder_flow(128, seed=2002)
    _check_full(snap, "mixed", order=order, tol=tol)


def test_options_bilinear_lift0_given_dS_offset_origin():
    snap = synth.cylinder_flow(64, diameter=0.3, centre=(0.5, 0.5), n_surface=101, seed=9)
    snap.x0, snap.y0 = -0.25, 0.125
    snap.points = snap.points + np.array([-0.25, 0.125])
    dS = oracle.default_dS(snap.points) * (1 + 0.1 * np.sin(np.arange(101)))
    g, r = _check_full(snap, "fp64", interp="bilinear", lift=0.0, dS=dS)
    ed, el = force_err(g["forces"], r["forces"])
    assert ed < 1e-8 and el < 1e-8


@pytest.mark.parametrize("precision,order,tol", [("fp64", 20, 1e-11), ("mixed", 12, 2e-6)])
def test_multipoles_match_oracle_expansions(precision, order, tol):
    """Leaf P2M (Eq. alphaK) and shifted parents (Eq. expandedBeta) vs the oracle's
    expansions about the same centres, after undoing the box-side scaling; the mixed path's
    FP32 multipoles (its source kernel, leaf multipoles and upward kernels) within a few FP32
    roundings of the oracle's FP64 ones (relative to the level's largest coefficient)."""
    n = 64
    snap = synth.cylinder_flow(n, diameter=0.3, centre=(0.5, 0.5), seed=3)
    plan = api.Plan(n, snap.h, order, 0.5, precision=precision)
    fields = [to_dev(a, plan.dtype) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    plan.rhs(*fields, snap.lam)
    cast = (lambda a: a) if precision == "fp64" else (lambda a: np.asarray(a, np.float32).astype(np.float64))
    f = oracle.rhs(*(cast(a) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)), h=snap.h, lam=snap.lam)
    q = oracle.source_weights(f, snap.h)
    X, Y = synth.cell_centres(n, snap.h)
    for level in (3, 2, 1):
        side = 2 ** level
        s = 1.0 / side
        got = plan.get_expansion("multipole", level).cpu().numpy()
        for b in (0, side + 1, side * side - 1, side * (side // 2) + side // 2):
            bx, by = b % side, b // side
            m = int(n / side)
            qq = q[by * m:(by + 1) * m, bx * m:(bx + 1) * m]
            zz = X[by * m:(by + 1) * m, bx * m:(bx + 1) * m] + 1j * Y[by * m:(by + 1) * m, bx * m:(bx + 1) * m]
            zc = (bx + 0.5) * s + 1j * (by + 0.5) * s
            S, al = oracle.p2m(qq, zz, zc, order)
            want = np.concatenate([[S], al / s ** np.arange(1, order + 1)])
            assert np.max(np.abs(got[b] - want)) < tol * max(1.0, np.max(np.abs(want))), (level, b)


@pytest.mark.parametrize("n", [512, 2048])
def test_mixed_upward_pass_matches_fp64_at_every_level(n):
    """The mixed path's one-launch upward pass (one CTA per subtree of up to four levels, the
    last CTA to finish shifting the levels above up to the root) against the FP64 plan's
    multipoles, every level down to the root: the FP32 arithmetic of the source, the leaf
    multipoles and the shifts, within 1e-5 of each level's largest coefficient."""
    snap = synth.cylinder_flow(n, seed=2000, n_surface=64)
    got = {}
    for precision in ("fp64", "mixed"):
        plan = api.Plan(n, snap.h, 12, 0.75, precision=precision, tile=128 if precision == "mixed" else 16)
        fields = [to_dev(a, plan.dtype) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
        plan.rhs(*fields, snap.lam)
        got[precision] = [plan.get_expansion("multipole", lev).cpu().numpy() for lev in range(int(np.log2(n // 8)) + 1)]
        plan.destroy()
    for lev, (a, b) in enumerate(zip(got["mixed"], got["fp64"])):
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert err < 1e-5, (lev, err)


@pytest.mark.parametrize("n", [256, 512, 2048])
def test_mixed_downward_pass_matches_fp64_at_every_level(n):
    """The mixed path's two-launch downward pass (every level's multipole-to-local part in one
    grid, then one CTA per subtree of the level L - 3 boxes shifting the locals down from
    level 2 and evaluating them) against the FP64 plan's locals at every level 2..L: n = 256
    has its subtree roots at level 2, 512 one shared ancestor level, 2048 three.  Within 1e-5
    of each level's largest coefficient; the pressure against the FP64 solve within 1e-5."""
    snap = synth.cylinder_flow(n, seed=2001, n_surface=64)
    L = int(np.log2(n // 8))
    got, P = {}, {}
    for precision in ("fp64", "mixed"):
        plan = api.Plan(n, snap.h, 12, 0.75, precision=precision, tile=128 if precision == "mixed" else 16)
        fields = [to_dev(a, plan.dtype) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
        out = torch.empty(n * n, dtype=plan.dtype, device="cuda")
        plan.rhs(*fields, snap.lam)
        plan.pressure_solve(out)
        got[precision] = [plan.get_expansion("local", lev).cpu().numpy() for lev in range(2, L + 1)]
        P[precision] = out.double().cpu().numpy()
        plan.destroy()
    for lev, (a, b) in enumerate(zip(got["mixed"], got["fp64"]), start=2):
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert err < 1e-5, (lev, err)
    assert rel_l2(P["mixed"], P["fp64"]) < 1e-5
    assert worst_cell(P["mixed"], P["fp64"]) < 1e-5


@pytest.mark.parametrize("n", [256, 1024])
def test_mixed_downward_pass_matches_the_per_level_kernels(n):
    """An output one element off 16-byte alignment takes the per-level translation kernels
    with the evaluation fused into the leaf level; an aligned one the two-launch pass.  The
    same sums in different FP32 orders: the pressures agree within 2e-6."""
    snap = synth.cylinder_flow(n, seed=2002, n_surface=64)
    nn = n * n
    plan = api.Plan(n, snap.h, 12, 0.75, precision="mixed", tile=128)
    fields = [to_dev(a, plan.dtype) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    out = {}
    for shift in (0, 1):
        big = torch.zeros(nn + 4, dtype=torch.float32, device="cuda")
        plan.rhs(*fields, snap.lam)
        plan.pressure_solve(big[shift:shift + nn])
        torch.cuda.synchronize()
        out[shift] = big[shift:shift + nn].double().cpu().numpy()
    plan.destroy()
    assert rel_l2(out[1], out[0]) < 2e-6
    assert worst_cell(out[1], out[0]) < 2e-6


@pytest.mark.parametrize("n,theta", [(256, 0.75), (2048, 0.75), (512, 0.6), (2048, 0.6), (1024, 0.5)])
def test_tensor_core_translations_match_fp32_cores(n, theta):
    """The multipole-to-local translations on the tensor cores (split FP16 operands, 128 target
    boxes of one child position a tile, halo margin 1 at theta 0.75 and 2 at 0.6 and 0.5, the
    longest lists at 0.5) against the FP32-core kernel on the same plan settings: every
    level's locals within 1e-5 of the level's largest coefficient of the FP64 plan's, the
    pressures within 2e-6 of each other, and no bounded device wait gave up."""
    snap = synth.cylinder_flow(n, seed=2003, n_surface=64)
    L = int(np.log2(n // 8))
    got, P = {}, {}
    for mode in ("fp64", "fp32", "tensor"):
        prec = "fp64" if mode == "fp64" else "mixed"
        plan = api.Plan(n, snap.h, 12, theta, precision=prec, tile=128 if prec == "mixed" else 16,
                        m2l_tensor=mode == "tensor")
        if mode == "tensor":
            assert plan.info().downward == 3
        fields = [to_dev(a, plan.dtype) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
        out = torch.empty(n * n, dtype=plan.dtype, device="cuda")
        plan.rhs(*fields, snap.lam)
        plan.pressure_solve(out)
        assert plan.device_status() == [0, 0, 0, 0]
        got[mode] = [plan.get_expansion("local", lev).cpu().numpy() for lev in range(2, L + 1)]
        P[mode] = out.double().cpu().numpy()
        plan.destroy()
    for lev, (a, b) in enumerate(zip(got["tensor"], got["fp64"]), start=2):
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert err < 1e-5, (lev, err)
    assert rel_l2(P["tensor"], P["fp32"]) < 2e-6
    assert worst_cell(P["tensor"], P["fp32"]) < 2e-6
    assert rel_l2(P["tensor"], P["fp64"]) < 1e-5


def test_call_order_and_dtype_errors():
    snap = synth.cylinder_flow(32, diameter=0.3, centre=(0.5, 0.5), seed=1)
    plan = api.Plan(32, snap.h, 20, 0.5, precision="fp64")
    with pytest.raises(api.PPError) as e:
        plan.pressure_solve(None)
    assert e.value.status == api.PP_ERR_STATE
    with pytest.raises(TypeError):
        plan.rhs(*[to_dev(a, torch.float32) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)], 1.0)
    fields = [to_dev(a, torch.float64) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    plan.rhs(*fields, snap.lam)
    plan.pressure_solve(None)  # passes without a grid output
    pts = to_dev(snap.points, torch.float64)
    forces = torch.zeros(6, dtype=torch.float64, device="cuda")
    assert plan.surface_traction(fields[0], fields[1], pts, to_dev(snap.normals, torch.float64), 1e-4,
                                 forces=forces) is None
    host = plan.surface_traction(fields[0], fields[1], pts, to_dev(snap.normals, torch.float64), 1e-4)
    assert np.allclose(forces.cpu().numpy(), host, rtol=0, atol=0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_graph_replays_match_direct_calls(precision):
    """pp_step_graph_create/launch: identical results to the three calls, also after the
    input buffers are refilled in place between replays."""
    snaps = [synth.cylinder_flow(128, seed=2003), synth.cylinder_flow(128, seed=2004)]
    direct = [run_gpu(s, precision) for s in snaps]
    s0 = snaps[0]
    plan = api.Plan(s0.n, s0.h, 20, 0.5, precision=precision, lift=s0.lift, uinf=s0.uinf)
    dt = plan.dtype
    fields = [to_dev(a, dt) for a in (s0.u, s0.v, s0.chi, s0.usx, s0.usy)]
    pts = to_dev(s0.points, torch.float64)
    nrm = to_dev(s0.normals, torch.float64)
    P = torch.empty(s0.n * s0.n, dtype=dt, device="cuda")
    per = torch.empty(len(s0.points) * 5, dtype=torch.float64, device="cuda")
    F = torch.empty(6, dtype=torch.float64, device="cuda")
    g = plan.capture_step(*fields, s0.lam, p_out=P, points=pts, normals=nrm, nu=s0.nu, per_point=per, forces=F)
    for s, d in zip(snaps, direct):
        for dst, a in zip(fields, (s.u, s.v, s.chi, s.usx, s.usy)):
            dst.copy_(to_dev(a, dt))
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(P.double().cpu().numpy().reshape(s.n, s.n), d["P"])
        assert np.array_equal(per.cpu().numpy().reshape(-1, 5), d["per_point"])
        assert np.array_equal(F.cpu().numpy(), d["forces"])
    g.destroy()


@pytest.mark.parametrize("tile", [8, 16, 128])
@pytest.mark.parametrize("theta", [0.4, 0.5, 0.75])
def test_mixed_near_field_tiles(tile, theta):
    """The near-field kernels of the mixed path (8 or 16 targets per thread on the FP32
    cores, 128-leaf tiles on the tensor cores), for near lists of radius 1, 2 and 3."""
    snap = synth.cylinder_flow(128, seed=2005, n_surface=257)
    _check_full(snap, "mixed", theta=theta, tile=tile)


@pytest.mark.parametrize("n", [256, 512])
def test_tensor_core_near_field_matches_fp32_cores(n):
    """Tile 128 (tcgen05, split TF32, per-offset accumulators drained into Kahan sums)
    is as accurate as tile 16 (FP32 FMAs): both measured against the FP64 solve with the
    same p and theta, so only the near-field rounding differs.  The two FP32 paths round
    independently, so each is bounded against FP64 rather than against the other: the
    tensor-core error may exceed the FP32-core error by at most 50% plus 2^-23 (one
    unit roundoff of the stored result)."""
    snap = synth.swimmer_snapshot(n, phase=0.7, seed=4007, n_surface=512)
    ref = run_gpu(snap, "fp64", 20, 0.5)["P"]
    P16 = run_gpu(snap, "mixed", 20, 0.5, tile=16)["P"]
    Ptc = run_gpu(snap, "mixed", 20, 0.5, tile=128)["P"]
    e_cores, e_tc = rel_l2(P16, ref), rel_l2(Ptc, ref)
    assert e_cores < 5e-6
    assert e_tc < 1.5 * e_cores + 2.0 ** -23
    assert worst_cell(Ptc, ref) < 1.5 * worst_cell(P16, ref) + 2.0 ** -23


@pytest.mark.parametrize("n", [64, 256])
def test_source_from_unaligned_fields_matches_aligned(n):
    """The mixed path's register-blocked source kernel needs 16-byte aligned fields; fields
    one element off that alignment take the shared-memory kernels.  Both compute Eq.
    PoissonFinal with the same differences, so the sources agree to rounding.  The two
    kernels sum the leaf multipoles in different FP32 orders; each mixed solve is within
    ~2e-6 of the FP64 solve (the near-field tests), so the pressures agree within 1e-5."""
    snap = synth.cylinder_flow(n, seed=2011, n_surface=128)
    nn = n * n
    plan = api.Plan(n, snap.h, 20, 0.5, precision="mixed", lift=snap.lift, uinf=snap.uinf)
    out = {}
    for shift in (0, 1):
        bufs = []
        for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy):
            big = torch.zeros(nn + 4, dtype=torch.float32, device="cuda")
            big[shift:shift + nn] = torch.from_numpy(np.ascontiguousarray(a).ravel()).float()
            bufs.append(big[shift:shift + nn])
        f = torch.empty(nn, dtype=torch.float32, device="cuda")
        P = torch.empty(nn, dtype=torch.float32, device="cuda")
        plan.rhs(*bufs, snap.lam, f_out=f)
        plan.pressure_solve(P)
        torch.cuda.synchronize()
        out[shift] = (f.double().cpu().numpy(), P.double().cpu().numpy())
    f0, P0 = out[0]
    f1, P1 = out[1]
    assert np.max(np.abs(f0 - f1)) <= 1e-6 * np.max(np.abs(f0))
    assert rel_l2(P1, P0) < 1e-5
    plan.destroy()


def test_surface_theta_option():
    """The surface tree-code's acceptance parameter is its own option: the default is
    min(theta, 0.6), bitwise equal to passing that value; a looser surface theta (the grid's
    0.75) changes only the surface part and is less accurate against the direct sum."""
    snap = synth.cylinder_flow(256, seed=2012, n_surface=512)

    def solve(ts):
        plan = api.Plan(256, snap.h, 12, 0.75, precision="mixed", lift=snap.lift, uinf=snap.uinf, tile=128,
                        theta_surface=ts)
        f = [to_dev(a, torch.float32) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
        P = torch.empty(256 * 256, dtype=torch.float32, device="cuda")
        per = torch.empty(512 * 5, dtype=torch.float64, device="cuda")
        plan.rhs(*f, snap.lam)
        plan.pressure_solve(P)
        forces = plan.surface_traction(f[0], f[1], to_dev(snap.points, torch.float64),
                                       to_dev(snap.normals, torch.float64), snap.nu, per_point=per)
        torch.cuda.synchronize()
        out = (P.cpu().numpy(), per.cpu().numpy().reshape(-1, 5), np.asarray(forces), plan.info().theta_surface)
        plan.destroy()
        return out

    d, e, loose = solve(0.0), solve(0.6), solve(0.75)
    assert d[3] == 0.6 and e[3] == 0.6 and loose[3] == 0.75
    assert np.array_equal(d[0], e[0]) and np.array_equal(d[1], e[1]) and np.array_equal(d[2], e[2])
    assert np.array_equal(d[0], loose[0])  # the grid solve does not depend on it
    r = run_oracle(snap, cells=np.array([0]))  # the surface points are what is compared
    err = lambda x: rel_l2(x[1][:, 0], r["P_surf"])
    assert err(d) < 1e-4
    assert err(d) < err(loose)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["cylinder", "swimmer"])
def test_penal_force_matches_oracle(precision, kind):
    """Eq. dragPenal: the penalisation force (rigid cylinder, u_s = 0; deforming swimmer,
    u_s != 0) against the oracle's FP64 sum.  FP64 plans sum in FP64 (1e-12); mixed plans
    form each cell's term in FP32 (one rounding, relative 6e-8) and sum with compensation,
    so 1e-6 of the force magnitude.  Host and device results agree bitwise, and a repeated
    call is identical (fixed reduction order)."""
    snap = (synth.cylinder_flow(512, seed=2000, n_surface=64) if kind == "cylinder"
            else synth.swimmer_snapshot(256, phase=0.3, seed=4003, n_surface=128))
    plan = api.Plan(snap.n, snap.h, 12, 0.6, precision=precision, uinf=snap.uinf, tile=16)
    dt = plan.dtype
    f = [to_dev(a, dt) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    host = plan.penal_force(*f, snap.lam)
    dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    plan.penal_force(*f, snap.lam, forces=dev)
    again = plan.penal_force(*f, snap.lam)
    torch.cuda.synchronize()
    ref = oracle.penal_force(*[np.asarray(a, np.float64) if precision == "fp64" else
                               np.asarray(a, np.float32).astype(np.float64)
                               for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)],
                             snap.h, snap.lam, uinf=snap.uinf)
    scale = max(np.hypot(ref[0], ref[1]), 1e-300)
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.max(np.abs(host - ref)) <= tol * scale, (host, ref)
    assert np.array_equal(host, dev.cpu().numpy()) and np.array_equal(host, again)
    plan.destroy()
