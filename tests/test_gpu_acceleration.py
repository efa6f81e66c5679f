"""The deforming body's acceleration over a sequence of snapshots (Sec. 3.3): Eq. aSF from the
surface forces and the body's mass, Eq. aPenal from the centred difference of its
centre-of-mass velocity.  pp_body_moments against the oracle's sums; the accelerations of a
swimmer sequence (phases dt apart) from the GPU's forces and moments against the oracle's.

Tolerances: moments 1e-12 (FP64 plans, same sums) and 1e-6 (mixed: each term one FP32
product, compensated sums) relative to max |value|; a_SF inherits the forces' bound (1e-4
mixed at p = 12, 1e-6 FP64 at p = 20); a_penal differences u_CM values that agree to the moments' bound, divided
by 2 dt of the phase, so 1e-6 |u_CM| / dt (mixed) absolute."""
import numpy as np
import pytest

import oracle
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
    oracle.build()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_body_moments_match_oracle(precision, tol):
    snap = synth.swimmer_snapshot(256, phase=0.37, seed=4011, n_surface=512)
    plan = api.Plan(256, snap.h, 12, 0.6, precision=precision, rho=1.3)
    dt = plan.dtype
    u, v, chi = (to_dev(a, dt) for a in (snap.u, snap.v, snap.chi))
    got = plan.body_moments(u, v, chi)
    dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    plan.body_moments(u, v, chi, out=dev)
    again = plan.body_moments(u, v, chi)
    cast = (lambda a: np.asarray(a, np.float64)) if precision == "fp64" else \
        (lambda a: np.asarray(a, np.float32).astype(np.float64))
    ref = oracle.body_moments(cast(snap.u), cast(snap.v), cast(snap.chi), snap.h, rho=1.3)
    assert abs(got[0] - ref[0]) <= tol * ref[0]
    assert np.max(np.abs(got[1:] - ref[1:])) <= tol * np.max(np.abs(ref[1:]))
    assert np.array_equal(got, dev.cpu().numpy()) and np.array_equal(got, again)
    plan.destroy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_swimmer_sequence_accelerations_match_oracle(precision):
    n, dt, t0 = 256, 0.02, 0.31
    snaps = [synth.swimmer_snapshot(n, phase=t0 + k * dt, seed=4020, n_surface=1024) for k in range(5)]
    F, m, F_ref, m_ref = [], [], [], []
    for s in snaps:
        g = run_gpu(s, precision, 20 if precision == "fp64" else 12, 0.5, with_grid=False)
        plan = g["plan"]
        dtp = plan.dtype
        F.append(g["forces"])
        m.append(plan.body_moments(*(to_dev(a, dtp) for a in (s.u, s.v, s.chi))))
        plan.destroy()
        q = oracle.source_weights(oracle.rhs(s.u, s.v, s.chi, s.usx, s.usy, h=s.h, lam=s.lam), s.h)
        Ps = oracle.green_sum_grid(q, s.h, s.points[:, 0], s.points[:, 1])
        _, Fr = oracle.traction(s.u, s.v, s.h, s.points, s.normals, Ps, s.nu, lift=s.lift, uinf=s.uinf)
        F_ref.append(Fr)
        m_ref.append(oracle.body_moments(s.u, s.v, s.chi, s.h))
    a_sf, a_pen = api.accelerations(F, m, dt)
    r_sf = np.array([oracle.acceleration_sf(F_ref[k], m_ref[k][0]) for k in range(1, 4)])
    r_pen = np.array([oracle.acceleration_penal(m_ref[k - 1][1:], m_ref[k + 1][1:], dt) for k in range(1, 4)])
    tol_f = 1e-6 if precision == "fp64" else 1e-4
    scale = np.max(np.abs(r_sf))
    print(f"{precision}: a_SF {a_sf.tolist()} a_penal {a_pen.tolist()}")
    assert np.max(np.abs(a_sf - r_sf)) <= tol_f * scale, (a_sf, r_sf)
    ucm = max(np.max(np.abs(np.array(m_ref)[:, 1:])), 1e-300)
    tol_p = (1e-12 if precision == "fp64" else 1e-6) * ucm / dt
    assert np.max(np.abs(a_pen - r_pen)) <= tol_p, (a_pen, r_pen)
