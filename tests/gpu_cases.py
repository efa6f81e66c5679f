"""Helpers shared by the GPU parity tests: run one snapshot through the CUDA path
(via the C ABI binding) and through the CPU oracle on the same seeded inputs."""
import numpy as np

import oracle
from paper_1610_04398_gb300 import api


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def worst_cell(a, b):
    """Largest pointwise error relative to the largest reference value: max|a - b| / max|b|.
    A relative L2 over millions of cells hides a few wrong cells; this bound does not."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def to_dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def run_gpu(snap, precision="fp64", order=20, theta=0.5, interp="nearest", lift=None, dS=None,
            with_grid=True, rho=1.0, tile=16, theta_surface=0.0):
    """Full path on the GPU.  Returns dict(f, P (n x n or None), per_point, forces)."""
    import torch
    plan = api.Plan(snap.n, snap.h, order, theta, x0=snap.x0, y0=snap.y0, rho=rho, precision=precision,
                    lift=snap.lift if lift is None else lift, interp=interp, uinf=snap.uinf, tile=tile,
                    theta_surface=theta_surface)
    dt = plan.dtype
    fields = [to_dev(a, dt) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    f = torch.empty(snap.n * snap.n, dtype=dt, device="cuda")
    plan.rhs(*fields, snap.lam, f_out=f)
    P = None
    if with_grid:
        P = torch.empty(snap.n * snap.n, dtype=dt, device="cuda")
        plan.pressure_solve(P)
    pts = to_dev(snap.points, torch.float64)
    nrm = to_dev(snap.normals, torch.float64)
    per = torch.empty(len(snap.points) * 5, dtype=torch.float64, device="cuda")
    dS_t = None if dS is None else to_dev(dS, torch.float64)
    forces = plan.surface_traction(fields[0], fields[1], pts, nrm, snap.nu, dS=dS_t, per_point=per)
    torch.cuda.synchronize()
    out = dict(f=f.double().cpu().numpy().reshape(snap.n, snap.n),
               P=None if P is None else P.double().cpu().numpy().reshape(snap.n, snap.n),
               per_point=per.cpu().numpy().reshape(-1, 5), forces=forces, plan=plan)
    return out


def run_oracle(snap, cells=None, rho=1.0, interp="nearest", lift=None, dS=None):
    """Oracle on the same snapshot.  ``cells``: None = all cells, else flat indices."""
    n, h = snap.n, snap.h
    f = oracle.rhs(snap.u, snap.v, snap.chi, snap.usx, snap.usy, h=h, rho=rho, lam=snap.lam)
    q = oracle.source_weights(f, h)
    c = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(snap.x0 + c, snap.y0 + c)
    if cells is None:
        cells = np.arange(n * n)
    Pc = oracle.green_sum_grid(q, h, X.ravel()[cells], Y.ravel()[cells], snap.x0, snap.y0)
    Ps = oracle.green_sum_grid(q, h, snap.points[:, 0], snap.points[:, 1], snap.x0, snap.y0)
    per, F = oracle.traction(snap.u, snap.v, h, snap.points, snap.normals, Ps, snap.nu, rho=rho,
                             lift=snap.lift if lift is None else lift, dS=dS, uinf=snap.uinf,
                             x0=snap.x0, y0=snap.y0, interp=interp)
    return dict(f=f, cells=cells, P_cells=Pc, P_surf=Ps, per_point=per, forces=F)


def force_err(Fg, Fr):
    """Errors of drag and lift relative to the magnitude of the reference total force."""
    scale = max(np.hypot(Fr[4], Fr[5]), 1e-12)
    return abs(Fg[4] - Fr[4]) / scale, abs(Fg[5] - Fr[5]) / scale
