"""Autotuner of the mixed-precision path: expansion order p, acceptance parameter
theta and near-field tile, chosen for speed under an accuracy bound.

For one snapshot it times every candidate (p, theta, tile) as a captured step graph
and measures its error against FP64 references of the same snapshot: the grid pressure
against the FP64 zero-padded FFT solve, which is the discrete sum of Eq. greenSum itself
with no truncation error (grids up to 4096^2; larger ones use an FP64 multipole solve at
p = 20, theta = 0.4, truncation error ~1e-9), and drag/lift against the FP64 tree-code
forces at p = 20, theta = 0.4.  The fastest candidate whose relative L2 pressure error
over all cells, whose worst cell (max |dP| / max |P|) and whose drag/lift errors (relative
to the force magnitude) stay below ``safety * tol`` wins.  The tests check the chosen
setting against the oracle's direct sum itself.
"""
from __future__ import annotations

import itertools
import time

import numpy as np

from . import api

DEFAULT_ORDERS = (12, 16, 20)
DEFAULT_THETAS = (0.4, 0.5, 0.6, 0.7, 0.75)
DEFAULT_TILES = (8, 16, 128)


def _fields(snap, dtype):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)
            for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]


def _run(snap, precision, order, theta, tile=16, steps=0, warmup=3, exact_grid=False):
    """One captured step of a plan; returns (P, surface P, forces, ms_per_step or None).  With
    ``exact_grid`` the grid pressure returned is the plan's zero-padded FFT solve of the
    same source instead of the multipole one."""
    import torch
    plan = api.Plan(snap.n, snap.h, order, theta, x0=snap.x0, y0=snap.y0, precision=precision,
                    lift=snap.lift, uinf=snap.uinf, tile=tile)
    f = _fields(snap, plan.dtype)
    pts = torch.from_numpy(np.ascontiguousarray(snap.points)).cuda()
    nrm = torch.from_numpy(np.ascontiguousarray(snap.normals)).cuda()
    P = torch.empty(snap.n * snap.n, dtype=plan.dtype, device="cuda")
    per = torch.empty(len(snap.points) * 5, dtype=torch.float64, device="cuda")
    F = torch.zeros(6, dtype=torch.float64, device="cuda")
    g = plan.capture_step(*f, snap.lam, p_out=P, points=pts, normals=nrm, nu=snap.nu, per_point=per, forces=F)
    g.launch()
    ms = None
    if steps > 0:
        for _ in range(warmup):
            g.launch()
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            g.launch()
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
    if exact_grid and snap.n <= 4096:
        plan.pressure_solve_fft(P)
    torch.cuda.synchronize()
    out = P.double().cpu().numpy(), per.view(-1, 5)[:, 0].cpu().numpy(), F.cpu().numpy()
    g.destroy()
    plan.destroy()
    return out[0], out[1], out[2], ms


def autotune(snaps, orders=DEFAULT_ORDERS, thetas=DEFAULT_THETAS, tiles=DEFAULT_TILES, tol=1e-4,
             safety=0.5, steps=10):
    """Return {"best": {...}, "table": [...], "reference": "..."} for the mixed path.

    ``snaps``: one snapshot or a list; a candidate's errors are the largest over the list
    (grid relative L2, worst grid cell, surface pressure relative L2, drag/lift) and its time
    the sum over the list."""
    t0 = time.perf_counter()
    snaps = list(snaps) if isinstance(snaps, (list, tuple)) else [snaps]
    refs = []
    for snap in snaps:
        P_ref, Ps_ref, F_ref, _ = _run(snap, "fp64", 20, 0.4, exact_grid=True)
        refs.append((P_ref, np.linalg.norm(P_ref), np.max(np.abs(P_ref)), Ps_ref, np.linalg.norm(Ps_ref), F_ref,
                     max(np.hypot(F_ref[4], F_ref[5]), 1e-300)))
    table = []
    for p, th, tile in itertools.product(orders, thetas, tiles):
        e_p = w_p = e_s = e_f = 0.0
        ms = 0.0
        for snap, (P_ref, nref, pmax, Ps_ref, nsref, F_ref, fscale) in zip(snaps, refs):
            P, Ps, F, t = _run(snap, "mixed", p, th, tile, steps=steps)
            ms += t
            e_p = max(e_p, float(np.linalg.norm(P - P_ref) / nref))
            w_p = max(w_p, float(np.max(np.abs(P - P_ref)) / pmax))
            e_s = max(e_s, float(np.linalg.norm(Ps - Ps_ref) / nsref))
            e_f = max(e_f, float(max(abs(F[4] - F_ref[4]), abs(F[5] - F_ref[5])) / fscale))
        table.append({"order": p, "theta": th, "tile": tile, "ms": ms, "err_p": e_p, "worst_p": w_p,
                      "err_surface": e_s, "err_force": e_f,
                      "ok": bool(max(e_p, w_p, e_s, e_f) <= safety * tol)})
    ok = [r for r in table if r["ok"]]
    best = min(ok, key=lambda r: r["ms"]) if ok else min(table, key=lambda r: r["err_p"])
    ref = ("grid: FP64 zero-padded FFT solve (the exact discrete sum); surface and forces: FP64 tree-code, "
           "p=20, theta=0.4" if max(s.n for s in snaps) <= 4096 else "FP64 multipole solve, p=20, theta=0.4")
    return {"best": best, "table": table, "tol": tol, "safety": safety, "reference": ref,
            "snapshots": [f"{s.meta.get('kind', 'snapshot')} {s.n}^2" for s in snaps],
            "seconds": time.perf_counter() - t0}


def batch_representatives(snaps, largest=1024):
    """One snapshot of every grid size up to ``largest`` from a batch (the first of each),
    the set a batch's setting is tuned on."""
    seen = {}
    for s in snaps:
        if s.n <= largest and s.n not in seen:
            seen[s.n] = s
    return [seen[n] for n in sorted(seen)]
