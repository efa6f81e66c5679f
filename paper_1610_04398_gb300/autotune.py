"""Autotuner of the mixed-precision path: expansion order p, acceptance parameter
theta and near-field tile, chosen for speed under an accuracy bound.

For one snapshot it times every candidate (p, theta, tile) as a captured step graph
and measures its error against a high-accuracy FP64 GPU solve of the same snapshot
(p = 20, theta = 0.4: truncation error ~1e-9, far below the bound).  The fastest
candidate whose relative L2 pressure error over all cells and whose drag/lift errors
(relative to the force magnitude) stay below ``safety * tol`` wins.  The FP64 GPU
solve stands in for the FP64 direct sum here; the tests check the chosen setting
against the direct sum itself.
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


def _run(snap, precision, order, theta, tile=16, steps=0, warmup=3):
    """One captured step of a plan; returns (P, forces, ms_per_step or None)."""
    import torch
    plan = api.Plan(snap.n, snap.h, order, theta, x0=snap.x0, y0=snap.y0, precision=precision,
                    lift=snap.lift, uinf=snap.uinf, tile=tile)
    f = _fields(snap, plan.dtype)
    pts = torch.from_numpy(np.ascontiguousarray(snap.points)).cuda()
    nrm = torch.from_numpy(np.ascontiguousarray(snap.normals)).cuda()
    P = torch.empty(snap.n * snap.n, dtype=plan.dtype, device="cuda")
    F = torch.zeros(6, dtype=torch.float64, device="cuda")
    g = plan.capture_step(*f, snap.lam, p_out=P, points=pts, normals=nrm, nu=snap.nu, forces=F)
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
    torch.cuda.synchronize()
    out = P.double().cpu().numpy(), F.cpu().numpy()
    g.destroy()
    plan.destroy()
    return out[0], out[1], ms


def autotune(snap, orders=DEFAULT_ORDERS, thetas=DEFAULT_THETAS, tiles=DEFAULT_TILES, tol=1e-4,
             safety=0.5, steps=10):
    """Return {"best": {...}, "table": [...], "reference": "..."} for the mixed path."""
    t0 = time.perf_counter()
    P_ref, F_ref, _ = _run(snap, "fp64", 20, 0.4)
    nref = np.linalg.norm(P_ref)
    fscale = max(np.hypot(F_ref[4], F_ref[5]), 1e-300)
    table = []
    for p, th, tile in itertools.product(orders, thetas, tiles):
        P, F, ms = _run(snap, "mixed", p, th, tile, steps=steps)
        e_p = float(np.linalg.norm(P - P_ref) / nref)
        e_f = float(max(abs(F[4] - F_ref[4]), abs(F[5] - F_ref[5])) / fscale)
        table.append({"order": p, "theta": th, "tile": tile, "ms": ms, "err_p": e_p, "err_force": e_f,
                      "ok": bool(e_p <= safety * tol and e_f <= safety * tol)})
    ok = [r for r in table if r["ok"]]
    best = min(ok, key=lambda r: r["ms"]) if ok else min(table, key=lambda r: r["err_p"])
    return {"best": best, "table": table, "tol": tol, "safety": safety,
            "reference": "FP64 GPU solve, p=20, theta=0.4", "seconds": time.perf_counter() - t0}
