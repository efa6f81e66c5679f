"""Autotuner of the mixed-precision path: expansion order p, acceptance parameter theta,
near-field tile and the surface tree-code's acceptance parameter, chosen for speed under an
accuracy bound.

For one snapshot or a set of them it times every candidate (p, theta, tile) as a captured
step graph and measures its errors against FP64 references of the same snapshots: the grid
pressure against the FP64 zero-padded FFT solve, which is the discrete sum of Eq. greenSum
itself with no truncation error (grids up to 4096^2; larger ones use an FP64 multipole solve
at p = 20, theta = 0.4, truncation error ~1e-9), the surface pressure and drag/lift against
the FP64 tree-code at p = 20, theta = 0.4.  A candidate's errors are the largest over the
set: relative L2 and worst cell (max |dP| / max |P|) of the grid and of the surface, and
drag/lift relative to the force magnitude; the fastest candidate whose errors all stay below
``safety * tol`` wins, the surface acceptance tuned in a second stage (see ``autotune``).
Snapshots of one grid size share one plan and one step graph per candidate.  The tests
check the chosen setting against the oracle's direct sum itself.
"""
from __future__ import annotations

import itertools
import time

import numpy as np

from . import api

DEFAULT_ORDERS = (12, 16, 20)
DEFAULT_THETAS = (0.4, 0.5, 0.6, 0.7, 0.75)
DEFAULT_TILES = (8, 16, 128)
DEFAULT_SURFACE_THETAS = (0.6, 0.5, 0.45, 0.4)


def _fields(snap, dtype):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)
            for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]


def _run_group(snaps, precision, order, theta, tile=16, theta_surface=0.0, steps=0, warmup=3, exact_grid=False):
    """Snapshots of one grid size and one surface point count through ONE plan and ONE captured
    step graph (the inputs are copied into the graph's buffers before each replay).  Returns
    per snapshot (P, surface P, forces) and the step time in ms of the first snapshot
    (``steps`` replays after ``warmup``), or None."""
    import torch
    s0 = snaps[0]
    plan = api.Plan(s0.n, s0.h, order, theta, x0=s0.x0, y0=s0.y0, precision=precision, lift=s0.lift,
                    uinf=s0.uinf, tile=tile, theta_surface=theta_surface)
    f = _fields(s0, plan.dtype)
    pts = torch.from_numpy(np.ascontiguousarray(s0.points)).cuda()
    nrm = torch.from_numpy(np.ascontiguousarray(s0.normals)).cuda()
    P = torch.empty(s0.n * s0.n, dtype=plan.dtype, device="cuda")
    per = torch.empty(len(s0.points) * 5, dtype=torch.float64, device="cuda")
    F = torch.zeros(6, dtype=torch.float64, device="cuda")
    g = plan.capture_step(*f, s0.lam, p_out=P, points=pts, normals=nrm, nu=s0.nu, per_point=per, forces=F)
    out, ms = [], None
    for j, snap in enumerate(snaps):
        if j > 0:
            for dst, a in zip(f, _fields(snap, plan.dtype)):
                dst.copy_(a)
            pts.copy_(torch.from_numpy(np.ascontiguousarray(snap.points)))
            nrm.copy_(torch.from_numpy(np.ascontiguousarray(snap.normals)))
        g.launch()
        if j == 0 and steps > 0:
            for _ in range(warmup):
                g.launch()
            st = torch.cuda.current_stream()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(steps):
                g.launch()
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
        Pf = None
        if exact_grid and snap.n <= 4096:
            Pf = torch.empty_like(P)
            plan.pressure_solve_fft(Pf)
        torch.cuda.synchronize()
        out.append(((Pf if Pf is not None else P).double().cpu().numpy(), per.view(-1, 5)[:, 0].cpu().numpy(),
                    F.cpu().numpy()))
    g.destroy()
    plan.destroy()
    return out, ms


def _groups(snaps):
    """Indices of the snapshots grouped by (grid side, surface point count), in first-seen order."""
    groups = {}
    for i, s in enumerate(snaps):
        groups.setdefault((s.n, len(s.points), s.lift, tuple(s.uinf)), []).append(i)
    return list(groups.values())


def _run_all(snaps, groups, precision, order, theta, tile=16, theta_surface=0.0, steps=0, exact_grid=False):
    """Every snapshot, one plan per group; the time is the sum over the snapshots of their
    group's step time."""
    res = [None] * len(snaps)
    total = 0.0
    for idx in groups:
        out, ms = _run_group([snaps[i] for i in idx], precision, order, theta, tile, theta_surface, steps,
                             exact_grid=exact_grid)
        for i, o in zip(idx, out):
            res[i] = o
        if ms is not None:
            total += ms * len(idx)
    return res, (total if steps > 0 else None)


def _errors(res, refs):
    """Largest errors over the snapshots: grid relative L2, worst grid cell, surface pressure
    relative L2, worst surface point, drag/lift (relative to the force magnitude)."""
    e = np.zeros(5)
    for (P, Ps, F), (P_ref, Ps_ref, F_ref) in zip(res, refs):
        fscale = max(np.hypot(F_ref[4], F_ref[5]), 1e-300)
        e = np.maximum(e, [np.linalg.norm(P - P_ref) / np.linalg.norm(P_ref),
                           np.max(np.abs(P - P_ref)) / np.max(np.abs(P_ref)),
                           np.linalg.norm(Ps - Ps_ref) / np.linalg.norm(Ps_ref),
                           np.max(np.abs(Ps - Ps_ref)) / np.max(np.abs(Ps_ref)),
                           max(abs(F[4] - F_ref[4]), abs(F[5] - F_ref[5])) / fscale])
    return [float(x) for x in e]


def autotune(snaps, orders=DEFAULT_ORDERS, thetas=DEFAULT_THETAS, tiles=DEFAULT_TILES, tol=1e-4, safety=0.5,
             steps=10, surface_thetas=DEFAULT_SURFACE_THETAS, finalists=3):
    """Return {"best": {...}, "table": [...], "reference": "..."} for the mixed path.

    ``snaps``: one snapshot or a list; a candidate's errors are the largest over the list and
    its time the sum over the list.  Stage 1 times every (p, theta, tile) with the default
    surface acceptance min(theta, 0.6) and keeps those whose grid errors (relative L2 and
    worst cell) stay below safety * tol; stage 2 tries the surface acceptance values
    ``surface_thetas`` on the ``finalists`` fastest of them (the grid solve does not depend on
    it) and keeps the settings whose surface pressure (relative L2, worst point) and drag/lift
    errors also stay below safety * tol.  The fastest of those wins."""
    t0 = time.perf_counter()
    snaps = list(snaps) if isinstance(snaps, (list, tuple)) else [snaps]
    groups = _groups(snaps)
    refs, _ = _run_all(snaps, groups, "fp64", 20, 0.4, theta_surface=0.4, exact_grid=True)
    lim = safety * tol
    table = []
    for p, th, tile in itertools.product(orders, thetas, tiles):
        res, ms = _run_all(snaps, groups, "mixed", p, th, tile, steps=steps)
        e = _errors(res, refs)
        table.append({"order": p, "theta": th, "tile": tile, "theta_surface": min(th, 0.6), "ms": ms,
                      "err_p": e[0], "worst_p": e[1], "err_surface": e[2], "worst_surface": e[3], "err_force": e[4],
                      "ok": bool(max(e) <= lim), "stage": 1})
    grid_ok = sorted((r for r in table if max(r["err_p"], r["worst_p"]) <= lim), key=lambda r: r["ms"])
    for r in grid_ok[:finalists]:
        for ts in surface_thetas:
            if ts == r["theta_surface"]:
                continue
            res, ms = _run_all(snaps, groups, "mixed", r["order"], r["theta"], r["tile"], ts, steps=steps)
            e = _errors(res, refs)
            table.append({"order": r["order"], "theta": r["theta"], "tile": r["tile"], "theta_surface": ts,
                          "ms": ms, "err_p": e[0], "worst_p": e[1], "err_surface": e[2], "worst_surface": e[3],
                          "err_force": e[4], "ok": bool(max(e) <= lim), "stage": 2})
    ok = [r for r in table if r["ok"]]
    best = min(ok, key=lambda r: r["ms"]) if ok else min(
        table, key=lambda r: max(r["err_p"], r["worst_p"], r["err_surface"], r["worst_surface"], r["err_force"]))
    ref = ("grid: FP64 zero-padded FFT solve (the exact discrete sum); surface and forces: FP64 tree-code, "
           "p=20, theta=0.4" if max(s.n for s in snaps) <= 4096 else "FP64 multipole solve, p=20, theta=0.4")
    kinds = {}
    for s in snaps:
        k = f"{s.meta.get('kind', 'snapshot')} {s.n}^2"
        kinds[k] = kinds.get(k, 0) + 1
    return {"best": best, "table": table, "tol": tol, "safety": safety, "reference": ref, "snapshots": kinds,
            "seconds": time.perf_counter() - t0}


def batch_representatives(snaps, largest=512):
    """The snapshots of a batch whose grids are no larger than ``largest``: the set a batch's
    setting is tuned on (every phase the batch holds at the small sizes; the errors of the
    multipole and tree-code truncation depend on the body's shape, not on the grid size)."""
    return [s for s in snaps if s.n <= largest]
