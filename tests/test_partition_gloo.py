"""Multi-GPU decomposition logic on CPU ranks (no GPU).

* Replicas: round-robin sharding covers every item once; the job rate is all units
  over the slowest rank.
* One grid over several ranks: leaf-row bands, near-field and multipole-to-local halos
  and the shared (all-reduced) levels cover every source a rank's targets need; with
  gloo ranks that really exchange halo rows point-to-point, the banded near field
  equals the single-domain near field.
"""
import math
import os
import socket

import numpy as np
import pytest

from paper_1610_04398_gb300 import api, partition, _build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    api.load()


def _lists(theta):
    return api.pp_near_offsets(theta), [api.pp_m2l_entries(theta, c) for c in range(4)]


def test_replica_sharding_and_weak_scaling_value():
    for world in (1, 2, 3, 8):
        shards = [partition.replica_shard(64, r, world) for r in range(world)]
        flat = sorted(x for s in shards for x in s)
        assert flat == list(range(64))
    assert partition.weak_scaling_value([10, 10], [2.0, 2.5]) == 20 / 2.5


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("theta", [0.5, 0.6, 0.4])
def test_halos_cover_every_needed_source(world, theta):
    nL = 32
    near, m2l = _lists(theta)
    L = int(math.log2(nL))
    bands = partition.leaf_row_bands(nL, world)
    assert bands[0][0] == 0 and bands[-1][1] == nL
    assert all(bands[i][1] == bands[i + 1][0] for i in range(world - 1))
    for r in range(world):
        gp = partition.GridPartition(nL, world, r, near, m2l)
        r0, r1 = gp.band()
        have = set(range(r0, r1)) | set(gp.near_halo_rows())
        for ly in range(r0, r1):
            for dx, dy in near:
                if 0 <= ly + dy < nL:
                    assert ly + dy in have
        shared = set(gp.shared_levels())
        assert L not in shared or world > nL
        for lev in range(2, L + 1):
            if lev in shared:
                continue
            b0, b1 = gp.box_rows(lev)
            halo = gp.m2l_halo_rows(lev)
            side = 1 << lev
            for by in range(b0, b1):
                for bx in range(side):
                    c = (bx & 1) + 2 * (by & 1)
                    for dx, dy, kind in m2l[c]:
                        sl = lev if kind == 0 else lev - 1
                        sx, sy = (bx + dx, by + dy) if kind == 0 else ((bx >> 1) + dx, (by >> 1) + dy)
                        if not (0 <= sx < (1 << sl) and 0 <= sy < (1 << sl)):
                            continue
                        own = gp.box_rows(sl)
                        if own is None or sl in shared:
                            continue  # all-reduced level: available everywhere
                        assert own[0] <= sy < own[1] or sy in halo.get(sl, [])
        # every level below the shared ones is owned by whole box rows
        assert all(gp.box_rows(lev) is not None for lev in range(max(shared, default=-1) + 1, L + 1))


def _near_field(q, near, h):
    """Near-field Green's sum per leaf with the cell-offset log table (test-side)."""
    n = q.shape[0]
    nL = n // 8
    rh = h * math.exp(math.pi / 4 - 1.5 - 0.5 * math.log(2))
    c = np.arange(8)
    out = np.zeros_like(q)
    for dx, dy in near:
        ox = 8 * dx + c[None, :] - c[:, None]   # [t, s] along x
        oy = 8 * dy + c[None, :] - c[:, None]
        r = h * np.sqrt(ox[None, :, None, :] ** 2 + oy[:, None, :, None] ** 2)  # [ty, tx, sy, sx]
        K = np.log(np.maximum(r, rh)).reshape(64, 64)
        for LY in range(nL):
            if not 0 <= LY + dy < nL:
                continue
            for LX in range(nL):
                if not 0 <= LX + dx < nL:
                    continue
                src = q[8 * (LY + dy):8 * (LY + dy) + 8, 8 * (LX + dx):8 * (LX + dx) + 8].reshape(64)
                out[8 * LY:8 * LY + 8, 8 * LX:8 * LX + 8] += (K @ src).reshape(8, 8)
    return out / (2 * math.pi)


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist
    import torch
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        nL, theta = 16, 0.5
        n, h = 8 * nL, 1.0 / (8 * nL)
        near, m2l = _lists(theta)
        q_global = np.random.default_rng(11).normal(size=(n, n))
        gp = partition.GridPartition(nL, world, rank, near, m2l)
        r0, r1 = gp.band()
        local = np.zeros((n, n))
        local[8 * r0:8 * r1] = q_global[8 * r0:8 * r1]   # only the own band is known
        plans = [None] * world
        dist.all_gather_object(plans, gp.exchange_plan())
        # point-to-point halo exchange of q leaf rows: send what others ask of us
        reqs = []
        for other in range(world):
            if other == rank:
                continue
            want = plans[other][("q", gp.levels)].get(rank, [])
            for y in want:
                buf = torch.from_numpy(np.ascontiguousarray(local[8 * y:8 * y + 8]))
                reqs.append(dist.isend(buf, dst=other, tag=y))
        for owner, rows in plans[rank][("q", gp.levels)].items():
            for y in rows:
                buf = torch.empty(8, n, dtype=torch.float64)
                dist.recv(buf, src=owner, tag=y)
                local[8 * y:8 * y + 8] = buf.numpy()
        for rq in reqs:
            rq.wait()
        mine = _near_field(local, near, h)[8 * r0:8 * r1]
        parts = [None] * world
        dist.all_gather_object(parts, (r0, r1, mine))
        if rank == 0:
            full = _near_field(q_global, near, h)
            err = max(float(np.max(np.abs(p[2] - full[8 * p[0]:8 * p[1]]))) for p in parts)
            with open(result_path, "w") as f:
                f.write(repr(err))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_banded_near_field_with_gloo_halo_exchange(tmp_path, world):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = tmp_path / "err.txt"
    mp.spawn(_rank_main, args=(world, port, str(out)), nprocs=world, join=True)
    err = float(out.read_text())
    assert err < 1e-12


# ------------------------------------------------------------- the far field in bands
_zc = lambda l, bx, by: ((bx + 0.5) + 1j * (by + 0.5)) / (1 << l)  # noqa: E731


def _upward(q, nL, p, rows, shared=(), allreduce=None):
    """Multipoles as one rank holds them after its upward pass on the leaf rows ``rows``
    (oracle P2M on its leaves, M2M up its own box rows); at the deepest of the ``shared``
    levels (those whose boxes straddle some band, the same on every rank) each rank has a
    partial sum (the children it holds), which ``allreduce`` completes, and every rank forms
    the levels above from complete data.  {level: (S, A)}."""
    import oracle
    n = q.shape[0]
    L = int(round(math.log2(nL)))
    h = 1.0 / n
    r0, r1 = rows
    S = {l: np.zeros((1 << l, 1 << l)) for l in range(L + 1)}
    A = {l: np.zeros((1 << l, 1 << l, p), np.complex128) for l in range(L + 1)}
    cx = (np.arange(8) + 0.5) * h
    for LY in range(r0, r1):
        for LX in range(nL):
            zs = (LX * 8 * h + cx[None, :]) + 1j * (LY * 8 * h + cx[:, None])
            S[L][LY, LX], A[L][LY, LX] = oracle.p2m(q[8 * LY:8 * LY + 8, 8 * LX:8 * LX + 8], zs, _zc(L, LX, LY), p)
    full = False
    for l in range(L - 1, -1, -1):
        sh = L - l
        own = None if l in shared else (r0 >> sh, r1 >> sh)
        for by in (range(1 << l) if (own is None or full) else range(*own)):
            for bx in range(1 << l):
                for c in range(4):  # children a rank does not hold are zero and add nothing
                    ux, uy = 2 * bx + (c & 1), 2 * by + (c >> 1)
                    s_c, beta = oracle.m2m(S[l + 1][uy, ux], A[l + 1][uy, ux], _zc(l + 1, ux, uy), _zc(l, bx, by))
                    S[l][by, bx] += s_c
                    A[l][by, bx] += beta
        if own is None and not full:
            S[l], A[l] = allreduce(l, S[l], A[l])
            full = True
    return {l: (S[l], A[l]) for l in range(L + 1)}


def _downward(mp, nL, m2l, p, rows, n, shared=()):
    """Translations of the interaction entries into the locals of the boxes over the leaf rows
    ``rows`` (every box at the levels that straddle bands), local-to-local shifts down, and the
    local expansion at the band's cells: the far field on the band's rows."""
    import oracle
    L = int(round(math.log2(nL)))
    h = 1.0 / n
    r0, r1 = rows
    loc = {l: np.zeros((1 << l, 1 << l, p + 1), np.complex128) for l in range(L + 1)}
    for l in range(2, L + 1):
        sh = L - l
        own = None if l in shared else (r0 >> sh, r1 >> sh)
        for by in (range(1 << l) if own is None else range(*own)):
            for bx in range(1 << l):
                c = (bx & 1) + 2 * (by & 1)
                if l >= 3:
                    loc[l][by, bx] += oracle.l2l(loc[l - 1][by >> 1, bx >> 1], _zc(l - 1, bx >> 1, by >> 1),
                                                 _zc(l, bx, by))
                for dx, dy, kind in m2l[c]:
                    sl = l if kind == 0 else l - 1
                    sx, sy = (bx + dx, by + dy) if kind == 0 else ((bx >> 1) + dx, (by >> 1) + dy)
                    if 0 <= sx < (1 << sl) and 0 <= sy < (1 << sl):
                        S, A = mp[sl]
                        loc[l][by, bx] += oracle.m2l(S[sy, sx], A[sy, sx], _zc(sl, sx, sy), _zc(l, bx, by))
    out = np.zeros((8 * (r1 - r0), n))
    cx = (np.arange(8) + 0.5) * h
    for LY in range(r0, r1):
        for LX in range(nL):
            zs = (LX * 8 * h + cx[None, :]) + 1j * (LY * 8 * h + cx[:, None])
            out[8 * (LY - r0):8 * (LY - r0) + 8, 8 * LX:8 * LX + 8] = oracle.l2p(loc[L][LY, LX], _zc(L, LX, LY), zs)
    return out


def _rank_far(rank, world, port, result_path):
    import torch.distributed as dist
    import torch
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        nL, theta, p = 16, 0.5, 8
        n = 8 * nL
        near, m2l = _lists(theta)
        q_global = np.random.default_rng(12).normal(size=(n, n)) / n ** 2
        gp = partition.GridPartition(nL, world, rank, near, m2l)
        r0, r1 = gp.band()
        local = np.zeros((n, n))
        local[8 * r0:8 * r1] = q_global[8 * r0:8 * r1]   # only the own band is known
        plans = [None] * world
        dist.all_gather_object(plans, gp.exchange_plan())

        def allreduce(level, S, A):  # partial multipoles of the boxes that straddle bands, summed
            buf = torch.from_numpy(np.concatenate([S.ravel(), A.real.ravel(), A.imag.ravel()]))
            dist.all_reduce(buf)
            b = buf.numpy()
            m = S.size
            return b[:m].reshape(S.shape).copy(), (b[m:m + A.size] + 1j * b[m + A.size:]).reshape(A.shape)

        shared = set(gp.shared_levels())
        mp = _upward(local, nL, p, (r0, r1), shared, allreduce)
        reqs = []
        for other in range(world):  # the multipole rows the other ranks' plans ask of this rank
            if other == rank:
                continue
            for (kind, sl), owners in plans[other].items():
                if kind != "multipole":
                    continue
                for y in owners.get(rank, []):
                    S, A = mp[sl]
                    buf = torch.from_numpy(np.concatenate([S[y], A[y].real.ravel(), A[y].imag.ravel()]))
                    reqs.append((dist.isend(buf, dst=other, tag=int(1000 * sl + y)), buf))
        for (kind, sl), owners in plans[rank].items():
            if kind != "multipole":
                continue
            side = 1 << sl
            for owner, ys in owners.items():
                for y in ys:
                    buf = torch.empty(side + 2 * side * p, dtype=torch.float64)
                    dist.recv(buf, src=owner, tag=int(1000 * sl + y))
                    b = buf.numpy()
                    mp[sl][0][y] = b[:side]
                    mp[sl][1][y] = (b[side:side + side * p] + 1j * b[side + side * p:]).reshape(side, p)
        for rq, _ in reqs:
            rq.wait()
        far = _downward(mp, nL, m2l, p, (r0, r1), n, shared)
        parts = [None] * world
        dist.all_gather_object(parts, (r0, r1, far))
        if rank == 0:
            ref = _downward(_upward(q_global, nL, p, (0, nL)), nL, m2l, p, (0, nL), n)
            err = max(float(np.max(np.abs(pt[2] - ref[8 * pt[0]:8 * pt[1]]))) for pt in parts) / np.max(np.abs(ref))
            with open(result_path, "w") as f:
                f.write(repr(float(err)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_banded_far_field_with_multipole_halos_and_allreduce(tmp_path, world):
    """The far field of the one-grid split: each gloo rank forms its band's multipoles, the
    first level whose boxes straddle bands is completed by an all-reduce of the partial
    multipoles, the multipole rows the rank's interaction lists reach are exchanged
    point-to-point (GridPartition.exchange_plan), and the rank's translations and local
    evaluation then reproduce the single-domain far field on its band (to rounding: the same
    steps, summed in another order)."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = tmp_path / "err.txt"
    mp.spawn(_rank_far, args=(world, port, str(out)), nprocs=world, join=True)
    err = float(out.read_text())
    assert err < 1e-12, err
