"""The 2048^2 mixed-precision cylinder in exactly the configuration bench.py times: order
p = 12, theta = 0.75 and the 128-leaf tensor-core near field (k_near_tc), the setting the
autotuner picks for this snapshot, with 2048 surface points lifted by 2h; the surface part at
every surface acceptance the autotuner may pick (0.6, 0.5, 0.45, 0.4).

Checked against the oracle (exact FP64 sums of Eq. greenSum over all n^2 sources, computed
one target at a time) at cells chosen where a tiling mistake would show: both sides of the
tensor-core tiles' seams (tiles of 8 x 16 leaves, i.e. 64 cells in x and 128 in y), the
four cells around tile corners, the corner cells of leaves, the domain's corners and edge
midpoints, a ring of cells next to the body, and 512 random cells; at every surface point;
and on drag and lift.  The whole grid is compared with the FP64 zero-padded FFT solve of the
same discrete sum (no truncation error; pinned to the oracle in tests/test_gpu_fft.py).
Bounds: relative L2 <= 1e-4 and worst cell max|dP| / max|P| <= 1e-4 (Appendix A.1,
Eq. greenSum; mixed-path tolerance 1e-4).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1610_04398_gb300 import api, synth
from gpu_cases import force_err, rel_l2, run_gpu, run_oracle, to_dev, worst_cell

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 2048
SETTING = dict(order=12, theta=0.75, tile=128)
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()
    oracle.build()


def structured_cells(n, centre=(0.3, 0.5), radius=0.05, seed=31):
    """Flat indices (j * n + i) of the cells listed in the module docstring."""
    rng = np.random.default_rng(seed)
    cells = set()
    for _ in range(24):
        x = 64 * int(rng.integers(1, n // 64))          # vertical seam between tiles
        y = int(rng.integers(0, n))
        cells |= {(x - 1, y), (x, y)}
        y = 128 * int(rng.integers(1, n // 128))        # horizontal seam
        x = int(rng.integers(0, n))
        cells |= {(x, y - 1), (x, y)}
    for _ in range(16):                                 # tile corners
        x, y = 64 * int(rng.integers(1, n // 64)), 128 * int(rng.integers(1, n // 128))
        cells |= {(x - 1, y - 1), (x, y - 1), (x - 1, y), (x, y)}
    for _ in range(32):                                 # leaf corners
        lx, ly = (int(v) for v in rng.integers(0, n // 8, 2))
        cells |= {(8 * lx + cx, 8 * ly + cy) for cx in (0, 7) for cy in (0, 7)}
    m = n - 1
    cells |= {(0, 0), (m, 0), (0, m), (m, m), (n // 2, 0), (0, n // 2), (m, n // 2), (n // 2, m)}
    h = 1.0 / n
    for k in range(64):                                 # just outside the body
        a = 2 * math.pi * k / 64
        r = radius + (1 + k % 4) * h
        cells.add((int((centre[0] + r * math.cos(a)) / h), int((centre[1] + r * math.sin(a)) / h)))
    flat = np.array(sorted(j * n + i for i, j in cells), np.int64)
    rand = rng.choice(n * n, size=512, replace=False)
    return np.unique(np.concatenate([flat, rand]))


def test_structured_cells_cover_seams_and_corners():
    c = structured_cells(N)
    i, j = c % N, c // N
    assert len(c) >= 384
    assert np.any((i % 64 == 63)) and np.any((i % 64 == 0) & (i > 0))
    assert np.any((j % 128 == 127)) and np.any((j % 128 == 0) & (j > 0))
    assert {0, N - 1, N * (N - 1), N * N - 1} <= set(c.tolist())


def test_bench_setting_2048_against_oracle_and_fft():
    snap = synth.cylinder_flow(N, seed=2000, n_surface=2048)
    g = run_gpu(snap, "mixed", **SETTING)
    plan = g["plan"]
    assert plan.info().near_kernel == 128  # the tensor-core near field ran
    cells = structured_cells(N)
    r = run_oracle(snap, cells=cells)
    Pg = g["P"].ravel()[cells]
    e_cells, w_cells = rel_l2(Pg, r["P_cells"]), worst_cell(Pg, r["P_cells"])
    print(f"2048^2 bench setting vs oracle: cells rel_l2 {e_cells:.2e} worst {w_cells:.2e} ({len(cells)} cells)")
    assert e_cells < TOL and w_cells < TOL, (e_cells, w_cells)
    from paper_1610_04398_gb300 import autotune
    for ts in autotune.DEFAULT_SURFACE_THETAS:
        gs = g if ts == 0.6 else run_gpu(snap, "mixed", **SETTING, theta_surface=ts)
        assert gs["plan"].info().theta_surface == ts
        e_surf, w_surf = rel_l2(gs["per_point"][:, 0], r["P_surf"]), worst_cell(gs["per_point"][:, 0], r["P_surf"])
        ed, el = force_err(gs["forces"], r["forces"])
        print(f"  surface theta {ts}: surface rel_l2 {e_surf:.2e} worst {w_surf:.2e}; drag {ed:.2e} lift {el:.2e}")
        assert e_surf < TOL and w_surf < TOL, (ts, e_surf, w_surf)
        assert ed < TOL and el < TOL, (ts, ed, el)
        if gs is not g:
            gs["plan"].destroy()
    e_f = np.max(np.abs(g["f"] - r["f"])) / np.max(np.abs(r["f"]))
    assert e_f < 1e-5, e_f
    # the whole grid against the FP64 FFT solve of the same discrete sum on the same inputs
    del r
    plan.destroy()
    p64 = api.Plan(N, snap.h, 12, 0.75, precision="fp64", lift=snap.lift, uinf=snap.uinf)
    fields = [to_dev(a, torch.float64) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    p64.rhs(*fields, snap.lam)
    Pf = torch.empty(N * N, dtype=torch.float64, device="cuda")
    p64.pressure_solve_fft(Pf)
    torch.cuda.synchronize()
    Pf = Pf.cpu().numpy()
    e_all, w_all = rel_l2(g["P"].ravel(), Pf), worst_cell(g["P"].ravel(), Pf)
    print(f"2048^2 bench setting vs FP64 FFT over all {N * N} cells: rel_l2 {e_all:.2e} worst {w_all:.2e}")
    assert e_all < TOL and w_all < TOL, (e_all, w_all)
    # where the largest difference sits: a seam or boundary effect would concentrate it
    k = int(np.argmax(np.abs(g["P"].ravel() - Pf)))
    print(f"largest difference at cell (i, j) = ({k % N}, {k // N})")
    p64.destroy()
