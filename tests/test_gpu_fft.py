"""The zero-padded FFT (Hockney) solve, pp_pressure_solve_fft, against the oracle's direct sum
of Eq. greenSum, and as a whole-grid check of the multipole solve.

Tolerance (derived from the FFT's rounding, not fitted): a transform of N = M^2 points in
precision eps has relative l2 error ~ eps log2 N (Higham, Accuracy and Stability of Numerical
Algorithms, Sec. 24.1), spread evenly over the spectrum; multiplied by the kernel spectrum
K^ it becomes, per output cell, an rms error ~ eps log2 N ||q||_2 ||K||_2 / M (Parseval:
sum |K^|^2 = M^2 ||K||_2^2).  The tests allow 4x that for the rms and 40x for the maximum,
with ||K||_2 over the (2n - 1)^2 kernel table of the sum."""
import math

import numpy as np
import pytest

import oracle
from paper_1610_04398_gb300 import api, synth
from gpu_cases import rel_l2, run_gpu, to_dev, worst_cell

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = {"fp64": 2.0 ** -53, "mixed": 2.0 ** -24}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()
    oracle.build()


def _fft_pressure(snap, precision, plan=None):
    """pp_rhs then pp_pressure_solve_fft; returns (P n x n float64, q n x n float64, plan)."""
    if plan is None:
        plan = api.Plan(snap.n, snap.h, 12, 0.75, x0=snap.x0, y0=snap.y0, precision=precision,
                        lift=snap.lift, uinf=snap.uinf)
    dt = plan.dtype
    fields = [to_dev(a, dt) for a in (snap.u, snap.v, snap.chi, snap.usx, snap.usy)]
    f = torch.empty(snap.n * snap.n, dtype=dt, device="cuda")
    plan.rhs(*fields, snap.lam, f_out=f)
    P = torch.empty(snap.n * snap.n, dtype=dt, device="cuda")
    plan.pressure_solve_fft(P)
    torch.cuda.synchronize()
    # q = f h^2 in the plan's precision, as the source kernels form it
    npdt = np.float64 if dt == torch.float64 else np.float32
    hh = npdt(snap.h) * npdt(snap.h)
    q = (f.cpu().numpy().reshape(snap.n, snap.n) * hh).astype(np.float64)
    return P.double().cpu().numpy().reshape(snap.n, snap.n), q, plan


def _bound(q, h, precision):
    """rms error bound of the FFT convolution (module docstring)."""
    n = q.shape[0]
    M = 2 * n
    d = np.arange(-(n - 1), n)
    DX, DY = np.meshgrid(d, d)
    K = np.log(np.maximum(h * np.hypot(DX, DY), oracle.rho_h(h))) / (2 * math.pi)
    return 4 * EPS[precision] * math.log2(M * M) * np.linalg.norm(q) * np.linalg.norm(K) / M


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [8, 16, 32, 64, 128, 256])
def test_fft_solve_matches_oracle_on_every_cell(n, precision):
    """Every radix schedule of the line transforms: 2n = 16 (16), 32 (16, 2), 64 (16, 4),
    128 (16, 8), 256 (16, 16), 512 (16, 16, 2); q taken from the GPU's own source so the
    comparison isolates the solve (the source has its own parity tests)."""
    snap = synth.cylinder_flow(n, seed=2000 + n)
    P, q, _ = _fft_pressure(snap, precision)
    X, Y = synth.cell_centres(n, snap.h, snap.x0, snap.y0)
    ref = oracle.green_sum_grid(q, snap.h, X.ravel(), Y.ravel(), snap.x0, snap.y0).reshape(n, n)
    err = P - ref
    b = _bound(q, snap.h, precision)
    rms = float(np.sqrt(np.mean(err ** 2)))
    print(f"n={n} {precision}: rms {rms:.3e} max {np.max(np.abs(err)):.3e} bound {b:.3e} "
          f"rel_l2 {rel_l2(P, ref):.3e}")
    assert rms <= b, (rms, b)
    assert np.max(np.abs(err)) <= 10 * b


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fft_solve_swimmer_matches_oracle(precision):
    snap = synth.swimmer_snapshot(256, phase=0.3, seed=4001, n_surface=1024)
    P, q, _ = _fft_pressure(snap, precision)
    X, Y = synth.cell_centres(256, snap.h, snap.x0, snap.y0)
    ref = oracle.green_sum_grid(q, snap.h, X.ravel(), Y.ravel(), snap.x0, snap.y0).reshape(256, 256)
    rms = float(np.sqrt(np.mean((P - ref) ** 2)))
    assert rms <= _bound(q, snap.h, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fft_solve_full_size_sampled(precision):
    """2048^2 (the size the bench times): sampled cells against the oracle's exact sums, and
    the whole multipole-solved grid against the FFT-solved one (two independent algorithms
    for the same discrete sum; the FMM's truncation error dominates the difference)."""
    n = 2048
    snap = synth.cylinder_flow(n, seed=2000)
    P, q, plan = _fft_pressure(snap, precision)
    rng = np.random.default_rng(23)
    cells = np.unique(np.concatenate([rng.choice(n * n, 256, replace=False), [0, n - 1, n * n - 1]]))
    X, Y = synth.cell_centres(n, snap.h, snap.x0, snap.y0)
    ref = oracle.green_sum_grid(q, snap.h, X.ravel()[cells], Y.ravel()[cells], snap.x0, snap.y0)
    err = P.ravel()[cells] - ref
    b = _bound(q, snap.h, precision)
    print(f"2048 {precision}: sampled rms {np.sqrt(np.mean(err ** 2)):.3e} bound {b:.3e}")
    assert float(np.sqrt(np.mean(err ** 2))) <= b
    # the FMM (same plan, same source) over the whole grid
    Pm = torch.empty(n * n, dtype=plan.dtype, device="cuda")
    plan.pressure_solve(Pm)
    torch.cuda.synchronize()
    Pm = Pm.double().cpu().numpy().reshape(n, n)
    e_fmm, w_fmm = rel_l2(Pm, P), worst_cell(Pm, P)
    print(f"2048 {precision}: FMM (p=12, theta=0.75) vs FFT over all cells rel_l2 {e_fmm:.3e} worst {w_fmm:.3e}")
    assert e_fmm < 1e-4 and w_fmm < 1e-4


def test_fmm_fp64_whole_grid_against_fft_fp64():
    """The FP64 multipole solve at p = 20, theta = 0.5 on every cell of a 1024^2 grid, checked
    against the FP64 FFT solve of the same source (the oracle can only sample this size)."""
    snap = synth.cylinder_flow(1024, seed=2000)
    g = run_gpu(snap, "fp64", 20, 0.5)
    P, q, _ = _fft_pressure(snap, "fp64")
    assert np.array_equal(q, g["f"] * (snap.h * snap.h))
    assert rel_l2(g["P"], P) < 1e-6
    assert worst_cell(g["P"], P) < 1e-6


def test_fft_solve_state_errors_repeatability_and_capture():
    n = 256
    snap = synth.cylinder_flow(n, seed=5)
    plan = api.Plan(n, snap.h, 12, 0.75, precision="mixed", lift=snap.lift)
    P = torch.empty(n * n, dtype=plan.dtype, device="cuda")
    with pytest.raises(api.PPError) as ei:
        plan.pressure_solve_fft(P)  # no source yet
    assert ei.value.status == api.PP_ERR_STATE
    P1, _, plan = _fft_pressure(snap, "mixed", plan)
    P2, _, _ = _fft_pressure(snap, "mixed", plan)
    assert np.array_equal(P1, P2)  # fixed arithmetic order: bitwise repeatable
    # after the first call the solve allocates nothing and can be captured
    out = torch.zeros(n * n, dtype=plan.dtype, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.pressure_solve_fft(out)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.double().cpu().numpy().reshape(n, n), P1)
    big = api.Plan(8192, 1.0 / 8192, 12, 0.75, precision="mixed")
    with pytest.raises(api.PPError) as ei:
        big.pressure_solve_fft(torch.empty(8192 * 8192, dtype=big.dtype, device="cuda"))
    assert ei.value.status == api.PP_ERR_ARG
    big.destroy()
