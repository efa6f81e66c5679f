"""The full-size cylinder workloads at the spec accuracy setting (p = 20, theta = 0.5,
near-field tile 16), checked on sampled outputs the oracle computes one by one (exact FP64
sums over all n^2 sources): the 1024^2 FP64 cylinder and the 2048^2 mixed cylinder.  The
configuration bench.py times (p = 12, theta = 0.75, tensor-core tile) is checked at full size
in tests/test_gpu_bench_setting.py."""
import numpy as np
import pytest

import oracle
from paper_1610_04398_gb300 import synth
from gpu_cases import force_err, rel_l2, run_gpu, run_oracle, worst_cell

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_04398_gb300 as pkg
    pkg.build()
    oracle.build()


def _sample(n, k, seed):
    rng = np.random.default_rng(seed)
    cells = rng.choice(n * n, size=k, replace=False)
    # always include the domain corners and a cell next to the body surface
    return np.unique(np.concatenate([cells, [0, n - 1, n * (n - 1), n * n - 1]]))


@pytest.mark.parametrize("n,precision,k", [(1024, "fp64", 768), (2048, "mixed", 384)])
def test_cylinder_full_size_sampled(n, precision, k):
    snap = synth.cylinder_flow(n, seed=2000)
    g = run_gpu(snap, precision, 20, 0.5)
    cells = _sample(n, k, 17)
    r = run_oracle(snap, cells=cells)
    tol = 1e-6 if precision == "fp64" else 1e-4
    e_cells = rel_l2(g["P"].ravel()[cells], r["P_cells"])
    e_surf = rel_l2(g["per_point"][:, 0], r["P_surf"])
    ed, el = force_err(g["forces"], r["forces"])
    w_cells = worst_cell(g["P"].ravel()[cells], r["P_cells"])
    w_surf = worst_cell(g["per_point"][:, 0], r["P_surf"])
    assert e_cells < tol and w_cells < tol, (e_cells, w_cells)
    assert e_surf < tol and w_surf < tol, (e_surf, w_surf)
    assert ed < tol and el < tol, (ed, el)
    # RHS everywhere (no sampling needed: it is local)
    e_f = np.max(np.abs(g["f"] - r["f"])) / np.max(np.abs(r["f"]))
    assert e_f < (1e-12 if precision == "fp64" else 1e-5), e_f
