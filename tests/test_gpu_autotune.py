"""The autotuner's chosen mixed-precision setting meets the accuracy bound against the
FP64 direct sum (oracle), not only against its own FP64 GPU reference."""
import numpy as np
import pytest

import oracle
from paper_1610_04398_gb300 import autotune, synth
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


def test_autotuned_setting_meets_tolerance_against_oracle():
    snap = synth.cylinder_flow(512, seed=2000)
    res = autotune.autotune(snap, steps=2)
    best = res["best"]
    assert best["ok"], res["table"]
    stage1 = [r for r in res["table"] if r["stage"] == 1]
    assert len(stage1) == (len(autotune.DEFAULT_ORDERS) * len(autotune.DEFAULT_THETAS) * len(autotune.DEFAULT_TILES))
    assert len(res["table"]) - len(stage1) <= 3 * len(autotune.DEFAULT_SURFACE_THETAS)
    g = run_gpu(snap, "mixed", best["order"], best["theta"], tile=best["tile"], theta_surface=best["theta_surface"])
    rng = np.random.default_rng(5)
    cells = rng.choice(512 * 512, size=512, replace=False)
    r = run_oracle(snap, cells=cells)
    assert rel_l2(g["P"].ravel()[cells], r["P_cells"]) < 1e-4
    assert worst_cell(g["P"].ravel()[cells], r["P_cells"]) < 1e-4
    assert rel_l2(g["per_point"][:, 0], r["P_surf"]) < 1e-4
    assert worst_cell(g["per_point"][:, 0], r["P_surf"]) < 1e-4
    ed, el = force_err(g["forces"], r["forces"])
    assert ed < 1e-4 and el < 1e-4
