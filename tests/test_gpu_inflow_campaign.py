"""End-to-end learned-inflow campaign on a small domain (GPU): precursor
record, generator training, the four flag runs (grid-resolved, generated,
uniform, white-noise inflow) and their comparison. Checks that every stage
runs through the library and yields finite statistics; the physics is only
meaningful at the production size."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08246_gb300 import binding, build
    build.build()
    return binding.load()


def test_small_campaign_runs(lib):
    from paper_2103_08246_gb300 import inflow, inputs
    h = 1.0 / 16.0
    base = inputs.PRODUCTION.replace(name="campaign-128x32x128", nx=128, ny=32, nz=128, lx=128 * h,
                                     ly=32 * h, lz=128 * h, flag_ns=17, flag_nt=17, flag_x_le=3.0)
    # 150 steps carry the bar wakes past x = 2 at this spacing
    out = inflow.campaign(spin=150, record=60, train_steps=10, run_steps=200, discard=150, blocks=1, batch=2,
                          base=base, sample_every=5, log=lambda *a: None, stride=2)
    json.dumps(out, default=str)
    assert out["train"]["n_params"] == inputs.generator_param_count(128, 1, 6)
    assert all(np.isfinite(out["train"]["train"])) and all(np.isfinite(out["train"]["val"]))
    runs = out["runs"]
    for key in ("R", "G", "U", "W"):
        assert len(runs[key]["tu"]) == 3 and all(np.isfinite(runs[key]["tu"]))
        assert np.isfinite(runs[key]["strouhal"]) and np.isfinite(runs[key]["y_rms"])
    # turbulence only where the inflow or the bars carry it
    assert runs["R"]["tu"][0] > 3 * runs["U"]["tu"][0]
    assert runs["W"]["tu"][0] > 3 * runs["U"]["tu"][0]
    assert runs["G"]["tu"][0] > 3 * runs["U"]["tu"][0]
    assert "G_within_bounds" in out["comparison"]
