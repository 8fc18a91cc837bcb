"""The paper's open-loop trends (Sec. 4) reproduced with the library on
seeded synthetic frames: 40x40 lenslets on a 128^2 grid, noise-free slopes
for the residual, unit white noise for the propagation coefficient. What the
paper shows as figures is checked as orderings with margins."""

import numpy as np
import pytest

from paper_1705_04298_gb300 import diagnostics as dg
from paper_1705_04298_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_LENSLETS, PAD = 40, 3.2


@pytest.fixture(scope="module")
def fwr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04298_gb300 import fwr as m
    m.load()
    return m


def reconstructor(fwr, mask, ext, k, periodic):
    plan = fwr.Plan(mask, PAD, fwr.LSQ, 0.0, 1.0, 1.0, periodic)
    plan.set_extension(ext)

    def run(slopes):
        s = torch.tensor(np.asarray(slopes), dtype=torch.float32, device="cuda")
        return plan.reconstruct(s, k).cpu().numpy()
    return run


def test_residual_trends(fwr):
    sl, truth, mask = synth.batch(N_LENSLETS, 200, 5000, 0.0)
    cm = dg.corner_mask(mask)
    bins = np.array([0.0, 0.05, 0.5001])
    res = {}
    for name, ext, k, per in (("none", fwr.EXT_ZERO, 0, 2), ("hudgin", fwr.EXT_HUDGIN, 0, 0),
                              ("gerch3", fwr.EXT_ZERO, 3, 2), ("gerch3_per", fwr.EXT_ZERO, 3, 0)):
        est = dg.pupil_corners(reconstructor(fwr, mask, ext, k, per)(sl), N_LENSLETS)
        f, psd = dg.residual_psd(est, truth, cm, bins=bins)
        res[name] = psd
    # without extension the aperture's cut-off leaves most of the error at the
    # lowest frequencies; every extension removes most of it
    for name in ("hudgin", "gerch3", "gerch3_per"):
        assert res["none"][0] > 10 * res[name][0], name
    # with the periodic condition, 3 Gerchberg iterations beat the Hudgin
    # extension and 3 iterations without it at low frequencies
    assert res["gerch3_per"][0] < 0.7 * res["hudgin"][0]
    assert res["gerch3_per"][0] < 0.5 * res["gerch3"][0]


def test_noise_propagation_trends(fwr):
    mask = synth.pupil_mask(N_LENSLETS)
    c = {}
    for name, ext, k, per in (("hudgin", fwr.EXT_HUDGIN, 0, 0), ("g1", fwr.EXT_ZERO, 1, 2),
                              ("g1_per", fwr.EXT_ZERO, 1, 0), ("g3", fwr.EXT_ZERO, 3, 2),
                              ("g3_per", fwr.EXT_ZERO, 3, 0), ("g10_per", fwr.EXT_ZERO, 10, 0)):
        c[name] = dg.noise_propagation(reconstructor(fwr, mask, ext, k, per), mask, 256, 1)
    # the Gerchberg extension propagates less noise than the Hudgin extension
    assert c["g3_per"] < 0.7 * c["hudgin"]
    # the periodic condition raises it slightly (same noise realisations)
    assert c["g1"] < c["g1_per"] and c["g3"] < c["g3_per"]
    # and so do more iterations
    assert c["g1_per"] < c["g3_per"] < c["g10_per"]
