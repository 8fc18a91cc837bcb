"""What the trained warm start gains: on held-out seeded frames (40x40
lenslets, 128^2 grid, 0.05 rad noise, Wiener), the network followed by one or
two Gerchberg iterations must reconstruct far closer to the true phase than
the same number of plain iterations, and come close to ten plain iterations.
The committed weights were trained on the GPU by the library's own kernels
(paper_1705_04298_gb300/learned.py; report beside the weights)."""

import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fwr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04298_gb300 import fwr as m
    m.load()
    return m


def test_trained_warm_start_gain(fwr):
    from paper_1705_04298_gb300 import learned, synth
    assert os.path.exists(learned.WEIGHTS)
    F = 128
    net = learned.load_net(fwr, learned.WEIGHTS, max_batch=F)
    slopes, truth = learned.frames(F, learned.EVAL_SEED0, learned.EVAL_SIGMA)
    mask = synth.pupil_mask(learned.N_LENSLETS)
    plan = learned.make_plan(fwr, fwr.WIENER, learned.EVAL_SIGMA)
    phase = torch.empty((F, 128, 128), device="cuda")
    res = {}
    for k in (1, 2, 10):
        plan.reconstruct(slopes, k, phase)
        res["plain%d" % k] = learned.residual_rms(fwr, phase, truth, mask)
    warm = net.forward(plan, slopes)
    for k in (1, 2):
        plan.reconstruct(slopes, k, phase, ext_init=warm)
        res["learned%d" % k] = learned.residual_rms(fwr, phase, truth, mask)
    print(res)
    assert res["learned1"] < 0.4 * res["plain1"]
    assert res["learned2"] < 0.6 * res["plain2"]
    assert res["learned2"] < 1.35 * res["plain10"]
