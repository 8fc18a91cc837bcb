"""The allocation-free entry point for 256x256 grids (fwr_reconstruct_static).

Some callers cannot allocate device memory once they run: a real-time control
loop that forbids allocations after start-up, or a process whose device memory
belongs to another allocator. For them the library offers a variant of the
256x256 kernel whose working memory is a static array inside the library. This
test calls it through the C ABI and checks that two calls in a row give the
same phase as the regular entry point: bitwise, since it is the same kernel on
the same tables, and within the FP32 bounds of the other GPU tests against the
FP64 oracle. It also checks that a plan with the Hudgin extension gets the
same result from both entry points, and that requests the array cannot serve
(too many frames in flight, another grid size, the DFT-as-GEMM transform) are
refused.

It runs last on purpose (file name), and passes both alone in a fresh process
and after the other tests.
"""

import pytest

import oracle
from paper_1705_04298_gb300 import synth
from parity_check import FP32_RMS, within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fwr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04298_gb300 import fwr as m
    m.load()
    return m


def test_static_scratch_matches_regular_entry_point(fwr):
    n, pad, k, F = 80, 3.2, 3, 37
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sl, _, mask = synth.batch(n, F, 515, 0.05)
    plan = fwr.Plan(mask, pad, fwr.WIENER, 0.05 ** 2, r0p, L0p)
    assert plan.N == 256
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    ref = plan.reconstruct(s, k)
    a = plan.reconstruct_static(s, k, ctas=fwr.STATIC_SCRATCH_GRIDS)
    b = plan.reconstruct_static(s, k, ctas=5)   # second call in a row, reusing the array
    torch.cuda.synchronize()
    assert torch.isfinite(a).all() and torch.isfinite(b).all()
    assert torch.equal(a, ref)
    assert torch.equal(b, ref)
    for f in (0, F - 1):
        orc, _ = oracle.reconstruct(sl[f], mask, pad, k, oracle.FILTER_WIENER, 0.05 ** 2, r0p, L0p)
        assert within(b[f].cpu().numpy(), orc, FP32_RMS, where="static f=%d" % f)
    assert plan.status() == "FWR_OK"


def test_static_scratch_with_hudgin_extension(fwr):
    n, pad, k, F = 128, 2.0, 1, 6
    sl, _, mask = synth.batch(n, F, 516, 0.05)
    plan = fwr.Plan(mask, pad, fwr.LSQ)
    plan.set_extension(fwr.EXT_HUDGIN)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    ref = plan.reconstruct(s, k)
    a = plan.reconstruct_static(s, k, ctas=3)
    b = plan.reconstruct_static(s, k, ctas=3)
    torch.cuda.synchronize()
    assert torch.equal(a, ref) and torch.equal(b, ref)


def test_static_scratch_refuses_what_it_cannot_hold(fwr):
    n = 80
    mask = synth.pupil_mask(n)
    plan = fwr.Plan(mask, 3.2, fwr.LSQ)
    s = torch.zeros((2, 2, n, n), dtype=torch.float32, device="cuda")
    for ctas in (0, fwr.STATIC_SCRATCH_GRIDS + 1):
        with pytest.raises(fwr.FwrError) as e:
            plan.reconstruct_static(s, 1, ctas=ctas)
        assert e.value.code == 1
    small = fwr.Plan(synth.pupil_mask(40), 3.2, fwr.LSQ)
    with pytest.raises(fwr.FwrError) as e:
        small.reconstruct_static(torch.zeros((1, 2, 40, 40), device="cuda"), 1)
    assert e.value.code == 2
    plan.set_transform(fwr.TRANSFORM_DFT_BF16X3)
    with pytest.raises(fwr.FwrError) as e:
        plan.reconstruct_static(s, 1)
    assert e.value.code == 2
