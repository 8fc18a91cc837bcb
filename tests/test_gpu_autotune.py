"""Launch-shape tuning (fwr_plan_autotune, FWR_OPT_SHAPE, FWR_OPT_CTAS,
FWR_OPT_L2_PERSIST and the batch's shape): every candidate shape,
persistent-grid size and L2 window gives
bitwise the phase of the default launch (each frame's arithmetic is fixed;
only the layout of the work on the GPU changes), the tuner records its
choice in the cache and a second plan with the same key takes it from
there without timing."""

import json

import pytest

from paper_1705_04298_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fwr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04298_gb300 import fwr as m
    m.load()
    return m


@pytest.mark.parametrize("n,pad,k", [(80, 3.2, 3), (40, 3.2, 2), (30, 2.0, 4), (12, 1.25, 2)])
def test_every_shape_is_bitwise_the_default(fwr, n, pad, k):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    F = sms + 37
    sl, _, mask = synth.batch(n, 8, 3000 + n, 0.05)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat(F // 8 + 1, 1, 1, 1)[:F].contiguous()
    plan = fwr.Plan(mask, pad, fwr.LSQ)
    ref = plan.reconstruct(s, k).clone()
    for shape in (0, 1, 2):
        for ctas in (0, 1, sms // 2, sms + 5):
            plan.set_shape(shape)
            plan.set_ctas(ctas)
            out = plan.reconstruct(s, k)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (plan.N, shape, ctas)
    assert plan.status() == "FWR_OK"


def test_autotune_records_and_reuses(fwr, tmp_path):
    n, k = 80, 2
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sl, _, mask = synth.batch(n, 8, 3100, 0.05)
    F = sms
    s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat(F // 8 + 1, 1, 1, 1)[:F].contiguous()
    out = torch.empty((F, 256, 256), device="cuda")
    cache = tmp_path / "plan_tune.jsonl"
    plan = fwr.Plan(mask, 3.2, fwr.LSQ)
    ref = plan.reconstruct(s, k).clone()
    shape, ctas = plan.autotune(s, k, out, cache)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1
    e = json.loads(lines[0])
    assert (e["shape"], e["ctas"]) == (shape, ctas) and shape in (1, 2)
    assert e["l2_persist"] in (0, 1) and plan.l2_persist == e["l2_persist"]
    assert "drv" in e["key"] and "|N256" in e["key"]
    assert torch.equal(plan.reconstruct(s, k), ref)
    other = fwr.Plan(mask, 3.2, fwr.LSQ)
    assert other.autotune(s, k, out, cache) == (shape, ctas)
    assert other.l2_persist == e["l2_persist"]
    assert len(cache.read_text().strip().splitlines()) == 1  # from the cache, not re-timed


@pytest.mark.parametrize("n,pad,k", [(80, 3.2, 3), (160, 3.2, 2)])
def test_l2_window_is_bitwise_the_default(fwr, n, pad, k):
    """FWR_OPT_L2_PERSIST on the 256^2 and 512^2 slab plans: the same phase,
    bit for bit, with and without the persisting window, in both shapes."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    F = sms + 9
    sl, _, mask = synth.batch(n, 4, 3200 + n, 0.05)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat(F // 4 + 1, 1, 1, 1)[:F].contiguous()
    plan = fwr.Plan(mask, pad, fwr.LSQ)
    assert plan.l2_persist == 0
    ref = plan.reconstruct(s, k).clone()
    plan.set_l2_persist(1)
    assert plan.l2_persist == 1
    for shape in ((0, 1, 2) if plan.N == 256 else (0,)):
        plan.set_shape(shape)
        out = plan.reconstruct(s, k)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (plan.N, shape)
    plan.set_l2_persist(0)
    assert plan.l2_persist == 0
    assert torch.equal(plan.reconstruct(s, k), ref)
    fwr.l2_persist_reset(torch.cuda.current_device())
    assert torch.equal(plan.reconstruct(s, k), ref)
    assert plan.status() == "FWR_OK"


def test_l2_window_refused_without_slab_memory(fwr):
    """Grids of 128^2 and below run without working memory in global memory:
    the window is refused (FWR_ERR_UNSUPPORTED), and a value other than 0 or 1
    is an argument error; the plan still works afterwards."""
    plan = fwr.Plan(synth.pupil_mask(40), 3.2, fwr.LSQ)
    with pytest.raises(fwr.FwrError):
        plan.set_l2_persist(1)
    assert plan.l2_persist == 0
    big = fwr.Plan(synth.pupil_mask(80), 3.2, fwr.LSQ)
    lib = fwr.load()
    assert lib.fwr_plan_set_option(big._h, fwr.OPT_L2_PERSIST, 2.0) == 1
    assert lib.fwr_plan_set_option(big._h, fwr.OPT_L2_PERSIST, 0.5) == 1
    assert big.l2_persist == 0


def test_batch_shapes_bitwise(fwr):
    sizes = [(40, 3.2), (80, 3.2)]
    plans = [fwr.Plan(synth.pupil_mask(n), pad, fwr.LSQ) for n, pad in sizes]
    fp = [0, 1, 1, 0, 1]
    slopes, phases = [], []
    for f, pl in enumerate(fp):
        n = sizes[pl][0]
        slopes.append(torch.tensor(synth.frame(n, 50 + f, 0.05)["slopes"], dtype=torch.float32, device="cuda"))
        phases.append(torch.empty((plans[pl].N,) * 2, device="cuda"))
    batch = fwr.Batch(plans, fp, 2)
    sp, pp = fwr.Batch.pointer_table(slopes), fwr.Batch.pointer_table(phases)
    assert batch.shape == 2
    batch.run(sp, pp)
    torch.cuda.synchronize()
    ref = [p.clone() for p in phases]
    batch.set_shape(1)
    batch.run(sp, pp)
    torch.cuda.synchronize()
    for a, b in zip(phases, ref):
        assert torch.equal(a, b)
    with pytest.raises(fwr.FwrError):
        batch.set_shape(3)
