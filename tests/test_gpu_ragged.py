"""Ragged batches on the GPU: one launch over 128^2 and 256^2 frames of four
plans (40, 64, 80 and 128 lenslets across) must give, frame by frame, the
result of the per-plan entry point (same per-frame code: bitwise) and match
the FP64 oracle; the launch replays identically from a CUDA graph; the
autotuner's cache round-trips."""

import json

import numpy as np
import pytest

import oracle
from paper_1705_04298_gb300 import synth
from parity_check import within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
SIZES = [(40, 3.2), (64, 2.0), (80, 3.2), (128, 2.0)]  # -> 128, 128, 256, 256


@pytest.fixture(scope="module")
def fwr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04298_gb300 import fwr as m
    m.load()
    return m


def make_batch(fwr, per_size, k, seed=7):
    plans = [fwr.Plan(synth.pupil_mask(n), pad, fwr.LSQ) for n, pad in SIZES]
    rng = np.random.default_rng(seed)
    frame_plan = rng.permutation(np.repeat(np.arange(len(SIZES)), per_size))
    slopes, phases, host = [], [], []
    for f, pl in enumerate(frame_plan):
        n = SIZES[pl][0]
        fr = synth.frame(n, 9000 + f, 0.05)
        host.append(fr["slopes"])
        slopes.append(torch.tensor(fr["slopes"], dtype=torch.float32, device="cuda"))
        N = plans[pl].N
        phases.append(torch.empty((N, N), dtype=torch.float32, device="cuda"))
    batch = fwr.Batch(plans, frame_plan, k)
    return plans, batch, frame_plan, host, slopes, phases


def test_ragged_matches_per_plan_and_oracle(fwr):
    k = 3
    plans, batch, frame_plan, host, slopes, phases = make_batch(fwr, 5, k)
    sp, pp = fwr.Batch.pointer_table(slopes), fwr.Batch.pointer_table(phases)
    batch.run(sp, pp)
    torch.cuda.synchronize()
    checked = set()
    for f, pl in enumerate(frame_plan):
        ref = plans[pl].reconstruct(slopes[f][None], k)[0]
        torch.cuda.synchronize()
        assert torch.equal(phases[f], ref), f
        if pl not in checked:
            n, pad = SIZES[pl]
            orc, _ = oracle.reconstruct(host[f], synth.pupil_mask(n), pad, k, oracle.FILTER_LSQ)
            assert within(phases[f].cpu().numpy(), orc, FP32_TOL, where="N=%d" % plans[pl].N)
            checked.add(pl)
    assert len(checked) == len(SIZES)


def test_ragged_graph_replay_and_schedules(fwr):
    k = 2
    plans, batch, frame_plan, host, slopes, phases = make_batch(fwr, 40, k, seed=11)
    sp, pp = fwr.Batch.pointer_table(slopes), fwr.Batch.pointer_table(phases)
    batch.run(sp, pp)
    torch.cuda.synchronize()
    eager = [p.clone() for p in phases]
    for p in phases:
        p.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.run(sp, pp, stream=s)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(phases, eager):
        assert torch.equal(a, b)
    # other schedules give the same frames (each frame's arithmetic is fixed)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for ctas, ratio in [(sms, 4.0), (max(1, sms // 3), 20.0), (1, 9.6)]:
        batch.schedule(ctas, ratio)
        assert batch.ctas == ctas
        batch.run(sp, pp)
        torch.cuda.synchronize()
        for a, b in zip(phases, eager):
            assert torch.equal(a, b)


def test_autotune_cache_round_trip(fwr, tmp_path):
    k = 1
    plans, batch, frame_plan, host, slopes, phases = make_batch(fwr, 8, k, seed=3)
    sp, pp = fwr.Batch.pointer_table(slopes), fwr.Batch.pointer_table(phases)
    cache = tmp_path / "tune.jsonl"
    ctas, ratio = batch.autotune(sp, pp, cache)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])
    assert entry["ctas"] == ctas and abs(entry["cost_ratio"] - ratio) < 1e-9
    other = fwr.Batch(plans, frame_plan, k)
    assert other.autotune(sp, pp, cache) == (ctas, ratio)
    assert len(cache.read_text().strip().splitlines()) == 1  # applied from the cache, not re-timed


def test_ragged_errors_and_status(fwr):
    small = fwr.Plan(synth.pupil_mask(16), 2.0, fwr.LSQ)  # 32^2: not a ragged size
    with pytest.raises(fwr.FwrError) as e:
        fwr.Batch([small], [0], 1)
    assert e.value.code == 2
    big = fwr.Plan(synth.pupil_mask(40), 3.2, fwr.LSQ)
    with pytest.raises(fwr.FwrError):
        fwr.Batch([big], [0, 1], 1)
    batch = fwr.Batch([big], [0, 0], 1)
    fr = synth.frame(40, 1, 0.05)["slopes"]
    bad = fr.copy()
    bad[1, 20, 20] = np.inf
    s = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in (fr, bad)]
    p = [torch.empty((128, 128), device="cuda") for _ in range(2)]
    batch.run(fwr.Batch.pointer_table(s), fwr.Batch.pointer_table(p))
    assert big.status() == "FWR_ERR_NONFINITE"


def test_reconstruct_ragged_one_call_against_oracle(fwr):
    """fwr_reconstruct_ragged (device frame table, one launch): every frame
    against the FP64 oracle, bitwise equal to the batch object's result and
    to a second (cached, allocation-free) call and its CUDA-graph replay."""
    k = 2
    plans, batch, frame_plan, host, slopes, phases = make_batch(fwr, 2, k, seed=21)
    sp, pp = fwr.Batch.pointer_table(slopes), fwr.Batch.pointer_table(phases)
    fpd = torch.tensor(frame_plan, dtype=torch.int32, device="cuda")
    fwr.reconstruct_ragged(plans, fpd, sp, pp, k)
    torch.cuda.synchronize()
    first = [p.clone() for p in phases]
    for f, pl in enumerate(frame_plan):
        n, pad = SIZES[pl]
        orc, _ = oracle.reconstruct(host[f], synth.pupil_mask(n), pad, k, oracle.FILTER_LSQ)
        assert within(first[f].cpu().numpy(), orc, FP32_TOL, where="frame %d N=%d" % (f, plans[pl].N))
    batch.run(sp, pp)
    torch.cuda.synchronize()
    for a, b in zip(phases, first):
        assert torch.equal(a, b)
    for p in phases:
        p.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fwr.reconstruct_ragged(plans, fpd, sp, pp, k, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(phases, first):
        assert torch.equal(a, b)
    fwr.ragged_release()


def test_reconstruct_ragged_rejects_bad_tables(fwr):
    big = fwr.Plan(synth.pupil_mask(40), 3.2, fwr.LSQ)
    fr = synth.frame(40, 1, 0.05)["slopes"]
    s = [torch.tensor(fr, dtype=torch.float32, device="cuda") for _ in range(2)]
    p = [torch.empty((128, 128), device="cuda") for _ in range(2)]
    sp, pp = fwr.Batch.pointer_table(s), fwr.Batch.pointer_table(p)
    with pytest.raises(fwr.FwrError) as e:
        fwr.reconstruct_ragged([big], torch.tensor([0, 1], dtype=torch.int32, device="cuda"), sp, pp, 1)
    assert e.value.code == 1
    # a table rewritten in place after the first call: the bad frame is skipped and reported
    fpd = torch.tensor([0, 0], dtype=torch.int32, device="cuda")
    fwr.reconstruct_ragged([big], fpd, sp, pp, 1)
    torch.cuda.synchronize()
    good = p[0].clone()
    p[0].zero_()
    fpd[1] = 5
    fwr.reconstruct_ragged([big], fpd, sp, pp, 1)
    torch.cuda.synchronize()
    assert torch.equal(p[0], good)
    assert big.status() == "FWR_ERR_ARG"
    assert big.status() == "FWR_OK"
    fwr.ragged_release()
