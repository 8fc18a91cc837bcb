"""The tcgen05 BF16 GEMM against an FP64 reference of the same BF16 inputs,
and the linear warm start built on it: its extension operator against the
oracle, its forward against an FP64 evaluation of the same BF16 factors, and
the reconstruction it starts (full rank, fitted to the extension: k = 1
reproduces k = 11; the default phase-weighted rank on the 40 x 40 workload:
within 1 % of the residual of 10 plain iterations)."""

import numpy as np
import pytest

import oracle
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


def bf16(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float32)).bfloat16().double().numpy()


@pytest.mark.parametrize("M,N,K", [(1, 128, 8), (100, 128, 64), (128, 256, 72), (300, 384, 1000),
                                   (257, 128, 2560), (1000, 1280, 2528), (600, 8192, 128), (1000, 32768, 64),
                                   (1000, 32768, 256), (256, 8192, 200)])
def test_gemm_matches_fp64_reference(fwr, M, N, K):
    """Rows beyond M and K beyond a multiple of 64 come from the TMA zero fill;
    N = 384 and 128 take 128-wide tiles, the rest 256-wide; (600, 8192, 128)
    and the 32768-wide shapes give some CTAs several tiles (both TMEM
    accumulators in turn). K <= 256 with a grid that is a multiple of the M
    tiles (or one tile per CTA) keeps A resident in shared memory: the small
    shapes, (1000, 32768, 64 / 256) over several tiles per CTA and
    (256, 8192, 200) with a partial last k-block."""
    g = torch.Generator().manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, generator=g).bfloat16()
    B = torch.randn(N, K, generator=g).bfloat16()
    D = fwr.gemm_bf16_tc(A.cuda(), B.cuda()).double().cpu()
    ref = A.double() @ B.double().T
    scale = (A.double().abs() @ B.double().abs().T).max()
    assert float((D - ref).abs().max()) <= 2e-6 * float(scale)


def test_gemm_argument_errors(fwr):
    A = torch.zeros(4, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(fwr.FwrError):
        fwr.gemm_bf16_tc(A, torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda"))   # N % 128
    A12 = torch.zeros(4, 12, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(fwr.FwrError):
        fwr.gemm_bf16_tc(A12, torch.zeros(128, 12, dtype=torch.bfloat16, device="cuda"))  # K % 8


def test_gemm_wait_timeout_reports_and_recovers(fwr):
    """The bounded-wait path of the tcgen05 GEMM: with a 16-cycle bound the MMA
    issuer gives up before the first TMA tiles land; the kernel drains its
    loads (full bound), frees its tensor memory and reports FWR_ERR_TIMEOUT.
    The context stays usable: the same product then comes out right."""
    g = torch.Generator().manual_seed(11)
    A = torch.randn(256, 512, generator=g).bfloat16()
    B = torch.randn(256, 512, generator=g).bfloat16()
    Ad, Bd = A.cuda(), B.cuda()
    with pytest.raises(fwr.FwrError) as e:
        fwr.gemm_bf16_tc(Ad, Bd, wait_cycles=16)
    assert e.value.code == 5
    D = fwr.gemm_bf16_tc(Ad, Bd).double().cpu()
    ref = A.double() @ B.double().T
    scale = (A.double().abs() @ B.double().abs().T).max()
    assert float((D - ref).abs().max()) <= 2e-6 * float(scale)
    with pytest.raises(fwr.FwrError) as e:
        fwr.gemm_bf16_tc(Ad, Bd, wait_cycles=0)
    assert e.value.code == 1


def small_setup(fwr):
    n, pad = 16, 2.0
    mask = synth.pupil_mask(n)
    plan = fwr.Plan(mask, pad, fwr.LSQ)
    return n, plan, mask


def test_operator_matches_oracle(fwr):
    from paper_1705_04298_gb300 import linws
    n, plan, mask = small_setup(fwr)
    E = linws.extension_operator(fwr, plan, mask, iters=10)
    assert E.shape == (2 * plan.valid_count, 2 * plan.N * plan.N)
    sl, _, _ = synth.batch(n, 3, 77, 0.05)
    X = linws.gathered(sl, mask)
    for f in range(3):
        s0x, s0y, P = oracle.embed(sl[f], mask, plan.N)
        sx, sy = oracle.gerchberg_extend(s0x, s0y, P, 10)
        ref = np.concatenate([sx.ravel(), sy.ravel()])
        got = X[f] @ E
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("F", [1, 5, 130, 200])
def test_forward_matches_fp64_of_bf16_factors(fwr, F):
    n, plan, mask = small_setup(fwr)
    K, r = 2 * plan.valid_count, 256
    rng = np.random.default_rng(F)
    A = rng.standard_normal((K, r)) / np.sqrt(K)
    V = rng.standard_normal((2 * plan.N * plan.N, r)) / np.sqrt(r)
    ws = fwr.LinearWarmStart(plan, A, V, max_batch=200)
    sl, _, _ = synth.batch(n, F, 300, 0.05)
    out = ws.forward(torch.tensor(sl, dtype=torch.float32, device="cuda"))
    ws.status()
    from paper_1705_04298_gb300 import linws
    C = bf16(bf16(linws.gathered(sl.astype(np.float32), mask)) @ bf16(A))
    ref = (C @ bf16(V).T).reshape(F, 2, plan.N, plan.N)
    got = out.double().cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max()


def test_full_rank_warm_start_reproduces_eleven_iterations(fwr):
    """E_10 at full rank (no truncation): one iteration from x0 = E_10 s is the
    eleventh plain iteration, up to the BF16 rounding of the factors."""
    from paper_1705_04298_gb300 import linws
    n, plan, mask = small_setup(fwr)
    K = 2 * plan.valid_count
    r = (K + 127) // 128 * 128
    ws, E = linws.build(fwr, plan, mask, rank=r, max_batch=64, frames=1024, weight="extension")
    sl, _, _ = synth.batch(n, 64, 900, 0.05)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    x0 = ws.forward(s)
    ws.status()
    ref_x0 = (linws.gathered(sl, mask) @ E).reshape(64, 2, plan.N, plan.N)
    assert np.linalg.norm(x0.double().cpu().numpy() - ref_x0) <= 1e-2 * np.linalg.norm(ref_x0)
    a = plan.reconstruct(s, 1, ext_init=x0).double().cpu().numpy()
    b = plan.reconstruct(s, 11).double().cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b)


def test_fused_entry_matches_forward_then_reconstruct(fwr):
    """fwr_linws_reconstruct keeps the warm start in BF16; against the FP32
    warm start through fwr_reconstruct_ex the phase differs by that rounding
    only. A plan with another pupil is refused."""
    n, plan, mask = small_setup(fwr)
    K = 2 * plan.valid_count
    rng = np.random.default_rng(4)
    A = rng.standard_normal((K, 256)) / np.sqrt(K)
    V = rng.standard_normal((2 * plan.N * plan.N, 256)) / 16.0
    ws = fwr.LinearWarmStart(plan, A, V, max_batch=40)
    sl, _, _ = synth.batch(n, 37, 500, 0.05)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    for k in (0, 1, 3):
        a = ws.reconstruct(s, k).double().cpu().numpy()
        b = plan.reconstruct(s, k, ext_init=ws.forward(s)).double().cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b), k
    ws.status()
    other = np.ones((n, n), dtype=bool)
    with pytest.raises(fwr.FwrError):
        ws.reconstruct(s, 1, plan=fwr.Plan(other, 2.0, fwr.LSQ))


def test_default_rank_within_one_percent_of_ten_iterations(fwr):
    """40 x 40 lenslets on 128^2 (Wiener, 0.05 rad), 256 held-out frames."""
    from paper_1705_04298_gb300 import learned, linws
    F = 256
    mask = synth.pupil_mask(learned.N_LENSLETS)
    plan = learned.make_plan(fwr, fwr.WIENER, learned.EVAL_SIGMA)
    ws, _ = linws.build(fwr, plan, mask, rank=linws.DEFAULT_RANK, max_batch=F)
    slopes, truth = learned.frames(F, learned.EVAL_SEED0, learned.EVAL_SIGMA)
    phase = torch.empty((F, 128, 128), device="cuda")
    plan.reconstruct(slopes, 10, phase)
    r10 = learned.residual_rms(fwr, phase, truth, mask)
    plan.reconstruct(slopes, 1, phase, ext_init=ws.forward(slopes))
    ws.status()
    r1 = learned.residual_rms(fwr, phase, truth, mask)
    ws.reconstruct(slopes, 1, phase)
    ws.status()
    r1h = learned.residual_rms(fwr, phase, truth, mask)
    print({"plain10": r10, "linear1": r1, "linear1_bf16_warm_start": r1h})
    assert r1 <= 1.01 * r10 and r1h <= 1.01 * r10


def test_reconstruct_replays_from_a_cuda_graph(fwr):
    """fwr_linws_reconstruct allocates nothing and does not synchronise, so it
    can be captured in a CUDA graph; the replay reproduces the direct call
    bit for bit (every kernel sums in a fixed order)."""
    n, plan, mask = small_setup(fwr)
    K = 2 * plan.valid_count
    rng = np.random.default_rng(8)
    ws = fwr.LinearWarmStart(plan, rng.standard_normal((K, 128)) / np.sqrt(K),
                             rng.standard_normal((2 * plan.N * plan.N, 128)) / 12.0, max_batch=24)
    sl, _, _ = synth.batch(n, 24, 700, 0.05)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    direct = ws.reconstruct(s, 2).clone()
    out = torch.empty_like(direct)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        ws.reconstruct(s, 2, out, stream=stream)
    g.replay()
    torch.cuda.synchronize()
    ws.status()
    assert torch.equal(out, direct)


def test_back_to_back_calls_keep_their_inputs(fwr):
    """The warm start's kernels are launched as programmatic dependents of
    their producers (gather -> X A -> (X A) V^T -> fused kernel), so each set-up
    overlaps the kernel before it. Two calls issued back to back on one stream,
    with different frames and no synchronisation between them, give bitwise
    the phases of the same calls run one at a time; so do three replays of a
    captured call whose input buffer changes between replays."""
    n, plan, mask = small_setup(fwr)
    K = 2 * plan.valid_count
    rng = np.random.default_rng(11)
    ws = fwr.LinearWarmStart(plan, rng.standard_normal((K, 256)) / np.sqrt(K),
                             rng.standard_normal((2 * plan.N * plan.N, 256)) / 16.0, max_batch=40)
    frames = [torch.tensor(synth.batch(n, 40, 900 + 10 * i, 0.05)[0], dtype=torch.float32, device="cuda")
              for i in range(3)]
    alone = []
    for s in frames:
        alone.append(ws.reconstruct(s, 1).clone())
        torch.cuda.synchronize()
    outs = [torch.empty_like(alone[0]) for _ in frames]
    for s, o in zip(frames, outs):
        ws.reconstruct(s, 1, o)
    torch.cuda.synchronize()
    ws.status()
    for a, b in zip(outs, alone):
        assert torch.equal(a, b)
    buf = frames[0].clone()
    out = torch.empty_like(alone[0])
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        ws.reconstruct(buf, 1, out, stream=stream)
    for s, a in zip(frames, alone):
        buf.copy_(s)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, a)
    ws.status()
