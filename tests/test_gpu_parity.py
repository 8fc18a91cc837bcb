"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances (relative phase rms, piston removed, full N x N grid):
  FP64 GPU path  <= 1e-11   (only summation order differs from the oracle)
  FP32 GPU path  <= 1e-5    (stated target for every FP32 path)
Index/bitwise facts (in-pupil slopes of the extended output, determinism,
host vs device entry points) are compared exactly.
"""

import math

import numpy as np
import pytest

import oracle
from paper_1705_04298_gb300 import synth
from parity_check import FP32_MAX_256_K10, FP32_MAX_512_K10, errors, max_tol_for, within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-11


@pytest.fixture(scope="module")
def fwr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04298_gb300 import fwr as m
    m.load()
    return m


def rel_rms(got, ref):
    return errors(got, ref)[0]


FILTERS = {"lsq": oracle.FILTER_LSQ, "wiener": oracle.FILTER_WIENER}


def run_oracle(slopes, mask, pad, iters, filt, noise_var, r0p, L0p, periodic, ext_init=None):
    return oracle.reconstruct(slopes, mask, pad, iters, filt, noise_var, r0p, L0p, periodic, ext_init)


def make_plan(fwr, mask, pad, filt, noise_var=0.0, r0p=1.0, L0p=100.0, periodic=0):
    return fwr.Plan(mask, pad, filt, noise_var, r0p, L0p, periodic)


# --------------------------------------------------------------- FFT ------

@pytest.mark.parametrize("N", [16, 32, 64, 128])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft2_matches_numpy(fwr, N, inverse):
    rng = np.random.Generator(np.random.PCG64(N + inverse))
    F = 7
    x = rng.standard_normal((F, N, N)) + 1j * rng.standard_normal((F, N, N))
    xt = torch.tensor(x.astype(np.complex64), device="cuda")
    y = fwr.fft2(xt, inverse=inverse).cpu().numpy().astype(np.complex128)
    ref = np.fft.ifft2(x) * N * N if inverse else np.fft.fft2(x)
    err = np.sqrt(np.sum(np.abs(y - ref) ** 2) / np.sum(np.abs(ref) ** 2))
    assert err < 2e-7 * math.log2(N * N)


# ------------------------------------------------ 16x16 -> 32^2 (1 frame) -

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_small_config_lsq_k10(fwr, precision):
    """16x16 lenslets, 32^2 grid, sigma = 0.05 rad, LSQ, 10 iterations."""
    n, pad, k = 16, 2.0, 10
    fr = synth.frame(n, 0, 0.05)
    ref, ref_ext = run_oracle(fr["slopes"], fr["mask"], pad, k, oracle.FILTER_LSQ, 0.0, 1.0, 1.0,
                              oracle.PERIODIC_BEFORE_EACH_FFT)
    plan = make_plan(fwr, fr["mask"], pad, fwr.LSQ)
    N = plan.N
    if precision == "fp64":
        s = torch.tensor(fr["slopes"][None], dtype=torch.float64, device="cuda")
        ext = torch.empty((1, 2, N, N), dtype=torch.float64, device="cuda")
        ph = plan.reconstruct_f64(s, k, ext_out=ext)
        tol = FP64_TOL
    else:
        s = torch.tensor(fr["slopes"][None], dtype=torch.float32, device="cuda")
        ext = torch.empty((1, 2, N, N), dtype=torch.float32, device="cuda")
        ph = plan.reconstruct(s, k, ext_out=ext)
        tol = FP32_TOL
    torch.cuda.synchronize()
    assert within(ph[0].cpu().numpy(), ref, tol, where=precision)
    e = ext[0].cpu().numpy().astype(np.float64)
    assert within(e, ref_ext, tol * 10, 10 * max_tol_for(tol), where=precision + " ext_out")
    # in-pupil slopes are the measurement (bitwise in the path's precision)
    s0x, s0y, P = oracle.embed(fr["slopes"], fr["mask"], N)
    dt = np.float64 if precision == "fp64" else np.float32
    assert np.array_equal(e[0][P].astype(dt), s0x[P].astype(dt))
    assert np.array_equal(e[1][P].astype(dt), s0y[P].astype(dt))
    assert plan.status() == "FWR_OK"


# --------------------------------------- periodic modes x filters (N=64) --

@pytest.mark.parametrize("periodic", [0, 1, 2])
@pytest.mark.parametrize("filt", ["lsq", "wiener"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_modes_and_filters(fwr, periodic, filt, precision):
    n, pad, k, sigma = 30, 2.0, 3, 0.1
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    F = 3
    sl, _, mask = synth.batch(n, F, 77, sigma)
    plan = make_plan(fwr, mask, pad, fwr.WIENER if filt == "wiener" else fwr.LSQ, sigma ** 2, r0p, L0p,
                     periodic)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    s = torch.tensor(sl, dtype=dtype, device="cuda")
    ph = (plan.reconstruct_f64 if precision == "fp64" else plan.reconstruct)(s, k)
    ph = ph.cpu().numpy()
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    for f in range(F):
        ref, _ = run_oracle(sl[f], mask, pad, k, FILTERS[filt], sigma ** 2, r0p, L0p, periodic)
        assert within(ph[f], ref, tol, where=str(f))


# ------------------------------ 40x40 -> 128^2, Wiener, every k, tail ------

@pytest.mark.parametrize("k", [0, 1, 2, 5, 10])
def test_40x40_wiener_iterations(fwr, k):
    n, pad = 40, 3.2
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sig = [0.02, 0.1]
    F = 4
    sl, _, mask = synth.batch(n, F, 1000, sig)
    for s_i in sig:
        plan = make_plan(fwr, mask, pad, fwr.WIENER, s_i ** 2, r0p, L0p)
        assert plan.N == 128
        ph = plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), k).cpu().numpy()
        for f in range(F):
            ref, _ = run_oracle(sl[f], mask, pad, k, oracle.FILTER_WIENER, s_i ** 2, r0p, L0p, 0)
            assert within(ph[f], ref, FP32_TOL, where=str((k, s_i, f)))


def test_persistent_tail_frames(fwr):
    """More frames than resident CTAs: every CTA loops, the last ones partly."""
    n, pad, k = 40, 3.2, 2
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    F = sms + 9
    sl, _, mask = synth.batch(n, F, 4242, 0.05)
    plan = make_plan(fwr, mask, pad, fwr.LSQ)
    ph = plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), k).cpu().numpy()
    for f in [0, 1, sms - 1, sms, sms + 8]:
        ref, _ = run_oracle(sl[f], mask, pad, k, oracle.FILTER_LSQ, 0.0, 1.0, 1.0, 0)
        assert within(ph[f], ref, FP32_TOL, where=str(f))


def test_full_size_40x40_1000_frames_sampled(fwr):
    """The benchmarked launch (1000 frames, k = 10, Wiener): sampled frames
    against the oracle, every frame for zero mean and finiteness."""
    n, pad, k, F, sigma = 40, 3.2, 10, 1000, 0.02
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sl, _, mask = synth.batch(n, F, 1000, [0.02, 0.1])
    plan = make_plan(fwr, mask, pad, fwr.WIENER, sigma ** 2, r0p, L0p)
    ph = plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), k)
    torch.cuda.synchronize()
    assert torch.isfinite(ph).all()
    means = ph.double().mean(dim=(1, 2)).abs().max().item()
    assert means < 1e-4 * ph.double().std().item()
    phn = ph.cpu().numpy()
    for f in [0, 1, 499, 998, 999]:
        ref, _ = run_oracle(sl[f], mask, pad, k, oracle.FILTER_WIENER, sigma ** 2, r0p, L0p, 0)
        assert within(phn[f], ref, FP32_TOL, where=str(f))


# ---------------------------------------------------- warm start / extras -

def test_warm_start_and_invariants(fwr):
    n, pad, k = 16, 2.0, 4
    F = 3
    sl, _, mask = synth.batch(n, F, 91, 0.05)
    N = 32
    rng = np.random.Generator(np.random.PCG64(5))
    ext_init = rng.standard_normal((F, 2, N, N))
    plan = make_plan(fwr, mask, pad, fwr.LSQ)
    ext_out = torch.empty((F, 2, N, N), dtype=torch.float64, device="cuda")
    ph = plan.reconstruct_f64(torch.tensor(sl, device="cuda"), k,
                              ext_init=torch.tensor(ext_init, device="cuda"), ext_out=ext_out)
    ph = ph.cpu().numpy()
    eo = ext_out.cpu().numpy()
    for f in range(F):
        ref, ref_ext = run_oracle(sl[f], mask, pad, k, oracle.FILTER_LSQ, 0.0, 1.0, 1.0, 0, ext_init[f])
        assert within(ph[f], ref, FP64_TOL, where=str(f))
        assert np.max(np.abs(eo[f] - ref_ext)) <= 1e-10 * np.max(np.abs(ref_ext))
        # Eq. PC: zero row sums of x slopes, zero column sums of y slopes
        assert np.max(np.abs(eo[f][0].sum(axis=1))) <= 1e-10
        assert np.max(np.abs(eo[f][1].sum(axis=0))) <= 1e-10


def test_zero_frames_and_argument_errors(fwr):
    mask = synth.pupil_mask(16)
    plan = make_plan(fwr, mask, 2.0, fwr.LSQ)
    s = torch.zeros((0, 2, 16, 16), dtype=torch.float32, device="cuda")
    plan.reconstruct(s, 3)
    with pytest.raises(fwr.FwrError):
        plan.reconstruct(torch.zeros((1, 2, 16, 16), device="cuda"), 65)
    with pytest.raises(fwr.FwrError):
        plan.set_periodic(3)
    big = make_plan(fwr, synth.pupil_mask(40), 3.2, fwr.LSQ)
    with pytest.raises(fwr.FwrError):
        big.reconstruct_f64(torch.zeros((1, 2, 40, 40), dtype=torch.float64, device="cuda"), 1)


def test_extreme_pupil_sizes(fwr):
    # smallest lenslet array, and the largest n that still leaves the fill
    # row/column outside the pupil (n = N - 2)
    for n, pad in [(2, 8.0), (30, 32 / 30)]:
        mask = synth.pupil_mask(n) if n > 2 else np.ones((2, 2), bool)
        sl, _, _ = synth.batch(n, 2, 31, 0.05)
        sl = np.where(mask[None, None], sl, 0.0)
        plan = make_plan(fwr, mask, pad, fwr.LSQ)
        ph = plan.reconstruct_f64(torch.tensor(sl, device="cuda"), 3).cpu().numpy()
        for f in range(2):
            ref, _ = run_oracle(sl[f], mask, pad, 3, oracle.FILTER_LSQ, 0.0, 1.0, 1.0, 0)
            assert within(ph[f], ref, FP64_TOL, where=str((n, f)))


def test_nonfinite_input_sets_status(fwr):
    mask = synth.pupil_mask(16)
    plan = make_plan(fwr, mask, 2.0, fwr.LSQ)
    sl, _, _ = synth.batch(16, 2, 5, 0.05)
    sl[1, 0, 8, 8] = np.nan
    plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), 1)
    assert plan.status() == "FWR_ERR_NONFINITE"
    assert plan.status() == "FWR_OK"  # read-and-clear


@pytest.mark.parametrize("n,pad", [(40, 3.2), (80, 3.2)])
def test_host_path_chunks_match_device_path(fwr, n, pad):
    """The host entry point pipelines its copies in chunks of whole SM-waves
    (several chunks and a partial last one here, on a side stream, two calls
    back to back): bit-identical to the device entry point."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    F = 4 * sms + 37 if n == 40 else 2 * sms + 5
    k = 2
    sl, _, mask = synth.batch(n, F, 11, 0.05)
    plan = make_plan(fwr, mask, pad, fwr.LSQ)
    ref = plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), k).cpu()
    sh = torch.tensor(sl, dtype=torch.float32).pin_memory()
    out1 = torch.full((F, plan.N, plan.N), float("nan"), dtype=torch.float32).pin_memory()
    out2 = torch.full((F, plan.N, plan.N), float("nan"), dtype=torch.float32).pin_memory()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        plan.reconstruct_host(sh, k, out1)
        plan.reconstruct_host(sh, k, out2)
    side.synchronize()
    assert torch.equal(out1, ref)
    assert torch.equal(out2, ref)


def test_deterministic_and_host_path_identical(fwr):
    n, pad, k, F = 40, 3.2, 5, 64
    sl, _, mask = synth.batch(n, F, 3, 0.05)
    plan = make_plan(fwr, mask, pad, fwr.LSQ)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    a = plan.reconstruct(s, k).cpu()
    b = plan.reconstruct(s, k).cpu()
    assert torch.equal(a, b)
    sh = torch.tensor(sl, dtype=torch.float32).pin_memory()
    out = torch.empty((F, plan.N, plan.N), dtype=torch.float32).pin_memory()
    plan.reconstruct_host(sh, k, out)
    torch.cuda.synchronize()
    assert torch.equal(out, a)


# ------------------------------------------- 256^2 grids (slab kernel) ----

@pytest.mark.parametrize("n,pad,k,periodic,filt", [
    (80, 3.2, 5, 0, "lsq"),
    (128, 2.0, 2, 1, "wiener"),
    (80, 3.2, 0, 0, "wiener"),
    (100, 2.56, 3, 2, "lsq"),
])
def test_256_grid(fwr, n, pad, k, periodic, filt):
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sigma = 0.05
    F = 3
    sl, _, mask = synth.batch(n, F, 2000 + n, sigma)
    plan = make_plan(fwr, mask, pad, fwr.WIENER if filt == "wiener" else fwr.LSQ, sigma ** 2, r0p, L0p,
                     periodic)
    assert plan.N == 256
    ph = plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), k).cpu().numpy()
    for f in range(F):
        ref, _ = run_oracle(sl[f], mask, pad, k, FILTERS[filt], sigma ** 2, r0p, L0p, periodic)
        assert within(ph[f], ref, FP32_TOL, where=str(f))


@pytest.mark.parametrize("case", ["256^2 frozen flow, 1000 frames", "512^2, 304 frames"])
def test_full_size_large_grids_sampled(fwr, case):
    """The benchmarked large-grid launches (k = 10, LSQ, the launch shape the
    tuner picks): 128x128 lenslets of frozen-flow frames on 256^2, 1000 frames,
    and 200x200 lenslets on 512^2, two frames per SM; sampled frames against
    the oracle, every frame finite with zero mean."""
    k = 10
    if case.startswith("256"):
        sl, _, mask = synth.frozen_flow(128, 32, 7, 0.05, r0=0.12, L0=25.0)
        pad, F, N = 2.0, 1000, 256
    else:
        sl, _, mask = synth.batch(200, 16, 7000, 0.05)
        pad, F, N = 2.56, 2 * torch.cuda.get_device_properties(0).multi_processor_count, 512
    reps = (F + len(sl) - 1) // len(sl)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat(reps, 1, 1, 1)[:F].contiguous()
    plan = make_plan(fwr, mask, pad, fwr.LSQ)
    assert plan.N == N
    out = torch.empty((F, N, N), device="cuda")
    plan.autotune(s, k, out)
    ph = plan.reconstruct(s, k, out)
    torch.cuda.synchronize()
    assert plan.status() == "FWR_OK"
    assert torch.isfinite(ph).all()
    means = ph.double().mean(dim=(1, 2)).abs().max().item()
    assert means < 1e-4 * ph.double().std().item()
    phn = ph.cpu().numpy()
    # element-wise bound of these ten-iteration large-grid launches (parity_check)
    max_tol = FP32_MAX_256_K10 if N == 256 else FP32_MAX_512_K10
    for f in [0, 1, F // 2, F - 2, F - 1]:
        ref, _ = run_oracle(sl[f % len(sl)], mask, pad, k, oracle.FILTER_LSQ, 0.0, 1.0, 100.0, 0)
        assert within(phn[f], ref, FP32_TOL, max_tol, where="%s frame %d" % (case, f))


def test_256_grid_persistent_tail_and_limits(fwr):
    n, pad, k = 80, 3.2, 1
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    F = sms + 5
    sl, _, mask = synth.batch(n, F, 77, 0.05)
    plan = make_plan(fwr, mask, pad, fwr.LSQ)
    ph = plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), k).cpu().numpy()
    for f in [0, sms, sms + 4]:
        ref, _ = run_oracle(sl[f], mask, pad, k, oracle.FILTER_LSQ, 0.0, 1.0, 1.0, 0)
        assert within(ph[f], ref, FP32_TOL, where=str(f))
    # 256^2: FP32 only, no extended-slope output
    with pytest.raises(fwr.FwrError):
        plan.reconstruct_f64(torch.zeros((1, 2, n, n), dtype=torch.float64, device="cuda"), 1)
    with pytest.raises(fwr.FwrError):
        plan.reconstruct(torch.zeros((1, 2, n, n), device="cuda"), 1,
                         ext_out=torch.empty((1, 2, 256, 256), device="cuda"))


# ------------------------------------ 512^2 grids (ELT scale, slab kernel) --

@pytest.mark.parametrize("n,pad,k,periodic,filt", [
    (200, 2.56, 2, 0, "wiener"),
    (160, 3.2, 1, 2, "lsq"),
    (256, 2.0, 1, 1, "lsq"),
])
def test_512_grid(fwr, n, pad, k, periodic, filt):
    """ELT-scale grids (the paper's case for the method, Sec. 1 and the
    operation count of Sec. 3.3): 160 to 256 lenslets across on 512^2, both
    launch shapes bitwise equal, against the FP64 oracle."""
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sigma = 0.05
    F = 2
    sl, _, mask = synth.batch(n, F, 5000 + n, sigma)
    plan = make_plan(fwr, mask, pad, fwr.WIENER if filt == "wiener" else fwr.LSQ, sigma ** 2, r0p, L0p,
                     periodic)
    assert plan.N == 512
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    ph = plan.reconstruct(s, k).clone()
    plan.set_shape(1)
    assert torch.equal(plan.reconstruct(s, k), ph)
    ph = ph.cpu().numpy()
    for f in range(F):
        ref, _ = run_oracle(sl[f], mask, pad, k, FILTERS[filt], sigma ** 2, r0p, L0p, periodic)
        assert within(ph[f], ref, FP32_TOL, where="N=512 f=%d" % f)
    assert plan.status() == "FWR_OK"


def test_512_grid_hudgin_and_tail(fwr):
    n, pad, k = 200, 2.56, 0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    F = sms + 3
    sl, _, mask = synth.batch(n, 4, 5500, 0.05)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat(F // 4 + 1, 1, 1, 1)[:F].contiguous()
    plan = make_plan(fwr, mask, pad, fwr.LSQ)
    plan.set_extension(fwr.EXT_HUDGIN)
    ph = plan.reconstruct(s, k)
    torch.cuda.synchronize()
    assert torch.equal(ph[0], ph[sms])  # same input in the first and the last wave
    ref, _ = oracle.reconstruct(sl[0], mask, pad, k, oracle.FILTER_LSQ, ext_init="hudgin")
    assert within(ph[0].cpu().numpy(), ref, FP32_TOL, where="N=512 hudgin")


def test_misaligned_phase_and_warm_start_are_refused(fwr):
    """The kernels store the phase and read the warm start with 16-byte
    vector accesses; pointers off that alignment are argument errors."""
    n = 16
    fr = synth.frame(n, 3, 0.05)
    plan = fwr.Plan(fr["mask"], 2.0, fwr.LSQ)
    N = plan.N
    s = torch.tensor(fr["slopes"][None], dtype=torch.float32, device="cuda")
    flat = torch.empty(N * N + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(fwr.FwrError):
        plan.reconstruct(s, 2, flat[1:].view(1, N, N))
    ext = torch.zeros(2 * N * N + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(fwr.FwrError):
        plan.reconstruct(s, 2, ext_init=ext[1:].view(1, 2, N, N))
    ok = plan.reconstruct(s, 2, flat[:N * N].view(1, N, N))
    assert torch.isfinite(ok).all()


# ------------------------------------------ measurement-model variants ----

MODELS = [(1, 0.0), (0, 1.0 / 6.0), (1, 1.0 / 6.0)]


@pytest.mark.parametrize("g_model,pixel", MODELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_model_variants_small(fwr, g_model, pixel, precision):
    """Fried geometry and the d - d_px pixel correction (FWR_OPT_G_MODEL,
    FWR_OPT_PIXEL) against the oracle with the same model: 30x30 lenslets on
    64^2, Wiener, every periodic mode."""
    n, pad, k, sigma = 30, 2.0, 4, 0.1
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sl, _, mask = synth.batch(n, 2, 91, sigma)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    for periodic in (0, 1, 2):
        plan = make_plan(fwr, mask, pad, fwr.WIENER, sigma ** 2, r0p, L0p, periodic)
        plan.set_model(g_model, pixel)
        s = torch.tensor(sl, dtype=dtype, device="cuda")
        ph = (plan.reconstruct_f64 if precision == "fp64" else plan.reconstruct)(s, k).cpu().numpy()
        for f in range(2):
            ref, _ = oracle.reconstruct(sl[f], mask, pad, k, oracle.FILTER_WIENER, sigma ** 2, r0p, L0p,
                                        periodic, g_model=g_model, pixel=pixel)
            assert within(ph[f], ref, tol, where=str((periodic, f)))


@pytest.mark.parametrize("n,pad,k", [(40, 3.2, 5), (80, 3.2, 2)])
def test_model_variants_large_grids(fwr, n, pad, k):
    """The same on 128^2 (fused kernel) and 256^2 (slab kernel), Fried with
    six pixels per lenslet; setting the default model back reproduces the
    default path bit for bit."""
    sigma = 0.05
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sl, _, mask = synth.batch(n, 3, 17, sigma)
    plan = make_plan(fwr, mask, pad, fwr.WIENER, sigma ** 2, r0p, L0p)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    base = plan.reconstruct(s, k).cpu()
    plan.set_model(fwr.G_FRIED, 1.0 / 6.0)
    ph = plan.reconstruct(s, k).cpu().numpy()
    for f in range(3):
        ref, _ = oracle.reconstruct(sl[f], mask, pad, k, oracle.FILTER_WIENER, sigma ** 2, r0p, L0p,
                                    g_model=oracle.G_FRIED, pixel=1.0 / 6.0)
        assert within(ph[f], ref, FP32_TOL, where=str(f))
    assert not torch.equal(torch.tensor(ph), base)
    plan.set_model(fwr.G_AVERAGED, 0.0)
    assert torch.equal(plan.reconstruct(s, k).cpu(), base)
    with pytest.raises(fwr.FwrError):
        plan.set_model(2, 0.0)
    with pytest.raises(fwr.FwrError):
        plan.set_model(fwr.G_AVERAGED, 0.6)


# ------------------------------------------------- Hudgin extension -------

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k,periodic", [(0, 0), (3, 0), (2, 2)])
def test_hudgin_extension_small(fwr, precision, k, periodic):
    """FWR_OPT_EXTENSION = FWR_EXT_HUDGIN against the oracle's Hudgin start:
    30x30 lenslets on 64^2, LSQ. k = 0 with the periodic condition is the
    paper's Hudgin method."""
    n, pad, sigma = 30, 2.0, 0.05
    sl, _, mask = synth.batch(n, 2, 123, sigma)
    plan = make_plan(fwr, mask, pad, fwr.LSQ, 0.0, 1.0, 1.0, periodic)
    plan.set_extension(fwr.EXT_HUDGIN)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    s = torch.tensor(sl, dtype=dtype, device="cuda")
    ph = (plan.reconstruct_f64 if precision == "fp64" else plan.reconstruct)(s, k).cpu().numpy()
    for f in range(2):
        ref, _ = oracle.reconstruct(sl[f], mask, pad, k, oracle.FILTER_LSQ, periodic=periodic, ext_init="hudgin")
        assert within(ph[f], ref, tol, where=str(f))


@pytest.mark.parametrize("n,pad,k", [(40, 3.2, 0), (40, 3.2, 2), (80, 3.2, 0), (80, 3.2, 1)])
def test_hudgin_extension_large_grids(fwr, n, pad, k):
    """The same on 128^2 (fused kernel) and 256^2 (slab kernel), Wiener; the
    host path and an explicit warm start (which takes precedence) behave as
    with the zero extension."""
    sigma = 0.05
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sl, _, mask = synth.batch(n, 3, 29, sigma)
    plan = make_plan(fwr, mask, pad, fwr.WIENER, sigma ** 2, r0p, L0p)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    zero = plan.reconstruct(s, k).cpu()
    plan.set_extension(fwr.EXT_HUDGIN)
    ph = plan.reconstruct(s, k).cpu()
    for f in range(3):
        ref, _ = oracle.reconstruct(sl[f], mask, pad, k, oracle.FILTER_WIENER, sigma ** 2, r0p, L0p,
                                    ext_init="hudgin")
        assert within(ph[f].numpy(), ref, FP32_TOL, where=str(f))
    assert not torch.equal(ph, zero)
    sh = torch.tensor(sl, dtype=torch.float32).pin_memory()
    out = torch.empty((3, plan.N, plan.N), dtype=torch.float32).pin_memory()
    plan.reconstruct_host(sh, k, out)
    torch.cuda.synchronize()
    assert torch.equal(out, ph)
    ext0 = torch.zeros((3, 2, plan.N, plan.N), device="cuda")
    assert torch.equal(plan.reconstruct(s, k, ext_init=ext0).cpu(), zero)
    plan.set_extension(fwr.EXT_ZERO)
    assert torch.equal(plan.reconstruct(s, k).cpu(), zero)


def test_hudgin_extension_unsupported_paths(fwr):
    n, pad = 40, 3.2
    sl, _, mask = synth.batch(n, 1, 3, 0.05)
    plan = make_plan(fwr, mask, pad, fwr.LSQ)
    plan.set_extension(fwr.EXT_HUDGIN)
    plan.set_transform(fwr.TRANSFORM_DFT_BF16X3)
    with pytest.raises(fwr.FwrError):
        plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), 1)
    with pytest.raises(fwr.FwrError):
        plan.set_extension(2)


# --------------------------- non-power-of-two windows (direct-DFT kernel) --

@pytest.mark.parametrize("N,k,periodic,filt", [(46, 10, 0, "wiener"), (52, 10, 0, "wiener"), (46, 2, 1, "lsq"),
                                               (52, 3, 2, "lsq"), (42, 1, 0, "lsq")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_window_grids_against_oracle(fwr, N, k, periodic, filt, precision):
    """40 lenslets on the paper's small windows (N = n + 2w, w = 3 and 6, Sec.
    4.1; and w = 1) through fwr_plan_create_grid: FP32 and FP64 against the
    FP64 oracle on the same grid, with the extended slopes' in-pupil cells
    bitwise equal to the measurement."""
    n, sigma = 40, 0.05
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    F = 3
    sl, _, mask = synth.batch(n, F, 4600 + N + k, sigma)
    fl = fwr.WIENER if filt == "wiener" else fwr.LSQ
    plan = fwr.Plan(mask, 1.0, fl, sigma ** 2, r0p, L0p, periodic, grid=N)
    assert plan.N == N
    dtype = torch.float64 if precision == "fp64" else torch.float32
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    s = torch.tensor(sl, dtype=dtype, device="cuda")
    ext = torch.empty((F, 2, N, N), dtype=dtype, device="cuda")
    ph = (plan.reconstruct_f64 if precision == "fp64" else plan.reconstruct)(s, k, ext_out=ext).cpu().numpy()
    eo = ext.cpu().numpy().astype(np.float64)
    for f in range(F):
        ref, ref_ext = oracle.reconstruct(sl[f], mask, 1.0, k, FILTERS[filt], sigma ** 2, r0p, L0p, periodic, N=N)
        assert within(ph[f], ref, tol, where="N=%d f=%d" % (N, f))
        assert within(eo[f], ref_ext, 10 * tol, 10 * max_tol_for(tol), where="N=%d ext f=%d" % (N, f))
        s0x, s0y, P = oracle.embed(sl[f], mask, N)
        dt = np.float64 if precision == "fp64" else np.float32
        assert np.array_equal(eo[f][0][P].astype(dt), s0x[P].astype(dt))
        assert np.array_equal(eo[f][1][P].astype(dt), s0y[P].astype(dt))
    assert plan.status() == "FWR_OK"


def test_window_grid_options_and_limits(fwr):
    mask = synth.pupil_mask(40)
    plan = fwr.Plan(mask, 1.0, fwr.LSQ, grid=46)
    with pytest.raises(fwr.FwrError) as e:
        plan.set_transform(fwr.TRANSFORM_DFT_BF16X3)
    assert e.value.code == 2
    plan.set_extension(fwr.EXT_HUDGIN)
    with pytest.raises(fwr.FwrError) as e:
        plan.reconstruct(torch.zeros((1, 2, 40, 40), device="cuda"), 1)
    assert e.value.code == 2
    for bad, code in ((47, 2), (66, 2), (41, 1)):
        with pytest.raises(fwr.FwrError) as e:
            fwr.Plan(mask, 1.0, fwr.LSQ, grid=bad)
        assert e.value.code == code
    # a power of two through the explicit-grid call is the regular plan
    p128 = fwr.Plan(mask, 1.0, fwr.LSQ, grid=128)
    ref = fwr.Plan(mask, 3.2, fwr.LSQ)
    s = torch.tensor(synth.batch(40, 2, 5, 0.05)[0], dtype=torch.float32, device="cuda")
    assert torch.equal(p128.reconstruct(s, 2), ref.reconstruct(s, 2))


def test_alternating_plans_of_one_kernel(fwr):
    """Plans of one grid whose shared-memory needs differ (the staged pupil
    grows with n) share the fused kernel; the launcher caches its occupancy
    per size and only ever raises the kernel's shared-memory limit, so calls
    alternating between them all launch and repeat bitwise."""
    plans, inputs, first = [], [], []
    for n in (64, 40, 24):
        sl, _, mask = synth.batch(n, 4, 1200 + n, 0.05)
        pl = fwr.Plan(mask, 128.0 / n if n != 24 else 5.0, fwr.LSQ)
        assert pl.N == 128
        plans.append(pl)
        inputs.append(torch.tensor(sl, dtype=torch.float32, device="cuda"))
    for pl, s in zip(plans, inputs):
        first.append(pl.reconstruct(s, 2).clone())
    for _ in range(2):
        for pl, s, ref in zip(plans[::-1], inputs[::-1], first[::-1]):
            assert torch.equal(pl.reconstruct(s, 2), ref)
    for pl in plans:
        assert pl.status() == "FWR_OK"
