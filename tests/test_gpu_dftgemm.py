"""Precision variant: 2-D transforms as dense DFT products on the tensor cores
with split-BF16 operands (FWR_TRANSFORM_DFT_BF16X3, grids 32^2 and 64^2).
The transform is checked against numpy's FFT, and whole reconstructions with
it against the FP64 oracle; the measured errors are printed (pytest -s) and
bounded here. A BF16 pair keeps 16 significant bits, so about 1e-5 per
transform and 1e-4 after the 22 transforms of 10 iterations is expected."""

import math

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


def rel_rms(got, ref):
    d = np.asarray(got, np.float64) - ref
    d -= d.mean()
    r = ref - ref.mean()
    return float(np.sqrt(np.sum(d * d) / np.sum(r * r)))


@pytest.mark.parametrize("N", [32, 64])
@pytest.mark.parametrize("inverse", [False, True])
def test_split_bf16_dft_matches_numpy(fwr, N, inverse):
    rng = np.random.default_rng(N + 10 * inverse)
    F = 9
    x = rng.standard_normal((F, N, N)) + 1j * rng.standard_normal((F, N, N))
    y = fwr.dft2_bf16x3(torch.tensor(x.astype(np.complex64), device="cuda"), inverse=inverse)
    y = y.cpu().numpy().astype(np.complex128)
    ref = np.fft.ifft2(x) * N * N if inverse else np.fft.fft2(x)
    err = np.sqrt(np.sum(np.abs(y - ref) ** 2) / np.sum(np.abs(ref) ** 2))
    print("split-BF16 DFT N=%d inverse=%d: relative error %.2e" % (N, inverse, err))
    assert err < 3e-5


@pytest.mark.parametrize("n,pad,k,filt", [(16, 2.0, 10, "lsq"), (30, 2.0, 3, "wiener"), (16, 2.0, 0, "lsq")])
def test_reconstruction_with_tensor_core_dft(fwr, n, pad, k, filt):
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sig = 0.05
    sl, _, mask = synth.batch(n, 3, 600 + n, sig)
    plan = fwr.Plan(mask, pad, fwr.WIENER if filt == "wiener" else fwr.LSQ, sig ** 2, r0p, L0p)
    plan.set_transform(fwr.TRANSFORM_DFT_BF16X3)
    ph = plan.reconstruct(torch.tensor(sl, dtype=torch.float32, device="cuda"), k).cpu().numpy()
    worst = 0.0
    for f in range(3):
        ref, _ = oracle.reconstruct(sl[f], mask, pad, k,
                                    oracle.FILTER_WIENER if filt == "wiener" else oracle.FILTER_LSQ,
                                    sig ** 2, r0p, L0p)
        worst = max(worst, rel_rms(ph[f], ref))
    print("split-BF16 DFT reconstruction n=%d N=%d k=%d: relative phase rms %.2e" % (n, plan.N, k, worst))
    assert worst < 1e-3


def test_transform_option_limits(fwr):
    plan = fwr.Plan(synth.pupil_mask(40), 3.2, fwr.LSQ)  # 128^2
    with pytest.raises(fwr.FwrError) as e:
        plan.set_transform(fwr.TRANSFORM_DFT_BF16X3)
    assert e.value.code == 2
    with pytest.raises(fwr.FwrError):
        plan.set_transform(7)
