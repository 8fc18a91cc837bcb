"""The CPU FFT baseline (cpu_baseline/, timed by bench.py beside the oracle)
against the FP64 direct-DFT oracle: FP64 to rounding, FP32 within the FP32
bound of the GPU paths, every periodic mode and both filters (Algorithm 1 of
Sec. 3.3, Eq. PC, Eqs. 2-3)."""

import numpy as np
import pytest

import cpu_baseline
import oracle
from paper_1705_04298_gb300 import synth
from parity_check import FP32_MAX, FP32_RMS, errors


@pytest.fixture(scope="module")
def lib():
    try:
        cpu_baseline.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    return cpu_baseline


@pytest.mark.parametrize("periodic", [0, 1, 2])
@pytest.mark.parametrize("filt", [oracle.FILTER_LSQ, oracle.FILTER_WIENER])
def test_fft_baseline_matches_oracle(lib, periodic, filt):
    n, pad, k, sigma = 12, 2.0, 3, 0.05
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sl, _, mask = synth.batch(n, 3, 41 + periodic, sigma)
    out64 = lib.reconstruct(sl, mask, pad, k, filt, sigma ** 2, r0p, L0p, periodic, precision=64, n_threads=2)
    out32 = lib.reconstruct(sl, mask, pad, k, filt, sigma ** 2, r0p, L0p, periodic, precision=32, n_threads=2)
    for f in range(3):
        ref, _ = oracle.reconstruct(sl[f], mask, pad, k, filt, sigma ** 2, r0p, L0p, periodic)
        rms, mx = errors(out64[f], ref)
        assert rms < 1e-12 and mx < 1e-12, (rms, mx)
        rms, mx = errors(out32[f], ref)
        assert rms < FP32_RMS and mx < FP32_MAX, (rms, mx)


def test_fft_baseline_40x40_128grid_k10(lib):
    """The benchmark workload's geometry (40x40 lenslets on 128^2, k = 10)."""
    n, pad, k, sigma = 40, 3.2, 10, 0.1
    r0p, L0p = synth.pitch_units(n, 0.15, 25.0)
    sl, _, mask = synth.batch(n, 2, 1000, sigma)
    out = lib.reconstruct(sl, mask, pad, k, oracle.FILTER_WIENER, sigma ** 2, r0p, L0p, 0, precision=32)
    assert out.shape == (2, 128, 128)
    ref, _ = oracle.reconstruct(sl[1], mask, pad, k, oracle.FILTER_WIENER, sigma ** 2, r0p, L0p, 0)
    rms, mx = errors(out[1], ref)
    assert rms < FP32_RMS and mx < FP32_MAX, (rms, mx)
    assert abs(out[1].mean()) < 1e-9 * np.abs(out[1]).max() + 1e-7
