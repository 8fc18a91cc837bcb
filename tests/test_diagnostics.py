"""The diagnostics' host-side arithmetic, checked on the CPU: the residual
PSD against known residuals, the noise propagation coefficient against its
exact expectation for a linear reconstructor built from the oracle."""

import math

import numpy as np

import oracle
from paper_1705_04298_gb300 import diagnostics as dg


def test_corner_mask():
    mask = np.zeros((3, 3), bool)
    mask[1, 1] = True
    cm = dg.corner_mask(mask)
    assert cm.sum() == 4 and cm[1, 1] and cm[2, 2] and cm[1, 2] and cm[2, 1]


def test_residual_psd_zero_for_exact_and_peaked_for_a_sinusoid():
    n = 15
    mask = np.ones((n, n), bool)
    cm = dg.corner_mask(mask)
    truth = np.random.default_rng(0).standard_normal((3, n + 1, n + 1))
    f, psd = dg.residual_psd(truth, truth, cm)
    assert np.all(psd == 0.0)
    # a residual at 0.3 cycles per pitch along x puts its power in that bin
    x = np.arange(n + 1)[None, :] * np.ones((n + 1, 1))
    est = truth + np.cos(2 * math.pi * 0.3 * x)[None]
    bins = np.array([0.0, 0.1, 0.2, 0.25, 0.35, 0.4, 0.5])
    f, psd = dg.residual_psd(est, truth, cm, pad=8, bins=bins)
    assert np.argmax(psd) == 3
    # (the 16-sample window leaks some power into every bin)
    assert psd[3] > 5 * max(psd[0], psd[1], psd[5])


def test_noise_propagation_matches_exact_expectation():
    """For a linear reconstructor R the expected coefficient is
    tr(C R R^T C) / (pupil corners), C the piston removal over the corners;
    R is built column by column from the oracle's impulse responses."""
    n, pad, k = 4, 2.0, 2
    mask = np.ones((n, n), bool)
    mask[0, 0] = False
    cm = dg.corner_mask(mask)

    def rec(slopes):
        return np.stack([oracle.reconstruct(s, mask, pad, k)[0] for s in slopes])

    basis = np.zeros((2 * n * n, 2, n, n))
    idx = [(c, i, j) for c in range(2) for i in range(n) for j in range(n) if mask[i, j]]
    for b, (c, i, j) in enumerate(idx):
        basis[b, c, i, j] = 1.0
    cols = dg.pupil_corners(rec(basis[:len(idx)]), n)[:, cm]      # (slopes, corners)
    Rm = cols.T                                                      # corners x slopes
    Cc = np.eye(Rm.shape[0]) - 1.0 / Rm.shape[0]
    exact = np.trace(Cc @ Rm @ Rm.T @ Cc) / Rm.shape[0]
    mc = dg.noise_propagation(rec, mask, n_frames=3000, seed=4)
    assert abs(mc - exact) < 0.05 * exact, (mc, exact)
