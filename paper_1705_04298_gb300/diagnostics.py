"""The paper's diagnostics of an extension method (Sec. 4, open loop):

* the power spectral density of the residual phase (reconstruction minus the
  true phase over the pupil), radially averaged, where the aperture's cut-off
  shows at low spatial frequencies and an enforced periodic condition at the
  waffle frequency 1/(2d);
* the noise propagation coefficient: the variance of the phase reconstructed
  from pure measurement noise over the pupil, per unit slope-noise variance.

Both are host-side analysis of reconstructions (numpy); the reconstructions
themselves go through the library (`Plan.reconstruct`). Phases are compared at
the lenslet corners inside the pupil, the samples the reconstruction and the
synthetic truth share (grid phase [m, n] is the lower-left corner of slope
cell [m, n]).
"""

import numpy as np


def corner_mask(mask):
    """(n+1, n+1) bool: the corners of the pupil's lenslets."""
    mask = np.asarray(mask, bool)
    n = mask.shape[0]
    cm = np.zeros((n + 1, n + 1), bool)
    cm[:n, :n] |= mask
    cm[1:, :n] |= mask
    cm[:n, 1:] |= mask
    cm[1:, 1:] |= mask
    return cm


def pupil_corners(phase, n):
    """(F, N, N) reconstructed phases -> (F, n+1, n+1) at the lenslet corners of
    the centred n x n array."""
    phase = np.asarray(phase, np.float64)
    N = phase.shape[-1]
    off = (N - n) // 2
    return phase[..., off:off + n + 1, off:off + n + 1]


def residual_psd(est, truth, cmask, pad=4, bins=None):
    """Radially averaged PSD of the residual est - truth over the pupil corners.

    est, truth: (F, n+1, n+1) phases (radians); cmask: (n+1, n+1) bool. Each
    frame's residual has its piston over the pupil removed and is zero outside
    it, zero-padded to pad (n+1) samples, transformed, and |X|^2 / (samples in
    the pupil) averaged over frames. Frequencies in cycles per lenslet pitch
    (0 .. 1/2; 1/2 is the waffle frequency 1/(2d)). Returns (f, psd) with
    psd[b] the mean over the frequencies in bin b; by Parseval the sum over all
    frequencies of |X|^2 / (samples in the pupil) is the mean-square residual.
    """
    est = np.asarray(est, np.float64)
    truth = np.asarray(truth, np.float64)
    cm = np.asarray(cmask, bool)
    M = pad * cm.shape[0]
    acc = np.zeros((M, M))
    for e, t in zip(est, truth):
        d = np.where(cm, e - t, 0.0)
        d[cm] -= d[cm].mean()
        x = np.zeros((M, M))
        x[:cm.shape[0], :cm.shape[1]] = d
        acc += np.abs(np.fft.fft2(x)) ** 2
    acc /= len(est) * cm.sum() * M * M
    u = np.fft.fftfreq(M)
    fr = np.sqrt(u[None, :] ** 2 + u[:, None] ** 2)
    if bins is None:
        bins = np.linspace(0.0, 0.5, 11)
    f = 0.5 * (bins[1:] + bins[:-1])
    psd = np.array([acc[(fr >= lo) & (fr < hi)].mean() for lo, hi in zip(bins[:-1], bins[1:])])
    return f, psd


def noise_propagation(reconstruct, mask, n_frames=256, seed=0):
    """Variance of the reconstructed phase over the pupil corners (piston
    removed, mean over frames) per unit slope-noise variance, for slopes that
    are unit-variance white noise in every pupil lenslet.

    reconstruct: callable taking float64 slopes (F, 2, n, n) and returning the
    phases (F, N, N); mask: (n, n) pupil. The coefficient is the quantity of
    the paper's error-propagation figure (noise variance in, phase variance
    out), in rad^2 per rad^2.
    """
    mask = np.asarray(mask, bool)
    n = mask.shape[0]
    rng = np.random.default_rng(seed)
    slopes = rng.standard_normal((n_frames, 2, n, n)) * mask
    phase = pupil_corners(reconstruct(slopes), n)
    cm = corner_mask(mask)
    v = []
    for p in phase:
        d = p[cm] - p[cm].mean()
        v.append(np.mean(d * d))
    return float(np.mean(v))
