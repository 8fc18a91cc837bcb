"""Seeded synthetic inputs for the reconstructor: pupil masks, von Karman
phase screens and Shack-Hartmann slopes.

This module feeds both the CUDA path and the FP64 oracle. It holds none of
the reconstruction's arithmetic (no measurement filter, no Gerchberg step, no
reconstructor): it only makes the data a wave-front sensor would deliver.

Workload recipe (stand-in for the paper's end-to-end simulations, Table 1):

* circular unobstructed pupil of diameter D = 8 m sampled by n x n lenslets of
  pitch d = D/n; lenslet (i, j) is valid when its centre lies within D/2 of
  the pupil centre;
* von Karman phase screen (r0 at 500 nm, outer scale L0) made by the FFT
  method on a periodic M x M grid at spacing d/2 (2x oversampling),
  M = next power of two >= 4n, zero-frequency term removed;
* slopes: for lenslet (i, j) the x slope is the difference between the
  screen's right and left lenslet edges, each edge averaged with the
  trapezoid weights (1/4, 1/2, 1/4) over its three samples; y likewise. This
  is a deliberate mismatch with the reconstructor's band-limited model and
  stands in for the aliasing of a real sensor;
* white Gaussian noise of standard deviation sigma (radians) on every slope;
* the true phase is the screen at the lenslet corners ((n+1) x (n+1)).

Every frame is generated from its own seed with numpy's PCG64 generator,
which gives the same numbers on every platform.
"""

import math

import numpy as np

TELESCOPE_D = 8.0


def _next_pow2(x):
    p = 1
    while p < x:
        p *= 2
    return p


def pupil_mask(n):
    """(n, n) bool: lenslet centre within D/2 of the pupil centre."""
    c = np.arange(n) + 0.5 - n / 2.0
    r2 = c[:, None] ** 2 + c[None, :] ** 2
    return r2 <= (n / 2.0) ** 2


def von_karman_screen(M, delta, r0, L0, rng):
    """Periodic M x M phase screen (radians) at sample spacing `delta` metres."""
    f = np.fft.fftfreq(M, d=delta)
    f2 = f[None, :] ** 2 + f[:, None] ** 2
    psd = 0.023 * r0 ** (-5.0 / 3.0) * (f2 + L0 ** -2.0) ** (-11.0 / 6.0)
    psd[0, 0] = 0.0
    df = 1.0 / (M * delta)
    c = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) * np.sqrt(psd) * df
    return np.real(np.fft.ifft2(c)) * (M * M)


def lenslet_slopes(screen, n, row0=0, col0=0):
    """(2, n, n) x/y slopes and (n+1, n+1) corner phase from a 2x-oversampled
    screen whose pupil origin is the sample (row0, col0)."""
    M = screen.shape[0]
    rows = (row0 + np.arange(2 * n + 1)) % M
    cols = (col0 + np.arange(2 * n + 1)) % screen.shape[1]
    s = screen[np.ix_(rows, cols)]
    w = (0.25, 0.5, 0.25)
    sx = np.zeros((n, n))
    sy = np.zeros((n, n))
    for r in range(3):
        # x: right edge (column 2j+2) minus left edge (column 2j), averaged down the edge
        sx += w[r] * (s[r:r + 2 * n:2, 2:2 * n + 1:2] - s[r:r + 2 * n:2, 0:2 * n:2])
        # y: top edge (row 2i+2) minus bottom edge (row 2i), averaged along the edge
        sy += w[r] * (s[2:2 * n + 1:2, r:r + 2 * n:2] - s[0:2 * n:2, r:r + 2 * n:2])
    corners = s[0:2 * n + 1:2, 0:2 * n + 1:2].copy()
    return np.stack([sx, sy]), corners


def frame(n, seed, sigma, r0=0.15, L0=25.0, D=TELESCOPE_D):
    """One seeded frame: dict(slopes (2,n,n), phase (n+1,n+1), mask (n,n))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = D / n
    M = _next_pow2(4 * n)
    screen = von_karman_screen(M, d / 2.0, r0, L0, rng)
    slopes, corners = lenslet_slopes(screen, n)
    slopes = slopes + sigma * rng.standard_normal(slopes.shape)
    mask = pupil_mask(n)
    slopes = np.where(mask[None], slopes, 0.0)
    return {"slopes": slopes, "phase": corners, "mask": mask}


def batch(n, F, seed0, sigma, r0=0.15, L0=25.0, D=TELESCOPE_D):
    """F frames with seeds seed0 .. seed0+F-1; sigma may be a scalar or a
    sequence that is cycled over the frames.  Returns (slopes (F,2,n,n),
    phases (F,n+1,n+1), mask (n,n)) in float64."""
    sig = np.atleast_1d(np.asarray(sigma, dtype=np.float64))
    slopes = np.empty((F, 2, n, n))
    phases = np.empty((F, n + 1, n + 1))
    mask = pupil_mask(n)
    for f in range(F):
        fr = frame(n, seed0 + f, float(sig[f % len(sig)]), r0, L0, D)
        slopes[f] = fr["slopes"]
        phases[f] = fr["phase"]
    return slopes, phases, mask


def pitch_units(n, r0, L0, D=TELESCOPE_D):
    """(r0/d, L0/d) for an n-lenslet pupil of diameter D."""
    d = D / n
    return r0 / d, L0 / d


def frozen_flow(n, T, seed, sigma, r0=0.12, L0=25.0, wind=10.0, rate=1000.0,
                D=TELESCOPE_D, length_factor=8):
    """T frames of a frozen-flow screen moving along x at `wind` m/s sampled at
    `rate` Hz.  The screen is length_factor*2n samples long in x (periodic) and
    is shifted by bilinear interpolation.  Returns (slopes (T,2,n,n),
    phases (T,n+1,n+1), mask)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = D / n
    delta = d / 2.0
    My = _next_pow2(4 * n)
    Mx = My * length_factor
    f_x = np.fft.fftfreq(Mx, d=delta)
    f_y = np.fft.fftfreq(My, d=delta)
    f2 = f_x[None, :] ** 2 + f_y[:, None] ** 2
    psd = 0.023 * r0 ** (-5.0 / 3.0) * (f2 + L0 ** -2.0) ** (-11.0 / 6.0)
    psd[0, 0] = 0.0
    dfx = 1.0 / (Mx * delta)
    dfy = 1.0 / (My * delta)
    c = (rng.standard_normal((My, Mx)) + 1j * rng.standard_normal((My, Mx))) * np.sqrt(psd * dfx * dfy)
    screen = np.real(np.fft.ifft2(c)) * (Mx * My)
    mask = pupil_mask(n)
    step = wind / rate / delta
    slopes = np.empty((T, 2, n, n))
    phases = np.empty((T, n + 1, n + 1))
    for t in range(T):
        shift = step * t
        s0 = int(math.floor(shift))
        fr = shift - s0
        a = np.roll(screen, -s0, axis=1)
        b = np.roll(screen, -s0 - 1, axis=1)
        sc = (1.0 - fr) * a + fr * b
        sl, ph = lenslet_slopes(sc, n)
        sl = sl + sigma * rng.standard_normal(sl.shape)
        slopes[t] = np.where(mask[None], sl, 0.0)
        phases[t] = ph
    return slopes, phases, mask
