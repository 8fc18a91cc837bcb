"""Pins of the oracle's measurement-model variants against definitions that do
not go through the oracle's formulas (Sec. 2, Eq. 4 and its pixel correction).

* G_FRIED: the phase is known at the lenslet corners and each slope is the mean
  of the lenslet's two edge differences. Checked by taking those finite
  differences of single Fourier modes sampled on the grid.
* pixel = d_px / d: the difference is taken over d - d_px between the
  transverse averages at the lenslet centre +- (d - d_px)/2, as a slope per
  lenslet. Checked by Gauss-Legendre quadrature of continuous Fourier modes.
* Either way the LSQ reconstruction filter inverts the model: slopes made by G
  from a phase without null components give that phase back.
"""

import math

import numpy as np
import pytest

import oracle

MODES = [(0, 1), (1, 0), (3, -2), (-5, 4), (7, 7), (8, 3), (2, 8), (-8, -8), (6, -1)]


def mode(N, kx, ky):
    m, n = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return np.exp(2j * math.pi * (kx * n + ky * m) / N)


@pytest.mark.parametrize("kx,ky", MODES)
def test_fried_model_is_the_mean_of_two_edge_differences(kx, ky):
    N = 16
    phi = mode(N, kx, ky)
    right = np.roll(phi, -1, axis=1)          # phi[m, n + 1]
    up = np.roll(phi, -1, axis=0)             # phi[m + 1, n]
    up_right = np.roll(up, -1, axis=1)        # phi[m + 1, n + 1]
    sx = 0.5 * ((right - phi) + (up_right - up))
    sy = 0.5 * ((up - phi) + (up_right - right))
    Gx, Gy = oracle.measurement_filters(N, oracle.G_FRIED)
    assert np.max(np.abs(sx - Gx[ky % N, kx % N] * phi)) < 1e-12
    assert np.max(np.abs(sy - Gy[ky % N, kx % N] * phi)) < 1e-12


def quadrature_slopes(u, v, pixel, x0, y0, order=24):
    """x and y slopes of exp(2i pi (u x + v y)) for the lenslet whose lower-left
    corner is (x0, y0), pitch 1: the difference of the transverse averages at
    the centre +- L/2, L = 1 - pixel, divided by L."""
    t, w = np.polynomial.legendre.leggauss(order)
    s = 0.5 * (t + 1.0)                       # nodes on [0, 1]
    w = 0.5 * w
    L = 1.0 - pixel
    f = lambda x, y: np.exp(2j * math.pi * (u * x + v * y))  # noqa: E731
    sx = np.sum(w * (f(x0 + 0.5 + L / 2, y0 + s) - f(x0 + 0.5 - L / 2, y0 + s))) / L
    sy = np.sum(w * (f(x0 + s, y0 + 0.5 + L / 2) - f(x0 + s, y0 + 0.5 - L / 2))) / L
    return sx, sy


@pytest.mark.parametrize("pixel", [0.0, 1.0 / 6.0, 0.3])
@pytest.mark.parametrize("kx,ky", [(1, 0), (0, 3), (3, -2), (-5, 4), (7, 7), (8, 3), (3, 8), (-7, 1)])
def test_pixel_corrected_model_matches_quadrature(pixel, kx, ky):
    N = 16
    u, v = kx / N, ky / N
    if kx == N // 2:
        u = -0.5
    if ky == N // 2:
        v = -0.5
    Gx, Gy = oracle.measurement_filters(N, oracle.G_AVERAGED, pixel)
    for x0, y0 in [(0, 0), (3, 5), (11, 2)]:
        sx, sy = quadrature_slopes(u, v, pixel, x0, y0)
        phi0 = np.exp(2j * math.pi * (u * x0 + v * y0))
        # the transverse average on the Nyquist bin is the mean of its two
        # aliases (0): the quadrature of one alias is compared only off it
        if ky != N // 2:
            assert abs(sx - Gx[ky % N, kx % N] * phi0) < 1e-12, (x0, y0)
        if kx != N // 2:
            assert abs(sy - Gy[ky % N, kx % N] * phi0) < 1e-12, (x0, y0)


def test_pixel_correction_vanishes_continuously():
    N = 32
    Gx0, Gy0 = oracle.measurement_filters(N)
    Gx1, Gy1 = oracle.measurement_filters(N, oracle.G_AVERAGED, 1e-9)
    assert np.max(np.abs(Gx1 - Gx0)) < 1e-8 and np.max(np.abs(Gy1 - Gy0)) < 1e-8
    # the correction lengthens the measured difference at high frequency:
    # |a(u)| grows with d_px at the Nyquist column, as sin(pi (1-e)/2) / (1-e)
    a0 = oracle.shift_factor(N)
    a1 = oracle.shift_factor(N, 1.0 / 6.0)
    e = 1.0 / 6.0
    assert abs(a1[N // 2] - (-2.0 * math.cos(math.pi * e / 2) / (1 - e))) < 1e-14
    assert abs(a0[N // 2] + 2.0) < 1e-14


@pytest.mark.parametrize("g_model,pixel", [(oracle.G_FRIED, 0.0), (oracle.G_AVERAGED, 1.0 / 6.0),
                                           (oracle.G_FRIED, 1.0 / 6.0)])
def test_lsq_filter_inverts_each_model(g_model, pixel):
    N = 32
    rng = np.random.default_rng(7)
    spec = np.zeros((N, N), complex)
    for ky in range(-6, 7):
        for kx in range(-6, 7):
            if (kx, ky) != (0, 0):
                spec[ky % N, kx % N] = rng.standard_normal() + 1j * rng.standard_normal()
    spec = 0.5 * (spec + np.conj(np.roll(np.flip(spec), 1, axis=(0, 1))))   # Hermitian: real phase
    phi = oracle.real_idft2(spec)
    Gx, Gy = oracle.measurement_filters(N, g_model, pixel)
    sx = oracle.real_idft2(Gx * oracle.dft2(phi))
    sy = oracle.real_idft2(Gy * oracle.dft2(phi))
    Rx, Ry = oracle.reconstruction_filters(N, oracle.FILTER_LSQ, g_model=g_model, pixel=pixel)
    rec = oracle.final_reconstruct(sx, sy, Rx, Ry)
    assert np.max(np.abs(rec - (phi - phi.mean()))) < 1e-10


def test_full_path_takes_the_model():
    """With slopes made by a variant model on the whole grid, the full path
    (Gerchberg loop with that model, final LSQ filter) returns the phase."""
    n, pad = 16, 2.0
    N = oracle.grid_size(n, pad)
    rng = np.random.default_rng(3)
    spec = np.zeros((N, N), complex)
    for ky in range(-4, 5):
        for kx in range(-4, 5):
            if (kx, ky) != (0, 0):
                spec[ky % N, kx % N] = rng.standard_normal() + 1j * rng.standard_normal()
    spec = 0.5 * (spec + np.conj(np.roll(np.flip(spec), 1, axis=(0, 1))))
    phi = oracle.real_idft2(spec)
    Gx, Gy = oracle.measurement_filters(N, oracle.G_FRIED, 0.2)
    sx = oracle.real_idft2(Gx * oracle.dft2(phi))
    sy = oracle.real_idft2(Gy * oracle.dft2(phi))
    off = oracle.pupil_offset(n, N)
    slopes = np.stack([sx[off:off + n, off:off + n], sy[off:off + n, off:off + n]])
    mask = np.ones((n, n), bool)
    # the consistent slopes of the whole grid are a fixed point of the loop
    # only when the extension already holds them: give it as the warm start
    rec, ext = oracle.reconstruct(slopes, mask, pad, 3, oracle.FILTER_LSQ, periodic=oracle.PERIODIC_NONE,
                                  ext_init=np.stack([sx, sy]), g_model=oracle.G_FRIED, pixel=0.2)
    assert np.max(np.abs(rec - (phi - phi.mean()))) < 1e-10
    assert np.max(np.abs(ext[0] - sx)) < 1e-10
