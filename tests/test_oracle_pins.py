"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
not by the oracle itself (CPU only).

P1  separable DFT = brute-force quadruple-sum DFT = numpy's FFT (library).
P2  measurement filters = exact lenslet-averaged slopes of single Fourier modes
    obtained by Gauss-Legendre quadrature of the continuous mode (Eq. 4),
    Hermitian symmetry, the Roddier Laplacian small-frequency limit (Sec. 2),
    the null set, Wiener (Eq. 3) with zero noise = LSQ.
P3  single-mode closed form: consistent slopes of one Fourier mode are a fixed
    point of the Gerchberg loop and reconstruct that mode exactly; from zero
    padding the slope error to the truth never increases (Fejer monotonicity
    of alternating projections).
P4  Gerchberg invariant: the in-pupil slopes are the measurement after every
    iteration (Algorithm 1 step 4).
P5  periodic condition (Eq. PC): zero row sums of x slopes and zero column
    sums of y slopes; the inverse-FFT output has them without any fill.
P6  alternating projections: a point of the intersection found by a dense
    solver on a projector built from numpy's FFT is a fixed point of the loop,
    and the distances to it and to range(G) never grow.
P7  linearity.  P8  the spectral step is an orthogonal projector.
"""

import math

import numpy as np
import pytest

import oracle
from paper_1705_04298_gb300 import synth


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- P1 -------

@pytest.mark.parametrize("N", [4, 8, 6, 10])  # 6, 10: non-power-of-two grids (the paper's windows)
def test_p1_dft_matches_bruteforce(N):
    rng = _rng(N)
    x = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    X = np.zeros((N, N), dtype=complex)
    for ky in range(N):
        for kx in range(N):
            acc = 0j
            for m in range(N):
                for n in range(N):
                    acc += x[m, n] * complex(math.cos(-2 * math.pi * (ky * m + kx * n) / N),
                                             math.sin(-2 * math.pi * (ky * m + kx * n) / N))
            X[ky, kx] = acc
    got = oracle.dft2(x)
    assert np.max(np.abs(got - X)) <= 1e-13 * np.max(np.abs(X)) * N


@pytest.mark.parametrize("N", [16, 32, 128])
def test_p1_dft_matches_numpy_fft(N):
    rng = _rng(100 + N)
    x = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    ref = np.fft.fft2(x)
    got = oracle.dft2(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    back = oracle.idft2(got)
    assert np.max(np.abs(back - x)) <= 1e-12 * np.max(np.abs(x))


def test_p1_impulse_and_plane_wave():
    N = 16
    d = np.zeros((N, N))
    d[0, 0] = 1.0
    assert np.allclose(oracle.dft2(d), np.ones((N, N)), atol=1e-14)
    m, n = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ky, kx = 3, 5
    wave = np.exp(2j * math.pi * (ky * m + kx * n) / N)
    X = oracle.dft2(wave)
    expect = np.zeros((N, N), dtype=complex)
    expect[ky, kx] = N * N
    assert np.max(np.abs(X - expect)) <= 1e-11


# ---------------------------------------------------------------- P2 -------

def _exact_mode_slopes(N, u, v, A=1.0 + 0.0j, nodes=24):
    """Exact Shack-Hartmann slopes of the continuous mode
    phi(x, y) = A exp(2 i pi (u x + v y)) (x = column, y = row, unit pitch):
    sx[m, n] = int_0^1 phi(n+1, m+t) - phi(n, m+t) dt, sy likewise, evaluated
    by Gauss-Legendre quadrature (independent of the filter formulas)."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    m, n = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    phi = lambda x, y: A * np.exp(2j * math.pi * (u * x + v * y))  # noqa: E731
    sx = np.zeros((N, N), dtype=complex)
    sy = np.zeros((N, N), dtype=complex)
    for tk, wk in zip(t, w):
        sx += wk * (phi(n + 1, m + tk) - phi(n, m + tk))
        sy += wk * (phi(n + tk, m + 1) - phi(n + tk, m))
    return sx, sy, phi(n, m)


@pytest.mark.parametrize("N", [8, 16, 10])
def test_p2_filters_match_exact_lenslet_average(N):
    Gx, Gy = oracle.measurement_filters(N)
    u_of = oracle.signed_freq(N)
    worst = 0.0
    for ky in range(N):
        for kx in range(N):
            if ky == N // 2 or kx == N // 2:
                continue  # Nyquist row/column: symmetrised, checked below
            u, v = u_of[kx], u_of[ky]
            sx, sy, phi = _exact_mode_slopes(N, u, v)
            worst = max(worst, np.max(np.abs(sx - Gx[ky, kx] * phi)),
                        np.max(np.abs(sy - Gy[ky, kx] * phi)))
    assert worst <= 1e-12


def test_p2_nyquist_is_alias_average():
    N = 16
    Gx, Gy = oracle.measurement_filters(N)
    u_of = oracle.signed_freq(N)
    for kx in range(N):
        if kx == N // 2:
            continue
        u = u_of[kx]
        sxa, _, phia = _exact_mode_slopes(N, u, -0.5)
        sxb, _, phib = _exact_mode_slopes(N, u, +0.5)
        # both aliases sample to the same grid values; G on the Nyquist row is
        # the mean of their two transfer values
        ga = (sxa / phia)[0, 0]
        gb = (sxb / phib)[0, 0]
        assert abs(Gx[N // 2, kx] - 0.5 * (ga + gb)) <= 1e-12
        # and the same for Gy on the Nyquist column
        _, sya, pa = _exact_mode_slopes(N, -0.5, u)
        _, syb, pb = _exact_mode_slopes(N, +0.5, u)
        assert abs(Gy[kx, N // 2] - 0.5 * ((sya / pa)[0, 0] + (syb / pb)[0, 0])) <= 1e-12


@pytest.mark.parametrize("N", [8, 32, 128])
def test_p2_hermitian_and_closed_form_modulus(N):
    Gx, Gy = oracle.measurement_filters(N)
    neg = (-np.arange(N)) % N
    assert np.max(np.abs(Gx[np.ix_(neg, neg)] - np.conj(Gx))) <= 1e-15
    assert np.max(np.abs(Gy[np.ix_(neg, neg)] - np.conj(Gy))) <= 1e-15
    u = oracle.signed_freq(N)
    U, V = np.meshgrid(u, u)  # U varies along columns (kx), V along rows (ky)
    gx2 = 4 * np.sin(math.pi * U) ** 2 * np.sinc(V) ** 2
    gx2[N // 2, :] = 0.0
    assert np.max(np.abs(np.abs(Gx) ** 2 - gx2)) <= 1e-14


def test_p2_roddier_laplacian_limit():
    N = 4096
    Gx, Gy = oracle.measurement_filters(N)
    g2 = np.abs(Gx) ** 2 + np.abs(Gy) ** 2
    for ky, kx in [(0, 1), (1, 0), (1, 1), (2, 3)]:
        u, v = kx / N, ky / N
        lap = (2 * math.pi) ** 2 * (u * u + v * v)
        assert abs(g2[ky, kx] / lap - 1.0) < 1e-4


@pytest.mark.parametrize("N", [16, 64])
def test_p2_null_set_and_wiener_limit(N):
    Gx, Gy = oracle.measurement_filters(N)
    g2 = np.abs(Gx) ** 2 + np.abs(Gy) ** 2
    nulls = set(zip(*np.nonzero(g2 < oracle.NULL_THRESHOLD)))
    assert nulls == {(0, 0), (N // 2, N // 2)}
    Rx, Ry = oracle.reconstruction_filters(N, oracle.FILTER_LSQ)
    Wx, Wy = oracle.reconstruction_filters(N, oracle.FILTER_WIENER, 0.0, 0.75, 125.0)
    assert np.array_equal(Rx, Wx) and np.array_equal(Ry, Wy)
    # Wiener gain is a shrinkage of LSQ that grows with the noise variance
    prev = np.abs(Rx)
    for nv in (1e-4, 1e-2, 1.0):
        Wx, _ = oracle.reconstruction_filters(N, oracle.FILTER_WIENER, nv, 0.75, 125.0)
        cur = np.abs(Wx)
        assert np.all(cur <= prev + 1e-15)
        prev = cur


# ---------------------------------------------------------------- P3 -------

def _mode_problem(N, n, u, v, A):
    """Real single-mode phase and its exact slopes on the N x N grid."""
    sx, sy, phi = _exact_mode_slopes(N, u, v, A)
    return sx.real, sy.real, phi.real


@pytest.mark.parametrize("mode", [oracle.PERIODIC_BEFORE_EACH_FFT, oracle.PERIODIC_FINAL_ONLY,
                                  oracle.PERIODIC_NONE])
def test_p3_single_mode_fixed_point(mode):
    N, n = 32, 16
    u, v = 3 / N, -5 / N
    sx, sy, phi = _mode_problem(N, n, u, v, 0.7 - 0.4j)
    mask = synth.pupil_mask(n)
    off = oracle.pupil_offset(n, N)
    slopes = np.stack([sx[off:off + n, off:off + n], sy[off:off + n, off:off + n]])
    slopes = np.where(mask[None], slopes, 0.0)
    hist = []
    phase, ext = oracle.reconstruct(slopes, mask, 2.0, 4, oracle.FILTER_LSQ, periodic=mode,
                                    ext_init=np.stack([sx, sy]), history=hist)
    for hx, hy in hist:
        assert np.max(np.abs(hx - sx)) <= 1e-12 and np.max(np.abs(hy - sy)) <= 1e-12
    assert np.max(np.abs(phase - (phi - phi.mean()))) <= 1e-12


@pytest.mark.parametrize("mode", [oracle.PERIODIC_BEFORE_EACH_FFT, oracle.PERIODIC_NONE])
def test_p3_single_mode_fixed_point_on_a_window_grid(mode):
    """The same fixed point on a non-power-of-two grid: 40 lenslets with a
    window of 3 lenslets on each side (N = 46, Sec. 4.1)."""
    N, n = 46, 40
    u, v = 5 / N, -7 / N
    sx, sy, phi = _mode_problem(N, n, u, v, 0.3 + 0.9j)
    mask = synth.pupil_mask(n)
    off = oracle.pupil_offset(n, N)
    assert off == 3
    slopes = np.stack([sx[off:off + n, off:off + n], sy[off:off + n, off:off + n]])
    slopes = np.where(mask[None], slopes, 0.0)
    hist = []
    phase, ext = oracle.reconstruct(slopes, mask, 1.0, 3, oracle.FILTER_LSQ, periodic=mode,
                                    ext_init=np.stack([sx, sy]), history=hist, N=N)
    assert phase.shape == (N, N)
    for hx, hy in hist:
        assert np.max(np.abs(hx - sx)) <= 1e-12 and np.max(np.abs(hy - sy)) <= 1e-12
    assert np.max(np.abs(phase - (phi - phi.mean()))) <= 1e-12


def test_p3_zero_padding_error_never_increases():
    N, n = 32, 16
    sx, sy, phi = _mode_problem(N, n, 2 / N, 1 / N, 1.0 + 0.3j)
    mask = synth.pupil_mask(n)
    off = oracle.pupil_offset(n, N)
    slopes = np.where(mask[None], np.stack([sx[off:off + n, off:off + n],
                                            sy[off:off + n, off:off + n]]), 0.0)
    hist = []
    oracle.reconstruct(slopes, mask, 2.0, 30, periodic=oracle.PERIODIC_NONE, history=hist)
    err = [math.sqrt(np.sum((hx - sx) ** 2 + (hy - sy) ** 2)) for hx, hy in hist]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(err, err[1:]))
    assert err[-1] < 0.99 * err[0]


# ---------------------------------------------------------------- P4/P5 ----

@pytest.mark.parametrize("mode", [oracle.PERIODIC_BEFORE_EACH_FFT, oracle.PERIODIC_NONE])
def test_p4_in_pupil_slopes_are_the_measurement(mode):
    fr = synth.frame(16, 7, 0.05)
    hist = []
    _, ext = oracle.reconstruct(fr["slopes"], fr["mask"], 2.0, 5, periodic=mode, history=hist)
    N = 32
    s0x, s0y, P = oracle.embed(fr["slopes"], fr["mask"], N)
    for hx, hy in hist + [(ext[0], ext[1])]:
        assert np.array_equal(hx[P], s0x[P]) and np.array_equal(hy[P], s0y[P])


def test_p5_periodic_fill_zero_sums():
    fr = synth.frame(16, 3, 0.05)
    _, ext = oracle.reconstruct(fr["slopes"], fr["mask"], 2.0, 3,
                                periodic=oracle.PERIODIC_BEFORE_EACH_FFT)
    scale = np.max(np.abs(ext))
    assert np.max(np.abs(ext[0].sum(axis=1))) <= 1e-12 * scale * 32
    assert np.max(np.abs(ext[1].sum(axis=0))) <= 1e-12 * scale * 32


def test_p5_projection_output_has_zero_sums():
    rng = _rng(5)
    sx, sy = rng.standard_normal((2, 32, 32))
    px, py = oracle.spectral_projection(sx, sy)
    assert np.max(np.abs(px.sum(axis=1))) <= 1e-12
    assert np.max(np.abs(py.sum(axis=0))) <= 1e-12


# ---------------------------------------------------------------- P6 -------

def test_p6_alternating_projection_fixed_point():
    """With no periodic fill the loop alternates the orthogonal projection
    onto range(G) and the projection onto {s : s = s0 in the pupil}.  A point
    of their intersection, found by a dense pseudo-inverse solve on a
    projector built from numpy's FFT, must be a fixed point of one oracle
    iteration; the iterates' distance to it and to range(G) never grow."""
    N, n = 16, 6
    mask = synth.pupil_mask(n)
    rng = _rng(11)
    slopes = np.where(mask[None], rng.standard_normal((2, n, n)), 0.0)
    s0x, s0y, P = oracle.embed(slopes, mask, N)
    Gx, Gy = oracle.measurement_filters(N)
    cols = []
    for idx in range(N * N):
        e = np.zeros((N, N))
        e.flat[idx] = 1.0
        E = np.fft.fft2(e)
        cols.append(np.concatenate([np.fft.ifft2(Gx * E).real.ravel(),
                                    np.fft.ifft2(Gy * E).real.ravel()]))
    B = np.array(cols).T
    Q, sv, _ = np.linalg.svd(B, full_matrices=False)
    Q = Q[:, sv > 1e-10 * sv[0]]
    Pi = Q @ Q.T
    out = np.concatenate([~P.ravel(), ~P.ravel()])
    s0 = np.concatenate([s0x.ravel(), s0y.ravel()])
    # fixed point: z = [Pi (s0 + E z)]_out  <=>  (I - Pi_oo) z = Pi_oi s0_in
    A = np.eye(int(out.sum())) - Pi[np.ix_(out, out)]
    z = np.linalg.pinv(A, rcond=1e-10) @ (Pi[out][:, ~out] @ s0[~out])
    s_star = s0.copy()
    s_star[out] = z
    ext = np.stack([s_star[:N * N].reshape(N, N), s_star[N * N:].reshape(N, N)])
    hist = []
    oracle.gerchberg_extend(s0x, s0y, P, 1, oracle.PERIODIC_NONE, ext_init=ext, history=hist)
    scale = np.max(np.abs(s_star))
    assert np.max(np.abs(hist[0][0] - ext[0])) <= 1e-12 * scale
    assert np.max(np.abs(hist[0][1] - ext[1])) <= 1e-12 * scale

    hist = []
    oracle.gerchberg_extend(s0x, s0y, P, 200, oracle.PERIODIC_NONE, history=hist)
    flat = [np.concatenate([hx.ravel(), hy.ravel()]) for hx, hy in hist]
    to_star = [np.linalg.norm(f - s_star) for f in flat]
    to_range = [np.linalg.norm(f - Pi @ f) for f in flat]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(to_star, to_star[1:]))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(to_range, to_range[1:]))
    assert to_range[-1] < 0.9 * to_range[0]


# ---------------------------------------------------------------- P7/P8 ----

def test_p7_linearity():
    fa = synth.frame(16, 21, 0.05)
    fb = synth.frame(16, 22, 0.05)
    mask = fa["mask"]
    args = dict(pad_factor=2.0, iters=3, filt=oracle.FILTER_WIENER, noise_var=0.0025,
                r0_pitch=0.3, L0_pitch=50.0)
    pa, _ = oracle.reconstruct(fa["slopes"], mask, **args)
    pb, _ = oracle.reconstruct(fb["slopes"], mask, **args)
    pab, _ = oracle.reconstruct(2.0 * fa["slopes"] - 0.5 * fb["slopes"], mask, **args)
    assert np.max(np.abs(pab - (2.0 * pa - 0.5 * pb))) <= 1e-12 * np.max(np.abs(pab))


def test_p8_projection_idempotent_and_nonexpansive():
    rng = _rng(8)
    sx, sy = rng.standard_normal((2, 16, 16))
    px, py = oracle.spectral_projection(sx, sy)
    qx, qy = oracle.spectral_projection(px, py)
    assert np.max(np.abs(qx - px)) <= 1e-12 and np.max(np.abs(qy - py)) <= 1e-12
    assert np.sum(px ** 2 + py ** 2) <= np.sum(sx ** 2 + sy ** 2)
    # orthogonality: the residual is orthogonal to the projection
    assert abs(np.sum((sx - px) * px + (sy - py) * py)) <= 1e-10


# ------------------------------------------------------- filter choice ----

@pytest.mark.parametrize("sigma", [0.3, 1.0])
def test_wiener_is_mse_optimal_among_scaled_noise_terms(sigma):
    """Eq. 3 with gamma = 1 minimises the expected residual.  On a periodic,
    fully measured grid whose phase is a von Karman screen generated at the
    grid spacing (band-limited, made by the input generator in metres) and
    whose slopes are G applied to it (G pinned above) plus white noise,
    scaling the noise term by 1/2, 2 or 4, or dropping it (LSQ), must give a
    larger residual.  This fixes the units of the PSD (r0 and L0 in pitches)
    and of the noise variance."""
    N = 32
    d = 0.5
    r0, L0 = 0.15, 25.0
    Gx, Gy = oracle.measurement_filters(N)
    full = np.ones((N, N), dtype=bool)
    errs = {}
    for name, scale in [("lsq", None), ("w/2", 0.5), ("w", 1.0), ("w*2", 2.0), ("w*4", 4.0)]:
        tot = 0.0
        for f in range(40):
            rng = _rng(7000 + f)
            ph = synth.von_karman_screen(N, d, r0, L0, rng)
            spec = np.fft.fft2(ph)
            sl = np.stack([np.fft.ifft2(Gx * spec).real, np.fft.ifft2(Gy * spec).real])
            sl = sl + sigma * rng.standard_normal(sl.shape)
            if scale is None:
                est, _ = oracle.reconstruct(sl, full, 1.0, 0, oracle.FILTER_LSQ,
                                            periodic=oracle.PERIODIC_NONE)
            else:
                est, _ = oracle.reconstruct(sl, full, 1.0, 0, oracle.FILTER_WIENER,
                                            scale * sigma ** 2, r0 / d, L0 / d,
                                            periodic=oracle.PERIODIC_NONE)
            res = est - ph
            res -= res.mean()
            tot += np.mean(res ** 2)
        errs[name] = tot
    for other in ("lsq", "w/2", "w*2", "w*4"):
        assert errs["w"] < errs[other], errs
