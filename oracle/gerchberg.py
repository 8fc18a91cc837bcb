"""Plain FP64 CPU oracle for iterative Fourier wave-front reconstruction.

TEST INFRASTRUCTURE. This module is the independent reference that the CUDA
path is checked against. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library itself never does,
and it shares no code, tables or constants with the CUDA sources.

It is deliberately slow and literal:

* every 2-D transform is a direct separable DFT (one dense DFT matrix applied
  to the rows and one to the columns, O(N^3) per transform);
* the x and y slopes are transformed as two separate real fields (no packing);
* the Gerchberg loop follows the four steps of Algorithm 1 (Sec. 3.3) in the
  paper's order, and the final phase comes from the Wiener / least-squares
  filter of Eq. 3.

Conventions (the paper leaves them open; each is a reading of it):

* Grid index [m, n]: m is the row (y), n the column (x). x slopes are summed
  along a row in Eq. PC, so this matches the paper's s_x(m, n).
* Frequencies u = kx/N, v = ky/N are signed in [-1/2, 1/2), in cycles per
  lenslet pitch d.
* Slopes are phase differences across one lenslet (radians); the phase sample
  [m, n] is the lower-left corner of slope cell [m, n].
* The discrete Shack-Hartmann model of Eq. 4 (lenslet sampling x lenslet
  averaging x gradient) is read as
      Gx(u, v) = (exp(2i pi u) - 1) * sinc(v) * exp(i pi v)
      Gy(u, v) = sinc(u) * exp(i pi u) * (exp(2i pi v) - 1)
  with the transverse factor set to 0 on the Nyquist row/column (the average
  of its two aliases), so that G is Hermitian on the grid.
* Measurement-model variants (options of the same model):
  - G_FRIED: the phase known at the lenslet corners, each slope the mean of
    the lenslet's two edge differences: transverse factor cos(pi v) exp(i pi v);
  - pixel = d_px / d > 0: the difference of Sec. 2 taken over d - d_px (the
    correction to Eq. 4 for a pixelated detector), between the transverse
    averages at the lenslet centre +- (d - d_px)/2 and scaled back to a slope
    per lenslet: exp(2i pi u) - 1 becomes
    2i sin(pi u (1 - pixel)) / (1 - pixel) exp(i pi u).
* 1/|G|^2 is set to 0 where |G|^2 < 1e-14 (piston and the (-1/2, -1/2)
  waffle bin), so every reconstructed phase has zero mean over the grid.
* The Wiener noise-to-signal ratio of Eq. 3 (gamma = 1) is
  noise_var / W_phi(kappa) with the von Karman PSD in pitch units
      W_phi = 0.023 (r0/d)^(-5/3) (kappa^2 + (d/L0)^2)^(-11/6).
"""

import math

import numpy as np

# Where the periodic condition of Eq. PC is applied (Sec. 3.2; Algorithm 1
# step 5).  BEFORE_EACH_FFT: before every forward transform, including the
# final one (so also at zero iterations).  FINAL_ONLY: only before the final
# reconstruction, as printed in Algorithm 1.  NONE: never.
PERIODIC_BEFORE_EACH_FFT = 0
PERIODIC_FINAL_ONLY = 1
PERIODIC_NONE = 2

FILTER_LSQ = 0
FILTER_WIENER = 1

NULL_THRESHOLD = 1e-14

# measurement models (transverse factor of G)
G_AVERAGED = 0   # lenslet-averaged gradient (Eq. 4): sinc
G_FRIED = 1      # corner samples, mean of the two edge differences: cos


def next_pow2(x):
    p = 1
    while p < x:
        p *= 2
    return p


def grid_size(n, pad_factor):
    """Padded grid size N = next power of two >= ceil(pad_factor * n)."""
    return next_pow2(int(math.ceil(pad_factor * n - 1e-9)))


def pupil_offset(n, N):
    """Centred embedding: lenslet (i, j) sits at grid cell (off + i, off + j)."""
    return (N - n) // 2


# ----------------------------------------------------------------------------
# Direct DFT (Sec. 3.1: the FFT assumes periodic data on a rectangular grid)
# ----------------------------------------------------------------------------

def dft_matrix(N, sign):
    """E[k, m] = exp(sign * 2 i pi k m / N); the product k m is reduced
    modulo N before the trigonometric call so large products stay exact."""
    k = np.arange(N)
    km = np.outer(k, k) % N
    ang = sign * 2.0 * math.pi * km / N
    return np.cos(ang) + 1j * np.sin(ang)


def dft2(x):
    """Forward 2-D DFT, X[ky, kx] = sum_{m,n} x[m, n] exp(-2i pi (ky m + kx n)/N),
    applied as a column transform and a row transform (separable)."""
    N = x.shape[0]
    F = dft_matrix(N, -1)
    return F @ np.asarray(x, dtype=np.complex128) @ F.T


def idft2(X):
    """Inverse 2-D DFT with the 1/N^2 normalisation."""
    N = X.shape[0]
    Fi = dft_matrix(N, +1)
    return (Fi @ np.asarray(X, dtype=np.complex128) @ Fi.T) / (N * N)


def real_idft2(X):
    """Inverse DFT of a Hermitian spectrum; checks that the imaginary part is
    at rounding level before dropping it."""
    x = idft2(X)
    scale = max(float(np.sqrt(np.mean(np.abs(x) ** 2))), 1e-300)
    assert float(np.max(np.abs(x.imag))) <= 1e-9 * scale + 1e-300, "spectrum not Hermitian"
    return x.real.copy()


# ----------------------------------------------------------------------------
# Measurement model and filters (Sec. 2: Eqs. 1-4)
# ----------------------------------------------------------------------------

def signed_freq(N):
    """u[k] = k/N for k < N/2 and (k - N)/N otherwise: values in [-1/2, 1/2)."""
    k = np.arange(N)
    return np.where(k < N // 2, k, k - N) / N


def shift_factor(N, pixel=0.0):
    """a(u) = exp(2i pi u) - 1: the difference across one pitch of a mode at
    frequency u (gradient x lenslet sampling in Eq. 4).  With pixel = d_px/d
    > 0 the difference spans d - d_px about the lenslet centre and is scaled
    by d / (d - d_px): 2i sin(pi u (1 - pixel)) / (1 - pixel) exp(i pi u)."""
    u = signed_freq(N)
    if pixel == 0.0:
        return np.exp(2j * math.pi * u) - 1.0
    L = 1.0 - pixel
    return 2j * np.sin(math.pi * u * L) / L * np.exp(1j * math.pi * u)


def average_factor(N, g_model=G_AVERAGED):
    """T(u) = sinc(u) exp(i pi u): the average of a mode over one pitch in the
    transverse direction (the box Pi of Eq. 4).  On the Nyquist bin u = -1/2
    the two aliases give -2i/pi and +2i/pi; their average, 0, is used.
    G_FRIED: the mean of the two corner samples, cos(pi u) exp(i pi u), which
    is 0 on the Nyquist bin."""
    u = signed_freq(N)
    if g_model == G_FRIED:
        T = np.cos(math.pi * u) * np.exp(1j * math.pi * u)
    elif g_model == G_AVERAGED:
        T = np.sinc(u) * np.exp(1j * math.pi * u)
    else:
        raise ValueError("unknown measurement model")
    T[N // 2] = 0.0
    return T


def measurement_filters(N, g_model=G_AVERAGED, pixel=0.0):
    """Gx[ky, kx] and Gy[ky, kx]: the discrete Shack-Hartmann model (Eq. 4)
    in the Fourier domain, s~ = G~ phi~ (Eq. 1)."""
    a = shift_factor(N, pixel)
    T = average_factor(N, g_model)
    Gx = np.outer(T, a)   # row factor depends on v (ky), column factor on u (kx)
    Gy = np.outer(a, T)
    return Gx, Gy


def lsq_weight(Gx, Gy):
    """iota = 1 / (|Gx|^2 + |Gy|^2), 0 at the nulls (LSQ filter of Sec. 3.3)."""
    g2 = np.abs(Gx) ** 2 + np.abs(Gy) ** 2
    iota = np.zeros_like(g2)
    ok = g2 >= NULL_THRESHOLD
    iota[ok] = 1.0 / g2[ok]
    return iota


def von_karman_psd(N, r0_pitch, L0_pitch):
    """Phase PSD per unit (cycles/pitch)^2 on the grid frequencies."""
    u = signed_freq(N)
    kappa2 = u[None, :] ** 2 + u[:, None] ** 2
    return 0.023 * r0_pitch ** (-5.0 / 3.0) * (kappa2 + L0_pitch ** -2.0) ** (-11.0 / 6.0)


def reconstruction_filters(N, filt, noise_var=0.0, r0_pitch=1.0, L0_pitch=1.0, g_model=G_AVERAGED,
                           pixel=0.0):
    """Rx, Ry of Eq. 2.  LSQ: G*/|G|^2.  Wiener (Eq. 3, gamma = 1):
    G* / (|G|^2 + noise_var / W_phi).  Both are 0 at the nulls of |G|^2."""
    Gx, Gy = measurement_filters(N, g_model, pixel)
    g2 = np.abs(Gx) ** 2 + np.abs(Gy) ** 2
    if filt == FILTER_LSQ:
        w = lsq_weight(Gx, Gy)
    elif filt == FILTER_WIENER:
        denom = g2 + noise_var / von_karman_psd(N, r0_pitch, L0_pitch)
        w = np.zeros_like(g2)
        ok = g2 >= NULL_THRESHOLD
        w[ok] = 1.0 / denom[ok]
    else:
        raise ValueError("unknown filter")
    return np.conj(Gx) * w, np.conj(Gy) * w


# ----------------------------------------------------------------------------
# Slope extension (Sec. 3.2 Eq. PC; Sec. 3.3 Algorithm 1)
# ----------------------------------------------------------------------------

def periodic_fill(sx, sy):
    """Eq. PC in 0-based indices: the last column of x slopes takes minus the
    sum of the other N-1 entries of its row; the last row of y slopes takes
    minus the sum of the other N-1 entries of its column."""
    N = sx.shape[0]
    sx = sx.copy()
    sy = sy.copy()
    for m in range(N):
        sx[m, N - 1] = -np.sum(sx[m, : N - 1])
    for n in range(N):
        sy[N - 1, n] = -np.sum(sy[: N - 1, n])
    return sx, sy


def embed(slopes, mask, N):
    """Dense (2, n, n) slopes -> two N x N fields, zero outside the pupil;
    also returns the N x N pupil indicator P."""
    n = mask.shape[0]
    off = pupil_offset(n, N)
    P = np.zeros((N, N), dtype=bool)
    P[off:off + n, off:off + n] = mask.astype(bool)
    sx = np.zeros((N, N))
    sy = np.zeros((N, N))
    sx[off:off + n, off:off + n] = np.where(mask, slopes[0], 0.0)
    sy[off:off + n, off:off + n] = np.where(mask, slopes[1], 0.0)
    return sx, sy, P


def hudgin_extension(s0x, s0y, P):
    """The Hudgin extension of Sec. 3.2 (from Poyneer et al.): outside the
    pupil, every x slope takes the measured x slope at the top or bottom edge
    of the pupil in its column (the nearer end, going up or down to the grid
    edge), and every y slope the measured y slope at the left or right edge of
    the pupil in its row. Gaps between two pupil cells of a column (row) and
    columns (rows) without pupil cells stay 0. Returns (2, N, N)."""
    N = s0x.shape[0]
    ex = np.zeros((N, N))
    ey = np.zeros((N, N))
    for col in range(N):
        rows = [m for m in range(N) if P[m, col]]
        if rows:
            top, bot = rows[0], rows[-1]
            for m in range(N):
                if m < top:
                    ex[m, col] = s0x[top, col]
                elif m > bot:
                    ex[m, col] = s0x[bot, col]
    for row in range(N):
        cols = [n for n in range(N) if P[row, n]]
        if cols:
            left, right = cols[0], cols[-1]
            for n in range(N):
                if n < left:
                    ey[row, n] = s0y[row, left]
                elif n > right:
                    ey[row, n] = s0y[row, right]
    return np.stack([ex, ey])


def gerchberg_iteration(sx, sy, s0x, s0y, P, Gx, Gy, iota):
    """One pass of Algorithm 1, steps 1-4."""
    # step 1: Fourier transform of both slope fields
    Sx = dft2(sx)
    Sy = dft2(sy)
    # step 2: LSQ phase estimate, then slopes re-synthesised through G
    phi_hat = (np.conj(Gx) * Sx + np.conj(Gy) * Sy) * iota
    Sx_new = Gx * phi_hat
    Sy_new = Gy * phi_hat
    # step 3: back to direct space
    sx_new = real_idft2(Sx_new)
    sy_new = real_idft2(Sy_new)
    # step 4: measured slopes inside the pupil, extrapolation outside
    sx_new = np.where(P, s0x, sx_new)
    sy_new = np.where(P, s0y, sy_new)
    return sx_new, sy_new


def gerchberg_extend(s0x, s0y, P, iters, periodic=PERIODIC_BEFORE_EACH_FFT,
                     ext_init=None, history=None, g_model=G_AVERAGED, pixel=0.0):
    """Run `iters` Gerchberg iterations from the embedded slopes (Algorithm 1).

    ext_init: optional (2, N, N) initial extension used outside the pupil, or
    the string "hudgin" for the Hudgin extension of the measured slopes.
    history: optional list; receives (sx, sy) after every iteration.
    Returns the slopes that enter the final reconstruction, after the
    periodic condition where the mode asks for it (Algorithm 1 step 5).
    """
    N = s0x.shape[0]
    Gx, Gy = measurement_filters(N, g_model, pixel)
    iota = lsq_weight(Gx, Gy)
    if isinstance(ext_init, str):
        if ext_init != "hudgin":
            raise ValueError("unknown extension")
        ext_init = hudgin_extension(s0x, s0y, P)
    if ext_init is None:
        sx, sy = s0x.copy(), s0y.copy()
    else:
        sx = np.where(P, s0x, ext_init[0])
        sy = np.where(P, s0y, ext_init[1])
    for _ in range(iters):
        if periodic == PERIODIC_BEFORE_EACH_FFT:
            sx, sy = periodic_fill(sx, sy)
        sx, sy = gerchberg_iteration(sx, sy, s0x, s0y, P, Gx, Gy, iota)
        if history is not None:
            history.append((sx.copy(), sy.copy()))
    if periodic in (PERIODIC_BEFORE_EACH_FFT, PERIODIC_FINAL_ONLY):
        sx, sy = periodic_fill(sx, sy)
    return sx, sy


def final_reconstruct(sx, sy, Rx, Ry):
    """Eq. 2: phi~ = Rx Sx + Ry Sy, then the inverse transform."""
    phi_hat = Rx * dft2(sx) + Ry * dft2(sy)
    return real_idft2(phi_hat)


def reconstruct(slopes, mask, pad_factor, iters, filt=FILTER_LSQ, noise_var=0.0,
                r0_pitch=1.0, L0_pitch=1.0, periodic=PERIODIC_BEFORE_EACH_FFT,
                ext_init=None, history=None, g_model=G_AVERAGED, pixel=0.0, N=None):
    """Whole path for one frame: embed -> Gerchberg extension -> final filter.

    slopes: (2, n, n) x then y slopes in radians per lenslet; mask: (n, n).
    g_model, pixel: the measurement model (G_AVERAGED or G_FRIED; d_px / d).
    N: the grid size itself (any N >= n + 2; the paper's windows of w
    lenslets around the pupil are N = n + 2w, Sec. 4.1) instead of the power
    of two that pad_factor gives.
    Returns (phase N x N, extended slopes (2, N, N)).
    """
    slopes = np.asarray(slopes, dtype=np.float64)
    mask = np.asarray(mask).astype(bool)
    n = mask.shape[0]
    if N is None:
        N = grid_size(n, pad_factor)
    s0x, s0y, P = embed(slopes, mask, N)
    sx, sy = gerchberg_extend(s0x, s0y, P, iters, periodic, ext_init, history, g_model, pixel)
    Rx, Ry = reconstruction_filters(N, filt, noise_var, r0_pitch, L0_pitch, g_model, pixel)
    phase = final_reconstruct(sx, sy, Rx, Ry)
    return phase, np.stack([sx, sy])


def spectral_projection(sx, sy):
    """Steps 1-3 of Algorithm 1 without the reinsertion: the orthogonal
    per-frequency projection of (sx, sy) onto the range of G."""
    N = sx.shape[0]
    Gx, Gy = measurement_filters(N)
    iota = lsq_weight(Gx, Gy)
    phi_hat = (np.conj(Gx) * dft2(sx) + np.conj(Gy) * dft2(sy)) * iota
    return real_idft2(Gx * phi_hat), real_idft2(Gy * phi_hat)
