"""Linear warm start: the extension operator of the Gerchberg loop, its
data-weighted rank-r truncation, and the evaluation driver.

Algorithm 1 (Sec. 3.3) is linear in the measured slopes: from a zero start,
the extended slopes after k iterations are E_k s for a fixed matrix E_k that
depends only on the pupil, the grid and the periodic mode. Its rows are the
loop's responses to unit slopes, taken here from the library's own FP32 path
(fwr_reconstruct_ex with ext_out), one frame per valid slope.

A warm start x0 = E_k s followed by one more iteration reproduces k + 1 plain
iterations. E_10 is 2 n_valid x 2 N^2 (2528 x 32768 for 40 x 40 lenslets on a
128^2 grid): 166 MFLOP per frame, which the tcgen05 tensor cores evaluate far
faster than the nine FP32 FFT iterations it replaces. A rank-r factorisation
E ~ A V^T cuts that further. It is fitted to data: over training frames X,
it minimises the error of the phase that the following iteration and the
final filter make at the pupil corners (fit_phase; the reconstruction is
linear, so that phase's dependence on the warm start is one more matrix P,
taken from the library), or of the extension itself (fit). The phase fit
needs a far smaller rank: the pupil phase after one iteration depends on the
warm start through a few hundred modes. The fit is off-line host work in FP64
(numpy); inference runs entirely in the library (fwr_linws_reconstruct).
bench.py measures it against the plain loop.
"""

import time

import numpy as np

from . import learned

TRAIN_FRAMES = 8192
OPERATOR_ITERS = 10
DEFAULT_RANK = 256


def valid_cells(mask):
    return np.flatnonzero(np.asarray(mask, dtype=bool).ravel())


def gathered(slopes, mask):
    """(F, 2, n, n) slopes -> X (F, 2 n_valid): x slopes of the valid cells
    (row-major), then y slopes."""
    s = np.asarray(slopes)
    cells = valid_cells(mask)
    F = s.shape[0]
    flat = s.reshape(F, 2, -1)
    return np.concatenate([flat[:, 0, cells], flat[:, 1, cells]], axis=1)


def extension_operator(fwr, plan, mask, iters=OPERATOR_ITERS, chunk=1024):
    """E (2 n_valid, 2 N^2) float64: row j is the extension after `iters`
    iterations for the unit slope vector e_j (library FP32 path)."""
    import torch
    cells = valid_cells(mask)
    nv = len(cells)
    K = 2 * nv
    n, N = plan.n, plan.N
    E = np.empty((K, 2 * N * N), dtype=np.float64)
    for a in range(0, K, chunk):
        b = min(K, a + chunk)
        imp = torch.zeros((b - a, 2, n * n), dtype=torch.float32, device="cuda")
        rows = torch.arange(b - a, device="cuda")
        j = torch.arange(a, b, device="cuda")
        ch = (j >= nv).long()
        cell = torch.tensor(cells, device="cuda")[j - ch * nv]
        imp[rows, ch, cell] = 1.0
        ext = torch.empty((b - a, 2, N, N), dtype=torch.float32, device="cuda")
        plan.reconstruct(imp.view(b - a, 2, n, n), iters, ext_out=ext)
        E[a:b] = ext.reshape(b - a, -1).double().cpu().numpy()
    return E


def fit(E, X, rank):
    """Reduced-rank factors (A, V) with E ~ A V^T minimising ||X E - X A V^T||_F:
    with X = Q R, V = the leading right singular vectors of R E, A = E V.
    rank: columns of A and V (the device wants a multiple of 128); columns
    beyond the rank of R E are zero."""
    r = int(rank)
    R = np.linalg.qr(np.asarray(X, dtype=np.float64), mode="r")
    KE = R @ E                                   # (min(F, K), 2N^2)
    lam, U = np.linalg.eigh(KE @ KE.T)           # ascending
    keep = min(r, KE.shape[0])
    lam = lam[::-1][:keep]
    U = U[:, ::-1][:, :keep]
    cols = np.flatnonzero(lam > lam[0] * 1e-20)
    V = np.zeros((E.shape[1], r))
    V[:, cols] = (KE.T @ U[:, cols]) / np.sqrt(lam[cols])
    A = E @ V
    return A.astype(np.float32), V.astype(np.float32)


def pupil_corners(mask, N):
    """Flat indices, in the N x N phase grid, of the phase corners that touch
    a valid lenslet (where the residual of a reconstruction is measured)."""
    n = mask.shape[0]
    off = (N - n) // 2
    g = np.zeros((N, N), dtype=bool)
    g[off:off + n + 1, off:off + n + 1] = learned.corner_mask(mask)
    return np.flatnonzero(g.ravel())


def phase_response(fwr, plan, mask, E, iters_after=1, chunk=1024):
    """P (K, n_corners): the phase at the pupil corners, piston removed, of
    `iters_after` iterations and the final filter of `plan` started from row
    j of E as the warm start with zero measured slopes (the reconstruction is
    linear: its phase is L s + P-part, and this is the warm start's part)."""
    import torch
    N = plan.N
    idx = torch.tensor(pupil_corners(mask, N), device="cuda")
    K = E.shape[0]
    P = np.empty((K, len(idx)))
    zeros = torch.zeros((chunk, 2, plan.n, plan.n), dtype=torch.float32, device="cuda")
    ph = torch.empty((chunk, N, N), dtype=torch.float32, device="cuda")
    for a in range(0, K, chunk):
        b = min(K, a + chunk)
        ext = torch.tensor(E[a:b].reshape(b - a, 2, N, N), dtype=torch.float32, device="cuda")
        plan.reconstruct(zeros[:b - a], iters_after, ph[:b - a], ext_init=ext)
        P[a:b] = ph[:b - a].reshape(b - a, -1)[:, idx].double().cpu().numpy()
    return P - P.mean(axis=1, keepdims=True)


def fit_phase(E, P, X, rank):
    """Rank-r factors (A, V), E ~ A V^T, that minimise the error of the
    reconstructed phase rather than of the extension: with X = Q R and the
    SVD R P = U S Z^T, the rank-r optimum of ||X P - X A V^T L^T|| (L the map
    from the warm start to P) is Q U_r S_r Z_r^T; it is reached by A = R^-1
    U_r S_r (minimum norm when there are fewer frames than slopes) and V =
    E^T (Z_r^T P^+)^T, which keeps the warm start in the row space of E."""
    r = int(rank)
    R = np.linalg.qr(np.asarray(X, dtype=np.float64), mode="r")
    U, S, Zt = np.linalg.svd(R @ P, full_matrices=False)
    keep = min(r, len(S))
    A = np.zeros((E.shape[0], r))
    # R is square (more frames than slopes) or wide: the minimum-norm solution of R A = U_r S_r
    A[:, :keep] = np.linalg.lstsq(R, U[:, :keep] * S[:keep], rcond=None)[0]
    Bt = Zt[:keep] @ np.linalg.pinv(P, rcond=1e-10)       # keep x K
    V = np.zeros((E.shape[1], r))
    V[:, :keep] = E.T @ Bt.T
    return A.astype(np.float32), V.astype(np.float32)


def build(fwr, plan, mask, rank=DEFAULT_RANK, max_batch=1000, frames=TRAIN_FRAMES, iters=OPERATOR_ITERS,
          weight="phase", iters_after=1, log=None):
    """Operator from the library, training slopes from the seeded generator
    (seeds 1e6 + i, noise cycling 0.02, 0.05, 0.1 rad; 8192 frames by default),
    fit, device object. weight="phase" (default) fits the phase that
    `iters_after` iterations and the plan's final filter make from the warm
    start (fit_phase); "extension" fits the extension itself (fit)."""
    from . import synth
    t0 = time.time()
    E = extension_operator(fwr, plan, mask, iters)
    t1 = time.time()
    sl, _, _ = synth.batch(plan.n, frames, learned.TRAIN_SEED0, list(learned.TRAIN_SIGMAS), learned.R0, learned.L0)
    X = gathered(sl, mask)
    t2 = time.time()
    if weight == "phase":
        A, V = fit_phase(E, phase_response(fwr, plan, mask, E, iters_after), X, rank)
    else:
        A, V = fit(E, X, rank)
    t3 = time.time()
    if log:
        log("operator %.1f s, training slopes %.1f s, fit %.1f s" % (t1 - t0, t2 - t1, t3 - t2))
    return fwr.LinearWarmStart(plan, A, V, max_batch), E
