"""The reduced-rank fit of the linear warm start (host code, no GPU): exact
at full rank, and at rank r it reaches the Eckart-Young optimum, the error of
the best rank-r approximation of X E given by its singular values."""

import numpy as np

from paper_1705_04298_gb300 import linws


def test_full_rank_is_exact():
    rng = np.random.default_rng(0)
    E = rng.standard_normal((40, 300))
    X = rng.standard_normal((100, 40))
    A, V = linws.fit(E, X, 128)
    assert A.shape == (40, 128) and V.shape == (300, 128)
    assert np.linalg.norm(X @ E - X @ A @ V.T) <= 1e-6 * np.linalg.norm(X @ E)


def test_rank_r_reaches_the_optimum():
    rng = np.random.default_rng(1)
    E = rng.standard_normal((40, 300)) * np.exp(-np.arange(300) / 60.0)
    X = rng.standard_normal((100, 40)) * np.exp(-np.arange(40) / 15.0)
    S = np.linalg.svd(X @ E, compute_uv=False)
    for r in (1, 5, 10, 25):
        A, V = linws.fit(E, X, r)
        err = np.linalg.norm(X @ E - X @ A.astype(np.float64) @ V.astype(np.float64).T)
        best = np.sqrt(np.sum(S[r:] ** 2))
        assert err <= best * (1 + 1e-4) + 1e-6 * S[0], (r, err, best)


def test_fewer_frames_than_slopes():
    rng = np.random.default_rng(2)
    E = rng.standard_normal((40, 300))
    X = rng.standard_normal((12, 40))
    A, V = linws.fit(E, X, 128)
    assert np.linalg.norm(X @ E - X @ A @ V.T) <= 1e-6 * np.linalg.norm(X @ E)
    assert np.all(V[:, 12:] == 0)


def test_gathered_order():
    mask = np.array([[0, 1], [1, 1]], dtype=bool)
    s = np.arange(2 * 2 * 2 * 2, dtype=float).reshape(2, 2, 2, 2)
    X = linws.gathered(s, mask)
    assert X.tolist() == [[1, 2, 3, 5, 6, 7], [9, 10, 11, 13, 14, 15]]


def test_phase_fit_reaches_the_phase_optimum():
    """fit_phase: with P = E L (L a linear map from the extension to the
    phase), the phase error of X A V^T L is the tail of the singular values
    of X P beyond the rank; and the warm start stays in the row space of E."""
    rng = np.random.default_rng(3)
    K, M, C = 30, 200, 60
    E = rng.standard_normal((K, M))
    L = rng.standard_normal((M, C)) * np.exp(-np.arange(C) / 8.0)
    P = E @ L
    for frames in (80, 20):   # more and fewer frames than slopes
        _check_phase_fit(E, L, P, rng.standard_normal((frames, K)))


def _check_phase_fit(E, L, P, X):
    S = np.linalg.svd(X @ P, compute_uv=False)
    for r in (2, 5, 12):
        A, V = linws.fit_phase(E, P, X, r)
        err = np.linalg.norm(X @ P - X @ A.astype(np.float64) @ V.astype(np.float64).T @ L)
        best = np.sqrt(np.sum(S[r:] ** 2))
        assert err <= best * (1 + 1e-3) + 1e-5 * S[0], (r, err, best)
        # V = E^T B for some B: projecting V onto the row space of E changes nothing
        proj = E.T @ np.linalg.lstsq(E.T, V.astype(np.float64), rcond=None)[0]
        assert np.linalg.norm(proj - V) <= 1e-4 * np.linalg.norm(V)


def test_pupil_corners_match_the_residual_region():
    mask = np.zeros((4, 4), dtype=bool)
    mask[1:3, 1:3] = True
    idx = linws.pupil_corners(mask, 8)
    g = np.zeros((8, 8), dtype=bool)
    g.ravel()[idx] = True
    # corners (rows/cols 1..3 of the 5 x 5 corner grid) at offset 2
    assert g.sum() == 9 and g[3:6, 3:6].all()
