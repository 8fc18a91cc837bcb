"""Pins of the oracle's Hudgin extension (Sec. 3.2): the closed form for a tilt
and its place in the full path (the hand-worked example is the fixture
tests/golden/hudgin_6x6.txt, checked in tests/test_golden.py)."""

import numpy as np

import oracle


def test_tilt_extends_to_every_column_and_row_of_the_pupil():
    n = 12
    mask = np.zeros((n, n), bool)
    c = (n - 1) / 2
    for i in range(n):
        for j in range(n):
            mask[i, j] = (i - c) ** 2 + (j - c) ** 2 <= (n / 2) ** 2
    N = 32
    slopes = np.stack([np.full((n, n), 0.7), np.full((n, n), -0.3)])
    s0x, s0y, P = oracle.embed(slopes, mask, N)
    ex, ey = oracle.hudgin_extension(s0x, s0y, P)
    cols = P.any(axis=0)
    rows = P.any(axis=1)
    sx = np.where(P, s0x, ex)
    sy = np.where(P, s0y, ey)
    # a tilt's x slopes fill every column through the pupil, its y slopes every
    # row through the pupil (a convex pupil has no gaps), and nothing else
    assert np.all(sx[:, cols] == 0.7) and np.all(sx[:, ~cols] == 0.0)
    assert np.all(sy[rows, :] == -0.3) and np.all(sy[~rows, :] == 0.0)


def test_hudgin_start_in_the_full_path():
    """ext_init="hudgin" with zero iterations is the Hudgin method: periodic
    fill of the extended slopes, then the final filter."""
    n, pad = 12, 2.0
    rng = np.random.default_rng(5)
    mask = np.ones((n, n), bool)
    mask[0, :3] = False
    slopes = rng.standard_normal((2, n, n))
    N = oracle.grid_size(n, pad)
    s0x, s0y, P = oracle.embed(slopes, mask, N)
    ex, ey = oracle.hudgin_extension(s0x, s0y, P)
    sx, sy = oracle.periodic_fill(np.where(P, s0x, ex), np.where(P, s0y, ey))
    Rx, Ry = oracle.reconstruction_filters(N, oracle.FILTER_LSQ)
    want = oracle.final_reconstruct(sx, sy, Rx, Ry)
    got, ext = oracle.reconstruct(slopes, mask, pad, 0, oracle.FILTER_LSQ, ext_init="hudgin")
    assert np.max(np.abs(got - want)) < 1e-12
    assert np.array_equal(ext[0][P], s0x[P])
