"""The closed-loop bookkeeping on the CPU with the FP64 oracle as the
reconstructor: the corrector slopes of a bilinear surface, and a small loop
that converges."""

import numpy as np

import oracle
from paper_1705_04298_gb300 import closed_loop, synth


def test_corrector_slopes_of_a_bilinear_surface():
    n = 5
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    # a tilt gives its gradient; the saddle x y gives the cell-centre gradient
    s = closed_loop.corrector_slopes((0.3 * j - 0.7 * i)[None])
    assert np.allclose(s[0, 0], 0.3) and np.allclose(s[0, 1], -0.7)
    s = closed_loop.corrector_slopes((i * j * 1.0)[None])
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    assert np.allclose(s[0, 0], ii + 0.5) and np.allclose(s[0, 1], jj + 0.5)


def test_small_loop_converges_with_the_oracle():
    n, pad = 12, 2.0

    mask = synth.pupil_mask(n)

    def rec(slopes):
        return np.stack([oracle.reconstruct(s, mask, pad, 1, periodic=oracle.PERIODIC_NONE)[0] for s in slopes])

    out = closed_loop.simulate(rec, n=n, steps=30, loops=4, gain=0.5, sigma=0.0)
    ol = float(np.mean(out["open_loop"]))
    tail = float(np.mean(out["residual"][15:]))
    assert out["residual"][0] == out["open_loop"][0]
    assert tail < 0.3 * ol, (tail, ol)
