"""Input generator checks (CPU): the von Karman screens have the textbook
small-separation structure function, the pupil is the stated circle, and the
slopes are reproducible from their seed."""

import numpy as np

from paper_1705_04298_gb300 import synth


def test_structure_function_matches_kolmogorov_at_small_lags():
    r0, L0, delta, M = 0.15, 25.0, 0.1, 256
    lags = [1, 2, 4]
    acc = np.zeros(len(lags))
    for s in range(20):
        rng = np.random.Generator(np.random.PCG64(300 + s))
        scr = synth.von_karman_screen(M, delta, r0, L0, rng)
        for i, l in enumerate(lags):
            acc[i] += 0.5 * (np.mean((np.roll(scr, -l, axis=1) - scr) ** 2)
                             + np.mean((np.roll(scr, -l, axis=0) - scr) ** 2))
    acc /= 20
    for i, l in enumerate(lags):
        r = l * delta
        kolmo = 6.88 * (r / r0) ** (5.0 / 3.0)
        # the finite outer scale lowers D(r) by 1 - 1.485 (r/L0)^(1/3) to first order
        vk = kolmo * (1.0 - 1.485 * (r / L0) ** (1.0 / 3.0))
        assert 0.85 < acc[i] / vk < 1.15, (l, acc[i], vk)


def test_pupil_counts_and_symmetry():
    for n in (16, 40, 64, 80, 128):
        m = synth.pupil_mask(n)
        assert np.array_equal(m, m[::-1]) and np.array_equal(m, m.T)
        frac = m.sum() / (n * n)
        assert abs(frac - np.pi / 4) < 0.03


def test_frames_are_seeded():
    a = synth.frame(16, 42, 0.05)
    b = synth.frame(16, 42, 0.05)
    c = synth.frame(16, 43, 0.05)
    assert np.array_equal(a["slopes"], b["slopes"])
    assert not np.array_equal(a["slopes"], c["slopes"])
    assert np.all(a["slopes"][:, ~a["mask"]] == 0.0)
