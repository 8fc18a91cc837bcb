"""Writes the oracle fixtures of tests/golden/ (calls only oracle/ and numpy).

    python tests/golden/make_golden.py

oracle_small.txt: the FP64 oracle on three fixed tiny inputs: 4x4 lenslets
with one corner cell masked, a 3/4 seeded Gaussian slope field, on an 8x8 grid
(pad 2). Per case, the final phase and extended slopes after k Gerchberg
iterations (Algorithm 1, Sec. 3.3) and the final filter (Eqs. 2-3), 17
significant digits. A later change to the oracle's arithmetic must rewrite
this file and say in its commit which passage of the paper justifies it.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

CASES = [
    # (name, iters, filter, noise_var, r0_pitch, L0_pitch, periodic, g_model, pixel, ext)
    ("lsq_k2_each_fft", 2, oracle.FILTER_LSQ, 0.0, 1.0, 1.0, oracle.PERIODIC_BEFORE_EACH_FFT, oracle.G_AVERAGED, 0.0,
     None),
    ("wiener_k3_final_only", 3, oracle.FILTER_WIENER, 0.01, 2.0, 40.0, oracle.PERIODIC_FINAL_ONLY,
     oracle.G_AVERAGED, 0.0, None),
    ("lsq_k1_fried_pixel_hudgin", 1, oracle.FILTER_LSQ, 0.0, 1.0, 1.0, oracle.PERIODIC_BEFORE_EACH_FFT,
     oracle.G_FRIED, 1.0 / 6.0, "hudgin"),
]


def inputs():
    rng = np.random.default_rng(20170512)
    slopes = 0.75 * rng.standard_normal((2, 4, 4))
    mask = np.ones((4, 4), bool)
    mask[0, 0] = False
    return slopes, mask


def compute():
    slopes, mask = inputs()
    out = {}
    for name, k, filt, nv, r0, L0, per, gm, px, ext in CASES:
        phase, extd = oracle.reconstruct(slopes, mask, 2.0, k, filt, nv, r0, L0, per, ext_init=ext, g_model=gm,
                                         pixel=px)
        out[name] = (phase, extd)
    return out


def main():
    with open(os.path.join(HERE, "oracle_small.txt"), "w") as fh:
        fh.write("# written by tests/golden/make_golden.py from the FP64 oracle; see its docstring\n")
        for name, (phase, extd) in compute().items():
            for label, arr in (("phase", phase), ("sx", extd[0]), ("sy", extd[1])):
                fh.write("%s %s\n" % (name, label))
                for row in arr:
                    fh.write(" ".join("%.17g" % v for v in row) + "\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
