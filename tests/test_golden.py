"""The oracle against the fixtures of tests/golden/: the hand-worked Hudgin
example, and the stored reconstructions of tests/golden/make_golden.py (which
catch any change to the oracle's arithmetic)."""

import os
import sys

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_blocks(path):
    blocks, name = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            name = line
            blocks[name] = []
        else:
            blocks[name].append([float(v) for v in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def test_hudgin_hand_worked_example():
    b = read_blocks(os.path.join(GOLDEN, "hudgin_6x6.txt"))
    P = b["mask"].astype(bool)
    m, n = np.meshgrid(np.arange(6), np.arange(6), indexing="ij")
    s0x = np.where(P, 10 * m + n + 0.5, 0.0)
    s0y = np.where(P, -(10 * m + n) - 0.25, 0.0)
    ex, ey = oracle.hudgin_extension(s0x, s0y, P)
    assert np.array_equal(ex, b["ext_sx"]) and np.array_equal(ey, b["ext_sy"])


def test_oracle_matches_stored_reconstructions():
    sys.path.insert(0, GOLDEN)
    try:
        import make_golden
    finally:
        sys.path.remove(GOLDEN)
    stored = read_blocks(os.path.join(GOLDEN, "oracle_small.txt"))
    for name, (phase, extd) in make_golden.compute().items():
        for label, arr in (("phase", phase), ("sx", extd[0]), ("sy", extd[1])):
            ref = stored["%s %s" % (name, label)]
            assert np.max(np.abs(arr - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref))), (name, label)
