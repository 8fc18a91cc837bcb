"""Pins of the FP64 warm-start network reference (CPU only): its backward pass
against central finite differences of its own forward pass (which is a plain
composition of textbook layers), the layer primitives against direct
definitions, and the data mapping against the pupil geometry."""

import numpy as np
import pytest

import oracle
from oracle import unet
from paper_1705_04298_gb300 import synth


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv(x, W, b)
    for (bb, i, j, co) in [(0, 0, 0, 0), (1, 4, 5, 3), (0, 2, 3, 1), (1, 0, 5, 2)]:
        acc = b[co]
        for dy in range(3):
            for dx in range(3):
                yy, xx = i + dy - 1, j + dx - 1
                if 0 <= yy < 5 and 0 <= xx < 6:
                    acc += np.dot(x[bb, yy, xx], W[co, dy, dx])
        assert abs(y[bb, i, j, co] - acc) < 1e-12


def test_pool_and_upsample_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 8, 3))
    g = rng.standard_normal((2, 4, 4, 3))
    # <pool(x), g> = <x, pool^T(g)>;  <up(g), x> = <g, up^T(x)>
    assert abs(np.sum(unet.avgpool2(x) * g) - np.sum(x * unet.avgpool2_backward(g))) < 1e-12
    assert abs(np.sum(unet.up2(g) * x) - np.sum(g * unet.up2_backward(x))) < 1e-12


def test_backward_matches_finite_differences():
    w = 2
    rng = np.random.default_rng(2)
    params = unet.init_params(w, 3) + 0.05 * rng.standard_normal(unet.param_count(w))
    x = rng.standard_normal((2, 32, 32, 3))
    target = rng.standard_normal((2, 32, 32, 2))
    lm = rng.random((2, 32, 32)) < 0.6

    def loss(p):
        out, _ = unet.forward(p, x, w)
        return unet.loss_and_grad(out, target, lm)[0]

    out, cache = unet.forward(params, x, w)
    _, dout = unet.loss_and_grad(out, target, lm)
    g = unet.backward(params, cache, dout, w)
    idx = rng.choice(len(params), 60, replace=False)
    # every layer's weights and biases are covered by the sample
    idx = np.unique(np.concatenate([idx, [0, len(params) - 1, len(params) // 2]]))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(params)
        e[i] = h
        fd = (loss(params + e) - loss(params - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_param_count_is_about_a_quarter_million_for_width_16():
    assert 200_000 < unet.param_count(16) < 350_000


def test_data_mapping_geometry():
    n, N = 40, 128
    off = oracle.pupil_offset(n, N)
    fr = synth.frame(n, 5, 0.05)
    x = unet.net_input(fr["slopes"], fr["mask"], off)
    assert x.shape == (32, 32, 3)
    # the mask channel is the pupil fraction of each 4x4 block
    assert abs(x[..., 2].sum() * 16 - fr["mask"].sum()) < 1e-9
    ext = np.random.default_rng(0).standard_normal((2, N, N))
    t, lm = unet.net_target(ext, fr["mask"], off)
    assert not np.any(lm & (x[..., 2] > 0))
    assert not lm[-1].any() and not lm[:, -1].any()
    ws = unet.warm_start(t)
    assert ws.shape == (2, N, N)
    assert np.allclose(ws[:, ::4, ::4] * unet.IN_SCALE, np.moveaxis(t, -1, 0))
