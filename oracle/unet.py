"""FP64 CPU reference of the warm-start network (test infrastructure).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. It shares no code
with the CUDA network (csrc/fwr_net.*).

The network predicts the extension of the slopes outside the pupil, used as
the warm start of the Gerchberg loop (Algorithm 1, Sec. 3.3), from the
measured slopes. Definition (shared, by specification only, with the CUDA
network):

* input, 3 channels on a 32 x 32 grid: the measured x and y slopes embedded
  in the 128 x 128 grid (zero outside the pupil) and the pupil indicator, each
  averaged over 4 x 4 blocks; slopes are multiplied by IN_SCALE;
* a 4-level U-Net with widths (w, 2w, 4w, 4w): two 3 x 3 convolutions with
  zero padding, bias and ReLU per level, 2 x 2 average pooling down,
  2 x nearest upsampling up, skip connections concatenated as
  [upsampled, skip] along channels, and a final 1 x 1 convolution to 2
  channels (no ReLU);
* layout NHWC; a 3 x 3 weight is W[cout][dy][dx][cin] applied to input pixel
  (y + dy - 1, x + dx - 1);
* output: the 2-channel 32 x 32 prediction divided by IN_SCALE, repeated over
  4 x 4 blocks to 128 x 128 (the warm start outside the pupil);
* training loss: mean squared error against the 4 x 4 block means of the
  target extended slopes (times IN_SCALE), over the blocks that contain no
  pupil cell and are not in the last block row or column (which hold the
  periodic-fill cells).
"""

import numpy as np

IN_SCALE = 0.5
GRID = 128
LOW = 32
POOL = GRID // LOW


def widths(w):
    return (w, 2 * w, 4 * w, 4 * w)


def layer_specs(w):
    """(name, cin, cout, k) in evaluation order."""
    w1, w2, w3, w4 = widths(w)
    return [("e1a", 3, w1, 3), ("e1b", w1, w1, 3),
            ("e2a", w1, w2, 3), ("e2b", w2, w2, 3),
            ("e3a", w2, w3, 3), ("e3b", w3, w3, 3),
            ("ba", w3, w4, 3), ("bb", w4, w4, 3),
            ("d3a", w4 + w3, w3, 3), ("d3b", w3, w3, 3),
            ("d2a", w3 + w2, w2, 3), ("d2b", w2, w2, 3),
            ("d1a", w2 + w1, w1, 3), ("d1b", w1, w1, 3),
            ("out", w1, 2, 1)]


def param_count(w):
    return sum(co * k * k * ci + co for _, ci, co, k in layer_specs(w))


def unpack(params, w):
    """Flat vector -> {name: (W[cout][k][k][cin], b[cout])}, layer by layer, W then b."""
    out, pos = {}, 0
    for name, ci, co, k in layer_specs(w):
        nW = co * k * k * ci
        W = params[pos:pos + nW].reshape(co, k, k, ci)
        pos += nW
        b = params[pos:pos + co]
        pos += co
        out[name] = (W, b)
    assert pos == len(params)
    return out


# ---------------------------------------------------------------- layers ---

def conv(x, W, b):
    """Same-padded convolution, x [B, H, W, Cin] -> [B, H, W, Cout]."""
    B, H, Wd, _ = x.shape
    co, k = W.shape[0], W.shape[1]
    p = k // 2
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    out = np.zeros((B, H, Wd, co))
    for dy in range(k):
        for dx in range(k):
            out += xp[:, dy:dy + H, dx:dx + Wd, :] @ W[:, dy, dx, :].T
    return out + b


def conv_backward(x, W, dout):
    """Gradients of conv(x, W, b) for the upstream gradient dout."""
    B, H, Wd, ci = x.shape
    k = W.shape[1]
    p = k // 2
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    d2 = dout.reshape(-1, dout.shape[-1])
    for dy in range(k):
        for dx in range(k):
            xs = xp[:, dy:dy + H, dx:dx + Wd, :].reshape(-1, ci)
            dW[:, dy, dx, :] = d2.T @ xs
            dxp[:, dy:dy + H, dx:dx + Wd, :] += (d2 @ W[:, dy, dx, :]).reshape(B, H, Wd, ci)
    db = d2.sum(axis=0)
    return dxp[:, p:p + H, p:p + Wd, :], dW, db


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(dout):
    return np.repeat(np.repeat(dout, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(dout):
    B, H, W, C = dout.shape
    return dout.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


# --------------------------------------------------------------- network ---

def forward(params, x, w, store=None):
    """x [B, 32, 32, 3] -> prediction [B, 32, 32, 2] and the cache for backward.

    store: optional function applied to every hidden activation as it is kept
    (the ReLU outputs and the pooled maps), e.g. a rounding to a storage
    format; the identity when None."""
    P = unpack(params, w)
    cache = {}
    keep = store if store is not None else (lambda a: a)

    def cr(name, h):
        z = conv(h, *P[name])
        cache[name] = (h, z)
        return keep(np.maximum(z, 0.0))

    def pool(a):
        return keep(avgpool2(a))

    s1 = cr("e1b", cr("e1a", x))
    s2 = cr("e2b", cr("e2a", pool(s1)))
    s3 = cr("e3b", cr("e3a", pool(s2)))
    bt = cr("bb", cr("ba", pool(s3)))
    d3 = cr("d3b", cr("d3a", np.concatenate([up2(bt), s3], axis=-1)))
    d2 = cr("d2b", cr("d2a", np.concatenate([up2(d3), s2], axis=-1)))
    d1 = cr("d1b", cr("d1a", np.concatenate([up2(d2), s1], axis=-1)))
    out = conv(d1, *P["out"])
    cache["out"] = (d1, out)
    cache["widths"] = widths(w)
    return out, cache


def backward(params, cache, dout, w):
    """Gradient of sum(dout * forward(params, x)) with respect to params (flat)."""
    P = unpack(params, w)
    w1, w2, w3, w4 = widths(w)
    grads = {}

    def conv_b(name, dz):
        h, _ = cache[name]
        dh, dW, db = conv_backward(h, P[name][0], dz)
        grads[name] = (dW, db)
        return dh

    def cr_b(name, dy):
        _, z = cache[name]
        return conv_b(name, dy * (z > 0))

    dd1 = conv_b("out", dout)
    dcat1 = cr_b("d1a", cr_b("d1b", dd1))
    dd2 = up2_backward(dcat1[..., :w2])
    ds1 = dcat1[..., w2:]
    dcat2 = cr_b("d2a", cr_b("d2b", dd2))
    dd3 = up2_backward(dcat2[..., :w3])
    ds2 = dcat2[..., w3:]
    dcat3 = cr_b("d3a", cr_b("d3b", dd3))
    dbt = up2_backward(dcat3[..., :w4])
    ds3 = dcat3[..., w4:]
    dp3 = cr_b("ba", cr_b("bb", dbt))
    ds3 = ds3 + avgpool2_backward(dp3)
    dp2 = cr_b("e3a", cr_b("e3b", ds3))
    ds2 = ds2 + avgpool2_backward(dp2)
    dp1 = cr_b("e2a", cr_b("e2b", ds2))
    ds1 = ds1 + avgpool2_backward(dp1)
    cr_b("e1a", cr_b("e1b", ds1))
    flat = []
    for name, _, _, _ in layer_specs(w):
        dW, db = grads[name]
        flat += [dW.ravel(), db]
    return np.concatenate(flat)


def loss_and_grad(pred, target, lmask):
    """Masked mean squared error over (B, 32, 32, 2); lmask [B, 32, 32]."""
    m = lmask[..., None].astype(np.float64)
    cnt = max(1.0, 2.0 * float(m.sum()))
    d = (pred - target) * m
    return float(np.sum(d * d) / cnt), 2.0 * d / cnt


# --------------------------------------------------------- data mapping ---

def net_input(slopes, mask, off):
    """Dense (2, n, n) slopes and mask -> [32, 32, 3] network input."""
    n = mask.shape[0]
    g = np.zeros((GRID, GRID, 3))
    m = mask.astype(np.float64)
    g[off:off + n, off:off + n, 0] = slopes[0] * m * IN_SCALE
    g[off:off + n, off:off + n, 1] = slopes[1] * m * IN_SCALE
    g[off:off + n, off:off + n, 2] = m
    return g.reshape(LOW, POOL, LOW, POOL, 3).mean(axis=(1, 3))


def net_target(ext, mask, off):
    """Extended slopes (2, 128, 128) -> block-mean target [32, 32, 2] and the
    loss mask [32, 32] (blocks without pupil cells, last block row/column out)."""
    n = mask.shape[0]
    t = np.stack([ext[0], ext[1]], axis=-1) * IN_SCALE
    t = t.reshape(LOW, POOL, LOW, POOL, 2).mean(axis=(1, 3))
    P = np.zeros((GRID, GRID))
    P[off:off + n, off:off + n] = mask
    lm = P.reshape(LOW, POOL, LOW, POOL).sum(axis=(1, 3)) == 0
    lm[LOW - 1, :] = False
    lm[:, LOW - 1] = False
    return t, lm


def warm_start(pred):
    """[32, 32, 2] prediction -> (2, 128, 128) warm start."""
    up = np.repeat(np.repeat(pred / IN_SCALE, POOL, axis=0), POOL, axis=1)
    return np.stack([up[..., 0], up[..., 1]])


def init_params(w, seed):
    """He-style initialisation with a seeded generator (biases 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    flat = []
    for _, ci, co, k in layer_specs(w):
        std = np.sqrt(2.0 / (ci * k * k))
        flat += [rng.standard_normal(co * k * k * ci) * std, np.zeros(co)]
    return np.concatenate(flat)
