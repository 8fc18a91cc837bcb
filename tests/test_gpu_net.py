"""The warm-start network's BF16 kernels against the FP64 reference network
(oracle/unet.py, pinned by finite differences) at the same BF16-rounded
weights and inputs, and a short training run that must lower the loss."""

import numpy as np
import pytest

import oracle
from oracle import unet
from paper_1705_04298_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fwr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04298_gb300 import fwr as m
    m.load()
    return m


def bf16_round(x):
    """Round float64 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def setup_problem(fwr, w, F, seed):
    n, pad = 40, 3.2
    N = 128
    off = oracle.pupil_offset(n, N)
    plan = fwr.Plan(synth.pupil_mask(n), pad, fwr.LSQ)
    sl, _, mask = synth.batch(n, F, seed, 0.05)
    rng = np.random.default_rng(seed)
    ext = rng.standard_normal((F, 2, N, N)) * 2.0
    params = unet.init_params(w, seed) + 0.02 * rng.standard_normal(unet.param_count(w))
    return plan, sl, mask, off, ext, params


def oracle_run(params, w, sl, mask, off, ext):
    pb = bf16_round(params)
    # the GPU keeps FP32 biases; only weights are BF16
    pos = 0
    for _, ci, co, k in unet.layer_specs(w):
        nW = co * k * k * ci
        pos += nW
        pb[pos:pos + co] = params[pos:pos + co]
        pos += co
    x = np.stack([bf16_round(unet.net_input(sl[f], mask, off)) for f in range(len(sl))])
    tl = [unet.net_target(ext[f], mask, off) for f in range(len(sl))]
    t = np.stack([a for a, _ in tl])
    lm = np.stack([b for _, b in tl])
    # the GPU keeps every hidden activation in BF16
    out, cache = unet.forward(pb, x, w, store=bf16_round)
    loss, dout = unet.loss_and_grad(out, t, lm)
    g = unet.backward(pb, cache, dout, w)
    return out, loss, g


@pytest.mark.parametrize("w,F", [(4, 3), (16, 2)])
def test_gradients_match_reference(fwr, w, F):
    plan, sl, mask, off, ext, params = setup_problem(fwr, w, F, 21)
    net = fwr.Net(w, F, params)
    assert net.param_count == unet.param_count(w)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    e = torch.tensor(ext, dtype=torch.float32, device="cuda")
    loss, g = net.gradients(plan, s, e)
    out_o, loss_o, g_o = oracle_run(params, w, sl, mask, off, ext)
    assert abs(loss - loss_o) <= 2e-2 * abs(loss_o)
    rel = np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
    cos = float(np.dot(g, g_o) / (np.linalg.norm(g) * np.linalg.norm(g_o)))
    assert rel <= 5e-2 and cos >= 0.998, (rel, cos)
    # per layer: every layer's gradient agrees in direction
    pos = 0
    for name, ci, co, k in unet.layer_specs(w):
        m = co * k * k * ci + co
        a, b = g[pos:pos + m], g_o[pos:pos + m]
        pos += m
        c = float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert c >= 0.99, (name, c)


@pytest.mark.parametrize("w,F", [(4, 2), (8, 3), (16, 5)])
def test_forward_matches_reference(fwr, w, F):
    """w = 4 and 8: a mix of CUDA-core and tensor-core convolutions (the
    levels with 16k channels go to the tensor cores); w = 16: all 3 x 3
    convolutions but the first. F = 5 at w = 16 leaves ragged CTA tiles at
    the 4 x 4 level (80 pixels)."""
    plan, sl, mask, off, ext, params = setup_problem(fwr, w, F, 5)
    net = fwr.Net(w, F, params)
    assert net.tc_layers == {4: 5, 8: 9, 16: 13}[w]
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    ws = net.forward(plan, s).cpu().numpy().astype(np.float64)
    out_o, _, _ = oracle_run(params, w, sl, mask, off, ext)
    for f in range(F):
        ref = unet.warm_start(out_o[f])
        assert np.linalg.norm(ws[f] - ref) <= 2e-2 * np.linalg.norm(ref)


@pytest.mark.parametrize("w,F", [(16, 7), (32, 2)])
def test_tensor_core_forward_matches_simt(fwr, w, F):
    """Same weights and inputs, tensor-core and CUDA-core convolutions: both
    sum in FP32 and differ only in order, so the predictions agree to a few
    BF16 roundings of the activations."""
    plan, sl, mask, off, ext, params = setup_problem(fwr, w, F, 9)
    net = fwr.Net(w, F, params)
    assert net.tc_layers == 13
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    a = net.forward(plan, s).clone()
    net.set_conv(fwr.NET_CONV_SIMT)
    b = net.forward(plan, s).clone()
    net.set_conv(fwr.NET_CONV_AUTO)
    c = net.forward(plan, s)
    assert torch.equal(a, c)
    rel = float((a - b).norm() / b.norm())
    assert rel <= 1e-2, rel
    with pytest.raises(RuntimeError):
        net.set_conv(7)


def test_training_lowers_the_loss(fwr):
    w, F = 8, 32
    n, pad = 40, 3.2
    plan = fwr.Plan(synth.pupil_mask(n), pad, fwr.LSQ)
    sl, _, mask = synth.batch(n, F, 123, 0.05)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    # targets: the FP32 path's extended slopes after 10 iterations
    ext = torch.empty((F, 2, 128, 128), device="cuda")
    plan.reconstruct(s, 10, ext_out=ext)
    net = fwr.Net(w, F, unet.init_params(w, 0))
    first = net.train_step(plan, s, ext, 1e-3)
    for _ in range(60):
        last = net.train_step(plan, s, ext, 1e-3)
    assert np.isfinite(last) and last < 0.8 * first, (first, last)
