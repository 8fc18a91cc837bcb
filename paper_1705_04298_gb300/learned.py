"""Learned warm start: data, training and evaluation of the U-Net (fwr_net_*).

The network predicts the slopes outside the pupil from the measured ones; the
Gerchberg loop (Algorithm 1, Sec. 3.3) then starts from that prediction
instead of zeros, so one or two iterations replace many. Every step runs in
the library's kernels: the targets are the FP32 path's extended slopes after
10 iterations (checked against the FP64 oracle by the tests), training is
fwr_net_train_step, inference fwr_net_forward + fwr_reconstruct_ex.

    python -m paper_1705_04298_gb300.learned train --frames 32768 --epochs 12 \\
        --width 16 --out paper_1705_04298_gb300/weights/warmstart_w16_n40.npz
    python -m paper_1705_04298_gb300.learned eval \\
        --weights paper_1705_04298_gb300/weights/warmstart_w16_n40.npz

Workload (40x40 lenslets on a 128^2 grid, D = 8 m, r0 = 0.15 m, L0 = 25 m):
training frames use seeds 1e6 + i with the noise level cycling through
0.02, 0.05, 0.1 rad; evaluation frames use seeds 2e6 + i at 0.05 rad.
"""

import argparse
import json
import os
import sys
import time

import numpy as np

N_LENSLETS, PAD, GRID = 40, 3.2, 128
R0, L0 = 0.15, 25.0
TRAIN_SEED0, EVAL_SEED0 = 1_000_000, 2_000_000
TRAIN_SIGMAS = (0.02, 0.05, 0.1)
EVAL_SIGMA = 0.05
TARGET_ITERS = 10
PLAIN_ITERS = (1, 2, 3, 4, 5, 6, 8, 10)
LEARNED_ITERS = (1, 2, 3)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart_w16_n40.npz")


def _torch():
    import torch
    return torch


def he_init(width, seed):
    """He-normal weights (fan-in), zero biases, in the library's flat order
    (e1a e1b e2a e2b e3a e3b ba bb d3a d3b d2a d2b d1a d1b out)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w1, w2, w3, w4 = width, 2 * width, 4 * width, 4 * width
    layers = [(3, w1, 3), (w1, w1, 3), (w1, w2, 3), (w2, w2, 3), (w2, w3, 3), (w3, w3, 3), (w3, w4, 3),
              (w4, w4, 3), (w4 + w3, w3, 3), (w3, w3, 3), (w3 + w2, w2, 3), (w2, w2, 3), (w2 + w1, w1, 3),
              (w1, w1, 3), (w1, 2, 1)]
    flat = []
    for ci, co, k in layers:
        flat.append(rng.standard_normal(co * k * k * ci) * np.sqrt(2.0 / (ci * k * k)))
        flat.append(np.zeros(co))
    return np.concatenate(flat).astype(np.float32)


def corner_mask(mask):
    """Phase corners touching a valid lenslet."""
    n = mask.shape[0]
    cm = np.zeros((n + 1, n + 1), dtype=bool)
    for i in range(n):
        for j in range(n):
            if mask[i, j]:
                cm[i:i + 2, j:j + 2] = True
    return cm


def make_plan(fwr, filt=None, sigma=0.0):
    from . import synth
    r0p, L0p = synth.pitch_units(N_LENSLETS, R0, L0)
    filt = fwr.LSQ if filt is None else filt
    return fwr.Plan(synth.pupil_mask(N_LENSLETS), PAD, filt, sigma ** 2, r0p, L0p)


def frames(F, seed0, sigma):
    """Seeded frames: (slopes float32 CUDA, true corner phases numpy)."""
    torch = _torch()
    from . import synth
    sl, ph, _ = synth.batch(N_LENSLETS, F, seed0, sigma, R0, L0)
    return torch.tensor(sl, dtype=torch.float32, device="cuda"), ph


def targets(fwr, slopes, chunk=4096):
    """Extended slopes after TARGET_ITERS iterations (FP32 path)."""
    torch = _torch()
    plan = make_plan(fwr)
    F = slopes.shape[0]
    ext = torch.empty((F, 2, GRID, GRID), dtype=torch.float32, device="cuda")
    for a in range(0, F, chunk):
        b = min(F, a + chunk)
        plan.reconstruct(slopes[a:b], TARGET_ITERS, ext_out=ext[a:b])
    torch.cuda.synchronize()
    return ext


def train(fwr, n_frames, epochs, width, batch=256, lr=2e-3, seed=0, log=print):
    torch = _torch()
    t0 = time.time()
    slopes, _ = frames(n_frames, TRAIN_SEED0, list(TRAIN_SIGMAS))
    ext = targets(fwr, slopes)
    log("data: %d frames in %.1f s" % (n_frames, time.time() - t0))
    plan = make_plan(fwr)
    net = fwr.Net(width, batch, he_init(width, seed))
    gen = torch.Generator(device="cpu").manual_seed(seed)
    steps = epochs * (n_frames // batch)
    step = 0
    hist = []
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(n_frames, generator=gen).cuda()
        tot = 0.0
        for i in range(n_frames // batch):
            idx = perm[i * batch:(i + 1) * batch]
            # cosine decay of the learning rate
            cur = lr * 0.5 * (1.0 + np.cos(np.pi * step / max(1, steps)))
            tot += net.train_step(plan, slopes[idx].contiguous(), ext[idx].contiguous(), max(cur, 1e-6))
            step += 1
        hist.append(tot / (n_frames // batch))
        log("epoch %d: loss %.5f (%.1f s)" % (ep, hist[-1], time.time() - t0))
    return net, {"width": width, "frames": n_frames, "epochs": epochs, "batch": batch, "lr": lr,
                 "loss_per_epoch": hist, "train_seconds": time.time() - t0}


def residual_rms(fwr, phase, truth, mask):
    """Residual rms (rad) between the reconstruction at the pupil corners and
    the true phase, piston removed, averaged over frames."""
    off = (GRID - N_LENSLETS) // 2
    cm = corner_mask(mask)
    est = phase[:, off:off + N_LENSLETS + 1, off:off + N_LENSLETS + 1].double().cpu().numpy()
    r = []
    for f in range(est.shape[0]):
        d = est[f][cm] - truth[f][cm]
        d -= d.mean()
        r.append(np.mean(d * d))
    return float(np.sqrt(np.mean(r)))


def evaluate(fwr, net, n_frames=1000, reps=20, log=print):
    """Residual and frames/s of the plain loop (k = 1, 2, 10) and of the
    network followed by k = 1, 2 iterations, on the evaluation frames."""
    torch = _torch()
    from . import synth
    slopes, truth = frames(n_frames, EVAL_SEED0, EVAL_SIGMA)
    mask = synth.pupil_mask(N_LENSLETS)
    plan = make_plan(fwr, fwr.WIENER, EVAL_SIGMA)
    phase = torch.empty((n_frames, GRID, GRID), device="cuda")
    warm = torch.empty((n_frames, 2, GRID, GRID), device="cuda")

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    for k in PLAIN_ITERS:
        ms = timed(lambda: plan.reconstruct(slopes, k, phase))
        out["plain_k%d" % k] = {"residual_rad": residual_rms(fwr, phase, truth, mask), "ms": ms,
                                "frames_per_s": n_frames / ms * 1e3}
    ms_net = timed(lambda: net.forward(plan, slopes, warm))
    for k in LEARNED_ITERS:
        def run():
            net.forward(plan, slopes, warm)
            plan.reconstruct(slopes, k, phase, ext_init=warm)
        ms = timed(run)
        r = residual_rms(fwr, phase, truth, mask)
        # the cheapest plain loop that reaches at least this residual
        match = [j for j in PLAIN_ITERS if out["plain_k%d" % j]["residual_rad"] <= r]
        ref = out["plain_k%d" % match[0]] if match else None
        out["learned_k%d" % k] = {"residual_rad": r, "ms": ms, "net_ms": ms_net,
                                  "frames_per_s": n_frames / ms * 1e3,
                                  "plain_iters_same_residual": match[0] if match else None,
                                  "speedup_same_residual": ref["ms"] / ms if ref else None}
    for key, v in out.items():
        log("%-11s residual %.4f rad  %.3f ms  %.0f frames/s" % (key, v["residual_rad"], v["ms"], v["frames_per_s"]))
    return out


def load_net(fwr, path=WEIGHTS, max_batch=1000):
    d = np.load(path)
    return fwr.Net(int(d["width"]), max_batch, d["weights"])


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--frames", type=int, default=32768)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--width", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--report", default=None)
    args = ap.parse_args(argv)
    from . import fwr
    fwr.load()
    if args.cmd == "train":
        net, info = train(fwr, args.frames, args.epochs, args.width, lr=args.lr)
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        np.savez(args.out, weights=net.weights(), width=args.width)
        info["eval"] = evaluate(fwr, load_net(fwr, args.out))
        if args.report:
            with open(args.report, "w") as fh:
                json.dump(info, fh, indent=1)
        print(json.dumps(info["eval"]))
    else:
        res = evaluate(fwr, load_net(fwr, args.weights))
        print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
