"""Batched closed-loop simulation around the reconstructor (the paper's
closed-loop study, Sec. 4.2: residual slopes, an integrator with a one-frame
delay, few Gerchberg iterations): many independent loops, one library call per
time step for all of them.

Each loop sees its own seeded frozen-flow von Karman screen. The corrector is
the phase at the lenslet corners (a bilinear surface), so its slopes over a
lenslet are exactly the mean of the lenslet's two edge differences (Fried
geometry). At step t the wave-front sensor measures the turbulence slopes
minus the corrector's, plus white noise; the reconstruction at the corners is
added, times the loop gain, to the corrector one frame later. The residual
phase is compared at the pupil corners, piston removed.

Host-side bookkeeping in numpy; each step's reconstruction of all loops is one
`Plan.reconstruct` call.
"""

from collections import deque

import numpy as np


def corrector_slopes(corners):
    """(L, n+1, n+1) corner phases -> (L, 2, n, n) slopes of their bilinear
    surface: for lenslet (i, j), the mean of its bottom and top (x) or left
    and right (y) edge differences."""
    p = np.asarray(corners, np.float64)
    sx = 0.5 * ((p[:, :-1, 1:] - p[:, :-1, :-1]) + (p[:, 1:, 1:] - p[:, 1:, :-1]))
    sy = 0.5 * ((p[:, 1:, :-1] - p[:, :-1, :-1]) + (p[:, 1:, 1:] - p[:, :-1, 1:]))
    return np.stack([sx, sy], axis=1)


def library_reconstructor(fwr, mask, pad, iters, periodic=2, extension=0, filt=None):
    """The library's FP32 path as a callable for `simulate`: float64 slopes
    (L, 2, n, n) in, phases (L, N, N) out (LSQ filter unless `filt`)."""
    import torch
    plan = fwr.Plan(mask, pad, fwr.LSQ if filt is None else filt, 0.0, 1.0, 1.0, periodic)
    plan.set_extension(extension)

    def run(slopes):
        s = torch.tensor(np.asarray(slopes), dtype=torch.float32, device="cuda")
        return plan.reconstruct(s, iters).double().cpu().numpy()
    return run


def turbulence(n=40, steps=60, loops=32, seed0=100, r0=0.12, L0=25.0):
    """Noise-free turbulence of `loops` seeded frozen-flow screens: slopes
    (loops, steps, 2, n, n), corner phases (loops, steps, n+1, n+1), mask."""
    from . import synth
    slopes, phases = [], []
    mask = None
    for l in range(loops):
        s, ph, mask = synth.frozen_flow(n, steps, seed0 + l, 0.0, r0=r0, L0=L0)
        slopes.append(s)
        phases.append(ph)
    return np.stack(slopes), np.stack(phases), mask


def simulate(reconstruct, n=40, steps=60, loops=32, gain=0.5, sigma=0.02, seed0=100, r0=0.12, L0=25.0,
             delay=1, data=None):
    """Run `loops` independent closed loops for `steps` frames.

    reconstruct: callable, float64 slopes (loops, 2, n, n) -> phases
    (loops, N, N) on the grid whose centred n x n lenslets the slopes fill
    (`library_reconstructor`, or the oracle on the CPU). sigma: slope noise
    (rad) of every measurement. data: the output of `turbulence` to reuse
    (else made from n, steps, loops, seed0, r0, L0). Returns a dict:
    'residual' (steps,) the residual rms (rad) at the pupil corners, averaged
    over loops, before each measurement; 'open_loop' the same for the
    turbulence alone.
    """
    from .diagnostics import corner_mask
    slopes, phases, mask = data if data is not None else turbulence(n, steps, loops, seed0, r0, L0)
    loops, steps = slopes.shape[0], slopes.shape[1]
    n = mask.shape[0]
    cm = corner_mask(mask)
    rng = np.random.default_rng(seed0 + 7919)
    dm = np.zeros((loops, n + 1, n + 1))
    pending = deque()

    def rms(p):
        d = p[:, cm]
        d = d - d.mean(axis=1, keepdims=True)
        return float(np.sqrt(np.mean(d * d)))

    residual = np.empty(steps)
    open_loop = np.empty(steps)
    for t in range(steps):
        residual[t] = rms(phases[:, t] - dm)
        open_loop[t] = rms(phases[:, t])
        meas = slopes[:, t] - corrector_slopes(dm) + sigma * rng.standard_normal((loops, 2, n, n))
        meas = np.where(mask[None, None], meas, 0.0)
        ph = reconstruct(meas)
        off = (ph.shape[-1] - n) // 2
        pending.append(ph[:, off:off + n + 1, off:off + n + 1])
        if len(pending) > delay:
            dm = dm + gain * pending.popleft()
    return {"residual": residual, "open_loop": open_loop}
