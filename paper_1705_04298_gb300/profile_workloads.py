"""Run one of the library's workloads a few times, for timing or under a
profiler (each one a plain sequence of library calls on seeded synthetic
frames; no measurement logic of its own beyond a CUDA-event mean).

    python -m paper_1705_04298_gb300.profile_workloads fused128 --reps 3
    python -m paper_1705_04298_gb300.profile_workloads slab256 --reps 3
    python -m paper_1705_04298_gb300.profile_workloads dftgemm256 --reps 2
    python -m paper_1705_04298_gb300.profile_workloads unet --reps 3

Workloads (1000 frames unless --frames):
  fused128     40x40 lenslets on 128^2, Wiener, k iterations (default 10)
  slab256      128x128 lenslets on 256^2 (frozen-flow frames), LSQ, k = 10
  dftgemm256   the same through the split-BF16 DFT-as-GEMM transform
  unet         the warm-start U-Net forward on 40x40 slopes (committed weights)
"""

import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["fused128", "slab256", "dftgemm256", "unet"])
    ap.add_argument("--frames", type=int, default=1000)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    import torch
    from . import fwr, learned, synth
    fwr.load()
    F, k = args.frames, args.iters
    if args.workload == "fused128":
        sl, _, mask = synth.batch(40, min(F, 64), 1000, 0.1)
        r0p, L0p = synth.pitch_units(40, 0.15, 25.0)
        plan = fwr.Plan(mask, 3.2, fwr.WIENER, 0.01, r0p, L0p)
        s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat((F + 63) // 64, 1, 1, 1)[:F].contiguous()
        out = torch.empty((F, plan.N, plan.N), device="cuda")
        run = lambda: plan.reconstruct(s, k, out)  # noqa: E731
    elif args.workload in ("slab256", "dftgemm256"):
        sl, _, mask = synth.frozen_flow(128, 32, 7, 0.05, r0=0.12, L0=25.0)
        plan = fwr.Plan(mask, 2.0, fwr.LSQ)
        if args.workload == "dftgemm256":
            plan.set_transform(fwr.TRANSFORM_DFT_BF16X3)
        s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat((F + 31) // 32, 1, 1, 1)[:F].contiguous()
        out = torch.empty((F, plan.N, plan.N), device="cuda")
        run = lambda: plan.reconstruct(s, k, out)  # noqa: E731
    else:
        net = learned.load_net(fwr, learned.WEIGHTS, max_batch=F)
        plan = learned.make_plan(fwr, fwr.WIENER, learned.EVAL_SIGMA)
        s, _ = learned.frames(F, learned.EVAL_SEED0, learned.EVAL_SIGMA)
        out = torch.empty((F, 2, 128, 128), device="cuda")
        run = lambda: net.forward(plan, s, out)  # noqa: E731
    run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    print("%s: %.4f ms per call of %d frames" % (args.workload, e0.elapsed_time(e1) / args.reps, F))
    return 0


if __name__ == "__main__":
    sys.exit(main())
