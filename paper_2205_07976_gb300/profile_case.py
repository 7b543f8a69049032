"""Run one named case of the library a few times, for kernel profilers.

    python -m paper_2205_07976_gb300.profile_case CASE [--n N] [--reps R]

Each case builds its shot, runs one untimed launch, then R launches of the
kernel it names, and prints one line with their mean CUDA-event time.  A
profiler skips the first launch (the table builders and the warm-up) with
its launch-skip option.  Cases:

  split   N x N window (N=512) of the large shot, warp-per-pixel kernel
  sinc    N x N window (N=256) of the 1024^2 precision sweep at Na=Nb=Nc=10
          (sinc, nearest lookup), thread-per-pixel kernel
  sinc200 the same at N=200
  f64     N x N window (N=64) of the large shot, the plain FP64 kernel
  adjoint the 64-panel differentiation shot (S=8, tricubic lookup): forward,
          Poisson loss and adjoint per repetition
  adjnear the same with nearest lookup
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["split", "sinc", "sinc200", "f64",
                                     "adjoint", "adjnear"])
    ap.add_argument("--n", type=int, default=0, help="window side")
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    from paper_2205_07976_gb300 import nbgb
    from paper_2205_07976_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    times = []

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        times.append(e0.elapsed_time(e1))

    if args.case in ("split", "f64", "sinc", "sinc200"):
        if args.case in ("split", "f64"):
            n = args.n or (512 if args.case == "split" else 64)
            shot = W.shrink(W.large_shot(), n, n, 1536 - n // 2,
                            1536 - n // 2)
            prec, variant = (("mixed", "warp") if args.case == "split"
                             else ("f64", "auto"))
        else:
            n = args.n or 256
            base = W.precision_shot(10 if args.case == "sinc" else 200)
            shot = W.shrink(base, n, n, 512 - n // 2, 512 - n // 2)
            prec, variant = "mixed", "thread"
        sim = nbgb.Sim(prec, stream=stream).set_shot(shot)
        sim.set_variant(variant)
        sim.add_spots()
        stream.synchronize()
        for _ in range(args.reps):
            timed(sim.add_spots)
        steps = shot.pixel_steps
        sim.close()
    else:
        shot = W.multipanel_shot(8)
        shot.interp = (W.INTERP_TRICUBIC if args.case == "adjoint"
                       else W.INTERP_NEAREST)
        sim = nbgb.Sim("mixed", stream=stream).set_shot(shot)
        # the differentiation leg's orientation and target
        U = W.random_orientation(np.random.default_rng(3))
        sim.set_params(U, [79.0, 79.0, 38.0], [0.0, 0.0, 0.0],
                       [15.0, 15.0, 15.0], 1.0)
        sim.add_spots()
        img = sim.image()
        y = torch.from_numpy(np.random.default_rng(7).poisson(
            img + 1.0).astype(np.float64)).to(dev)
        dL = torch.empty_like(y)
        gF = torch.zeros(shot.F.size, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()

        def step():
            sim.zero()
            sim.add_spots()
            sim.poisson_loss(y.data_ptr(), 1.0, dL.data_ptr())
            sim.adjoint(dL.data_ptr(), gF.data_ptr())

        step()
        for _ in range(args.reps):
            timed(step)
        steps = shot.pixel_steps
        sim.close()
    ms = sum(times) / len(times)
    print(f"{args.case}: {ms:.3f} ms per repetition, {steps} pixel-steps",
          flush=True)


if __name__ == "__main__":
    main()
