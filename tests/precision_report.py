"""Per-configuration report (not a test): time and error against the FP64
oracle of every form on the single shot, the precision sweep (N = 10, 50,
200) and the multi-panel shot, and both variants on the large shot.

Run on a GPU machine from the repository root:
    python tests/precision_report.py
Errors are per pixel on pixels above 1e-3 of the oracle image's maximum
(max and median); times are CUDA events around one launch (best and median
of a few).  Prints one line per case.
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_2205_07976_gb300 import nbgb  # noqa: E402
from paper_2205_07976_gb300 import workloads as W  # noqa: E402


def timed(sim, reps):
    sim.zero()
    sim.add_spots()
    sim.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        sim.zero()
        sim.synchronize()
        ev0.record()
        sim.add_spots()
        ev1.record()
        torch.cuda.synchronize()
        ts.append(ev0.elapsed_time(ev1) / 1e3)
    return min(ts), float(np.median(ts))


def errors(got, ref):
    m = ref > 1e-3 * ref.max()
    r = np.abs(got[m] - ref[m]) / ref[m]
    return r.max(), float(np.median(r)), int(m.sum())


def report(name, shot, forms, reps, ref=None):
    for p in forms:
        sim = nbgb.Sim(p).set_shot(shot)
        best, med = timed(sim, reps)
        line = (f"{name} {p}: best {best * 1e3:.3f} ms median "
                f"{med * 1e3:.3f} ms {shot.pixel_steps / med:.3e} "
                "pixel-steps/s")
        if ref is not None:
            e = errors(sim.image(), ref)
            line += f" maxrel {e[0]:.2e} medrel {e[1]:.2e} (n={e[2]})"
        print(line, flush=True)
        sim.close()


def main():
    c0 = W.single_shot_small()
    report("single 256^2", c0, ("f64", "mixed", "f32"), 5, oracle.image(c0))
    for N in (10, 50, 200):
        s = W.precision_shot(N)
        t0 = time.time()
        ref = oracle.image(s)
        dt = time.time() - t0
        print(f"precision N={N} oracle: {dt:.1f} s "
              f"({s.pixel_steps / dt:.3e} pixel-steps/s, "
              f"{oracle.max_threads()} threads)", flush=True)
        report(f"precision N={N}", s, ("f64", "mixed", "f32"), 3, ref)
    for S in (1, 2, 4, 8):
        report(f"multipanel S={S}", W.multipanel_shot(S), ("f64", "mixed"), 3)
    c1 = W.large_shot()
    for v in ("warp", "thread"):
        sim = nbgb.Sim("mixed").set_shot(c1).set_variant(v)
        best, med = timed(sim, 2)
        print(f"large mixed {v}: best {best * 1e3:.3f} ms median "
              f"{med * 1e3:.3f} ms {c1.pixel_steps / med:.3e} pixel-steps/s",
              flush=True)
        sim.close()


if __name__ == "__main__":
    main()
