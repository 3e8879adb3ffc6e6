"""Run one of the synthetic channels and print its observables.

  python -m paper_2410_11129_gb300.run --workload 1600x200 --steps 100 [--precision fp32]

Workloads: 200x40, 1600x200, 2400x300, 800x100, 9600x1200, 900x150-open
(see workloads.py).
With FCD_NO_GRAPH=1 in the environment the potential-solve loop is driven from
the host instead of a CUDA-graph while node (same kernels; profilers that do
not follow conditional graph nodes can then see every launch).
"""
import argparse
import json
import sys
import time

from . import fcd
from . import workloads as W

NAMED = {"200x40": W.C1, "1600x200": W.C2, "2400x300": W.C3, "800x100": W.C5,
         "9600x1200": W.ROOF, "900x150-open": W.PAPER}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="1600x200", choices=sorted(NAMED))
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--every", type=int, default=0, help="print observables every N steps")
    ap.add_argument("--precision", default=None, choices=sorted(fcd.PRECISION))
    args = ap.parse_args(argv)
    import torch
    cfg = dict(NAMED[args.workload])
    if args.precision:
        cfg["precision"] = args.precision
    ch = fcd.Channel(cfg)
    done = 0
    t0 = time.perf_counter()
    while done < args.steps:
        n = min(args.every or args.steps, args.steps - done)
        ch.step(n)
        done += n
        if args.every:
            print(json.dumps(ch.observe(allow=(fcd.FCD_ENOCONV,))), flush=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = ch.observe(allow=(fcd.FCD_ENOCONV,))
    out["wall_s"] = dt
    out["solver"] = ch.solver_stats()
    print(json.dumps(out), flush=True)
    ch.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
