"""Gradient of the shell deformation: tangent-linear run and discrete adjoint
against central differences of the plain FP64 method, on the same GPU.

  python -m paper_2410_11129_gb300.gradient --steps 20000
  python -m paper_2410_11129_gb300.gradient --steps 500 --h 1e-4 --checkpoint 500
  python -m paper_2410_11129_gb300.gradient --steps 20 --checkpoint 20 --only adjoint

The tangent context advances the state and its derivatives along
(Bo_m, Ca, alpha, nu_r) together; the adjoint context runs the plain step with
a checkpoint every `checkpoint` steps, then one reverse sweep per functional
(T_o, then the overlap); central differences need two plain runs per
direction (eight in all) with theta_j +- h * max(|theta_j|, 1). All report
dT_o/dtheta and d overlap/dtheta (overlap = sum phi_1 phi_3) at the final
step; the wall time of each includes every run it needs.
"""
import argparse
import json
import sys
import time

import numpy as np

from . import fcd
from . import workloads as W


def _overlap(ch):
    p1, p2 = ch.field("phi1"), ch.field("phi2")
    return float(np.sum(p1 * (1.0 - p1 - p2)))


def tangent_gradient(cfg, steps):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ch = fcd.Tangent(cfg)
    ch.step(steps)
    o = ch.tangent_observe(allow=(fcd.FCD_ENOCONV,))
    stats = ch.solver_stats()
    ch.close()
    torch.cuda.synchronize()
    return o, time.perf_counter() - t0, stats


def adjoint_gradient(cfg, steps, checkpoint):
    """Forward pass with checkpoints, then the sweep for T_o and the sweep for
    the overlap; seconds: the forward pass plus the T_o sweep, and the total."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ch = fcd.Adjoint(cfg, checkpoint)
    ch.step(steps)
    torch.cuda.synchronize()
    tf = time.perf_counter()
    aT = ch.gradient(1.0, 0.0, allow=(fcd.FCD_ENOCONV,))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    aO = ch.gradient(0.0, 1.0, allow=(fcd.FCD_ENOCONV,))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ch.close()
    return ({"dT_o": aT["grad"], "doverlap": aO["grad"], "T_o": aT["T_o"],
             "capped_solves": aT["capped_solves"] + aO["capped_solves"],
             "recomputed_steps": [aT["recomputed_steps"], aO["recomputed_steps"]],
             "solve_cycles": [aT["solve_cycles"], aO["solve_cycles"]],
             "seconds_forward": tf - t0, "seconds_sweeps": [t1 - tf, t2 - t1]},
            t1 - t0, t2 - t0)


def difference_gradient(cfg, steps, h_rel):
    import torch
    theta = list(fcd.parameters_of(cfg))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dT, dO = [], []
    for j in range(4):
        h = h_rel * max(abs(theta[j]), 1.0)
        vals = []
        for s in (1.0, -1.0):
            th = list(theta)
            th[j] += s * h
            ch = fcd.Channel(fcd.with_parameters(cfg, th))
            ch.step(steps)
            ob = ch.observe(allow=(fcd.FCD_ENOCONV,))
            vals.append((ob["T_o"], _overlap(ch)))
            ch.close()
        dT.append((vals[0][0] - vals[1][0]) / (2 * h))
        dO.append((vals[0][1] - vals[1][1]) / (2 * h))
    torch.cuda.synchronize()
    return {"dT_o": dT, "doverlap": dO}, time.perf_counter() - t0


def compare(cfg, steps, h_rel=1e-4, checkpoint=500, only=None):
    cfg = dict(cfg, precision="fp64")
    if only == "adjoint":  # the adjoint alone (profiling runs)
        adj, t_adj1, t_adj2 = adjoint_gradient(cfg, steps, checkpoint)
        return {"steps": steps, "adjoint": dict(adj, checkpoint=checkpoint,
                                                seconds_one_functional=t_adj1, seconds_both=t_adj2)}
    if only == "tangent,adjoint":  # both exact forms, no difference runs
        o, t_tan, stats = tangent_gradient(cfg, steps)
        adj, t_adj1, t_adj2 = adjoint_gradient(cfg, steps, checkpoint)
        out = {"steps": steps, "T_o": o["T_o"], "overlap": o["overlap"],
               "tangent": {"dT_o": o["dT_o"], "doverlap": o["doverlap"], "seconds": t_tan,
                           "solver": stats},
               "adjoint": dict(adj, checkpoint=checkpoint, seconds_one_functional=t_adj1,
                               seconds_both=t_adj2)}
        for q in ("dT_o", "doverlap"):
            a, c = np.array(o[q]), np.array(adj[q])
            out["max_rel_diff_adjoint_tangent_" + q] = float(
                np.abs(c - a).max() / max(np.abs(a).max(), 1e-300))
        return out
    o, t_tan, stats = tangent_gradient(cfg, steps)
    adj, t_adj1, t_adj2 = adjoint_gradient(cfg, steps, checkpoint)
    fd, t_fd = difference_gradient(cfg, steps, h_rel)
    out = {"workload": cfg.get("name", "%dx%d" % (cfg["nx"], cfg["ny"])), "steps": steps,
           "directions": list(fcd.DIRECTIONS), "mag_tol": cfg["mag_tol"], "h_rel": h_rel,
           "T_o": o["T_o"], "overlap": o["overlap"],
           "tangent": {"dT_o": o["dT_o"], "doverlap": o["doverlap"], "seconds": t_tan,
                       "solver": stats},
           "adjoint": dict(adj, checkpoint=checkpoint, seconds_one_functional=t_adj1,
                           seconds_both=t_adj2),
           "central_differences": dict(fd, seconds=t_fd, runs=8),
           "speedup": t_fd / t_tan,
           "speedup_adjoint_one_functional": t_fd / t_adj1,
           "speedup_adjoint_both": t_fd / t_adj2}
    for q in ("dT_o", "doverlap"):
        a, b, c = np.array(o[q]), np.array(fd[q]), np.array(adj[q])
        scale = max(np.abs(a).max(), 1e-300)
        out["max_rel_diff_" + q] = float(np.abs(a - b).max() / scale)
        out["max_rel_diff_adjoint_tangent_" + q] = float(np.abs(c - a).max() / scale)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=W.C5["steps"])
    ap.add_argument("--h", type=float, default=1e-4, help="relative step of the differences")
    ap.add_argument("--checkpoint", type=int, default=W.C5.get("checkpoint", 500),
                    help="checkpoint interval of the adjoint")
    ap.add_argument("--only", choices=["adjoint", "tangent,adjoint"], default=None,
                    help="run only the adjoint, or only the tangent and the adjoint")
    args = ap.parse_args(argv)
    print(json.dumps(compare(W.C5, args.steps, args.h, args.checkpoint, args.only), indent=1),
          flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
