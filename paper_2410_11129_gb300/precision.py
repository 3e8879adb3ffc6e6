"""Storage-precision study of the coupled step: FP32 and FP32 weight-offset
populations against FP64.

  python -m paper_2410_11129_gb300.precision --workload 2400x300 --checkpoints 10000,50000
  python -m paper_2410_11129_gb300.precision --workload 1600x200 --checkpoints 100000 --every 1000

Every form starts from the same initial state and advances to each checkpoint;
at each checkpoint the report gives, per form, the relative drift of the three
phase masses since step 0, the max-norm velocity error relative to max |u| of
the FP64 run, the max-norm phase-field error, and the error of each observable
(deformations, centroids) against FP64. With --every, the observable histories
are compared at that interval as well. The FP64 form itself is the
parity-tested path (it matches the CPU oracle to round-off).
"""
import argparse
import json
import sys

import numpy as np

from . import fcd
from . import workloads as W

NAMED = {"200x40": W.C1, "1600x200": W.C2, "2400x300": W.C3, "800x100": W.C5}
OBS_KEYS = ("T_o", "T_i", "xc_core", "yc_core", "xc_shell", "yc_shell")
FORMS = ("fp64", "fp32", "fp32_offset")


def snapshot(ch):
    ob = ch.observe(allow=(fcd.FCD_ENOCONV,))
    return {"obs": ob, "ux": ch.field("ux"), "uy": ch.field("uy"),
            "phi": np.stack([ch.field("phi1"), ch.field("phi2")])}


def run_form(cfg, form, checkpoints, every):
    cfg = dict(cfg, precision=form)
    if form == "fp64":
        cfg["mag_tol"] = min(cfg["mag_tol"], 1e-10)
    ch = fcd.Channel(cfg)
    m0 = np.array(ch.observe(allow=(fcd.FCD_ENOCONV,))["mass"])
    snaps, hist, done = {}, [], 0
    marks = sorted(set(checkpoints) | (set(range(every, max(checkpoints) + 1, every)) if every else set()))
    for m in marks:
        ch.step(m - done)
        done = m
        if m in checkpoints:
            snaps[m] = snapshot(ch)
        if every and m % every == 0:
            ob = ch.observe(allow=(fcd.FCD_ENOCONV,))
            hist.append({k: ob[k] for k in OBS_KEYS + ("step",)})
    ch.close()
    return m0, snaps, hist


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="2400x300", choices=sorted(NAMED))
    ap.add_argument("--checkpoints", default="10000,50000")
    ap.add_argument("--every", type=int, default=0)
    ap.add_argument("--forms", default=",".join(FORMS))
    args = ap.parse_args(argv)
    cfg = dict(NAMED[args.workload])
    checkpoints = [int(c) for c in args.checkpoints.split(",")]
    forms = args.forms.split(",")
    assert forms[0] == "fp64", "the first form is the reference"
    results = {f: run_form(cfg, f, checkpoints, args.every) for f in forms}
    m0_ref, ref, ref_hist = results["fp64"]
    report = {"workload": cfg["name"], "checkpoints": {}}
    for c in checkpoints:
        row = {}
        umax = max(np.abs(ref[c]["ux"]).max(), np.abs(ref[c]["uy"]).max())
        for f in forms:
            m0, snaps, _ = results[f]
            s = snaps[c]
            m = np.array(s["obs"]["mass"])
            entry = {"mass_drift_rel": list((m - m0) / np.abs(m0))}
            if f != "fp64":
                entry["u_err_rel"] = float(max(np.abs(s["ux"] - ref[c]["ux"]).max(),
                                               np.abs(s["uy"] - ref[c]["uy"]).max()) / umax)
                entry["phi_err"] = float(np.abs(s["phi"] - ref[c]["phi"]).max())
                entry["obs_err"] = {k: s["obs"][k] - ref[c]["obs"][k] for k in OBS_KEYS}
            entry["breakup"] = [s["obs"]["breakup"], s["obs"]["b_step"]]
            row[f] = entry
        report["checkpoints"][c] = row
    if args.every:
        report["history_max_err"] = {}
        for f in forms[1:]:
            h = results[f][2]
            report["history_max_err"][f] = {
                k: float(max(abs(a[k] - b[k]) for a, b in zip(h, ref_hist))) for k in OBS_KEYS}
    print(json.dumps(report, indent=1), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
