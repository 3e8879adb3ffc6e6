"""The storage forms on the 2400 x 300 precision-study channel against the FP64
oracle itself (not against the GPU's FP64 form), per field and per observable.

The oracle runs row-parallel on every host core (bitwise the same as one
thread); the GPU FP64 form must match it to round-off on this channel too, and
the FP32 forms within 1e-4 (phase fields absolute, velocity relative to its
maximum, T_o and T_i, centroids relative to the channel length). The FP32
forms solve the potential to 1e-6 (the hi + lo pair), FP64 to 1e-10. The
channel's eps_n (1e-4) keeps the interface normal above the rounding of
either form; with 1e-12 the FP32 phase fields part from the oracle's by 1e-3
within 100 steps on the ridge of the thick shell, while u and every
observable still agree to 1e-5.
"""
import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 40


@pytest.fixture(scope="module")
def oracle_state(orc):
    cfg = dict(W.C3, mag_tol=1e-10, mag_max_iter=100000)
    orc.set_threads(orc.max_threads())
    try:
        sim = orc.Sim(cfg)
        sim.step(STEPS)
        ob = sim.observe()
        return {"phi": sim.phi()[:2].copy(), "ux": sim.macro[0].copy(), "uy": sim.macro[1].copy(),
                "obs": ob}
    finally:
        orc.set_threads(1)


@pytest.mark.parametrize("prec,tol_field", [("fp64", 1e-8), ("fp32_offset", 1e-4), ("fp32", 1e-4)])
def test_forms_against_the_oracle_on_the_precision_channel(oracle_state, prec, tol_field):
    import torch
    assert torch.cuda.is_available()
    from paper_2410_11129_gb300 import fcd
    cfg = dict(W.C3, precision=prec, mag_tol=1e-10 if prec == "fp64" else 1e-6, mag_max_iter=300)
    ch = fcd.Channel(cfg)
    ch.step(STEPS)
    phi = np.stack([ch.field("phi1"), ch.field("phi2")])
    ux, uy = ch.field("ux"), ch.field("uy")
    ob = ch.observe()
    ch.close()
    ref = oracle_state
    umax = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
    err = {"phi": float(np.abs(phi - ref["phi"]).max()),
           "u": float(max(np.abs(ux - ref["ux"]).max(), np.abs(uy - ref["uy"]).max()) / umax)}
    for k in ("T_o", "T_i"):
        err[k] = abs(ob[k] - ref["obs"][k])
    for k in ("xc_core", "yc_core", "xc_shell", "yc_shell"):
        err[k] = abs(ob[k] - ref["obs"][k]) / cfg["nx"]
    print(prec, STEPS, "steps vs the FP64 oracle:", err)
    assert err["phi"] <= tol_field and err["u"] <= tol_field
    for k in ("T_o", "T_i", "xc_core", "yc_core", "xc_shell", "yc_shell"):
        assert err[k] <= max(tol_field, 1e-9), (k, err[k])
