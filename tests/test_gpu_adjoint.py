"""Discrete adjoint (reverse mode) of the coupled step (needs a GB300).

The reverse sweep's gradients of J = w_T T_o + w_overlap sum phi_1 phi_3 are
checked against (1) the tangent-linear context, which differentiates the same
discrete step forwards (agreement up to the potential-solve tolerance),
(2) Richardson-extrapolated central differences of the FP64 CPU oracle,
(3) central differences of the plain FP64 GPU path and of the oracle along
random directions of the initial populations (the state adjoint
dJ/d(f0, g0)), (4) the FP64 CPU adjoint of oracle/torch_step.py, element by
element, and (5) the exact
zero of dT_o/dalpha at alpha = 0 for a droplet on the centre line. The
checkpoint interval must not change a bit.
"""
import math

import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 30


@pytest.fixture(scope="module")
def fcd():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2410_11129_gb300 import fcd as F
    F.load()
    return F


def grad_cfg(**kw):
    base = dict(nx=48, ny=20, r1=3.0, r2=6.0, xc=14.0, xi=4.0, Ca=0.1, Bo_m=2.0,
                alpha_deg=math.degrees(0.3), nu_r=1.5, ferro="shell", chi_ferro=1.0,
                mag_tol=1e-13, mag_max_iter=300)
    base.update(kw)
    return dict(W.small(**base), precision="fp64")


def overlap_of(phi1, phi2):
    return float(np.sum(phi1 * (1.0 - phi1 - phi2)))


def richardson(fun, theta, j, rel=1e-3):
    h = rel * max(abs(theta[j]), 1.0)

    def D(hh):
        tp, tm = list(theta), list(theta)
        tp[j] += hh
        tm[j] -= hh
        return (fun(tp) - fun(tm)) / (2 * hh)

    return (4 * D(h / 2) - D(h)) / 3


def adjoint_grads(F, cfg, steps, checkpoint, initial=False, weights=((1.0, 0.0), (0.0, 1.0))):
    ch = F.Adjoint(cfg, checkpoint)
    ch.step(steps)
    out = [ch.gradient(wT, wO, initial=initial) for wT, wO in weights]
    assert ch.observe()["step"] == steps  # back at the final state
    ch.close()
    return out


def tangent_obs(F, cfg, steps):
    ch = F.Tangent(cfg)
    ch.step(steps)
    o = ch.tangent_observe()
    ch.close()
    return o


@pytest.mark.parametrize("open_x", [0, 1])
def test_adjoint_matches_tangent(fcd, open_x):
    """Four segments (8, 8, 8, 6 steps): reverse and forward mode agree, in the
    periodic and in the open channel (Eq. 37 inlet, convective outlet)."""
    cfg = grad_cfg(open_x=open_x)
    t = tangent_obs(fcd, cfg, STEPS)
    aT, aO = adjoint_grads(fcd, cfg, STEPS, 8)
    for a, ref, name in ((aT, t["dT_o"], "T_o"), (aO, t["doverlap"], "overlap")):
        scale = max(abs(v) for v in ref)
        assert scale > 0
        err = max(abs(x - y) for x, y in zip(a["grad"], ref))
        assert err <= 1e-9 * scale, (name, a["grad"], ref)
        assert a["capped_solves"] == 0
    # the forward pass kept the last segment (steps 24-29); the first sweep
    # recomputes the other three, the second finds the slots reused and
    # recomputes all four
    assert aT["recomputed_steps"] == 24 and aO["recomputed_steps"] == 30
    assert aT["solve_cycles"] > 0
    assert abs(aT["T_o"] - t["T_o"]) <= 1e-13
    assert abs(aO["overlap"] - t["overlap"]) <= 1e-10 * max(1.0, t["overlap"])
    assert aT["J"] == aT["T_o"] and aO["J"] == aO["overlap"]


def test_checkpoint_interval_does_not_change_bits(fcd):
    """Recomputed segments are bitwise the forward states, so the sweep gives
    the same bits for any interval (one step per segment, ragged, one segment)."""
    cfg = grad_cfg()
    w = ((1.0, 0.5),)
    ref = adjoint_grads(fcd, cfg, STEPS, 1, initial=True, weights=w)[0]
    for K in (7, 64):
        o = adjoint_grads(fcd, cfg, STEPS, K, initial=True, weights=w)[0]
        assert o["grad"] == ref["grad"]
        assert np.array_equal(o["df0"], ref["df0"]) and np.array_equal(o["dg0"], ref["dg0"])


def test_adjoint_graph_and_host_loop_agree(fcd, monkeypatch):
    """The captured adjoint step (solve loop as a graph while node) and the
    host-driven loop: same values, gradients equal to round-off (measured
    1e-13 relative; the plain and tangent steps agree bitwise)."""
    cfg = grad_cfg(mag_tol=1e-10)
    a = adjoint_grads(fcd, cfg, 20, 6, weights=((1.0, 1.0),))[0]
    monkeypatch.setenv("FCD_NO_GRAPH", "1")
    b = adjoint_grads(fcd, cfg, 20, 6, weights=((1.0, 1.0),))[0]
    assert a["T_o"] == b["T_o"] and a["overlap"] == b["overlap"]
    scale = max(abs(v) for v in a["grad"])
    assert max(abs(x - y) for x, y in zip(a["grad"], b["grad"])) <= 1e-11 * scale


@pytest.mark.parametrize("open_x", [0, 1])
def test_adjoint_against_oracle_differences(fcd, orc, open_x):
    cfg = grad_cfg(open_x=open_x)
    theta = list(fcd.parameters_of(cfg))
    aT, aO = adjoint_grads(fcd, cfg, STEPS, 16)

    def run(th):
        sim = orc.Sim(fcd.with_parameters(cfg, th))
        sim.step(STEPS)
        ob = sim.observe()
        phi = sim.phi()
        return np.array([ob["T_o"], overlap_of(phi[0], phi[1])])

    fd = np.array([richardson(run, theta, j) for j in range(4)])  # 4 x 2
    for q, a in enumerate((aT, aO)):
        scale = np.abs(fd[:, q]).max()
        assert scale > 0
        assert np.abs(np.array(a["grad"]) - fd[:, q]).max() <= 1e-5 * scale, (a["grad"], fd[:, q])


def test_initial_state_adjoint_against_gpu_differences(fcd):
    """<dJ/dg0, d> and <dJ/df0, e> against central differences of plain FP64
    runs started from perturbed populations (seeded random directions). The
    step clamps phi to [0, 1] (kinks at the bulk values), so the phase-field
    direction is relative: d phi_i = phi_i phi_3 r_i with random r_i keeps the
    sign of phi_1, phi_2 and phi_3 at every node, and no difference straddles
    a kink; f needs no such care."""
    cfg = grad_cfg()
    wT, wO = 1.0, 2.0
    o = adjoint_grads(fcd, cfg, STEPS, 10, initial=True, weights=((wT, wO),))[0]
    base = fcd.Channel(cfg)
    f0, g0, psi0 = base.populations()
    base.close()
    rng = np.random.default_rng(2024)
    p1, p2 = g0[0].sum(axis=0), g0[1].sum(axis=0)
    p3 = 1.0 - p1 - p2
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]

    def J(f, g):
        ch = fcd.Channel(cfg)
        ch.set_populations(f, g, psi0, step=0)
        ch.step(STEPS)
        val = wT * ch.observe()["T_o"] + wO * overlap_of(ch.field("phi1"), ch.field("phi2"))
        ch.close()
        return val

    for which in ("g", "f"):
        if which == "g":
            r = rng.standard_normal((2,) + p1.shape)
            d = np.stack([w * (p1 * p3 * r[0]), w * (p2 * p3 * r[1])])
        else:
            d = rng.standard_normal(f0.shape)
        h = 1e-6
        if which == "g":
            fd = (J(f0, g0 + h * d) - J(f0, g0 - h * d)) / (2 * h)
            ad = float(np.sum(o["dg0"] * d))
            mag = float(np.sum(np.abs(o["dg0"] * d)))
        else:
            fd = (J(f0 + h * d, g0) - J(f0 - h * d, g0)) / (2 * h)
            ad = float(np.sum(o["df0"] * d))
            mag = float(np.sum(np.abs(o["df0"] * d)))
        assert mag > 0
        assert abs(fd - ad) <= 1e-6 * mag + 1e-7 * abs(ad), (which, fd, ad, mag)


def test_initial_state_adjoint_against_oracle_differences(fcd, orc):
    """The same directional derivatives along the initial populations, the
    differences taken with the FP64 CPU oracle instead of the GPU path."""
    cfg = grad_cfg()
    wT, wO = 1.0, 2.0
    o = adjoint_grads(fcd, cfg, STEPS, 10, initial=True, weights=((wT, wO),))[0]
    base = orc.Sim(cfg)
    g0 = base.g.copy()
    p1, p2 = g0[0].sum(axis=0), g0[1].sum(axis=0)
    p3 = 1.0 - p1 - p2
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    rng = np.random.default_rng(7)

    def J(df, dg):
        sim = orc.Sim(cfg)
        sim.f += df
        sim.g += dg
        sim.step(STEPS)
        phi = sim.phi()
        return wT * sim.observe()["T_o"] + wO * overlap_of(phi[0], phi[1])

    h = 1e-6
    r = rng.standard_normal((2,) + p1.shape)
    dg = np.stack([w * (p1 * p3 * r[0]), w * (p2 * p3 * r[1])])
    df = rng.standard_normal(base.f.shape)
    zf, zg = np.zeros_like(df), np.zeros_like(dg)
    for name, a, b, bar in (("g", zf, dg, o["dg0"]), ("f", df, zg, o["df0"])):
        fd = (J(h * a, h * b) - J(-h * a, -h * b)) / (2 * h)
        d = b if name == "g" else a
        ad = float(np.sum(bar * d))
        mag = float(np.sum(np.abs(bar * d)))
        assert mag > 0
        assert abs(fd - ad) <= 1e-6 * mag + 1e-7 * abs(ad), (name, fd, ad, mag)


@pytest.mark.parametrize("open_x", [0, 1])
def test_adjoint_against_cpu_adjoint(fcd, orc, open_x):
    """The GPU sweep against the FP64 CPU adjoint (oracle/torch_step.py: the
    oracle's step in PyTorch float64 with an exact potential solve, reverse
    mode by torch.autograd): the four parameter derivatives, and the fields
    dJ/d(f0, g0) element by element."""
    from oracle import torch_step as TS
    cfg = grad_cfg(open_x=open_x)
    o = adjoint_grads(fcd, cfg, STEPS, 8, initial=True, weights=((1.0, 2.0),))[0]
    sim = orc.Sim(cfg)
    r = TS.gradients(cfg, STEPS, sim.f.copy(), sim.g.copy(), 1.0, 2.0)
    assert abs(o["J"] - r["J"]) <= 1e-10 * max(1.0, abs(r["J"]))
    scale = max(abs(v) for v in r["grad"])
    assert max(abs(a - b) for a, b in zip(o["grad"], r["grad"])) <= 1e-8 * scale, (o["grad"], r["grad"])
    for key in ("df0", "dg0"):
        ref, got = r[key], o[key]
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), key


def test_state_seed_reproduces_the_overlap_functional(fcd):
    """Seeding the sweep with dJ/dg_N of the overlap (phi_3 - phi_1 on the
    core planes, -phi_1 on the shell planes) gives the built-in gradient."""
    cfg = grad_cfg()
    ch = fcd.Adjoint(cfg, 8)
    ch.step(STEPS)
    o1 = ch.gradient(0.0, 1.0, initial=True)
    f, g, _ = ch.populations()
    p1, p2 = g[0].sum(axis=0), g[1].sum(axis=0)
    sg = np.stack([np.repeat((1.0 - 2.0 * p1 - p2)[None], 9, axis=0),
                   np.repeat((-p1)[None], 9, axis=0)])
    o2 = ch.gradient_state(None, sg, initial=True)
    ch.close()
    scale = max(abs(v) for v in o1["grad"])
    assert max(abs(a - b) for a, b in zip(o1["grad"], o2["grad"])) <= 1e-12 * scale
    assert np.abs(o1["dg0"] - o2["dg0"]).max() <= 1e-12 * np.abs(o1["dg0"]).max()
    assert o2["J"] == 0.0 and o2["overlap"] == o1["overlap"]


def test_final_state_autograd_against_cpu_adjoint(fcd, orc):
    """A torch loss of the final populations back-propagated through
    fcd.final_state (one GPU sweep) against the same loss through the FP64
    CPU adjoint."""
    import torch
    from oracle import torch_step as TS
    cfg = grad_cfg()
    rng = np.random.default_rng(5)
    S = torch.from_numpy(rng.standard_normal((9, 20, 48)))
    R = torch.from_numpy(rng.standard_normal((2, 9, 20, 48)))
    th = torch.tensor(fcd.parameters_of(cfg), dtype=torch.float64, requires_grad=True)
    f, g = fcd.final_state(th, cfg, STEPS, checkpoint=8)
    loss = (f * S).sum() + (g * R).sum()
    loss.backward()
    sim = orc.Sim(cfg)
    theta = torch.tensor(TS.parameters_of(cfg), dtype=torch.float64, requires_grad=True)
    _, (fc, gc) = TS.run(cfg, theta, STEPS, sim.f.copy(), sim.g.copy())
    lc = (fc * S.reshape(9, -1)).sum() + (gc * R.reshape(2, 9, -1)).sum()
    lc.backward()
    assert abs(loss.item() - lc.item()) <= 1e-10 * max(1.0, abs(lc.item()))
    ref, got = theta.grad.numpy(), th.grad.numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), (got, ref)
    # a GPU-resident theta gets its gradient on its own device
    thd = torch.tensor(fcd.parameters_of(cfg), dtype=torch.float64, device="cuda",
                       requires_grad=True)
    f, g = fcd.final_state(thd, cfg, STEPS, checkpoint=8)
    ((f * S).sum() + (g * R).sum()).backward()
    assert thd.grad.device == thd.device
    assert np.abs(thd.grad.cpu().numpy() - got).max() <= 1e-12 * np.abs(got).max()


def test_adjoint_alpha_derivative_vanishes_by_symmetry(fcd):
    cfg = grad_cfg(alpha_deg=0.0, yc=9.5)
    aT, aO = adjoint_grads(fcd, cfg, STEPS, 10)
    ia = fcd.DIRECTIONS.index("alpha")
    for a in (aT, aO):
        other = max(abs(v) for v in a["grad"])
        assert other > 0
        assert abs(a["grad"][ia]) <= 1e-11 * other


def test_adjoint_autograd_matches_tangent(fcd):
    import torch
    cfg = grad_cfg(Ca=0.12, Bo_m=1.5, alpha_deg=20.0, nu_r=0.8)
    theta = list(fcd.parameters_of(cfg))
    t = tangent_obs(fcd, cfg, STEPS)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    out = fcd.droplet_observables(th, cfg, STEPS, method="adjoint", checkpoint=12)
    assert abs(out[0].item() - t["T_o"]) <= 1e-13
    (out[0] + 2.0 * out[1]).backward()
    expect = np.array(t["dT_o"]) + 2.0 * np.array(t["doverlap"])
    assert np.abs(th.grad.numpy() - expect).max() <= 1e-9 * np.abs(expect).max()


def test_adjoint_rejects_bad_input(fcd):
    for bad, K in ((dict(Bo_m=0.0), 10), ({}, 0)):
        with pytest.raises(fcd.FcdError) as e:
            fcd.Adjoint(grad_cfg(**bad), K)
        assert e.value.status == fcd.FCD_EINVAL
    ch = fcd.Adjoint(grad_cfg(), 5)
    with pytest.raises(fcd.FcdError) as e:
        ch.get_state(np.zeros(16, np.uint8))
    assert e.value.status == fcd.FCD_ESTATE
    ch.close()
    plain = fcd.Channel(grad_cfg())
    o = fcd.fcd_adjoint_out()
    import ctypes as C
    assert fcd.load().fcd_adjoint_gradient(plain.h, 1.0, 0.0, C.byref(o), None, None) == fcd.FCD_EINVAL
    plain.close()
