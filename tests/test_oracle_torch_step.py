"""The FP64 CPU adjoint (oracle/torch_step.py: the oracle's step in plain
PyTorch float64, reverse mode by torch.autograd) pinned to the C oracle: the
same states after 30 steps (periodic and open channel), parameter gradients
equal to Richardson-extrapolated central differences of the C oracle, and
directional derivatives along the initial populations equal to its central
differences."""
import math

import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W

torch = pytest.importorskip("torch")

STEPS = 30


def grad_cfg(**kw):
    base = dict(nx=48, ny=20, r1=3.0, r2=6.0, xc=14.0, xi=4.0, Ca=0.1, Bo_m=2.0,
                alpha_deg=math.degrees(0.3), nu_r=1.5, ferro="shell", chi_ferro=1.0,
                mag_tol=1e-13, mag_max_iter=300)
    base.update(kw)
    return dict(W.small(**base), precision="fp64")


def with_theta(cfg, th):
    out = dict(cfg)
    out["Bo_m"], out["Ca"], out["alpha"] = th[0], th[1], th[2]
    nu = list(cfg["nu"])
    nu[1] = nu[2] / th[3]
    out["nu"] = nu
    return out


def overlap_of(g):
    p1, p2 = g[0].sum(axis=0), g[1].sum(axis=0)
    return float(np.sum(p1 * (1.0 - p1 - p2)))


@pytest.mark.parametrize("open_x", [0, 1])
def test_torch_step_reproduces_the_oracle(orc, open_x):
    from oracle import torch_step as TS
    cfg = grad_cfg(open_x=open_x)
    sim = orc.Sim(cfg)
    f0, g0 = sim.f.copy(), sim.g.copy()
    theta = torch.tensor(TS.parameters_of(cfg), dtype=torch.float64)
    (To, ov), (f, g) = TS.run(cfg, theta, STEPS, f0, g0)
    sim.step(STEPS)
    assert np.abs(f.numpy().reshape(sim.f.shape) - sim.f).max() <= 1e-13
    assert np.abs(g.numpy().reshape(sim.g.shape) - sim.g).max() <= 1e-13
    assert abs(float(To) - sim.observe()["T_o"]) <= 1e-12
    assert abs(float(ov) - overlap_of(sim.g)) <= 1e-11


@pytest.mark.parametrize("open_x", [0, 1])
def test_cpu_adjoint_against_oracle_differences(orc, open_x):
    from oracle import torch_step as TS
    cfg = grad_cfg(open_x=open_x)
    sim = orc.Sim(cfg)
    f0, g0 = sim.f.copy(), sim.g.copy()
    rT = TS.gradients(cfg, STEPS, f0, g0, 1.0, 0.0)
    rO = TS.gradients(cfg, STEPS, f0, g0, 0.0, 1.0)
    theta = TS.parameters_of(cfg)

    def J(th):
        s = orc.Sim(with_theta(cfg, th))
        s.step(STEPS)
        return np.array([s.observe()["T_o"], overlap_of(s.g)])

    def richardson(j, rel=1e-3):
        h = rel * max(abs(theta[j]), 1.0)

        def D(hh):
            tp, tm = list(theta), list(theta)
            tp[j] += hh
            tm[j] -= hh
            return (J(tp) - J(tm)) / (2 * hh)

        return (4 * D(h / 2) - D(h)) / 3

    fd = np.array([richardson(j) for j in range(4)])  # 4 x 2
    for q, r in enumerate((rT, rO)):
        scale = np.abs(fd[:, q]).max()
        assert scale > 0
        assert np.abs(np.array(r["grad"]) - fd[:, q]).max() <= 1e-5 * scale, (r["grad"], fd[:, q])


def test_cpu_adjoint_initial_state_against_oracle_differences(orc):
    """Relative phase-field direction d phi_i = phi_i phi_3 r_i (no difference
    straddles a clamp kink), random direction for f."""
    from oracle import torch_step as TS
    cfg = grad_cfg()
    sim = orc.Sim(cfg)
    f0, g0 = sim.f.copy(), sim.g.copy()
    r = TS.gradients(cfg, STEPS, f0, g0, 1.0, 2.0)
    p1, p2 = g0[0].sum(axis=0), g0[1].sum(axis=0)
    p3 = 1.0 - p1 - p2
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    rng = np.random.default_rng(11)
    rr = rng.standard_normal((2,) + p1.shape)
    dg = np.stack([w * (p1 * p3 * rr[0]), w * (p2 * p3 * rr[1])])
    df = rng.standard_normal(f0.shape)

    def J(df_, dg_):
        s = orc.Sim(cfg)
        s.f += df_
        s.g += dg_
        s.step(STEPS)
        return s.observe()["T_o"] + 2.0 * overlap_of(s.g)

    h = 1e-6
    for a, b, bar in ((np.zeros_like(df), dg, r["dg0"]), (df, np.zeros_like(dg), r["df0"])):
        fd = (J(h * a, h * b) - J(-h * a, -h * b)) / (2 * h)
        d = b if bar is r["dg0"] else a
        ad = float(np.sum(bar * d))
        mag = float(np.sum(np.abs(bar * d)))
        assert mag > 0
        assert abs(fd - ad) <= 1e-6 * mag + 1e-7 * abs(ad), (fd, ad, mag)


def test_cpu_adjoint_alpha_derivative_vanishes_by_symmetry(orc):
    """alpha = 0 with the droplet on the centre line: T_o(alpha) = T_o(-alpha)."""
    from oracle import torch_step as TS
    cfg = grad_cfg(alpha_deg=0.0, yc=9.5)
    sim = orc.Sim(cfg)
    r = TS.gradients(cfg, STEPS, sim.f.copy(), sim.g.copy(), 1.0, 0.0)
    other = max(abs(v) for v in r["grad"])
    assert other > 0
    assert abs(r["grad"][2]) <= 1e-12 * other


def test_torch_step_total_spreading_matches_the_oracle(orc):
    """eta > 0 with a negative spreading coefficient (sigma_13 = 3 sigma_12)."""
    from oracle import torch_step as TS
    cfg = grad_cfg(s13_over_s12=3.0, eta=0.02)
    sim = orc.Sim(cfg)
    f0, g0 = sim.f.copy(), sim.g.copy()
    theta = torch.tensor(TS.parameters_of(cfg), dtype=torch.float64)
    (To, _), (f, g) = TS.run(cfg, theta, STEPS, f0, g0)
    sim.step(STEPS)
    assert np.abs(g.numpy().reshape(sim.g.shape) - sim.g).max() <= 1e-13
    assert abs(float(To) - sim.observe()["T_o"]) <= 1e-12
