"""Tangent-linear (forward-mode) derivatives of the coupled step (needs a GB300).

The derivatives of the shell deformation T_o (Eq. 42) and of the core-carrier
overlap sum phi_1 phi_3 along (Bo_m, Ca, alpha, nu_r) are checked against
(1) Richardson-extrapolated central differences of the FP64 CPU oracle,
(2) central differences of the plain FP64 GPU path, and (3) the exact zero of
dT_o/dalpha at alpha = 0 for a droplet on the centre line (mirror symmetry:
T_o(alpha) = T_o(-alpha)). The primal part of a tangent context reproduces the
plain FP64 context.
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
    """sum over nodes of phi_1 phi_3, phi_3 = 1 - phi_1 - phi_2."""
    return float(np.sum(phi1 * (1.0 - phi1 - phi2)))


def richardson(fun, theta, j, rel=1e-3):
    """(4 D(h/2) - D(h)) / 3 with D(h) the central difference along theta_j."""
    h = rel * max(abs(theta[j]), 1.0)

    def D(hh):
        tp, tm = list(theta), list(theta)
        tp[j] += hh
        tm[j] -= hh
        fp, fm = fun(tp), fun(tm)
        return (fp - fm) / (2 * hh)

    return (4 * D(h / 2) - D(h)) / 3


def tangent_run(F, cfg, steps):
    ch = F.Tangent(cfg)
    ch.step(steps)
    o = ch.tangent_observe()
    plain_obs = ch.observe()
    fields = {k: ch.field(k) for k in ("phi1", "phi2", "ux", "uy", "psi")}
    ch.close()
    return o, plain_obs, fields


@pytest.mark.parametrize("open_x", [0, 1])
def test_tangent_primal_matches_plain(fcd, open_x):
    cfg = grad_cfg(open_x=open_x)
    o, ob, fields = tangent_run(fcd, cfg, STEPS)
    ch = fcd.Channel(cfg)
    ch.step(STEPS)
    ref = ch.observe()
    for k in ("phi1", "phi2", "ux", "uy", "psi"):
        r = ch.field(k)
        scale = max(np.abs(r).max(), 1e-300)
        assert np.abs(fields[k] - r).max() <= 1e-12 * max(scale, 1.0), k
    ch.close()
    for k in ("T_o", "lx_o", "ly_o"):
        assert abs(ob[k] - ref[k]) <= 1e-12, (k, ob[k], ref[k])
    assert abs(o["T_o"] - ref["T_o"]) <= 1e-12
    phi1, phi2 = fields["phi1"], fields["phi2"]
    assert abs(o["overlap"] - overlap_of(phi1, phi2)) <= 1e-10 * max(1.0, o["overlap"])


@pytest.mark.parametrize("open_x", [0, 1])
def test_tangent_against_oracle_differences(fcd, orc, open_x):
    """Forward-mode derivatives vs Richardson central differences of the oracle,
    in the periodic and in the open channel."""
    cfg = grad_cfg(open_x=open_x)
    theta = list(fcd.parameters_of(cfg))
    o, _, _ = tangent_run(fcd, cfg, STEPS)

    def run(th):
        sim = orc.Sim(fcd.with_parameters(cfg, th))
        sim.step(STEPS)
        ob = sim.observe()
        phi = sim.phi()
        return np.array([ob["T_o"], overlap_of(phi[0], phi[1])])

    fd = np.array([richardson(run, theta, j) for j in range(4)])  # 4 x 2
    tan = np.array([o["dT_o"], o["doverlap"]]).T
    for q, name in enumerate(("T_o", "overlap")):
        scale = np.abs(fd[:, q]).max()
        err = np.abs(tan[:, q] - fd[:, q]).max()
        assert scale > 0, name
        assert err <= 1e-5 * scale, (name, tan[:, q], fd[:, q])


def test_tangent_against_gpu_differences_and_autograd(fcd):
    """Forward-mode derivatives vs central differences of the plain FP64 GPU path,
    and the torch.autograd wrapper returning the same gradient."""
    import torch
    cfg = grad_cfg(Ca=0.12, Bo_m=1.5, alpha_deg=20.0, nu_r=0.8)
    theta = list(fcd.parameters_of(cfg))
    o, _, _ = tangent_run(fcd, cfg, STEPS)

    def run(th):
        ch = fcd.Channel(fcd.with_parameters(cfg, th))
        ch.step(STEPS)
        ob = ch.observe()
        val = np.array([ob["T_o"], overlap_of(ch.field("phi1"), ch.field("phi2"))])
        ch.close()
        return val

    fd = np.array([richardson(run, theta, j) for j in range(4)])
    tan = np.array([o["dT_o"], o["doverlap"]]).T
    for q, name in enumerate(("T_o", "overlap")):
        scale = np.abs(fd[:, q]).max()
        assert np.abs(tan[:, q] - fd[:, q]).max() <= 1e-5 * scale, (name, tan[:, q], fd[:, q])

    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    out = fcd.droplet_observables(th, cfg, STEPS)
    (out[0] + 2.0 * out[1]).backward()
    expect = np.array(o["dT_o"]) + 2.0 * np.array(o["doverlap"])
    assert np.allclose(th.grad.numpy(), expect, rtol=1e-12, atol=0.0)
    assert abs(out[0].item() - o["T_o"]) <= 1e-14


def test_alpha_derivative_vanishes_by_symmetry(fcd):
    """alpha = 0 with the droplet on the centre line: the state is mirror
    symmetric and T_o(alpha) = T_o(-alpha), so dT_o/dalpha = 0 exactly."""
    cfg = grad_cfg(alpha_deg=0.0, yc=9.5)
    o, _, _ = tangent_run(fcd, cfg, STEPS)
    other = max(abs(v) for v in o["dT_o"])
    assert other > 0
    assert abs(o["dT_o"][fcd.DIRECTIONS.index("alpha")]) <= 1e-12 * other
    oth = max(abs(v) for v in o["doverlap"])
    assert abs(o["doverlap"][fcd.DIRECTIONS.index("alpha")]) <= 1e-12 * oth


def test_tangent_rejects_bad_input(fcd):
    with pytest.raises(fcd.FcdError):
        fcd.Tangent(grad_cfg(Bo_m=0.0))
    ch = fcd.Tangent(grad_cfg())
    with pytest.raises(fcd.FcdError):
        ch.get_state(np.zeros(16, np.uint8))
    ch.close()


def test_tangent_graph_and_host_loop_agree(fcd, monkeypatch):
    """The captured tangent step (five solve loops as graph while nodes) and
    the host-driven loop give the same bits."""
    cfg = grad_cfg(mag_tol=1e-10)
    a = fcd.Tangent(cfg)
    a.step(20)
    oa = a.tangent_observe()
    monkeypatch.setenv("FCD_NO_GRAPH", "1")
    b = fcd.Tangent(cfg)
    b.step(20)
    ob = b.tangent_observe()
    for x, y in zip(a.populations(), b.populations()):
        assert np.array_equal(x, y)
    assert oa == ob
    a.close()
    b.close()
