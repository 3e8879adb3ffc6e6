"""GPU path against the FP64 oracle, element by element (needs a GB300).

Tolerances: FP64 storage and arithmetic match the oracle to 1e-10 (phase
fields absolute, velocity relative to its maximum) with both potential
solves at 1e-13; the FP32 forms match the FP64 oracle to 1e-4.
"""
import os

import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcd():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2410_11129_gb300 import fcd as F
    F.load()
    return F


def parity_cfg(**kw):
    base = dict(nx=48, ny=20, r1=3.0, r2=6.0, xc=14.0, xi=4.0, Ca=0.1, Bo_m=2.0,
                ferro="shell", chi_ferro=1.0, mag_tol=1e-13, mag_max_iter=300)
    base.update(kw)
    return W.small(**base)


def compare_fp64(orc, cfg, steps, tol=1e-10):
    from paper_2410_11129_gb300 import fcd as F
    sim = orc.Sim(cfg)
    ch = F.Channel(dict(cfg, precision="fp64"))
    sim.step(steps)
    ch.step(steps)
    f, g, psi = ch.populations()
    ux, uy = ch.field("ux"), ch.field("uy")
    phi = np.stack([ch.field("phi1"), ch.field("phi2")])
    ophi = sim.phi()[:2]
    umax = np.abs(sim.macro[:2]).max()
    err = {
        "phi": np.abs(phi - ophi).max(),
        "u_rel": max(np.abs(ux - sim.macro[0]).max(), np.abs(uy - sim.macro[1]).max()) / umax,
        "f": np.abs(f - sim.f).max(),
        "g": np.abs(g - sim.g).max(),
        "pstar": np.abs(ch.field("pstar") - sim.macro[2]).max(),
        "psi_rel": np.abs(psi - sim.psi).max() / max(np.abs(sim.psi).max(), 1e-300),
    }
    ob, oo = ch.observe(), sim.observe()
    ch.close()
    assert err["phi"] <= tol, err
    assert err["u_rel"] <= tol, err
    assert err["f"] <= tol and err["g"] <= tol and err["pstar"] <= tol, err
    assert err["psi_rel"] <= 1e-8 or np.abs(sim.psi).max() == 0, err
    for k in ("T_o", "T_i", "xc_core", "yc_core", "xc_shell", "yc_shell", "lx_o", "ly_o"):
        assert abs(ob[k] - oo[k]) <= 1e-8 * max(1.0, abs(oo[k])), (k, ob[k], oo[k])
    for i in range(3):
        assert abs(ob["mass"][i] - oo["mass"][i]) <= 1e-9 * abs(oo["mass"][i])
    assert ob["breakup"] == oo["breakup"] and ob["b_step"] == oo["b_step"]
    return err


@pytest.mark.parametrize("kw", [
    dict(),                                                           # shell ferro, alpha 0
    dict(ferro="core", chi_ferro=2.0, alpha=np.pi / 2, rho_r=2.0, nu_r=2.0, Ca=0.2, Bo_m=3.0),
    dict(nx=38, ny=13, xc=11.0, yc=6.3, alpha=0.6),                   # ragged tiles, odd ny, off-centre
    dict(nx=8, ny=6, r1=1.0, r2=2.0, xc=3.0, yc=2.5),                 # brute-force tiny grids
    dict(nx=12, ny=10, r1=2.0, r2=3.5, xc=5.0, yc=4.5, alpha=0.4),
])
def test_fp64_parity_small(orc, fcd, kw):
    compare_fp64(orc, parity_cfg(**kw), 120)


def test_fp64_parity_no_field_and_static(orc, fcd):
    compare_fp64(orc, parity_cfg(Bo_m=0.0), 60)
    compare_fp64(orc, parity_cfg(u_max=0.0, sigma23=0.01, Ca=0.0), 60)


def test_fp64_parity_minimal_grid(orc, fcd):
    compare_fp64(orc, parity_cfg(nx=4, ny=2, r1=-1000.0, r2=-1000.0, xc=0.0, yc=0.0,
                                 Bo_m=0.0, ferro="none"), 50)


def test_fp64_parity_200x40_channel(orc, fcd):
    """The 200x40 FP64 channel (shell ferrofluid, Ca 0.1, Bo_m 1) over its 1000
    steps, both solves at 1e-13."""
    cfg = dict(W.C1, mag_tol=1e-13, mag_max_iter=300)
    err = compare_fp64(orc, cfg, 1000)
    print("200x40 parity", err)


def test_solver_matches_oracle_and_layered_exact(orc, fcd):
    """fcd_solve_magnetic on a droplet state reaches the oracle's CG answer."""
    cfg = parity_cfg(ferro="core", chi_ferro=2.0, alpha=0.9, Bo_m=4.0)
    from paper_2410_11129_gb300 import fcd as F
    ch = F.Channel(dict(cfg, precision="fp64"))
    it, res, st = ch.solve_magnetic(1e-13, 300)
    assert st == F.FCD_OK and res <= 1e-13
    f, g, psi = ch.populations()
    phi, k = orc.phase(cfg, g)
    ref, st2, _, _ = orc.mag_solve(k, ch.derived()["H0"], cfg["alpha"], tol=1e-13)
    assert st2 == 0
    assert np.abs(psi - ref).max() <= 1e-10 * np.abs(ref).max()
    ch.close()


@pytest.mark.parametrize("kw", [
    dict(),                                                             # shell ferro
    dict(ferro="core", chi_ferro=2.0, alpha=0.7, rho_r=2.0, nu_r=2.0, Bo_m=3.0, xc=10.0),
])
def test_fp64_parity_open_channel(orc, fcd, kw):
    """Open channel: Eq. 37 inlet and convective outlet, droplet and field."""
    compare_fp64(orc, parity_cfg(open_x=1, **kw), 120)


def test_open_channel_poiseuille_gpu(fcd):
    """The open channel's developed flow on the GPU: the inlet parabola and the
    closed-form pressure gradient, as pinned on the oracle."""
    from paper_2410_11129_gb300 import fcd as F
    nx, ny = 48, 12
    cfg = W.channel(nx, ny, -1000.0, -1000.0, xc=0.0, yc=0.0, xi=4.0, Bo_m=0.0, ferro="none",
                    u_max=0.01, open_x=1)
    cfg["nu"] = [1 / 8] * 3
    ch = F.Channel(dict(cfg, precision="fp64"))
    ch.step(12000)
    u, p = ch.field("ux"), ch.field("pstar")
    ch.close()
    y = np.arange(ny)
    exact = 0.01 * 4 * (y + 0.5) * (ny - 0.5 - y) / ny**2
    assert max(np.abs(u[:, x] - exact).max() for x in range(10, nx - 10)) <= 1e-6 * exact.max()
    slope = np.polyfit(np.arange(nx // 4, 3 * nx // 4), p[ny // 2, nx // 4:3 * nx // 4], 1)[0]
    assert abs(slope / (-8 * (1 / 8) * 0.01 / ny**2 / (1 / 3)) - 1) <= 1e-6


@pytest.mark.parametrize("prec", ["fp32", "fp32_offset"])
@pytest.mark.parametrize("open_x", [0, 1])
def test_fp32_forms_against_fp64_oracle(orc, fcd, prec, open_x):
    """Both FP32 storage forms within 1e-4 of the FP64 oracle after 200 steps:
    phase fields absolute, velocity relative to its maximum, observables. The
    FP32 potential (hi + lo pair) is solved to 1e-6."""
    cfg = parity_cfg(mag_tol=1e-6, open_x=open_x)
    sim = orc.Sim(dict(cfg, mag_tol=1e-13))
    from paper_2410_11129_gb300 import fcd as F
    ch = F.Channel(dict(cfg, precision=prec))
    sim.step(200)
    ch.step(200)
    phi = np.stack([ch.field("phi1"), ch.field("phi2")])
    err_phi = np.abs(phi - sim.phi()[:2]).max()
    umax = np.abs(sim.macro[:2]).max()
    err_u = np.abs(ch.field("ux") - sim.macro[0]).max() / umax
    ob, oo = ch.observe(), sim.observe()
    print(prec, "phi", err_phi, "u_rel", err_u, {k: ob[k] - oo[k] for k in ("T_o", "T_i", "xc_shell")})
    assert err_phi <= 1e-4 and err_u <= 1e-4
    for k in ("T_o", "T_i", "xc_core", "yc_core", "xc_shell", "yc_shell"):
        assert abs(ob[k] - oo[k]) <= 1e-4 * max(1.0, abs(oo[k])), k
    ch.close()


def test_mass_conservation_gpu(fcd):
    """FP64: exact to round-off. The plain FP32 form rounds every stored
    population every step, with a bias that does not average out in a
    quasi-steady state (about 1e-5 over these 300 steps); the offset form's
    rest population takes each node's exact remainder, rounded without bias,
    which leaves a random walk of one rounding per node and step (5e-8 here)."""
    from paper_2410_11129_gb300 import fcd as F
    for prec, tol in (("fp64", 1e-12), ("fp32", 3e-5), ("fp32_offset", 3e-7)):
        ch = F.Channel(dict(parity_cfg(mag_tol=1e-6 if prec != "fp64" else 1e-10), precision=prec))
        m0 = np.array(ch.observe()["mass"])
        ch.step(300)
        m1 = np.array(ch.observe()["mass"])
        print(prec, "relative mass drift over 300 steps", (m1 - m0) / np.abs(m0))
        assert np.all(np.abs(m1 - m0) <= tol * np.abs(m0)), (prec, m1 - m0)
        ch.close()


@pytest.mark.parametrize("case", ["non-engulfing", "complete engulfing-type 1"])
def test_fp64_parity_total_spreading(orc, fcd, case):
    """Table 2 topologies with a negative spreading coefficient and eta > 0
    (Eqs. 27-28): the GPU path against the oracle, element by element."""
    cfg = W.topology(case, 0.005, nx=48, ny=20, r1=3.0, r2=6.0, xc=14.0, xi=4.0, Bo_m=2.0,
                     ferro="shell", chi_ferro=1.0, mag_tol=1e-13, mag_max_iter=300)
    compare_fp64(orc, cfg, 60)


def test_offset_form_conserves_phase_mass(fcd):
    """The FP32 offset form stores each node's rest population as the exact
    remainder of its pre-collision sum, rounded without bias, so its phase
    masses only random-walk by one rounding per node and step (measured 5e-8
    over these 5000 steps); the plain FP32 form, which rounds every stored
    population, drifts coherently (1.7e-4 on this channel)."""
    from paper_2410_11129_gb300 import fcd as F
    drift = {}
    for prec in ("fp32", "fp32_offset"):
        ch = F.Channel(dict(W.C2, precision=prec))
        m0 = np.array(ch.observe()["mass"][:2])
        ch.step(5000)
        m1 = np.array(ch.observe(allow=(F.FCD_ENOCONV,))["mass"][:2])
        ch.close()
        drift[prec] = np.abs(m1 - m0) / np.abs(m0)
    print("relative drift of phi_1, phi_2 over 5000 steps", drift)
    assert np.all(drift["fp32_offset"] <= 5e-7), drift
    assert np.all(drift["fp32_offset"] <= 0.01 * drift["fp32"]), drift


def test_checkpoint_resume_bitwise(fcd):
    from paper_2410_11129_gb300 import fcd as F
    for prec, tol in (("fp64", 1e-10), ("fp32_offset", 1e-4)):
        cfg = dict(parity_cfg(mag_tol=tol), precision=prec)
        a = F.Channel(cfg)
        a.step(30)
        snap = np.zeros(a.state_bytes(), np.uint8)
        a.get_state(snap)
        a.step(40)
        fa, ga, pa = a.populations()
        b = F.Channel(cfg)
        b.set_state(snap)
        b.step(40)
        fb, gb, pb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb) and np.array_equal(pa, pb)
        assert a.observe()["step"] == b.observe()["step"] == 70
        a.close()
        b.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp64", 1e-5), ("fp32", 1e-4),
                                      ("fp32", 1e-5), ("fp32_offset", 1e-5)])
def test_graph_and_host_loop_agree(fcd, monkeypatch, prec, tol):
    """The graph's cycle loop (the while form below a tolerance of 1e-5, the IF
    form from 1e-5 on) and the host-driven loop run the same kernels in the same
    order: bitwise the same state, and the same cycle counts, after 25 steps that
    include solves needing more than their first cycle head."""
    from paper_2410_11129_gb300 import fcd as F
    cfg = dict(parity_cfg(mag_tol=tol), precision=prec)
    a = F.Channel(cfg)
    s0 = a.solver_stats()
    a.step(25)
    sa = a.solver_stats()
    monkeypatch.setenv("FCD_NO_GRAPH", "1")
    b = F.Channel(cfg)
    t0 = b.solver_stats()
    b.step(25)
    sb = b.solver_stats()
    for x, y in zip(a.populations(), b.populations()):
        assert np.array_equal(x, y)
    assert {k: sa[k] - s0[k] for k in sa} == {k: sb[k] - t0[k] for k in sb}
    print(prec, tol, {k: sa[k] - s0[k] for k in sa})
    if tol <= 1e-5:
        assert sa["heads"] - s0["heads"] > 25  # some solve ran a cycle after its first head
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp32_offset"])
@pytest.mark.parametrize("open_x", [0, 1])
def test_collide_tile_heights_agree_bitwise(fcd, monkeypatch, prec, open_x):
    """The FP32 collide's two tile heights (4 and 8 rows) do the same arithmetic
    per node: the state after 60 steps is the same to the bit, so the height
    timed at create cannot change a result. 38 x 13 leaves ragged tiles in both
    directions for both heights."""
    from paper_2410_11129_gb300 import fcd as F
    cfg = dict(parity_cfg(nx=38, ny=13, xc=11.0, yc=6.3, alpha=0.6, mag_tol=1e-6, open_x=open_x),
               precision=prec)
    out = []
    for h in (4, 8):
        monkeypatch.setenv("FCD_COLLIDE_TILE_H", str(h))
        ch = F.Channel(cfg)
        assert ch.collide_tile_height() == h
        ch.step(60)
        out.append(ch.populations() + (ch.field("ux"), ch.field("pstar")))
        ch.close()
    for x, y in zip(*out):
        assert np.array_equal(x, y)
    monkeypatch.delenv("FCD_COLLIDE_TILE_H")
    ch = F.Channel(cfg)  # timed at create: one of the two
    assert ch.collide_tile_height() in (4, 8)
    ch.close()


def test_poiseuille_magic_parameter_gpu(fcd):
    """tau = 3/8 puts the half-way wall exactly: the parabola to round-off."""
    from paper_2410_11129_gb300 import fcd as F
    cfg = W.channel(8, 16, -1000.0, -1000.0, xc=0.0, yc=0.0, xi=4.0, Bo_m=0.0, ferro="none")
    cfg["nu"] = [1 / 8] * 3
    ch = F.Channel(dict(cfg, precision="fp64"))
    ch.step(12000)
    y = np.arange(16)
    exact = 0.01 * 4 * (y + 0.5) * (16 - 0.5 - y) / 256.0
    assert np.abs(ch.field("ux")[:, 3] - exact).max() < 1e-10
    ch.close()


def test_breakup_record_gpu(orc, fcd):
    """A thin shell touches at once: step 0 and the smallest (y, x), as the oracle."""
    cfg = parity_cfg(r1=4.0, r2=5.0, Bo_m=0.0, ferro="none")
    from paper_2410_11129_gb300 import fcd as F
    ch = F.Channel(dict(cfg, precision="fp64"))
    sim = orc.Sim(cfg)
    ch.step(3)
    sim.step(3)
    ob, oo = ch.observe(), sim.observe()
    assert ob["breakup"] == oo["breakup"] == 1
    assert (ob["b_step"], ob["xb"], ob["yb"]) == (oo["b_step"], oo["xb"], oo["yb"])
    ch.close()


def test_full_size_1600x200_fp32_sampled(orc, fcd):
    """The benchmark's 1600x200 FP32 channel in the same launch path: a few
    steps against the FP64 oracle on whole fields."""
    cfg = dict(W.C2)
    from paper_2410_11129_gb300 import fcd as F
    ch = F.Channel(cfg)
    sim = orc.Sim(dict(cfg, mag_tol=1e-10, mag_max_iter=20000))
    ch.step(3)
    sim.step(3)
    phi = np.stack([ch.field("phi1"), ch.field("phi2")])
    err_phi = np.abs(phi - sim.phi()[:2]).max()
    umax = np.abs(sim.macro[:2]).max()
    err_u = np.abs(ch.field("ux") - sim.macro[0]).max() / umax
    print("1600x200 FP32 after 3 steps: phi", err_phi, "u_rel", err_u)
    assert err_phi <= 1e-4 and err_u <= 1e-4
    ob = ch.observe()
    assert ob["mag_resid"] <= cfg["mag_tol"] and ob["mag_iters"] >= 0
    ch.close()


BATCH_CFGS = [
    dict(precision="fp32", mag_tol=1e-6),
    dict(precision="fp32_offset", nx=64, ny=24, xc=20.0, ferro="core", chi_ferro=2.0, mag_tol=1e-4),
    dict(precision="fp64", nx=38, ny=13, xc=11.0, yc=6.3, mag_tol=1e-10),
    dict(precision="fp32", nx=256, ny=64, r1=8.0, r2=16.0, xc=60.0, mag_tol=1e-6),
    dict(precision="fp32", Bo_m=0.0),
    dict(precision="fp32_offset", nx=96, ny=28, xc=30.0, alpha=0.5, mag_tol=1e-5),
]


def _batch_cfgs():
    out = []
    for kw in BATCH_CFGS:
        kw = dict(kw)
        prec = kw.pop("precision")
        out.append(dict(parity_cfg(**kw), precision=prec))
    return out


def _batch_vs_alone(F, mode, same, groups=3):
    """30 batch steps, then one instance stepped alone (its group falls out of
    phase and steps instance by instance) and 5 more batch steps; each
    instance against the same steps run alone: same(a, b) on every array."""
    cfgs = _batch_cfgs()
    b = F.Batch(cfgs)
    b.set_mode(mode)
    t = b.tuning()
    assert t["batched"] == 5 and t["groups"] == groups and all(h in (4, 8, 16) for h in t["tile_h"])
    b.step(30)
    got = [inst.populations() for inst in b.instances]
    obs = b.observe()
    b.instances[1].step(1)
    b.step(5)
    got2 = [inst.populations() for inst in b.instances]
    b.close()
    for k, (cfg, g1, ob, g2) in enumerate(zip(cfgs, got, obs, got2)):
        ch = F.Channel(cfg)
        ch.step(30)
        for x, y in zip(ch.populations(), g1):
            same(x, y, k)
        assert ob["step"] == 30
        ch.step(6 if k == 1 else 5)
        for x, y in zip(ch.populations(), g2):
            same(x, y, k)
        ch.close()


def test_batch_on_instance_streams_is_bitwise_alone(fcd):
    """Mode 0 (every instance's own graph on its own stream) is bit-identical
    to stepping each instance alone; the instances differ in size, physics
    and form."""
    from paper_2410_11129_gb300 import fcd as F

    def same(x, y, k):
        assert np.array_equal(x, y), k
    _batch_vs_alone(F, 0, same)


@pytest.mark.parametrize("split", [0, 2])
def test_batched_kernels_match_instances_alone(fcd, monkeypatch, split):
    """Mode 1 (one launch per kernel over a work list spanning the instances
    of a storage form, one multigrid loop for all, the 256 x 64 instance with
    a grid-wide coarse level) against each instance alone: the same arithmetic
    up to the fused multiply-adds of each compiled kernel variant, so equal to
    FP32 round-off (FP64 instances step alone: bitwise). Groups are per storage
    form and level-0 form of the potential (one FP32 plane below a tolerance of
    1e-4, else the hi + lo pair): three here; split = 2 puts each such set's
    instances into up to two groups on their own streams (four here)."""
    from paper_2410_11129_gb300 import fcd as F
    if split:
        monkeypatch.setenv("FCD_BATCH_GROUPS", str(split))

    def same(x, y, k):
        scale = max(np.abs(x).max(), 1e-30)
        assert np.abs(x - y).max() <= 1e-5 * scale, (k, np.abs(x - y).max(), scale)
        if k == 2:
            assert np.array_equal(x, y)
    _batch_vs_alone(F, 1, same, 4 if split else 3)


def test_batch_times_both_modes_then_keeps_one(fcd, monkeypatch):
    monkeypatch.delenv("FCD_BATCH_MODE", raising=False)
    from paper_2410_11129_gb300 import fcd as F
    b = F.Batch(_batch_cfgs()[:2])
    assert b.tuning()["mode"] == -1
    b.step(4)
    assert b.tuning()["mode"] == -1
    b.step(3)
    assert b.tuning()["mode"] in (0, 1)
    assert all(o["step"] == 7 for o in b.observe())
    b.close()


def test_batched_instances_against_fp64_oracle(orc, fcd):
    """Two batched FP32 instances of different sizes and physics (the larger
    with a grid-wide coarse multigrid level) against the FP64 oracle, after
    120 steps: phase fields and velocity within 1e-4, as the plain FP32 form."""
    from paper_2410_11129_gb300 import fcd as F
    cfgs = [parity_cfg(mag_tol=1e-6),
            parity_cfg(nx=256, ny=64, r1=8.0, r2=16.0, xc=60.0, ferro="core", chi_ferro=2.0,
                       alpha=np.pi / 2, mag_tol=1e-6)]
    b = F.Batch([dict(c, precision="fp32_offset") for c in cfgs])
    b.set_mode(1)
    assert b.tuning()["batched"] == 2
    b.step(120)
    orc.set_threads(orc.max_threads())
    try:
        for cfg, inst in zip(cfgs, b.instances):
            sim = orc.Sim(dict(cfg, mag_tol=1e-13))
            sim.step(120)
            phi = np.stack([inst.field("phi1"), inst.field("phi2")])
            err_phi = np.abs(phi - sim.phi()[:2]).max()
            umax = np.abs(sim.macro[:2]).max()
            err_u = max(np.abs(inst.field("ux") - sim.macro[0]).max(),
                        np.abs(inst.field("uy") - sim.macro[1]).max()) / umax
            print("batched", cfg["nx"], "x", cfg["ny"], "phi", err_phi, "u_rel", err_u)
            assert err_phi <= 1e-4 and err_u <= 1e-4
    finally:
        orc.set_threads(1)
        b.close()
