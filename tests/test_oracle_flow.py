"""Whole-step pins of the oracle (no GPU): analytic flows, interface equilibria,
conservation and symmetry (Secs. 2.2-2.5)."""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import curve_fit

from paper_2410_11129_gb300 import workloads as W

NO_DROP = dict(xc=0.0, yc=0.0, Bo_m=0.0, ferro="none")


def _single_phase(nx, ny, nu, u_max, **kw):
    cfg = W.channel(nx, ny, -1000.0, -1000.0, xi=4.0, u_max=u_max, **NO_DROP, **kw)
    cfg["nu"] = [nu, nu, nu]
    return cfg


def _poiseuille(ny, y, u_max):
    return u_max * 4 * (y + 0.5) * (ny - 0.5 - y) / ny ** 2


@pytest.mark.parametrize("nu", [1 / 8, 1 / 6, 0.1])
def test_poiseuille(orc, nu):
    """Body-force channel flow between half-way bounce-back walls (Eqs. 12-22).
    With the stress rate 1/(1/2 + tau) and every other rate 1 (Eq. 13) the
    two-rate bounce-back slip is the known uniform offset
    u_max (16 L - 3) / (3 ny^2), L = tau (1/s_q - 1/2) = tau/2: zero at tau = 3/8."""
    ny = 16
    s = orc.Sim(_single_phase(4, ny, nu, 0.01))
    s.step(12000)
    y = np.arange(ny)
    tau = 3 * nu
    slip = 0.01 * (16 * tau / 2 - 3) / (3 * ny ** 2)
    err = s.macro[0][:, 0] - _poiseuille(ny, y, 0.01)
    assert np.abs(err - slip).max() < 1e-10
    assert np.abs(s.macro[1]).max() < 1e-14


def test_layered_two_fluid_channel(orc):
    """Steady layered flow of two fluids (rho and nu ratio 2) driven by G solves
    d/dy(rho nu du/dy) = -G; the density-gradient forces F_p, F_mu of Eq. 19 and
    the viscosity mixing make the LBM match the quadrature of that ODE."""
    nx, ny, xi = 4, 48, 4.0
    cfg = W.channel(nx, ny, -1000.0, -1000.0, xi=xi, u_max=0.01, rho_r=2.0, nu_r=2.0,
                    sigma23=0.001, **NO_DROP)
    s = orc.Sim(cfg)
    y = np.arange(ny, dtype=float)
    y1, y2 = 14.0, 33.0
    band = lambda t: 0.5 * (np.tanh(2 * (t - y1) / xi) - np.tanh(2 * (t - y2) / xi))
    G9 = orc.gamma(0.0, 0.0)
    s.g[:] = 0.0
    for a in range(9):
        s.g[1, a] = band(y)[:, None] * G9[a]
    s.step(30000)
    d = s.derived()
    mu = lambda t: (1.0 - 0.5 * band(t)) * (d.tau[2] + (d.tau[1] - d.tau[2]) * band(t)) / 3.0
    yc = 0.5 * (ny - 1)
    ua = np.array([quad(lambda t: -d.G * (t - yc) / mu(t), -0.5, v, limit=200)[0] for v in y])
    assert np.abs(s.macro[0][:, 0] - ua).max() / ua.max() < 0.005


def test_flat_interface_equilibrium(orc):
    """A planar interface keeps the profile (1 + tanh(2x/xi))/2 of Eq. 23 (this
    fixes the scaling of the phase-field source term) and conserves mass."""
    nx, ny, xi = 64, 2, 4.0
    cfg = W.channel(nx, ny, -1000.0, -1000.0, xi=xi, u_max=0.0, sigma23=0.01, **NO_DROP)
    s = orc.Sim(cfg)
    x = np.arange(nx, dtype=float)
    prof = lambda t, w, c1, c2: 0.5 * (np.tanh(2 * (t - c1) / w) - np.tanh(2 * (t - c2) / w))
    phi0 = prof(x, xi, 16.0, 48.0)
    G9 = orc.gamma(0.0, 0.0)
    s.g[:] = 0.0
    for a in range(9):
        s.g[0, a] = phi0[None, :] * G9[a]
    m0 = s.phi()[0].sum()
    s.step(3000)
    p1 = s.phi()[0]
    assert abs(p1.sum() - m0) / m0 < 1e-12
    assert np.abs(p1[0] - phi0).max() < 0.01
    (w, c1, c2), _ = curve_fit(prof, x, p1[0], p0=[xi, 16.0, 48.0])
    assert abs(w / xi - 1) < 0.03
    assert abs(c1 - 16.0) < 1e-3 and abs(c2 - 48.0) < 1e-3


@pytest.mark.parametrize("pair", ["13", "23", "12"])
def test_laplace_law(orc, pair):
    """Static drop: pressure jump sigma_ij / R (2D) for each pair, with unequal
    sigma_12 = 0.005, sigma_13 = 0.0075, sigma_23 = 0.01 (Eqs. 25-28, 36).
    The lattice converges to the law as xi grows; at xi = 8 within 3%."""
    n, R, xi = 64, 16.0, 8.0
    kw = dict(xc=n / 2 - 0.5, yc=n / 2 - 0.5, xi=xi, Bo_m=0.0, ferro="none", u_max=0.0,
              sigma23=0.01, s13_over_s12=1.5, s23_over_s12=2.0)
    if pair == "13":
        cfg = W.channel(n, n, R, R, **kw)           # phase 1 in phase 3
    elif pair == "23":
        cfg = W.channel(n, n, -1000.0, R, **kw)     # phase 2 in phase 3
    else:
        cfg = W.channel(n, n, R, 1000.0, **kw)      # phase 1 in phase 2
    s = orc.Sim(cfg)
    s.step(3000)
    d = s.derived()
    i, j = int(pair[0]) - 1, int(pair[1]) - 1
    p = s.macro[2] / 3.0  # p = rho c_s^2 p*, rho = 1
    dp = p[n // 2, n // 2] - p[2, 2]
    assert abs(dp * R / d.sigma[i][j] - 1) < 0.03


@pytest.mark.parametrize("case,pair", [("complete engulfing-type 1", "13"),
                                       ("complete engulfing-type 2", "23")])
def test_laplace_law_total_spreading(orc, case, pair):
    """Table 2 total-spreading ratios: the absent phase has gamma < 0 and eta > 0
    (Eq. 28), yet a binary interface carries exactly sigma_ij, since the eta term
    and the absent phase's gradient term vanish where its phi is zero."""
    n, R, xi = 64, 16.0, 8.0
    kw = dict(nx=n, ny=n, xc=n / 2 - 0.5, yc=n / 2 - 0.5, xi=xi, Bo_m=0.0, ferro="none",
              u_max=0.0)
    if pair == "13":
        cfg = W.topology(case, 0.005, r1=R, r2=R, **kw)        # phase 1 in phase 3
    else:
        cfg = W.topology(case, 0.005, r1=-1000.0, r2=R, **kw)  # phase 2 in phase 3
    s = orc.Sim(cfg)
    d = s.derived()
    i, j = int(pair[0]) - 1, int(pair[1]) - 1
    assert min(d.gamma[k] for k in range(3)) < 0 and cfg["eta"] > 0
    s.step(3000)
    p = s.macro[2] / 3.0
    dp = p[n // 2, n // 2] - p[2, 2]
    assert abs(dp * R / d.sigma[i][j] - 1) < 0.03


def _drop_cfg(**kw):
    base = dict(nx=40, ny=20, r1=3.0, r2=6.0, xc=14.0, xi=4.0, Ca=0.1, Bo_m=2.0,
                ferro="shell", chi_ferro=1.0, mag_tol=1e-13, mag_max_iter=5000)
    base.update(kw)
    return W.small(**base)


def test_mass_conservation(orc):
    """Sum_a of the source term vanishes and sum_a g^eq = phi (Eqs. 29-32), and the
    walls bounce back, so each phase's mass is conserved to round-off."""
    for cfg in (_drop_cfg(), _drop_cfg(ferro="core", rho_r=2.0, nu_r=2.0, alpha=1.0)):
        s = orc.Sim(cfg)
        m0 = s.phi().reshape(3, -1).sum(1)
        s.step(150)
        m1 = s.phi().reshape(3, -1).sum(1)
        assert np.all(np.abs(m1 - m0) / np.abs(m0) < 1e-12)


@pytest.mark.parametrize("alpha_deg", [0.0, 90.0])
def test_mirror_symmetry(orc, alpha_deg):
    """A droplet on the centre line with the field along or across the channel
    keeps y -> ny-1-y mirror symmetry."""
    cfg = _drop_cfg(alpha=np.radians(alpha_deg), rho_r=2.0)
    s = orc.Sim(cfg)
    s.step(60)
    phi = s.phi()
    assert np.abs(phi - phi[:, ::-1]).max() < 1e-12
    assert np.abs(s.macro[0] - s.macro[0][::-1]).max() < 1e-12
    assert np.abs(s.macro[1] + s.macro[1][::-1]).max() < 1e-12


def test_translation_invariance(orc):
    """Periodic x: shifting the droplet shifts the solution."""
    a = orc.Sim(_drop_cfg())
    b = orc.Sim(_drop_cfg(xc=14.0 + 7))
    a.step(40)
    b.step(40)
    assert np.abs(np.roll(a.phi(), 7, axis=2) - b.phi()).max() < 1e-12
    assert np.abs(np.roll(a.macro[0], 7, axis=1) - b.macro[0]).max() < 1e-12


def test_kelvin_force_limits(orc):
    """Eq. 7: Bo_m = 0 gives F_m = 0; with only the core magnetic, F_m vanishes
    wherever grad phi_1 does (Sec. 3.1.1), here where phi_1 is identically 0."""
    cfg = _drop_cfg(Bo_m=0.0)
    s = orc.Sim(cfg)
    F = orc.forces(cfg, s.f, s.g, s.psi)
    assert np.all(F["Fm_x"] == 0) and np.all(F["Fm_y"] == 0)
    cfg = _drop_cfg(ferro="core", Bo_m=3.0, chi_ferro=2.0, xi=2.0)
    s = orc.Sim(cfg)
    phi = s.phi()
    ny, nx = phi.shape[1:]
    y, x = np.mgrid[0:ny, 0:nx]
    cut = np.hypot(x - cfg["xc"], y - cfg["yc"]) > cfg["r1"] + 2.0
    g = s.g.copy()
    g[0][:, cut] = 0.0  # compact core: phi_1 == 0 outside
    F = orc.forces(cfg, s.f, g, s.psi)
    ph1 = g[0].sum(0)
    zero = np.ones_like(cut)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            zero &= np.roll(np.roll(ph1, dy, 0), dx, 1) == 0
    zero[0] = zero[-1] = False
    assert zero.sum() > 100
    assert np.all(F["Fm_x"][zero] == 0) and np.all(F["Fm_y"][zero] == 0)
    assert np.abs(F["Fm_x"]).max() > 0


def test_kelvin_force_matches_permeability_gradient(orc):
    """Eq. 9 (analytic grad chi) against the isotropic gradient of the Eq. 8
    permeability field, for a smooth ferro core; and F_m points out of the drop
    (from high to low chi) where the field is tangential... here radially outward
    along the field axis."""
    cfg = _drop_cfg(ferro="core", Bo_m=3.0, chi_ferro=2.0, xi=6.0, r1=5.0, r2=8.0)
    s = orc.Sim(cfg)
    F = orc.forces(cfg, s.f, s.g, s.psi)
    phi, k = orc.phase(cfg, s.g)
    gx, gy = orc.grad(k)
    H2 = F["Hx"] ** 2 + F["Hy"] ** 2
    ref_x, ref_y = -0.5 * H2 * gx, -0.5 * H2 * gy
    scale = np.abs(ref_x).max()
    assert np.abs(F["Fm_x"] - ref_x).max() < 0.05 * scale
    assert np.abs(F["Fm_y"] - ref_y).max() < 0.05 * scale
    yc, xc = int(round(cfg["yc"])), int(cfg["xc"])
    assert F["Fm_x"][yc, xc + 5] > 0 and F["Fm_x"][yc, xc - 5] < 0


def test_oracle_threads_give_identical_bits(orc):
    """The row-parallel loops write disjoint outputs and the sums stay serial,
    so any thread count reproduces the single-thread run bit for bit."""
    from paper_2410_11129_gb300 import workloads as W
    cfg = W.small(nx=48, ny=20, r1=3.0, r2=6.0, xc=14.0, xi=4.0, Bo_m=2.0, mag_tol=1e-12)
    runs = []
    for n in (1, 4):
        orc.set_threads(n)
        sim = orc.Sim(cfg)
        sim.step(15)
        runs.append((sim.f.copy(), sim.g.copy(), sim.psi.copy()))
    orc.set_threads(1)
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def _open_poiseuille(orc, steps):
    nx, ny = 48, 12
    cfg = W.channel(nx, ny, -1000.0, -1000.0, xc=0.0, yc=0.0, xi=4.0, Bo_m=0.0, ferro="none",
                    u_max=0.01, open_x=1)
    cfg["nu"] = [1 / 8] * 3  # tau = 3/8: half-way bounce-back exact for the parabola
    orc.set_threads(orc.max_threads())
    try:
        s = orc.Sim(cfg)
        s.step(steps)
    finally:
        orc.set_threads(1)
    return s, nx, ny


def test_open_channel_poiseuille(orc):
    """Velocity inlet (Eq. 37) + convective outlet: the developed flow is the
    inlet parabola with the closed-form pressure gradient -G / c_s^2,
    G = 8 rho nu u_max / ny^2 (the body force of the periodic channel), the
    same flux through every column, and the outlet holds the reference p* = 0."""
    s, nx, ny = _open_poiseuille(orc, 12000)
    u, p = s.macro[0], s.macro[2]
    y = np.arange(ny)
    exact = 0.01 * 4 * (y + 0.5) * (ny - 0.5 - y) / ny**2
    inner = range(10, nx - 10)  # away from the entrance and exit layers
    assert max(np.abs(u[:, x] - exact).max() for x in inner) <= 1e-6 * exact.max()
    flux = u.sum(axis=0)
    assert np.abs(flux / exact.sum() - 1).max() <= 1e-9
    slope = np.polyfit(np.arange(nx // 4, 3 * nx // 4), p[ny // 2, nx // 4:3 * nx // 4], 1)[0]
    expect = -8 * (1 / 8) * 0.01 / ny**2 / (1 / 3)
    assert abs(slope / expect - 1) <= 1e-6
    assert abs(p[ny // 2, nx - 1]) <= 1e-6


def test_open_channel_drop_leaves_through_outlet(orc):
    """A drop advected through the convective outlet leaves completely (no
    reflection), and the inflow carries no phase 1."""
    nx, ny = 64, 16
    cfg = W.channel(nx, ny, 4.0, 4.0, xc=44.0, yc=7.5, xi=4.0, Bo_m=0.0, ferro="none",
                    u_max=0.05, Ca=0.1, open_x=1)
    orc.set_threads(orc.max_threads())
    try:
        s = orc.Sim(cfg)
        m0 = s.phi()[0].sum()
        s.step(3000)
    finally:
        orc.set_threads(1)
    ph = s.phi()[0]
    assert np.isfinite(s.f).all() and np.isfinite(s.g).all()
    assert abs(ph.sum()) <= 1e-9 * m0
    assert np.abs(ph).max() <= 1e-8
