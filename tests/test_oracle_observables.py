"""Pins of the oracle's observables (Eq. 42, Eq. 38, breakup metrics of Sec. 2.5)
on constructed phase fields with known geometry (no GPU)."""
import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W


def _state_from_phi(orc, phi1, phi2):
    ny, nx = phi1.shape
    G9 = orc.gamma(0.0, 0.0)
    g = np.zeros((2, 9, ny, nx))
    for a in range(9):
        g[0, a] = phi1 * G9[a]
        g[1, a] = phi2 * G9[a]
    return g


def _observe(orc, cfg, g, step=0, track=None):
    p = orc.make_params(cfg)
    o = orc.Obs()
    import ctypes as C
    t = track or orc.Track(-1, 0, 0)
    orc.lib().orc_observe(C.byref(p), orc.oracle._p(np.ascontiguousarray(g)), C.byref(t), step,
                          C.byref(o))
    return o.as_dict()


def _ellipse(nx, ny, xc, yc, a, b, w=2.0):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    dx = (x - xc + nx / 2) % nx - nx / 2
    # signed distance scaled to the ellipse: zero level exactly on the ellipse
    s = np.hypot(dx / a, (y - yc) / b)
    return 0.5 * (1 - np.tanh(2 * (s - 1) * min(a, b) / w))


def test_deformation_index_of_ellipses(orc):
    """T = (l_y - l_x)/(l_y + l_x) of the 1/2-level sets of two ellipses (Eq. 42);
    extents read off the centre line and the widest column within interpolation
    error (about 0.05 node for these tanh profiles)."""
    nx, ny = 120, 41
    cfg = W.channel(nx, ny, 5, 10, u_max=0.01)
    outer = _ellipse(nx, ny, 40.0, 20.0, 16.0, 11.0)
    inner = _ellipse(nx, ny, 40.0, 20.0, 5.0, 8.0)
    o = _observe(orc, cfg, _state_from_phi(orc, inner, outer - inner))
    assert abs(o["lx_o"] - 32.0) < 0.1 and abs(o["ly_o"] - 22.0) < 0.1
    assert abs(o["lx_i"] - 10.0) < 0.1 and abs(o["ly_i"] - 16.0) < 0.1
    assert abs(o["T_o"] - (22 - 32) / 54.0) < 3e-3
    assert abs(o["T_i"] - (16 - 10) / 26.0) < 3e-3
    assert abs(o["xc_shell"] - 40.0) < 1e-9 and abs(o["yc_shell"] - 20.0) < 1e-9
    assert abs(o["xc_core"] - 40.0) < 1e-9 and abs(o["yc_core"] - 20.0) < 1e-9
    assert o["breakup"] == 0
    m = o["mass"]
    assert abs(m[0] - inner.sum()) < 1e-9 and abs(m[1] - (outer - inner).sum()) < 1e-9
    assert abs(sum(m) - nx * ny) < 1e-9


def test_droplet_across_periodic_seam(orc):
    """A droplet straddling x = 0 keeps its extents and its centroid (mod nx)."""
    nx, ny = 96, 40
    cfg = W.channel(nx, ny, 5, 10, u_max=0.01)
    outer = _ellipse(nx, ny, 2.0, 19.5, 12.0, 9.0)
    inner = _ellipse(nx, ny, 2.0, 19.5, 5.0, 4.0)
    o = _observe(orc, cfg, _state_from_phi(orc, inner, outer - inner))
    assert abs(o["lx_o"] - 24.0) < 0.1 and abs(o["ly_o"] - 18.0) < 0.1
    assert abs(o["xc_shell"] - 2.0) < 1e-9 and abs(o["xc_core"] - 2.0) < 1e-9


def test_breakup_detection_and_metrics(orc):
    """Breakup = the core touches the carrier (Sec. 2.5): first node in (y, x)
    order with phi_1 >= 1/2 next to phi_3 >= 1/2; t_b* by Eq. 38, L_b* = x/H,
    y_b* = distance from the centre line over H."""
    nx, ny = 64, 30
    cfg = W.channel(nx, ny, 5, 10, u_max=0.03)
    phi1 = np.zeros((ny, nx))
    phi2 = np.ones((ny, nx))
    phi2[:, :] = 1.0
    phi1[20:23, 30:34] = 1.0   # core block
    phi2[20:23, 30:34] = 0.0
    phi2[23, 31] = 0.0         # a carrier node right above the block (phi3 = 1)
    g = _state_from_phi(orc, phi1, phi2)
    o = _observe(orc, cfg, g, step=123)
    assert o["breakup"] == 1 and o["b_step"] == 123
    assert (o["xb"], o["yb"]) == (30.0, 22.0)   # (30,22) is diagonal to (31,23)
    u_avg = 2 * 0.03 / 3
    assert abs(o["tb_star"] - 123 * u_avg / 20.0) < 1e-15
    assert abs(o["Lb_star"] - 30 / 30.0) < 1e-15
    assert abs(o["yb_star"] - abs(22 - 14.5) / 30.0) < 1e-15
    phi2[23, 31] = 1.0
    o = _observe(orc, cfg, _state_from_phi(orc, phi1, phi2), step=5)
    assert o["breakup"] == 0


def test_breakup_is_sticky_through_steps(orc):
    """The step loop records the first step at which the touch is seen."""
    cfg = W.small(r1=4.0, r2=5.0, xi=4.0, Bo_m=0.0, ferro="none")
    s = orc.Sim(cfg)
    o = s.observe()
    assert o["breakup"] == 1 and o["b_step"] == 0   # a 1-node shell already touches
    s.step(3)
    o = s.observe()
    assert o["breakup"] == 1 and o["b_step"] == 0 and o["step"] == 3


def _run_history(orc, cfg, chunk, n):
    orc.set_threads(orc.max_threads())
    try:
        s = orc.Sim(cfg)
        out = []
        for _ in range(n):
            s.step(chunk)
            out.append(s.observe())
    finally:
        orc.set_threads(1)
    return out


@pytest.mark.parametrize("alpha_deg,sign", [(0.0, -1), (90.0, 1)])
def test_ferrofluid_drop_elongates_along_the_field(orc, alpha_deg, sign):
    """A ferrofluid drop at rest in a uniform field stretches along the field
    (the Kelvin force of Eq. 7 pulls hardest where the field crosses the
    interface): T = (l_y - l_x)/(l_y + l_x) < 0 for alpha = 0, > 0 for 90 deg."""
    n = 64
    cfg = W.channel(n, n, 12.0, 12.0, xc=n / 2 - 0.5, yc=n / 2 - 0.5, xi=4.0, Bo_m=3.0,
                    alpha_deg=alpha_deg, ferro="core", chi_ferro=2.0, u_max=0.0, sigma23=0.005,
                    Ca=0.0, mag_tol=1e-7)
    T = _run_history(orc, cfg, 1500, 1)[-1]["T_i"]
    assert sign * T > 0.05, T


def test_deformation_trends_of_the_paper(orc):
    """Sec. 3.1-3.2, on 200x40 channels before the shell breaks:
    - no field: the drag stretches the shell along the flow, T_o < 0;
    - shell ferrofluid, alpha = 0: field and drag both act along x, T_o falls
      further as Bo_m grows;
    - core ferrofluid, alpha = 0: the field stretches the core along x, T_i
      falls as Bo_m grows."""
    def cfg(ferro, bo):
        return W.channel(200, 40, 6, 12, xc=50, xi=4.0, Ca=0.1, Bo_m=bo, alpha_deg=0.0,
                         ferro=ferro, chi_ferro=1.0, mag_tol=1e-7)
    shell0, shell2 = (_run_history(orc, cfg("shell", b), 750, 2) for b in (0.0, 2.0))
    core0, core3 = (_run_history(orc, cfg("core", b), 750, 2) for b in (0.0, 3.0))
    assert shell0[-1]["T_o"] < 0
    assert all(b["T_o"] < a["T_o"] for a, b in zip(shell0, shell2))
    assert all(b["T_i"] < a["T_i"] for a, b in zip(core0, core3))
