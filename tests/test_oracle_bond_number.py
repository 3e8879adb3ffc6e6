"""Pins of the magnetic Bond number mapping (Sec. 2.5, Eq. 41), CPU only.

Eq. 41 defines Bo_m through mu0 H0^2, so the oracle inverts it for H0. The
pin measures mu0 H0^2 physically instead of reading it back: across a flat
layer of ferrofluid lying along a uniform field (alpha = 0) the tangential H is
continuous (psi' = 0 exactly), and the Kelvin force of Eq. 7 integrated
through one interface is the magnetic traction (1/2) mu0 chi H0^2. With that
traction, the paper's printed form of Eq. 41 gives Bo_m back:

  core  (inner droplet ferrofluid):  Bo_m = traction r1 / sigma12
  shell (outer droplet ferrofluid):  Bo_m = traction (r2^2 - r1^2) / (sigma12 r1 + sigma23 r2)

The cases use sigma12 != sigma23 and r1 != r2 (r2 = 3 r1), so a swapped radius
or surface tension, or a lost factor 2, misses by 29% or more; the sigma_ij
themselves are pinned by the Laplace law (test_oracle_flow.py). The library's
own mapping (fcd_derive_params, host code) must equal the oracle's.
"""
import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W

CASES = {
    "core": dict(ferro="core", chi_ferro=0.5, r1=4.0, r2=12.0, Bo_m=2.5),
    "shell": dict(ferro="shell", chi_ferro=0.7, r1=3.0, r2=9.0, Bo_m=1.5),
}


def _cfg(case):
    kw = dict(CASES[case])
    return W.channel(4, 96, kw.pop("r1"), kw.pop("r2"), xc=2.0, xi=8.0, Ca=0.12,
                     s23_over_s12=0.6, s13_over_s12=1.3, **kw)


def _traction(orc, cfg):
    """-sum_y F_m,y through the lower interface of a flat ferrofluid layer (rows
    30-65, width 8) with the field along x; psi' is the exact solution 0."""
    phase = cfg["ferro_phase"] - 1
    ny, nx = cfg["ny"], cfg["nx"]
    y = np.arange(ny, dtype=float)
    layer = 0.5 * (np.tanh(2 * (y - 30) / cfg["xi"]) - np.tanh(2 * (y - 65) / cfg["xi"]))
    G9 = orc.gamma(0.0, 0.0)
    f = np.zeros((9, ny, nx))
    g = np.zeros((2, 9, ny, nx))
    for a in range(9):
        g[phase, a] = layer[:, None] * G9[a]
    phi, k = orc.phase(cfg, g)
    d = orc.derive(cfg)
    assert np.abs(orc.mag_rhs(k, d.H0, cfg["alpha"])).max() < 1e-14 * d.H0
    F = orc.forces(cfg, f, g, np.zeros((ny, nx)))
    assert np.abs(F["Hx"] - d.H0).max() < 1e-14 and np.abs(F["Hy"]).max() < 1e-14
    return -F["Fm_y"][: ny // 2, 0].sum(), d


@pytest.mark.parametrize("case", sorted(CASES))
def test_bond_number_from_magnetic_traction(orc, case):
    cfg = _cfg(case)
    traction, d = _traction(orc, cfg)
    chi = cfg["chi"][cfg["ferro_phase"] - 1]
    # the layer's traction is (1/2) chi mu0 H0^2 up to the stencils' error (< 1%)
    assert abs(traction / (0.5 * chi * d.mu0H0sq) - 1) < 0.01
    s12, s23 = d.sigma[0][1], d.sigma[1][2]
    assert abs(s12 / s23 - 1 / 0.6) < 1e-12  # unequal surface tensions
    r1, r2 = cfg["r1"], cfg["r2"]
    if case == "core":
        bo = traction * r1 / s12
    else:
        bo = traction * (r2 * r2 - r1 * r1) / (s12 * r1 + s23 * r2)
    assert abs(bo / cfg["Bo_m"] - 1) < 0.01, (case, bo, cfg["Bo_m"])


@pytest.mark.parametrize("case", sorted(CASES))
def test_bond_number_scaling(orc, case):
    """mu0 H0^2 is linear in Bo_m and in 1/chi (Eq. 41, both branches)."""
    cfg = _cfg(case)
    m = orc.derive(cfg).mu0H0sq
    assert abs(orc.derive(dict(cfg, Bo_m=3 * cfg["Bo_m"])).mu0H0sq / m - 3) < 1e-13
    chi = list(cfg["chi"])
    chi[cfg["ferro_phase"] - 1] *= 2
    assert abs(orc.derive(dict(cfg, chi=chi)).mu0H0sq / m - 0.5) < 1e-13
    assert orc.derive(dict(cfg, Bo_m=0.0)).H0 == 0.0


@pytest.mark.parametrize("case", sorted(CASES) + ["none"])
def test_library_mapping_equals_the_oracle(orc, case):
    """fcd_derive_params (the mapping fcd_create uses, host code only) against
    the oracle's, every derived quantity."""
    from paper_2410_11129_gb300 import fcd
    cfg = _cfg(case) if case != "none" else W.small(Bo_m=0.0, ferro="none")
    lib = fcd.derive_params(cfg)
    d = orc.derive(cfg)
    ref = {"u_avg": d.u_avg, "sigma12": d.sigma[0][1], "sigma13": d.sigma[0][2],
           "sigma23": d.sigma[1][2], "gammaT": d.gammaT, "tau_phi": d.tau_phi,
           "mu0H0sq": d.mu0H0sq, "H0": d.H0, "G": d.G}
    for i in range(3):
        ref["gamma%d" % (i + 1)] = d.gamma[i]
        ref["tau%d" % (i + 1)] = d.tau[i]
    for k, v in ref.items():
        assert abs(lib[k] - v) <= 1e-14 * max(1.0, abs(v)), (k, lib[k], v)


def test_library_mapping_rejects_what_create_rejects():
    from paper_2410_11129_gb300 import fcd
    with pytest.raises(fcd.FcdError) as e:
        fcd.derive_params(dict(W.small(), r1=9.0, r2=6.0))
    assert e.value.status == fcd.FCD_EINVAL
    assert "fcd_derive_params:" in str(e.value)
