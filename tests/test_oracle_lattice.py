"""Pins of the oracle's node-level pieces against closed forms (no GPU).

Each test names the equation it pins; none re-types the oracle's formula: they
check moments, limits, library routines or finite differences instead.
"""
import math

import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W

CS2 = 1.0 / 3.0


def test_d2q9_velocities_and_weights(orc):
    """Eq. 20 (cos/sin construction) and Eq. 17, plus lattice isotropy."""
    w, ex, ey, _, _ = orc.tables()
    e = np.stack([ex, ey], 1).astype(float)
    assert np.all(e[0] == 0)
    for a in range(1, 5):
        ang = (a - 1) * math.pi / 2
        assert np.allclose(e[a], [math.cos(ang), math.sin(ang)], atol=1e-15)
    for a in range(5, 9):
        ang = (2 * a - 9) * math.pi / 4
        assert np.allclose(e[a], [math.sqrt(2) * math.cos(ang), math.sqrt(2) * math.sin(ang)],
                           atol=1e-12)
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ e, 0)
    assert np.allclose(np.einsum("a,ai,aj->ij", w, e, e), CS2 * np.eye(2))
    m4 = np.einsum("a,ai,aj,ak,al->ijkl", w, e, e, e, e)
    d = np.eye(2)
    iso = CS2 ** 2 * (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
                      + np.einsum("il,jk->ijkl", d, d))
    assert np.allclose(m4, iso)


def test_moment_matrix(orc):
    """Lallemand-Luo orthogonal basis (ref. [48]); inverse against numpy."""
    w, ex, ey, M, Mi = orc.tables()
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.allclose(np.diag(G), [9, 36, 36, 6, 12, 6, 12, 4, 4])
    assert np.allclose(M[0], 1) and np.allclose(M[3], ex) and np.allclose(M[5], ey)
    assert np.allclose(M[7], ex ** 2 - ey ** 2) and np.allclose(M[8], ex * ey)
    assert np.allclose(Mi, np.linalg.inv(M), atol=1e-14)


def test_mrt_relaxation(orc):
    """Eq. 12-13: with all rates equal the MRT operator is BGK; the stress moments
    relax at s_nu and every other moment at 1."""
    _, _, _, M, Mi = orc.tables()
    rng = np.random.default_rng(1)
    h = rng.normal(size=9)
    assert np.allclose(orc.mrt_apply(h, 1.0), h, atol=1e-14)
    for s in (0.4, 1.3, 1.9):
        m = M @ h
        want = Mi @ (np.r_[m[:7], s * m[7:]])
        assert np.allclose(orc.mrt_apply(h, s), want, atol=1e-14)
        assert np.allclose(orc.mrt_apply(M[7], s), s * M[7], atol=1e-14)
        assert np.allclose(orc.mrt_apply(M[4], s), M[4], atol=1e-14)


@pytest.mark.parametrize("ux,uy,ps", [(0.0, 0.0, 0.0), (0.03, -0.02, 0.004), (-0.05, 0.07, -0.01)])
def test_equilibrium_moments(orc, ux, uy, ps):
    """Eqs. 16-18: zeroth moment p*, first moment u, second p* c_s^2 I + u u.
    sum_a Gamma_a = 1 fixes the factor 2 of the u.u term in Eq. 18."""
    w, ex, ey, _, _ = orc.tables()
    e = np.stack([ex, ey], 1).astype(float)
    G = orc.gamma(ux, uy)
    assert abs(G.sum() - 1.0) < 1e-15
    f = orc.feq(ps, ux, uy)
    u = np.array([ux, uy])
    assert abs(f.sum() - ps) < 1e-15
    assert np.allclose(f @ e, u, atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj->ij", f, e, e), ps * CS2 * np.eye(2) + np.outer(u, u),
                       atol=1e-15)


def _poly_field(nx, ny, c):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    return (c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
            + c[6] * x ** 3 + c[7] * x * x * y + c[8] * y ** 3), x, y


def test_isotropic_stencils_polynomial_exactness(orc):
    """Eq. 34 is exact for quadratics and Eq. 35 for cubics (away from the walls
    and the seam); on x^3 the gradient carries the central-difference term
    (third derivative)/6 = 1."""
    rng = np.random.default_rng(2)
    c = rng.normal(size=9)
    a, x, y = _poly_field(24, 16, c)
    lp = orc.lap(a)
    ex_lp = 2 * c[3] + 2 * c[5] + 6 * c[6] * x + 2 * c[7] * y + 6 * c[8] * y
    s = (slice(1, -1), slice(1, -1))
    assert np.allclose(lp[s], ex_lp[s], atol=1e-9)
    q = c.copy()
    q[6:] = 0
    a, x, y = _poly_field(24, 16, q)
    gx, gy = orc.grad(a)
    assert np.allclose(gx[s], (q[1] + 2 * q[3] * x + q[4] * y)[s], atol=1e-10)
    assert np.allclose(gy[s], (q[2] + q[4] * x + 2 * q[5] * y)[s], atol=1e-10)
    gx, _ = orc.grad(x ** 3)
    assert np.allclose(gx[s], (3 * x * x + 1)[s], atol=1e-10)


def test_stencil_boundaries(orc):
    """Periodic seam in x; mirrored ghost rows at the half-way walls."""
    ny, nx = 6, 10
    x = np.arange(nx)
    a = np.tile(np.sin(2 * np.pi * x / nx), (ny, 1))
    gx, gy = orc.grad(a)
    lp = orc.lap(a)
    k = 2 * np.pi / nx
    # the 1D stencil of a pure x-mode: (a_E - a_W)/2 and a_E + a_W - 2a
    assert np.allclose(gx, np.cos(k * x) * np.sin(k), atol=1e-14)
    assert np.allclose(gy, 0, atol=1e-15)
    assert np.allclose(lp, np.sin(k * x) * (2 * np.cos(k) - 2), atol=1e-14)
    b = np.tile(np.arange(ny, dtype=float)[:, None] ** 2, (1, nx))
    gx, gy = orc.grad(b)
    assert np.allclose(gy[0], (b[1, 0] - b[0, 0]) / 2)  # mirror: b(-1) = b(0)
    assert np.allclose(gy[-1], (b[-1, 0] - b[-2, 0]) / 2)


def _cfg(**kw):
    c = W.channel(16, 8, 3, 5, sigma23=0.013, s13_over_s12=1.3, s23_over_s12=0.9, xi=4.0)
    c.update(kw)
    return c


def test_free_energy_derivatives(orc):
    """Eq. 28 partial derivatives against central finite differences."""
    cfg = _cfg(eta=0.7)
    rng = np.random.default_rng(3)
    for _ in range(5):
        ph = rng.uniform(-0.1, 1.1, 3)
        d = orc.dH(cfg, ph)
        h = 1e-6
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            fd = (orc.free_energy(cfg, ph + e) - orc.free_energy(cfg, ph - e)) / (2 * h)
            assert abs(fd - d[i]) < 1e-8


def test_spreading_coefficients(orc):
    """Eqs. 26-27 and the Eq. 40 surface tension."""
    cfg = W.channel(16, 8, 3, 5, Ca=0.2, u_max=0.03, s13_over_s12=1.3, s23_over_s12=0.9)
    d = orc.derive(cfg)
    s23 = 1.0 * (1 / 6) * 0.02 / 0.2
    s12 = s23 / 0.9
    s13 = 1.3 * s12
    assert abs(d.sigma[1][2] - s23) < 1e-15
    g = [d.gamma[i] for i in range(3)]
    # each sigma_ij is recovered as (gamma_i + gamma_j)/2
    assert abs((g[0] + g[1]) / 2 - s12) < 1e-15
    assert abs((g[0] + g[2]) / 2 - s13) < 1e-15
    assert abs((g[1] + g[2]) / 2 - s23) < 1e-15
    assert abs(3 / d.gammaT - sum(1 / x for x in g)) < 1e-9
    assert abs(d.tau_phi - 0.9) < 1e-15  # M = 0.3, c_s^2 = 1/3


@pytest.mark.parametrize("phi", [0.1, 0.37, 0.5, 0.82])
def test_chemical_potential_binary_limit(orc, phi):
    """Eq. 25 with phi_2 = 0 reduces to the two-phase model with
    beta = 12 sigma13 / xi, kappa = 3 sigma13 xi / 2."""
    cfg = _cfg()
    d = orc.derive(cfg)
    s13, xi = d.sigma[0][2], cfg["xi"]
    lap1 = 0.013
    mu = orc.chem(cfg, [phi, 0.0, 1 - phi], [lap1, 0.0, -lap1])
    binary = 24 * s13 / xi * phi * (1 - phi) * (1 - 2 * phi) - 1.5 * s13 * xi * lap1
    assert abs((mu[0] - mu[2]) - binary) < 1e-15


def test_phase_recovery_and_permeability(orc):
    """Eqs. 32, 24 and 8 (harmonic mixing of 1 + chi)."""
    cfg = W.channel(4, 3, 1, 2, ferro="shell", chi_ferro=1.5)
    cfg["chi"] = [0.5, 1.5, 0.0]
    rng = np.random.default_rng(4)
    p1 = rng.uniform(0, 1, (3, 4))
    p2 = rng.uniform(0, 1 - p1)
    g = np.zeros((2, 9, 3, 4))
    wts = rng.dirichlet(np.ones(9))
    for a in range(9):
        g[0, a] = p1 * wts[a]
        g[1, a] = p2 * wts[8 - a] if a != 4 else p2 * wts[4]
    g[1] *= (p2 / g[1].sum(0))
    phi, k = orc.phase(cfg, g.ravel())
    assert np.allclose(phi[0], p1) and np.allclose(phi[1], p2)
    assert np.allclose(phi[2], 1 - p1 - p2)
    assert np.allclose(k, 1 / (p1 / 1.5 + p2 / 2.5 + (1 - p1 - p2)))
