"""Pins of the oracle's magnetic-potential discretisation and solver (no GPU).

Sec. 2.1, Eqs. 5-9: the potential equation div[(1+chi) grad psi] = 0 with
psi = psi0 + psi', psi0 = -H0 (x cos(alpha) + y sin(alpha)).
"""
import math

import numpy as np
import scipy.linalg

from paper_2410_11129_gb300 import workloads as W


def _assemble(orc, k):
    ny, nx = k.shape
    N = nx * ny
    A = np.zeros((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[:] = 0
        e[j] = 1
        A[:, j] = orc.mag_apply(k, e.reshape(ny, nx), 0.0, 0.0).ravel()
    return A


def _smooth_k(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    k = 1.5 + 0.4 * np.sin(2 * np.pi * x / nx + rng.uniform(0, 6)) * np.cos(0.3 * y + rng.uniform())
    return k


def test_operator_closed_forms(orc):
    """Uniform k: L = k * (Eq. 35 Laplacian), exact on quadratics; k linear in x
    and psi' linear in x: div(k grad psi') = dk/dx * dpsi'/dx exactly."""
    ny, nx = 12, 16
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    k = np.full((ny, nx), 1.7)
    a, b, c = 0.3, -0.2, 0.45
    psi = a * x * x + b * x * y + c * y * y
    out = orc.mag_apply(k, psi, 0.0, 0.0)
    s = (slice(1, -1), slice(1, -1))
    assert np.allclose(out[s], 2 * 1.7 * (a + c), atol=1e-11)
    k2 = 1.0 + 0.05 * x
    out = orc.mag_apply(k2, 0.7 * x, 0.0, 0.0)
    assert np.allclose(out[s], 0.05 * 0.7, atol=1e-12)


def test_operator_symmetric_negative_definite(orc):
    k = _smooth_k(8, 6, 0)
    A = _assemble(orc, k)
    assert np.allclose(A, A.T, atol=1e-14)
    assert np.linalg.eigvalsh(A).max() < 0


def test_uniform_medium_is_undisturbed(orc):
    """No permeability contrast: psi = psi0, i.e. H = H0 everywhere."""
    k = np.full((10, 14), 2.0)
    for al in (0.0, 0.7, math.pi / 2):
        b = orc.mag_rhs(k, 0.1, al)
        assert np.abs(b).max() < 1e-16
        psi, st, it, res = orc.mag_solve(k, 0.1, al)
        assert st == 0 and np.abs(psi).max() < 1e-15


def test_field_along_layers_is_undisturbed(orc):
    """Layers k(y) with the field along x: tangential H is continuous, psi' = 0."""
    ny, nx = 20, 8
    k = np.tile(1.0 + 0.5 * np.tanh(np.arange(ny) - 9.5)[:, None] + 0.5, (1, nx))
    assert np.abs(orc.mag_rhs(k, 0.2, 0.0)).max() < 1e-16


def test_layered_medium_exact_1d(orc):
    """Field across layers k(y) (alpha = 90 deg): the 9-point operator collapses to
    the 3-point conservative scheme with link coefficient (k_j + k_j+1)/2 (the
    diagonal and axial weights add to 1/6 per link); psi' = 0 on the wall faces."""
    ny, nx, H0 = 30, 6, 0.3
    yy = np.arange(ny)
    kk = 1.0 + 1.0 / (1 + np.exp(-(yy - 12.0))) - 0.6 / (1 + np.exp(-(yy - 21.0)))
    k = np.tile(kk[:, None], (1, nx))
    psi, st, it, res = orc.mag_solve(k, H0, math.pi / 2, tol=1e-14)
    assert st == 0
    # tridiagonal solve of  cN (p_j+1 - p_j - H0) + cS (p_j-1 - p_j + H0) = 0
    kN = 0.5 * (kk + np.r_[kk[1:], kk[-1]])
    kS = 0.5 * (kk + np.r_[kk[0], kk[:-1]])
    diag = -(kN + kS)
    diag[0] -= kS[0]      # ghost psi'(-1) = -psi'(0)
    diag[-1] -= kN[-1]    # ghost psi'(ny) = -psi'(ny-1)
    ab = np.zeros((3, ny))
    ab[0, 1:] = kN[:-1]
    ab[1] = diag
    ab[2, :-1] = kS[1:]
    rhs = H0 * (kN - kS)
    exact = scipy.linalg.solve_banded((1, 1), ab, rhs)
    assert np.abs(psi - exact[:, None]).max() < 1e-12


def test_dense_direct_solve_tiny(orc):
    """Conjugate gradients reach the dense Gaussian-elimination answer."""
    for (nx, ny, al) in ((12, 10, 0.0), (9, 7, 1.1)):
        k = _smooth_k(nx, ny, nx)
        A = _assemble(orc, k)
        b = orc.mag_rhs(k, 0.08, al).ravel()
        exact = np.linalg.solve(A, b).reshape(ny, nx)
        psi, st, it, res = orc.mag_solve(k, 0.08, al, tol=1e-14)
        assert st == 0 and res <= 1e-14
        assert np.abs(psi - exact).max() < 1e-12


def test_permeable_cylinder_interior_field(orc):
    """A cylinder of susceptibility chi in a uniform field H0 carries the uniform
    interior field 2 H0 / (2 + chi) (sharp-interface closed form); the diffuse
    interface and the walls make the lattice value converge as R grows."""
    n, R, xi = 256, 16.0, 2.0
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - (n / 2 - 0.5), y - (n / 2 - 0.5))
    phi = 0.5 * (1 - np.tanh(2 * (r - R) / xi))
    for chi, tol in ((1.0, 0.02), (2.0, 0.035)):
        k = 1.0 / (phi / (1 + chi) + (1 - phi))  # Eq. 8 with chi_out = 0
        H0 = 0.05
        psi, st, it, res = orc.mag_solve(k, H0, 0.0, tol=1e-10)
        assert st == 0
        gx, gy = orc.grad(psi)
        c = n // 2
        Hin = (H0 - gx[c - 1:c + 1, c - 1:c + 1]).mean()
        want = 2 * H0 / (2 + chi)
        assert abs(Hin / want - 1) < tol
        assert np.abs(gy[c - 1:c + 1, c - 1:c + 1]).max() < 1e-6 * H0


def test_phase_field_permeability_is_harmonic(orc):
    """Eq. 8 through orc_phase on a real droplet state: pure phases give 1 + chi_i."""
    cfg = W.small(chi_ferro=2.0, ferro="core", r1=6.0, r2=9.0, xi=1.0, ny=24)
    s = orc.Sim(cfg)
    phi, k = orc.phase(cfg, s.g)
    core = phi[0] > 0.999999
    far = phi[2] > 0.999999
    assert core.any() and far.any()
    assert np.allclose(k[core], 3.0, atol=1e-5) and np.allclose(k[far], 1.0, atol=1e-5)
