"""Synthetic workloads shaped like the paper's channels (arXiv 2410.11129, Sec. 2.5-2.6).

Plain parameter dictionaries and the seeded draw of the batched sweep; no
arithmetic of the method lives here, so both the CUDA path and the CPU oracle
read their inputs from this one module. Per-phase values follow Eq. 39's
ratio convention: rho_r = rho1/rho2 = rho3/rho2 and nu_r = nu1/nu2 = nu3/nu2,
with the carrier at rho3 = 1, nu3 = 1/6 (tau3 = 1/2).
"""
import math

import numpy as np

NU3 = 1.0 / 6.0


def _phases(rho_r=1.0, nu_r=1.0):
    return {"rho": [1.0, 1.0 / rho_r, 1.0], "nu": [NU3, NU3 / nu_r, NU3]}


def channel(nx, ny, r1, r2, xc=None, yc=None, xi=5.0, rho_r=1.0, nu_r=1.0, Ca=0.15,
            Bo_m=0.0, alpha_deg=0.0, ferro="shell", chi_ferro=1.0, u_max=0.01,
            mag_tol=1e-10, mag_max_iter=200, s13_over_s12=1.0, s23_over_s12=1.0, **extra):
    """A compound droplet in a periodic, body-force-driven channel."""
    chi = [0.0, 0.0, 0.0]
    fp = 0
    if ferro == "core":
        chi[0], fp = chi_ferro, 1
    elif ferro == "shell":
        chi[1], fp = chi_ferro, 2
    cfg = {
        "nx": int(nx), "ny": int(ny), "r1": float(r1), "r2": float(r2),
        "xc": float(4 * r1 if xc is None else xc),
        "yc": float(0.5 * (ny - 1) if yc is None else yc),
        "xi": float(xi), "mobility": 0.3, "eta": 0.0, "chi": chi, "ferro_phase": fp,
        "Ca": float(Ca), "Bo_m": float(Bo_m), "alpha": math.radians(alpha_deg),
        "u_max": float(u_max), "mag_tol": float(mag_tol), "mag_max_iter": int(mag_max_iter),
        "s13_over_s12": float(s13_over_s12), "s23_over_s12": float(s23_over_s12),
        "sigma23": 0.0, "eps_n": 1e-12,
    }
    cfg.update(_phases(rho_r, nu_r))
    cfg.update(extra)
    return cfg


# 200x40 FP64 parity channel: shell ferrofluid (chi = 1), Ca 0.1, Bo_m 1, alpha 0.
C1 = dict(channel(200, 40, 6, 12, xc=50, xi=4.0, Ca=0.1, Bo_m=1.0, alpha_deg=0.0,
                  ferro="shell", chi_ferro=1.0), name="channel-200x40-fp64", steps=1000,
          precision="fp64")

# eps_n of the interface normal grad(phi) / (|grad(phi)| + eps_n) in the source
# of Eq. 23, on the production and precision-study channels: above the gradient
# rounding of either storage form (~1e-8 in FP32), so that the normal on the
# ridge of a thick shell (grad(phi_2) -> 0 with phi_2 near 1) does not turn
# with the rounding; the source term moves by at most eps_n.
EPS_N = 1e-4

# 1600x200 FP32 production channel: core ferrofluid (chi = 2), rho_r = nu_r = 2,
# Ca 0.2, Bo_m 3, alpha 90 deg; droplet centre 4 r1 from the inlet.
C2 = dict(channel(1600, 200, 30, 60, Ca=0.2, Bo_m=3.0, alpha_deg=90.0, ferro="core",
                  chi_ferro=2.0, rho_r=2.0, nu_r=2.0, mag_tol=1e-4, eps_n=EPS_N),
          name="channel-1600x200-fp32", steps=100000, precision="fp32")
# FP32 forms solve to 1e-4: psi' held in one FP32 plane carries ~6e-8 relative
# rounding, which floors ||L psi||_inf / H0 near 2e-5 on this channel (below
# 1e-4 the context keeps psi' as a hi + lo pair).

# 2400x300 precision-study channel: the 1600x200 case scaled by 1.5.
C3 = dict(channel(2400, 300, 45, 90, Ca=0.2, Bo_m=3.0, alpha_deg=90.0, ferro="core",
                  chi_ferro=2.0, rho_r=2.0, nu_r=2.0, mag_tol=1e-4, eps_n=EPS_N),
          name="channel-2400x300", steps=50000, precision="fp32")

# 800x100 gradient channel: shell ferrofluid, Ca 0.15, Bo_m 2, alpha 0.
# eps_n = 1e-6 (as in the FP32 forms): with 1e-12 the normal grad(phi)/|grad(phi)|
# of the bulk, where grad(phi) is round-off, has a Jacobian of order
# theta / eps_n ~ 100 per step, and the tangent of the step grows without bound.
C5 = dict(channel(800, 100, 15, 30, Ca=0.15, Bo_m=2.0, alpha_deg=0.0, ferro="shell", eps_n=1e-6),
          name="channel-800x100", steps=20000, checkpoint=500, precision="fp64")

# The paper's own channel (Sec. 2.6: H x L = 150 x 900, L = 6H) as an open channel
# (Eq. 37 inlet, convective outlet), with the parameters of its grid study (Fig. 4):
# shell ferrofluid, Ca 0.15, alpha 0, r2/r1 = 1.75, Bo_m 2. r2 = 0.3 H is an
# assumption (no radius is given); centre 4 r1 from the inlet (Sec. 2.5).
PAPER = dict(channel(900, 150, 45.0 / 1.75, 45.0, xc=4 * 45.0 / 1.75, Ca=0.15, Bo_m=2.0,
                     alpha_deg=0.0, ferro="shell", mag_tol=1e-4, open_x=1, eps_n=EPS_N),
             name="open-channel-900x150-fp32", steps=20000, precision="fp32")

# L2-busting roofline channel: the 1600x200 physics on 9600x1200 (droplet x6).
# The FP32 residual floor grows with the droplet (|psi'| ~ H0 r1): 1e-3 here.
ROOF = dict(channel(9600, 1200, 180, 360, Ca=0.2, Bo_m=3.0, alpha_deg=90.0, ferro="core",
                    chi_ferro=2.0, rho_r=2.0, nu_r=2.0, mag_tol=1e-3, eps_n=EPS_N),
            name="channel-9600x1200-fp32", steps=200, precision="fp32")


def regime_sweep(seed=12345, n_len_align=32):
    """96 instances: Bo_m x Ca x {core, shell}; lengths U[800, 2400] (rounded down
    to a multiple of n_len_align), height 200, r1/r2 U[0.3, 0.7] with r2 = 60."""
    rng = np.random.default_rng(seed)
    out = []
    for ferro in ("core", "shell"):
        for Bo in (0.0, 0.5, 1.0, 2.0, 4.0, 8.0):
            for Ca in (0.05, 0.1, 0.15, 0.2, 0.3, 0.4, 0.5, 0.6):
                L = int(rng.uniform(800, 2400)) // n_len_align * n_len_align
                rr = float(rng.uniform(0.3, 0.7))
                r2 = 60.0
                out.append(channel(L, 200, rr * r2, r2, xc=2 * r2 + 10, Ca=Ca, Bo_m=Bo,
                                   ferro=ferro, mag_tol=1e-4, eps_n=EPS_N))
    return out


# Table 2 surface-tension ratios (sigma23/sigma12, sigma13/sigma12); sigma23 is
# the one set by Ca (Eq. 40), so sigma12 = sigma23 / (sigma23/sigma12).
TABLE2 = {"non-engulfing": (0.30, 0.30), "complete engulfing-type 1": (0.50, 1.70),
          "partial engulfing": (1.0, 1.0), "complete engulfing-type 2": (1.70, 0.50)}


def topology(case, sigma23, eta_over_s12=1.0, **kw):
    """A channel with the Table 2 ratios of `case` and sigma23 given directly.
    Three of the four cases are total spreading (one gamma_i < 0), which needs
    eta > 0 in Eq. 28; eta = eta_over_s12 * sigma12 (the paper gives no value)."""
    r23, r13 = TABLE2[case]
    cfg = channel(**kw)
    cfg.update(sigma23=float(sigma23), s23_over_s12=r23, s13_over_s12=r13,
               eta=float(eta_over_s12) * sigma23 / r23)
    return cfg


def small(nx=48, ny=20, **kw):
    """Small droplet channel for parity tests: spans several tiles and a ragged tail."""
    base = dict(r1=3.0, r2=6.0, xc=14.0, xi=4.0, Ca=0.1, Bo_m=1.0, ferro="shell",
                chi_ferro=1.0)
    base.update(kw)
    return channel(nx, ny, **base)
