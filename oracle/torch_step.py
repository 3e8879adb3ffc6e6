"""FP64 CPU reference for the gradients of the coupled step (test
infrastructure, like the rest of oracle/; never imported by the product).

The oracle's coupled step (fcd_oracle.c, arXiv 2410.11129 Secs. 2.1-2.5) is
restated here with plain PyTorch CPU operations in float64, so that
torch.autograd's reverse mode differentiates it: an FP64 CPU adjoint that
shares no code with the CUDA path. Same readings as the C oracle:
  - phases, permeability, density: Eqs. 32, 24, 8, 33 (clamped phases in the
    material laws, raw phases in the collision);
  - potential: the 9-point link operator of Eq. 6 with mirrored k and odd psi'
    at the half-way walls, periodic in x; solved exactly (dense LU) instead of
    by conjugate gradients, which the oracle runs to a tolerance;
  - forces: Eqs. 5, 7, 9 (Kelvin), 25-28 and 36 (surface tension, the full
    Eq. 25 form with gamma_T), 19 and 21 (pressure), the local non-equilibrium
    viscous force, the driving force, Eq. 22 (velocity);
  - collisions: Eqs. 12-18 with the Lallemand-Luo matrix (explicit M and its
    inverse), Eqs. 29-31 with the phase-field source;
  - streaming with half-way bounce-back; the open channel's Eq. 37 inlet and
    convective outlet;
  - observables: T_o of Eq. 42 through the crossing interpolation of the 1/2
    level set, and the unclamped overlap sum phi_1 phi_3.

The parameters theta = (Bo_m, Ca, alpha, nu_r) enter as tensors (nu_r =
nu_3 / nu_2, Eq. 39; sigma_23 = rho_3 nu_3 u_avg / Ca, Eq. 40; mu0 H0^2 from
Eq. 41), so d(T_o, overlap)/d(theta) and d/d(initial populations) come from
one backward pass. Clamps follow torch.clamp (derivative 1 on the closed
interval), sqrt and the crossing choice follow the primal values.
"""
import torch

Q = 9
EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
W = [4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
CS2 = 1.0 / 3.0
DT = torch.float64


def moment_matrix():
    """Lallemand-Luo orthogonal D2Q9 moments (rho, e, eps, jx, qx, jy, qy, pxx,
    pxy) as rows, and its inverse."""
    rows = []
    for a in range(Q):
        ex, ey = EX[a], EY[a]
        e2 = ex * ex + ey * ey
        rows.append([1.0, 3 * e2 - 4, (9 * e2 * e2 - 21 * e2 + 8) / 2, ex, (3 * e2 - 5) * ex, ey,
                     (3 * e2 - 5) * ey, ex * ex - ey * ey, ex * ey])
    M = torch.tensor(rows, dtype=DT).T.contiguous()
    return M, torch.linalg.inv(M)


class Grid:
    """Index tables of one channel: neighbour reads (periodic or clamped x,
    mirrored y), odd reads of psi', streaming sources."""

    def __init__(self, nx, ny, open_x):
        self.nx, self.ny, self.open = nx, ny, bool(open_x)
        N = nx * ny
        ys, xs = torch.meshgrid(torch.arange(ny), torch.arange(nx), indexing="ij")
        self.nb, self.nb_odd, self.sign_odd = [], [], []
        for a in range(Q):
            X, Y = xs + EX[a], ys + EY[a]
            Xm = X.clamp(0, nx - 1) if self.open else X % nx
            Ym = Y.clamp(0, ny - 1)
            self.nb.append((Ym * nx + Xm).reshape(-1))
            self.nb_odd.append((Ym * nx + X % nx).reshape(-1))
            ghost = (Y < 0) | (Y >= ny)
            self.sign_odd.append(torch.where(ghost, -1.0, 1.0).to(DT).reshape(-1))
        # streaming: destination population a at node m comes from
        #   source row inside: fpost[a] at m - e_a (x periodic, or absent when open)
        #   source row outside (wall): fpost[opp(a)] at m itself
        self.src, self.kind = [], []
        for a in range(Q):
            X, Y = xs - EX[a], ys - EY[a]
            wall = (Y < 0) | (Y >= ny)
            outside = (X < 0) | (X >= nx)
            kind = torch.where(wall, 1, torch.where(outside & self.open, 2, 0))
            src = (Y.clamp(0, ny - 1) * nx + X % nx)
            self.src.append(src.reshape(-1))
            self.kind.append(kind.reshape(-1))
        self.N = N


def shifted(a, grid, b):
    """a (N,) read at node + e_b (mirrored / periodic or clamped)."""
    return a[grid.nb[b]]


def grad(a, grid):
    gx = sum(W[b] * EX[b] * shifted(a, grid, b) for b in range(Q) if EX[b]) / CS2
    gy = sum(W[b] * EY[b] * shifted(a, grid, b) for b in range(Q) if EY[b]) / CS2
    return gx, gy


def lap(a, grid):
    return 2.0 / CS2 * sum(W[b] * (shifted(a, grid, b) - a) for b in range(1, Q))


def grad_odd(a, grid):
    """Eq. 34 for psi' (periodic in x, odd at the walls)."""
    gx = sum(W[b] * EX[b] * grid.sign_odd[b] * a[grid.nb_odd[b]] for b in range(Q) if EX[b]) / CS2
    gy = sum(W[b] * EY[b] * grid.sign_odd[b] * a[grid.nb_odd[b]] for b in range(Q) if EY[b]) / CS2
    return gx, gy


def derive(cfg, theta):
    """Lattice constants from cfg and theta = (Bo_m, Ca, alpha, nu_r) (tensors)."""
    bo, ca, alpha, nr = theta
    rho = [float(v) for v in cfg["rho"]]
    nu3 = float(cfg["nu"][2])
    nu = [float(cfg["nu"][0]), nu3 / nr, nu3]
    u_avg = 2.0 * cfg["u_max"] / 3.0
    if cfg.get("sigma23", 0.0) > 0:
        s23 = torch.tensor(float(cfg["sigma23"]), dtype=DT)
    else:
        s23 = rho[2] * nu3 * u_avg / ca  # Eq. 40
    s12 = s23 / cfg["s23_over_s12"]
    s13 = cfg["s13_over_s12"] * s12
    gam = [s12 + s13 - s23, s12 + s23 - s13, s13 + s23 - s12]  # Eq. 27
    gamT = 3.0 / (1.0 / gam[0] + 1.0 / gam[1] + 1.0 / gam[2])  # Eq. 26
    tau = [n / CS2 for n in nu]  # Eq. 14
    chi = [float(v) for v in cfg["chi"]]
    fp = cfg.get("ferro_phase", 0)
    r1, r2 = float(cfg["r1"]), float(cfg["r2"])
    if fp == 1:
        mu0H0sq = bo * 2.0 * s12 / (chi[0] * r1)  # Eq. 41, core
    elif fp == 2:
        mu0H0sq = bo * 2.0 * (s12 * r1 + s23 * r2) / (chi[1] * (r2 * r2 - r1 * r1))  # shell
    else:
        mu0H0sq = torch.zeros((), dtype=DT)
    H0 = torch.sqrt(mu0H0sq)
    G = 0.0 if cfg.get("open_x", 0) else 8.0 * rho[2] * nu3 * cfg["u_max"] / cfg["ny"] ** 2
    return dict(rho=rho, nu=nu, tau=tau, chi=chi, s12=s12, s13=s13, s23=s23, gam=gam, gamT=gamT,
                H0=H0, alpha=alpha, G=G, u_avg=u_avg, tau_phi=cfg["mobility"] / CS2,
                eta=float(cfg.get("eta", 0.0)), xi=float(cfg["xi"]), eps_n=float(cfg["eps_n"]))


def mag_solve(k, d, grid):
    """psi' with L(k) psi' = -L(k) psi0 (Eq. 6), dense and exact."""
    N, nx, ny = grid.N, grid.nx, grid.ny
    H0, al = d["H0"], d["alpha"]
    rows, cols, vals = [], [], []
    b = torch.zeros(N, dtype=DT)
    idx = torch.arange(N)
    for a in range(1, Q):
        kn = k[grid.nb[a]] if not grid.open else k[_nb_periodic(grid, a)]
        c = 2.0 / CS2 * W[a] * 0.5 * (k + kn)
        # (psi_nbr - psi_0): psi_nbr = sign * psi'[nb_odd]
        rows += [idx, idx]
        cols += [grid.nb_odd[a], idx]
        vals += [c * grid.sign_odd[a], -c]
        b = b + c * H0 * (EX[a] * torch.cos(al) + EY[a] * torch.sin(al))
    L = torch.zeros(N, N, dtype=DT).index_put((torch.cat(rows), torch.cat(cols)), torch.cat(vals),
                                              accumulate=True)
    return torch.linalg.solve(L, b)


def _nb_periodic(grid, a):
    """neighbour index with x periodic and y mirrored (k of the potential)."""
    nx, ny = grid.nx, grid.ny
    ys, xs = torch.meshgrid(torch.arange(ny), torch.arange(nx), indexing="ij")
    X, Y = (xs + EX[a]) % nx, (ys + EY[a]).clamp(0, ny - 1)
    return (Y * nx + X).reshape(-1)


def gamma9(ux, uy):
    """Eq. 18 with the u.u term over 2 c_s^2."""
    uu = ux * ux + uy * uy
    out = []
    for a in range(Q):
        eu = EX[a] * ux + EY[a] * uy
        out.append(W[a] * (1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2)))
    return torch.stack(out)


def feq9(ps, ux, uy):
    """Eq. 16."""
    G = gamma9(ux, uy)
    return torch.stack([ps * W[a] + (G[a] - W[a]) for a in range(Q)])


def mrt(h, s_nu, M, Mi):
    """M^-1 Lambda M h, Lambda = (1, ..., 1, s_nu, s_nu) per node."""
    m = M @ h
    m = torch.cat([m[:7], m[7:] * s_nu], dim=0)
    return Mi @ m


def step(f, g, d, grid, M, Mi, cfg):
    """One coupled step in the oracle's order; f (9, N), g (2, 9, N)."""
    N = grid.N
    phi = [g[0].sum(0), g[1].sum(0)]
    phi.append(1.0 - phi[0] - phi[1])
    phc = [p.clamp(0.0, 1.0) for p in phi]
    chi = d["chi"]
    k = 1.0 / sum(phc[i] / (1.0 + chi[i]) for i in range(3))
    rhof = sum(d["rho"][i] * phc[i] for i in range(3))  # Eq. 33
    psi = mag_solve(k, d, grid) if bool(d["H0"].detach() > 0) else torch.zeros(N, dtype=DT)

    gph = [grad(phi[0], grid), grad(phi[1], grid)]
    lph = [lap(phi[0], grid), lap(phi[1], grid)]
    gph.append((-(gph[0][0] + gph[1][0]), -(gph[0][1] + gph[1][1])))
    lph.append(-(lph[0] + lph[1]))
    # Eqs. 25, 28: chemical potentials from the free energy
    s12, s13, s23, gam, eta = d["s12"], d["s13"], d["s23"], d["gam"], d["eta"]
    p1, p2, p3 = phi
    gp = gam[0] * p1 + gam[1] * p2 + gam[2] * p3
    ppp = p1 * p2 * p3
    dH = [2 * s12 * p1 * p2 * p2 + 2 * s13 * p1 * p3 * p3 + p2 * p3 * gp + ppp * gam[0]
          + 2 * eta * p1 * p2 * p2 * p3 * p3,
          2 * s12 * p1 * p1 * p2 + 2 * s23 * p2 * p3 * p3 + p1 * p3 * gp + ppp * gam[1]
          + 2 * eta * p1 * p1 * p2 * p3 * p3,
          2 * s13 * p1 * p1 * p3 + 2 * s23 * p2 * p2 * p3 + p1 * p2 * gp + ppp * gam[2]
          + 2 * eta * p1 * p1 * p2 * p2 * p3]
    mu = []
    for i in range(3):
        s = sum((dH[i] - dH[j]) / gam[j] for j in range(3) if j != i)
        mu.append(4.0 * d["gamT"] / d["xi"] * s - 0.75 * d["xi"] * gam[i] * lph[i])
    Fs = [sum(mu[i] * gph[i][0] for i in range(3)), sum(mu[i] * gph[i][1] for i in range(3))]
    # Kelvin force (Eqs. 5, 7, 9)
    inv = sum(phc[i] / (1.0 + chi[i]) for i in range(3))
    sgx = sum(gph[i][0] / (1.0 + chi[i]) for i in range(3))
    sgy = sum(gph[i][1] / (1.0 + chi[i]) for i in range(3))
    gchi = (-sgx / (inv * inv), -sgy / (inv * inv))
    dpx, dpy = grad_odd(psi, grid)
    Hx = d["H0"] * torch.cos(d["alpha"]) - dpx
    Hy = d["H0"] * torch.sin(d["alpha"]) - dpy
    H2 = Hx * Hx + Hy * Hy
    Fm = (-0.5 * H2 * gchi[0], -0.5 * H2 * gchi[1])
    # pressure, predictor velocity, viscous force, velocity (Eqs. 19, 21, 22)
    ps = f.sum(0)
    jx = sum(EX[a] * f[a] for a in range(Q) if EX[a])
    jy = sum(EY[a] * f[a] for a in range(Q) if EY[a])
    grx, gry = grad(rhof, grid)
    F0x = Fs[0] + Fm[0] - ps * CS2 * grx + d["G"]
    F0y = Fs[1] + Fm[1] - ps * CS2 * gry
    upx, upy = jx + F0x / (2 * rhof), jy + F0y / (2 * rhof)
    tau = sum(phc[i] * d["tau"][i] for i in range(3))
    s_nu = 1.0 / (0.5 + tau)
    mh = mrt(f - feq9(ps, upx, upy), s_nu, M, Mi)
    Pxx = sum(EX[a] * EX[a] * mh[a] for a in range(Q) if EX[a])
    Pyy = sum(EY[a] * EY[a] * mh[a] for a in range(Q) if EY[a])
    Pxy = sum(EX[a] * EY[a] * mh[a] for a in range(Q) if EX[a] * EY[a])
    Fmx = -tau * (Pxx * grx + Pxy * gry)
    Fmy = -tau * (Pxy * grx + Pyy * gry)
    Ftx, Fty = F0x + Fmx, F0y + Fmy
    ux, uy = upx + Fmx / (2 * rhof), upy + Fmy / (2 * rhof)
    # MRT collision of f (Eqs. 12, 15, 16, 19)
    Fa = torch.stack([W[a] * (EX[a] * Ftx + EY[a] * Fty) / (rhof * CS2) for a in range(Q)])
    fpost = f - mrt(f - (feq9(ps, ux, uy) - 0.5 * Fa), s_nu, M, Mi) + Fa
    # phase fields (Eqs. 29-31)
    th, nn = [], []
    for j in range(3):
        th.append(4.0 / d["xi"] * phc[j] * (1.0 - phc[j]))
        mag = torch.sqrt(gph[j][0] ** 2 + gph[j][1] ** 2) + d["eps_n"]
        nn.append((gph[j][0] / mag, gph[j][1] / mag))
    mx = sum(th[j] * nn[j][0] for j in range(3))
    my = sum(th[j] * nn[j][1] for j in range(3))
    G9 = gamma9(ux, uy)
    taup = 0.5 + d["tau_phi"]
    gpost = []
    for i in range(2):
        qx, qy = th[i] * nn[i][0] - mx / 3.0, th[i] * nn[i][1] - my / 3.0
        Fp = torch.stack([W[a] * (EX[a] * qx + EY[a] * qy) for a in range(Q)])
        geq = phi[i] * G9 - 0.5 * Fp
        gpost.append(g[i] - (g[i] - geq) / taup + Fp)
    gpost = torch.stack(gpost)
    # streaming with half-way bounce-back
    fn = stream(fpost, grid)
    gn = torch.stack([stream(gpost[0], grid), stream(gpost[1], grid)])
    if grid.open:
        fn, gn = open_boundaries(f, g, fn, gn, d, grid, cfg)
    return fn, gn


def stream(post, grid):
    out = []
    for a in range(Q):
        kind = grid.kind[a]
        v = torch.where(kind == 0, post[a][grid.src[a]], post[OPP[a]])
        out.append(torch.where(kind == 2, torch.zeros_like(v), v))
    return torch.stack(out)


def open_boundaries(f, g, fn, gn, d, grid, cfg):
    """Eq. 37 inlet (Zou-He, corner solves) and the convective outlet on
    f - w p* (outlet reference p* = 0) and on g, as in the oracle."""
    nx, ny = grid.nx, grid.ny
    U = d["u_avg"]
    fn = fn.clone()
    gn = gn.clone()
    fa, fb_, ga, gb_ = [], [], [], []  # (index tuples, values) for index_put
    for y in range(ny):
        u = cfg["u_max"] * 4.0 * (y + 0.5) * (ny - 0.5 - y) / (ny * ny)
        n = y * nx
        fl = [fn[a, n] for a in range(Q)]
        if y == 0:
            fl[8] = fl[2] - fl[4] + fl[5] + fl[6] - fl[7]
        elif y == ny - 1:
            fl[5] = fl[4] - fl[2] - fl[6] + fl[7] + fl[8]
        else:
            fl[5] = fl[7] + 6 * W[5] * u - 0.5 * (fl[2] - fl[4])
            fl[8] = fl[6] + 6 * W[8] * u + 0.5 * (fl[2] - fl[4])
        if y in (0, ny - 1):
            fl[1] = u + fl[3] - fl[5] + fl[6] + fl[7] - fl[8]
        else:
            fl[1] = fl[3] + 6 * W[1] * u
        for a in (1, 5, 8):
            fa.append((a, n))
            fb_.append(fl[a])
        for i in range(2):
            for a in (1, 5, 8):
                if (a == 5 and y == 0) or (a == 8 and y == ny - 1):
                    continue
                ga.append((i, a, n))
                gb_.append(torch.zeros((), dtype=DT))
        o, b = n + nx - 1, n + nx - 2
        pb = sum(fn[a, b] for a in range(Q))
        po = sum(f[a, o] for a in range(Q))
        for a in (3, 6, 7):
            if (a == 6 and y == 0) or (a == 7 and y == ny - 1):
                continue
            fa.append((a, o))
            fb_.append(((f[a, o] - W[a] * po) + U * (fn[a, b] - W[a] * pb)) / (1 + U))
            for i in range(2):
                ga.append((i, a, o))
                gb_.append((g[i, a, o] + U * gn[i, a, b]) / (1 + U))
    ia = torch.tensor([t[0] for t in fa]), torch.tensor([t[1] for t in fa])
    fn = fn.index_put(ia, torch.stack(fb_))
    ig = (torch.tensor([t[0] for t in ga]), torch.tensor([t[1] for t in ga]),
          torch.tensor([t[2] for t in ga]))
    gn = gn.index_put(ig, torch.stack(gb_))
    return fn, gn


def _crossings(v):
    """First upward and last downward 1/2-crossing of v (1D tensor, zero
    padded outside): (lo, hi) tensors or None. The crossing choice follows
    the values; lo, hi are differentiable in v."""
    n = v.shape[0]
    vals = v.detach().tolist()
    first = last = None
    for i in range(-1, n):
        a = 0.0 if i < 0 else vals[i]
        b = vals[i + 1] if i + 1 < n else 0.0
        if a < 0.5 <= b and first is None:
            first = i
        if a >= 0.5 > b:
            last = i
    if first is None or last is None:
        return None
    zero = torch.zeros((), dtype=DT)
    a = zero if first < 0 else v[first]
    b = v[first + 1] if first + 1 < n else zero
    lo = first + (0.5 - a) / (b - a)
    a = zero if last < 0 else v[last]
    b = v[last + 1] if last + 1 < n else zero
    hi = last + (a - 0.5) / (a - b)
    return lo, hi


def observables(g, grid):
    """(T_o, overlap): Eq. 42 for the shell indicator, and sum phi_1 phi_3."""
    nx, ny = grid.nx, grid.ny
    p1, p2 = g[0].sum(0), g[1].sum(0)
    overlap = (p1 * (1.0 - p1 - p2)).sum()
    so = (p1.clamp(0, 1) + p2.clamp(0, 1)).reshape(ny, nx)
    # frame of l_x: from the emptiest column (the inlet in the open channel)
    xcut = 0
    if not grid.open:
        cols = so.detach().sum(0).tolist()
        best = None
        for x, s in enumerate(cols):
            if best is None or s < best:
                best, xcut = s, x
    order = [(xcut + j) % nx for j in range(nx)]
    if ny % 2:
        line = so[ny // 2, order]
    else:
        line = 0.5 * (so[ny // 2 - 1, order] + so[ny // 2, order])
    c = _crossings(line)
    lx = c[1] - c[0] if c else torch.zeros((), dtype=DT)
    ly = torch.zeros((), dtype=DT)
    for x in range(nx):
        c = _crossings(so[:, x])
        if c and bool((c[1] - c[0]).detach() > ly.detach()):
            ly = c[1] - c[0]
    s = lx + ly
    To = (ly - lx) / s if bool(s.detach() > 0) else torch.zeros((), dtype=DT)
    return To, overlap


def run(cfg, theta, steps, f0, g0):
    """(T_o, overlap) after `steps` steps from the populations (f0, g0),
    numpy arrays (9, ny, nx) and (2, 9, ny, nx) in the oracle's layout;
    theta a float64 tensor of 4 (may require grad); f0, g0 may be tensors
    that require grad."""
    nx, ny = cfg["nx"], cfg["ny"]
    grid = Grid(nx, ny, cfg.get("open_x", 0))
    M, Mi = moment_matrix()
    d = derive(cfg, (theta[0], theta[1], theta[2], theta[3]))
    f = torch.as_tensor(f0, dtype=DT).reshape(Q, nx * ny)
    g = torch.as_tensor(g0, dtype=DT).reshape(2, Q, nx * ny)
    for _ in range(steps):
        f, g = step(f, g, d, grid, M, Mi, cfg)
    return observables(g, grid), (f, g)


def parameters_of(cfg):
    """theta = (Bo_m, Ca, alpha, nu_r) of a configuration (nu_r = nu_3 / nu_2)."""
    return [float(cfg["Bo_m"]), float(cfg["Ca"]), float(cfg["alpha"]),
            float(cfg["nu"][2]) / float(cfg["nu"][1])]


def gradients(cfg, steps, f0, g0, w_T=1.0, w_overlap=0.0):
    """J = w_T T_o + w_overlap overlap after `steps` steps and its gradients
    with respect to theta, f0 and g0 (reverse mode through the whole run)."""
    theta = torch.tensor(parameters_of(cfg), dtype=DT, requires_grad=True)
    f = torch.tensor(f0, dtype=DT, requires_grad=True)
    g = torch.tensor(g0, dtype=DT, requires_grad=True)
    (To, ov), _ = run(cfg, theta, steps, f, g)
    J = w_T * To + w_overlap * ov
    J.backward()
    return {"T_o": float(To.detach()), "overlap": float(ov.detach()), "J": float(J.detach()),
            "grad": theta.grad.tolist(), "df0": f.grad.numpy(), "dg0": g.grad.numpy()}
