// fcd_adjoint.cuh -- the per-node part of the coupled step (arXiv 2410.11129)
// written out for reverse-mode differentiation: node_forward evaluates the
// collision of one lattice node from its stencil values and populations, as the
// collide kernel does (Eqs. 7-9 Kelvin force, Eqs. 25-28 and 36 surface
// tension, Eq. 19 pressure, viscous and driving forces, Eq. 22 velocity,
// Eqs. 12-18 MRT collision of f, Eqs. 29-31 collision of g^1, g^2) and keeps
// every intermediate; node_reverse is its hand-written adjoint: given the
// adjoints of the 27 post-collision populations it returns the adjoints of the
// node's inputs and of the constants that depend on (Bo_m, Ca, alpha, nu_r).
//
// The inputs are the reduced stencil values (the centre value, the isotropic
// gradient of Eq. 34 and the Laplacian of Eq. 35 of phi_1 and phi_2, the centre
// value and gradient of the mixture density, the gradient of psi') and the
// node's populations; the stencils are linear, so the kernels that call these
// functions apply their transposes.
//
// Both functions are host-and-device code so that the reverse can be checked
// against dual-number derivatives of the forward on the CPU.
#pragma once

#include "fcd_internal.cuh"

namespace fcd {

// Adjoints of the constants: sigma_ij and gamma_i (Eqs. 27-28), eta, the
// Laplacian coefficients (3/4) xi gamma_i (Eq. 25), H0 (cos alpha, sin alpha)
// and the relaxation times tau_i (Eq. 14).
enum ParamBar {
    PB_S12, PB_S13, PB_S23, PB_GAM0, PB_GAM1, PB_GAM2, PB_ETA,
    PB_LC0, PB_LC1, PB_LC2, PB_H0C, PB_H0S, PB_TAU0, PB_TAU1, PB_TAU2, NPB
};

// clamp to [0, 1]; derivative 1 on the closed interval (the value branch)
template <typename R>
__host__ __device__ inline R cl01(const R &v) {
    return v < 0.0 ? R(0.0) : (v > 1.0 ? R(1.0) : v);
}
__host__ __device__ inline double dcl01(double v) { return (v >= 0.0 && v <= 1.0) ? 1.0 : 0.0; }

// second-order moment rows of the MRT basis: p_xx (rows 1, 3 minus 2, 4),
// p_xy (rows 5, 7 minus 6, 8), energy e (-4, -1 on the axes, 2 on diagonals)
__host__ __device__ constexpr int rxx(int a) { return (a == 1 || a == 3) ? 1 : ((a == 2 || a == 4) ? -1 : 0); }
__host__ __device__ constexpr int rxy(int a) { return (a == 5 || a == 7) ? 1 : ((a == 6 || a == 8) ? -1 : 0); }
__host__ __device__ constexpr int ren(int a) { return a == 0 ? -4 : (a <= 4 ? -1 : 2); }

template <typename R>
struct NodeFwd {
    // inputs
    R ph1, g1x, g1y, l1, ph2, g2x, g2y, l2, rho, grx, gry, dpx, dpy;
    R f[9], g[18];
    // intermediates
    R ph3, g3x, g3y, l3, h1, h2, h3;
    R gp, q3, a1, a2, a3, X1, X2, X3, m1, m2, m3;
    R kk, gcx, gcy, Hx, Hy, hh;
    R pst, jx, jy, mpxx, mpxy, me;
    R Fx0, Fy0;  // surface tension + Kelvin + pressure + driving force
    R inv_rho, upx, upy, tau, snu, hxx, hxy, Pxx, Pyy, Pxy;
    R Fx, Fy;    // ... plus the viscous force
    R ux, uy, eu[9], dev[9], dxx, dxy, fr;
    R rn[3], nrm[3], iv[3];
    // outputs: post-collision populations (before streaming)
    R fout[9], gout[18];
};

template <typename R>
__host__ __device__ inline void node_forward(NodeFwd<R> &F, const Phys<R> &P) {
    F.ph3 = 1.0 - F.ph1 - F.ph2;
    F.g3x = -(F.g1x + F.g2x);
    F.g3y = -(F.g1y + F.g2y);
    F.l3 = -(F.l1 + F.l2);
    F.h1 = cl01(F.ph1);
    F.h2 = cl01(F.ph2);
    F.h3 = cl01(F.ph3);

    // surface tension (Eqs. 25, 28, 36)
    F.gp = P.gam[0] * F.ph1 + P.gam[1] * F.ph2 + P.gam[2] * F.ph3;
    F.q3 = F.ph1 * F.ph2 * F.ph3;
    F.a1 = F.ph1 * F.ph1;
    F.a2 = F.ph2 * F.ph2;
    F.a3 = F.ph3 * F.ph3;
    F.X1 = P.s12 * F.a2 + P.s13 * F.a3;
    F.X2 = P.s12 * F.a1 + P.s23 * F.a3;
    F.X3 = P.s13 * F.a1 + P.s23 * F.a2;
    const R d1 = 2.0 * F.ph1 * F.X1 + F.ph2 * F.ph3 * F.gp + P.gam[0] * F.q3 +
                 2.0 * P.eta * F.ph1 * F.a2 * F.a3;
    const R d2 = 2.0 * F.ph2 * F.X2 + F.ph1 * F.ph3 * F.gp + P.gam[1] * F.q3 +
                 2.0 * P.eta * F.a1 * F.ph2 * F.a3;
    const R d3 = 2.0 * F.ph3 * F.X3 + F.ph1 * F.ph2 * F.gp + P.gam[2] * F.q3 +
                 2.0 * P.eta * F.a1 * F.a2 * F.ph3;
    F.m1 = P.twelve_over_xi * d1 - P.lap_coef[0] * F.l1;
    F.m2 = P.twelve_over_xi * d2 - P.lap_coef[1] * F.l2;
    F.m3 = P.twelve_over_xi * d3 - P.lap_coef[2] * F.l3;
    R Fx = F.m1 * F.g1x + F.m2 * F.g2x + F.m3 * F.g3x;
    R Fy = F.m1 * F.g1y + F.m2 * F.g2y + F.m3 * F.g3y;

    // Kelvin force (Eqs. 5, 7, 9)
    F.kk = 1.0 / (P.ik[0] * F.h1 + P.ik[1] * F.h2 + P.ik[2] * F.h3);
    F.gcx = -F.kk * F.kk * (P.dk1 * F.g1x + P.dk2 * F.g2x);
    F.gcy = -F.kk * F.kk * (P.dk1 * F.g1y + P.dk2 * F.g2y);
    F.Hx = P.H0c - F.dpx;
    F.Hy = P.H0s - F.dpy;
    F.hh = 0.5 * (F.Hx * F.Hx + F.Hy * F.Hy);
    Fx = Fx - F.hh * F.gcx;
    Fy = Fy - F.hh * F.gcy;

    // moments of f
    F.pst = R(0.0);
    F.jx = R(0.0);
    F.jy = R(0.0);
    F.mpxx = R(0.0);
    F.mpxy = R(0.0);
    F.me = R(0.0);
    for (int a = 0; a < 9; a++) {
        F.pst = F.pst + F.f[a];
        if (cx(a)) F.jx = F.jx + double(cx(a)) * F.f[a];
        if (cy(a)) F.jy = F.jy + double(cy(a)) * F.f[a];
        if (rxx(a)) F.mpxx = F.mpxx + double(rxx(a)) * F.f[a];
        if (rxy(a)) F.mpxy = F.mpxy + double(rxy(a)) * F.f[a];
        F.me = F.me + double(ren(a)) * F.f[a];
    }

    // pressure and driving force, predictor velocity, viscous force (Eq. 19)
    F.Fx0 = Fx - F.pst * (1.0 / 3.0) * F.grx + P.G;
    F.Fy0 = Fy - F.pst * (1.0 / 3.0) * F.gry;
    F.inv_rho = 1.0 / F.rho;
    const R hir = 0.5 * F.inv_rho;
    F.upx = F.jx + F.Fx0 * hir;
    F.upy = F.jy + F.Fy0 * hir;
    F.tau = P.tau[0] * F.h1 + P.tau[1] * F.h2 + P.tau[2] * F.h3;
    F.snu = 1.0 / (0.5 + F.tau);
    const R he = F.me - (3.0 * (F.upx * F.upx + F.upy * F.upy) - 2.0 * F.pst);
    F.hxx = F.mpxx - (F.upx * F.upx - F.upy * F.upy);
    F.hxy = F.mpxy - F.upx * F.upy;
    F.Pxx = he * (1.0 / 6.0) + 0.5 * F.snu * F.hxx;
    F.Pyy = he * (1.0 / 6.0) - 0.5 * F.snu * F.hxx;
    F.Pxy = F.snu * F.hxy;
    F.Fx = F.Fx0 - F.tau * (F.Pxx * F.grx + F.Pxy * F.gry);
    F.Fy = F.Fy0 - F.tau * (F.Pxy * F.grx + F.Pyy * F.gry);

    // velocity (Eq. 22), equilibria and MRT collision of f (Eqs. 12-18)
    F.ux = F.jx + F.Fx * hir;
    F.uy = F.jy + F.Fy * hir;
    const R uu = 1.5 * (F.ux * F.ux + F.uy * F.uy);
    for (int a = 0; a < 9; a++) {
        F.eu[a] = double(cx(a)) * F.ux + double(cy(a)) * F.uy;
        F.dev[a] = 3.0 * F.eu[a] + 4.5 * F.eu[a] * F.eu[a] - uu;
    }
    F.dxx = F.mpxx - (F.ux * F.ux - F.uy * F.uy);
    F.dxy = F.mpxy - F.ux * F.uy;
    const R rel = (1.0 - F.snu) * 0.25;
    F.fr = 3.0 * F.inv_rho;
    const R Ftx = 0.5 * F.Fx * F.fr, Fty = 0.5 * F.Fy * F.fr;
    for (int a = 0; a < 9; a++) {
        F.fout[a] = wgt<double>(a) * ((F.pst + F.dev[a]) + (double(cx(a)) * Ftx + double(cy(a)) * Fty)) +
                    rel * (double(rxx(a)) * F.dxx + double(rxy(a)) * F.dxy);
    }

    // phase fields (Eqs. 29-31)
    const R hv[3] = {F.h1, F.h2, F.h3};
    const R gxv[3] = {F.g1x, F.g2x, F.g3x}, gyv[3] = {F.g1y, F.g2y, F.g3y};
    for (int i = 0; i < 3; i++) {
        const R t = P.four_over_xi * hv[i] * (1.0 - hv[i]);
        F.rn[i] = sqrt(gxv[i] * gxv[i] + gyv[i] * gyv[i]);
        F.nrm[i] = F.rn[i] + P.eps_n;
        F.iv[i] = t / F.nrm[i];
    }
    const R mx = (F.iv[0] * F.g1x + F.iv[1] * F.g2x + F.iv[2] * F.g3x) * (1.0 / 3.0);
    const R my = (F.iv[0] * F.g1y + F.iv[1] * F.g2y + F.iv[2] * F.g3y) * (1.0 / 3.0);
    for (int i = 0; i < 2; i++) {
        const R phi = i == 0 ? F.ph1 : F.ph2;
        const R qx = F.iv[i] * gxv[i] - mx, qy = F.iv[i] * gyv[i] - my;
        const R sqx = P.src_phi * qx, sqy = P.src_phi * qy;
        for (int a = 0; a < 9; a++) {
            F.gout[i * 9 + a] = P.keep_phi * F.g[i * 9 + a] +
                                wgt<double>(a) * (P.om_phi * phi * (1.0 + F.dev[a]) +
                                                  (double(cx(a)) * sqx + double(cy(a)) * sqy));
        }
    }
}

// Adjoints of the node's inputs (and of the constants, added into p[]).
struct NodeBar {
    double ph1, g1x, g1y, l1, ph2, g2x, g2y, l2, rho, grx, gry, dpx, dpy;
    double f[9], g[18];
};

// fb[a], gb[i*9 + a]: adjoints of the post-collision populations fout, gout.
__host__ __device__ inline void node_reverse(const NodeFwd<double> &F, const Phys<double> &P,
                                             const double *fb, const double *gb, NodeBar &B,
                                             double *p) {
    double ph1b = 0.0, ph2b = 0.0, ph3b = 0.0, h1b = 0.0, h2b = 0.0, h3b = 0.0;
    double g1xb = 0.0, g1yb = 0.0, g2xb = 0.0, g2yb = 0.0, g3xb = 0.0, g3yb = 0.0;
    double devb[9];
    for (int a = 0; a < 9; a++) devb[a] = 0.0;

    // ---- phase fields: g* = keep g + w (om phi (1 + dev) + e . src q)
    double qxb[2], qyb[2];
    for (int i = 0; i < 2; i++) {
        const double phi = i == 0 ? F.ph1 : F.ph2;
        double ob = 0.0, sxb = 0.0, syb = 0.0;
        for (int a = 0; a < 9; a++) {
            const double v = gb[i * 9 + a], w = wgt<double>(a);
            B.g[i * 9 + a] = P.keep_phi * v;
            ob += v * w * (1.0 + F.dev[a]);
            devb[a] += v * w * P.om_phi * phi;
            sxb += v * w * cx(a);
            syb += v * w * cy(a);
        }
        if (i == 0) ph1b += P.om_phi * ob;
        else ph2b += P.om_phi * ob;
        qxb[i] = P.src_phi * sxb;
        qyb[i] = P.src_phi * syb;
    }
    // q_i = iv_i grad phi_i - m, m = (1/3) sum_j iv_j grad phi_j
    double ivb[3];
    {
        const double mxb = -(qxb[0] + qxb[1]) * (1.0 / 3.0), myb = -(qyb[0] + qyb[1]) * (1.0 / 3.0);
        ivb[0] = qxb[0] * F.g1x + qyb[0] * F.g1y + mxb * F.g1x + myb * F.g1y;
        ivb[1] = qxb[1] * F.g2x + qyb[1] * F.g2y + mxb * F.g2x + myb * F.g2y;
        ivb[2] = mxb * F.g3x + myb * F.g3y;
        g1xb += (qxb[0] + mxb) * F.iv[0];
        g1yb += (qyb[0] + myb) * F.iv[0];
        g2xb += (qxb[1] + mxb) * F.iv[1];
        g2yb += (qyb[1] + myb) * F.iv[1];
        g3xb += mxb * F.iv[2];
        g3yb += myb * F.iv[2];
    }
    // iv_i = theta_i / (|grad phi_i| + eps_n), theta_i = (4/xi) h_i (1 - h_i)
    {
        const double hv[3] = {F.h1, F.h2, F.h3};
        const double gxv[3] = {F.g1x, F.g2x, F.g3x}, gyv[3] = {F.g1y, F.g2y, F.g3y};
        double gxb[3] = {0.0, 0.0, 0.0}, gyb[3] = {0.0, 0.0, 0.0}, hb[3];
        for (int i = 0; i < 3; i++) {
            const double tb = ivb[i] / F.nrm[i];
            const double nb = -ivb[i] * F.iv[i] / F.nrm[i];
            if (F.rn[i] > 0.0) {
                gxb[i] = nb * gxv[i] / F.rn[i];
                gyb[i] = nb * gyv[i] / F.rn[i];
            }
            hb[i] = tb * P.four_over_xi * (1.0 - 2.0 * hv[i]);
        }
        g1xb += gxb[0]; g1yb += gyb[0];
        g2xb += gxb[1]; g2yb += gyb[1];
        g3xb += gxb[2]; g3yb += gyb[2];
        h1b += hb[0]; h2b += hb[1]; h3b += hb[2];
    }

    // ---- f: f* = w (p* + dev + e . Ft) + rel (rxx dxx + rxy dxy)
    const double rel = (1.0 - F.snu) * 0.25;
    double pstb = 0.0, Ftxb = 0.0, Ftyb = 0.0, relb = 0.0, sxx = 0.0, sxy = 0.0;
    for (int a = 0; a < 9; a++) {
        const double v = fb[a], w = wgt<double>(a);
        pstb += v * w;
        devb[a] += v * w;
        Ftxb += v * w * cx(a);
        Ftyb += v * w * cy(a);
        relb += v * (rxx(a) * F.dxx + rxy(a) * F.dxy);
        sxx += v * rxx(a);
        sxy += v * rxy(a);
    }
    const double dxxb = rel * sxx, dxyb = rel * sxy;
    double snub = -0.25 * relb;
    double Fxb = 0.5 * F.fr * Ftxb, Fyb = 0.5 * F.fr * Ftyb;
    double irb = 3.0 * 0.5 * (F.Fx * Ftxb + F.Fy * Ftyb);  // through fr = 3 / rho
    // dev_a = 3 eu + 4.5 eu^2 - 1.5 |u|^2
    double uxb = 0.0, uyb = 0.0, uub = 0.0;
    for (int a = 0; a < 9; a++) {
        const double eub = devb[a] * (3.0 + 9.0 * F.eu[a]);
        uub -= devb[a];
        uxb += eub * cx(a);
        uyb += eub * cy(a);
    }
    uxb += 3.0 * F.ux * uub;
    uyb += 3.0 * F.uy * uub;
    // dxx = m_pxx - (ux^2 - uy^2), dxy = m_pxy - ux uy
    double mpxxb = dxxb, mpxyb = dxyb;
    uxb += -2.0 * F.ux * dxxb - F.uy * dxyb;
    uyb += 2.0 * F.uy * dxxb - F.ux * dxyb;
    // u = j + F / (2 rho)
    const double hir = 0.5 * F.inv_rho;
    double jxb = uxb, jyb = uyb;
    Fxb += uxb * hir;
    Fyb += uyb * hir;
    double hirb = uxb * F.Fx + uyb * F.Fy;
    // F = F0 - tau (Pi . grad rho)
    double Fx0b = Fxb, Fy0b = Fyb;
    double taub = -(Fxb * (F.Pxx * F.grx + F.Pxy * F.gry) + Fyb * (F.Pxy * F.grx + F.Pyy * F.gry));
    const double Pxxb = -F.tau * Fxb * F.grx, Pyyb = -F.tau * Fyb * F.gry;
    const double Pxyb = -F.tau * (Fxb * F.gry + Fyb * F.grx);
    double grxb = -F.tau * (Fxb * F.Pxx + Fyb * F.Pxy);
    double gryb = -F.tau * (Fxb * F.Pxy + Fyb * F.Pyy);
    // Pxx = he/6 + snu hxx/2, Pyy = he/6 - snu hxx/2, Pxy = snu hxy
    const double heb = (Pxxb + Pyyb) * (1.0 / 6.0);
    const double hxxb = 0.5 * F.snu * (Pxxb - Pyyb), hxyb = F.snu * Pxyb;
    snub += 0.5 * F.hxx * (Pxxb - Pyyb) + F.hxy * Pxyb;
    // he = m_e - 3 |u'|^2 + 2 p*, hxx = m_pxx - (u'x^2 - u'y^2), hxy = m_pxy - u'x u'y
    double meb = heb;
    pstb += 2.0 * heb;
    mpxxb += hxxb;
    mpxyb += hxyb;
    const double upxb = -6.0 * F.upx * heb - 2.0 * F.upx * hxxb - F.upy * hxyb;
    const double upyb = -6.0 * F.upy * heb + 2.0 * F.upy * hxxb - F.upx * hxyb;
    // snu = 1 / (1/2 + tau), tau = sum_i tau_i h_i
    taub -= snub * F.snu * F.snu;
    h1b += taub * P.tau[0];
    h2b += taub * P.tau[1];
    h3b += taub * P.tau[2];
    p[PB_TAU0] += taub * F.h1;
    p[PB_TAU1] += taub * F.h2;
    p[PB_TAU2] += taub * F.h3;
    // u' = j + F0 / (2 rho)
    jxb += upxb;
    jyb += upyb;
    Fx0b += upxb * hir;
    Fy0b += upyb * hir;
    hirb += upxb * F.Fx0 + upyb * F.Fy0;
    irb += 0.5 * hirb;
    B.rho = -irb * F.inv_rho * F.inv_rho;
    // F0 = Fs + Fm - p*/3 grad rho + G
    pstb -= (Fx0b * F.grx + Fy0b * F.gry) * (1.0 / 3.0);
    grxb -= Fx0b * F.pst * (1.0 / 3.0);
    gryb -= Fy0b * F.pst * (1.0 / 3.0);
    B.grx = grxb;
    B.gry = gryb;
    for (int a = 0; a < 9; a++)
        B.f[a] = pstb + cx(a) * jxb + cy(a) * jyb + rxx(a) * mpxxb + rxy(a) * mpxyb + ren(a) * meb;

    // ---- Kelvin force: Fm = -hh grad chi
    {
        const double hhb = -(Fx0b * F.gcx + Fy0b * F.gcy);
        const double gcxb = -F.hh * Fx0b, gcyb = -F.hh * Fy0b;
        const double Hxb = hhb * F.Hx, Hyb = hhb * F.Hy;
        p[PB_H0C] += Hxb;
        p[PB_H0S] += Hyb;
        B.dpx = -Hxb;
        B.dpy = -Hyb;
        const double k2 = F.kk * F.kk;
        const double cxs = P.dk1 * F.g1x + P.dk2 * F.g2x, cys = P.dk1 * F.g1y + P.dk2 * F.g2y;
        const double kkb = -2.0 * F.kk * (gcxb * cxs + gcyb * cys);
        g1xb -= k2 * P.dk1 * gcxb;
        g2xb -= k2 * P.dk2 * gcxb;
        g1yb -= k2 * P.dk1 * gcyb;
        g2yb -= k2 * P.dk2 * gcyb;
        const double skb = -kkb * k2;
        h1b += skb * P.ik[0];
        h2b += skb * P.ik[1];
        h3b += skb * P.ik[2];
    }

    // ---- surface tension: Fs = sum_i m_i grad phi_i, m_i = (12/xi) d_i - LC_i lap phi_i
    double l1b, l2b, l3b;
    {
        const double m1b = Fx0b * F.g1x + Fy0b * F.g1y;
        const double m2b = Fx0b * F.g2x + Fy0b * F.g2y;
        const double m3b = Fx0b * F.g3x + Fy0b * F.g3y;
        g1xb += Fx0b * F.m1; g1yb += Fy0b * F.m1;
        g2xb += Fx0b * F.m2; g2yb += Fy0b * F.m2;
        g3xb += Fx0b * F.m3; g3yb += Fy0b * F.m3;
        l1b = -P.lap_coef[0] * m1b;
        l2b = -P.lap_coef[1] * m2b;
        l3b = -P.lap_coef[2] * m3b;
        p[PB_LC0] -= m1b * F.l1;
        p[PB_LC1] -= m2b * F.l2;
        p[PB_LC2] -= m3b * F.l3;
        const double d1b = P.twelve_over_xi * m1b, d2b = P.twelve_over_xi * m2b,
                     d3b = P.twelve_over_xi * m3b;
        double a1b = 0.0, a2b = 0.0, a3b = 0.0, gpb = 0.0, q3b = 0.0;
        // d1 = 2 ph1 X1 + ph2 ph3 gp + gam1 q3 + 2 eta ph1 a2 a3
        ph1b += d1b * (2.0 * F.X1 + 2.0 * P.eta * F.a2 * F.a3);
        {
            const double Xb = 2.0 * F.ph1 * d1b;
            p[PB_S12] += Xb * F.a2; a2b += Xb * P.s12;
            p[PB_S13] += Xb * F.a3; a3b += Xb * P.s13;
        }
        ph2b += d1b * F.ph3 * F.gp; ph3b += d1b * F.ph2 * F.gp; gpb += d1b * F.ph2 * F.ph3;
        p[PB_GAM0] += d1b * F.q3; q3b += d1b * P.gam[0];
        p[PB_ETA] += d1b * 2.0 * F.ph1 * F.a2 * F.a3;
        a2b += d1b * 2.0 * P.eta * F.ph1 * F.a3;
        a3b += d1b * 2.0 * P.eta * F.ph1 * F.a2;
        // d2 = 2 ph2 X2 + ph1 ph3 gp + gam2 q3 + 2 eta a1 ph2 a3
        ph2b += d2b * (2.0 * F.X2 + 2.0 * P.eta * F.a1 * F.a3);
        {
            const double Xb = 2.0 * F.ph2 * d2b;
            p[PB_S12] += Xb * F.a1; a1b += Xb * P.s12;
            p[PB_S23] += Xb * F.a3; a3b += Xb * P.s23;
        }
        ph1b += d2b * F.ph3 * F.gp; ph3b += d2b * F.ph1 * F.gp; gpb += d2b * F.ph1 * F.ph3;
        p[PB_GAM1] += d2b * F.q3; q3b += d2b * P.gam[1];
        p[PB_ETA] += d2b * 2.0 * F.a1 * F.ph2 * F.a3;
        a1b += d2b * 2.0 * P.eta * F.ph2 * F.a3;
        a3b += d2b * 2.0 * P.eta * F.a1 * F.ph2;
        // d3 = 2 ph3 X3 + ph1 ph2 gp + gam3 q3 + 2 eta a1 a2 ph3
        ph3b += d3b * (2.0 * F.X3 + 2.0 * P.eta * F.a1 * F.a2);
        {
            const double Xb = 2.0 * F.ph3 * d3b;
            p[PB_S13] += Xb * F.a1; a1b += Xb * P.s13;
            p[PB_S23] += Xb * F.a2; a2b += Xb * P.s23;
        }
        ph1b += d3b * F.ph2 * F.gp; ph2b += d3b * F.ph1 * F.gp; gpb += d3b * F.ph1 * F.ph2;
        p[PB_GAM2] += d3b * F.q3; q3b += d3b * P.gam[2];
        p[PB_ETA] += d3b * 2.0 * F.a1 * F.a2 * F.ph3;
        a1b += d3b * 2.0 * P.eta * F.a2 * F.ph3;
        a2b += d3b * 2.0 * P.eta * F.a1 * F.ph3;
        // a_i = ph_i^2, q3 = ph1 ph2 ph3, gp = sum_i gam_i ph_i
        ph1b += 2.0 * F.ph1 * a1b + q3b * F.ph2 * F.ph3 + gpb * P.gam[0];
        ph2b += 2.0 * F.ph2 * a2b + q3b * F.ph1 * F.ph3 + gpb * P.gam[1];
        ph3b += 2.0 * F.ph3 * a3b + q3b * F.ph1 * F.ph2 + gpb * P.gam[2];
        p[PB_GAM0] += gpb * F.ph1;
        p[PB_GAM1] += gpb * F.ph2;
        p[PB_GAM2] += gpb * F.ph3;
    }

    // ---- phase 3 from phases 1, 2; clamps
    ph1b += h1b * dcl01(F.ph1);
    ph2b += h2b * dcl01(F.ph2);
    ph3b += h3b * dcl01(F.ph3);
    B.ph1 = ph1b - ph3b;
    B.ph2 = ph2b - ph3b;
    B.g1x = g1xb - g3xb;
    B.g1y = g1yb - g3yb;
    B.g2x = g2xb - g3xb;
    B.g2y = g2yb - g3yb;
    B.l1 = l1b - l3b;
    B.l2 = l2b - l3b;
}

}  // namespace fcd
