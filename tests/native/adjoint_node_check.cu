// Host-side check of the hand-written per-node adjoint of the collision
// (node_reverse) against forward-mode derivatives of its own forward
// (node_forward evaluated in dual numbers). For random nodes, including phase
// values outside [0, 1] and vanishing gradients, and random adjoints ybar of
// the 27 post-collision populations, every input x_k (40 node inputs) and
// every constant c_k (15) must satisfy
//     node_reverse(ybar)_k == sum_j ybar_j dy_j/dx_k
// Prints the worst relative mismatch and exits 1 above 1e-12.
#include <cmath>
#include <cstdio>
#include <random>

#include "fcd_adjoint.cuh"

using namespace fcd;
using D1 = Dual<1>;

template <typename R>
static R *input(NodeFwd<R> &F, int k) {
    R *s[13] = {&F.ph1, &F.g1x, &F.g1y, &F.l1, &F.ph2, &F.g2x, &F.g2y,
                &F.l2,  &F.rho, &F.grx, &F.gry, &F.dpx, &F.dpy};
    if (k < 13) return s[k];
    if (k < 22) return &F.f[k - 13];
    return &F.g[k - 22];
}

static double input_bar(const NodeBar &B, int k) {
    const double s[13] = {B.ph1, B.g1x, B.g1y, B.l1, B.ph2, B.g2x, B.g2y,
                          B.l2,  B.rho, B.grx, B.gry, B.dpx, B.dpy};
    if (k < 13) return s[k];
    if (k < 22) return B.f[k - 13];
    return B.g[k - 22];
}

template <typename R>
static R *constant(Phys<R> &P, int k) {
    R *c[NPB] = {&P.s12, &P.s13, &P.s23, &P.gam[0], &P.gam[1], &P.gam[2], &P.eta, &P.lap_coef[0],
                 &P.lap_coef[1], &P.lap_coef[2], &P.H0c, &P.H0s, &P.tau[0], &P.tau[1], &P.tau[2]};
    return c[k];
}

static void to_dual(Phys<D1> &Q, const Phys<double> &P) {
    Q.nx = P.nx; Q.ny = P.ny; Q.pitch = P.pitch; Q.ps = P.ps;
    for (int i = 0; i < 3; i++) {
        Q.rho[i] = D1(P.rho[i]); Q.tau[i] = D1(P.tau[i]); Q.ik[i] = D1(P.ik[i]);
        Q.gam[i] = D1(P.gam[i]); Q.lap_coef[i] = D1(P.lap_coef[i]);
    }
    Q.dk1 = D1(P.dk1); Q.dk2 = D1(P.dk2); Q.s12 = D1(P.s12); Q.s13 = D1(P.s13); Q.s23 = D1(P.s23);
    Q.eta = D1(P.eta); Q.twelve_over_xi = D1(P.twelve_over_xi); Q.four_over_xi = D1(P.four_over_xi);
    Q.eps_n = D1(P.eps_n); Q.om_phi = D1(P.om_phi); Q.keep_phi = D1(P.keep_phi);
    Q.src_phi = D1(P.src_phi); Q.H0c = D1(P.H0c); Q.H0s = D1(P.H0s); Q.G = D1(P.G);
}

int main() {
    std::mt19937_64 rng(20241015);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    // constants of a three-phase channel with eta != 0 and unequal chi, tau
    Phys<double> P{};
    P.rho[0] = 1.0; P.rho[1] = 0.5; P.rho[2] = 1.0;
    P.tau[0] = 0.5; P.tau[1] = 0.6; P.tau[2] = 0.7;
    P.ik[0] = 0.5; P.ik[1] = 1.0 / 3.0; P.ik[2] = 1.0;
    P.dk1 = P.ik[0] - P.ik[2]; P.dk2 = P.ik[1] - P.ik[2];
    P.s12 = 0.011; P.s13 = 0.013; P.s23 = 0.009;
    P.gam[0] = P.s12 + P.s13 - P.s23; P.gam[1] = P.s12 + P.s23 - P.s13; P.gam[2] = P.s13 + P.s23 - P.s12;
    P.eta = 0.004; P.twelve_over_xi = 3.0; P.four_over_xi = 1.0; P.eps_n = 1e-12;
    for (int i = 0; i < 3; i++) P.lap_coef[i] = 0.75 * 4.0 * P.gam[i];
    const double om = 1.0 / 1.4;
    P.om_phi = om; P.keep_phi = 1.0 - om; P.src_phi = 1.0 - 0.5 * om;
    P.H0c = 0.05; P.H0s = 0.02; P.G = 1e-6;
    double worst = 0.0;
    int bad = 0;
    for (int trial = 0; trial < 200; trial++) {
        double in[40];
        double p1 = 0.5 + 0.6 * U(rng), p2 = 0.3 + 0.6 * U(rng);
        if (trial % 4 == 1) { p1 = 1.02; p2 = -0.01; }  // outside the clamp range
        if (trial % 4 == 2) p2 = 0.0;                     // on the clamp edge
        in[0] = p1; in[1] = 0.1 * U(rng); in[2] = 0.1 * U(rng); in[3] = 0.05 * U(rng);
        in[4] = p2; in[5] = 0.1 * U(rng); in[6] = 0.1 * U(rng); in[7] = 0.05 * U(rng);
        if (trial % 8 == 3) { in[5] = 0.0; in[6] = 0.0; }  // vanishing grad phi_2
        in[8] = 0.8 + 0.2 * U(rng); in[9] = 0.05 * U(rng); in[10] = 0.05 * U(rng);
        in[11] = 0.05 * U(rng); in[12] = 0.05 * U(rng);
        for (int a = 0; a < 9; a++) in[13 + a] = 0.01 * U(rng);
        for (int q = 0; q < 18; q++) in[22 + q] = wgt<double>(q % 9) * (q < 9 ? p1 : p2) + 0.01 * U(rng);
        double fb[9], gb[18];
        for (int a = 0; a < 9; a++) fb[a] = U(rng);
        for (int q = 0; q < 18; q++) gb[q] = U(rng);

        NodeFwd<double> F;
        for (int k = 0; k < 40; k++) *input(F, k) = in[k];
        node_forward(F, P);
        NodeBar B;
        double pb[NPB] = {0.0};
        node_reverse(F, P, fb, gb, B, pb);

        for (int k = 0; k < 40 + NPB; k++) {
            NodeFwd<D1> G;
            for (int j = 0; j < 40; j++) *input(G, j) = D1(in[j]);
            Phys<D1> Q;
            to_dual(Q, P);
            if (k < 40) input(G, k)->d[0] = 1.0;
            else constant(Q, k - 40)->d[0] = 1.0;
            node_forward(G, Q);
            double dot = 0.0, mag = 0.0;
            for (int a = 0; a < 9; a++) {
                dot += fb[a] * G.fout[a].d[0];
                mag += std::fabs(fb[a] * G.fout[a].d[0]);
            }
            for (int q = 0; q < 18; q++) {
                dot += gb[q] * G.gout[q].d[0];
                mag += std::fabs(gb[q] * G.gout[q].d[0]);
            }
            const double r = k < 40 ? input_bar(B, k) : pb[k - 40];
            const double err = mag > 0.0 ? std::fabs(r - dot) / mag : std::fabs(r);
            if (err > worst) worst = err;
            if (!(err <= 1e-12)) {
                if (bad < 10) printf("trial %d input %d: reverse %.17g forward %.17g\n", trial, k, r, dot);
                bad++;
            }
        }
    }
    printf("worst relative mismatch %.3e over 200 nodes x 55 inputs\n", worst);
    return bad ? 1 : 0;
}
