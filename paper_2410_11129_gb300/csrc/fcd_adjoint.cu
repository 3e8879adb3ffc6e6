// fcd_adjoint.cu -- kernels of the discrete adjoint (reverse-mode) step of the
// coupled method (arXiv 2410.11129), FP64, periodic or open channel.
//
// One forward step maps the state (f_n, g_n) to (f_{n+1}, g_{n+1}) through
//   phi_i = sum_a g^i_a (Eq. 32), k = 1/sum_i phi^_i/(1 + chi_i) (Eq. 8),
//   psi' = L(k)^-1 b(k, H0 e_alpha) (Eq. 6, the 9-point link operator),
//   the collision of every node from its 3 x 3 stencil (Eqs. 7-36), push
//   streaming with half-way bounce-back.
// The adjoint step runs it backwards for given adjoints (fb_{n+1}, gb_{n+1}):
//   adj_collide : per node, pull the adjoints of the 27 outgoing populations,
//                 reverse the collision (node_reverse) -> adjoints of f_n, of
//                 the direct g_n term, of the reduced stencil values and of
//                 the constants (accumulated per block);
//   adj_gather  : transposed stencils (with the mirrored wall rows and the
//                 negated psi' ghosts) -> adjoints of phi_1, phi_2 (incl. the
//                 density) and of psi', the right-hand side of L(k) lam = psib
//                 (L is symmetric);
//   multigrid   : the adjoint potential lam (same hierarchy code as the plain
//                 solve, explicit right-hand side);
//   adj_kbar    : kb = (d r / d k)^T lam with r = b(k) - L(k) psi', phib +=
//                 kb dk/dphi, gb_n += phib (Eq. 32 transposed), and the adjoint
//                 of H0 (cos alpha, sin alpha) through b.
// The states of a segment of steps are recomputed from a checkpoint and kept in
// slots (f 9 planes, g 18 planes, psi' 1 plane); the kernels read the slot whose
// index sits in device memory, so one captured graph serves every step.
#include <climits>

#include "fcd_adjoint.cuh"

namespace fcd {

namespace {

constexpr int ATY = 4;  // adjoint collide tile: 32 x 4 nodes

__device__ __forceinline__ int wrapx(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }
__device__ __forceinline__ int mrow(int y, int ny) { return y < 0 ? 0 : (y >= ny ? ny - 1 : y); }

// weights of the reduced stencils on the value at x + e_b (Eqs. 34, 35)
__device__ __forceinline__ double wgx(int b) { return b == 0 ? 0.0 : cx(b) * (b <= 4 ? 1.0 / 3.0 : 1.0 / 12.0); }
__device__ __forceinline__ double wgy(int b) { return b == 0 ? 0.0 : cy(b) * (b <= 4 ? 1.0 / 3.0 : 1.0 / 12.0); }
__device__ __forceinline__ double wlp(int b) { return b == 0 ? -20.0 / 6.0 : (b <= 4 ? 4.0 / 6.0 : 1.0 / 6.0); }

__device__ __forceinline__ const double *slot_base(const double *seg, const int *slot, long long stride) {
    return seg + (long long)(*slot) * stride;
}

template <int NT_>
__device__ __forceinline__ void block_sum_add(double (&v)[NT_], double *acc) {
    __shared__ double red[NT_][32];
    const int t = threadIdx.y * blockDim.x + threadIdx.x, nw = (blockDim.x * blockDim.y + 31) / 32;
#pragma unroll
    for (int k = 0; k < NT_; k++) {
        double s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((t & 31) == 0) red[k][t >> 5] = s;
    }
    __syncthreads();
    if (t < NT_) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += red[t][w];
        acc[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * NT_ + t] += s;
    }
}

// phi_1, phi_2, k of the slot's state
__global__ void __launch_bounds__(256) adj_phase_kernel(Phys<double> P, const double *seg, const int *slot,
                                                        long long stride, double *phi1, double *phi2,
                                                        double *k) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const double *g = slot_base(seg, slot, stride) + 9 * P.ps;
    const long long n = (long long)y * P.pitch + x;
    double p1 = 0.0, p2 = 0.0;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        p1 += g[a * P.ps + n];
        p2 += g[(9 + a) * P.ps + n];
    }
    phi1[n] = p1;
    phi2[n] = p2;
    k[n] = 1.0 / (P.ik[0] * cl01(p1) + P.ik[1] * cl01(p2) + P.ik[2] * cl01(1.0 - p1 - p2));
}

// OPEN: the channel's x ends are an inlet and an outlet: phi-like halo columns
// mirrored there, populations leaving through them dropped (zero adjoint).
template <bool OPEN>
__global__ void __launch_bounds__(TX *ATY) adj_collide_kernel(AdjArgs A) {
    __shared__ double s1[ATY + 2][TX + 2], s2[ATY + 2][TX + 2], sr[ATY + 2][TX + 2], sp[ATY + 2][TX + 2];
    const Phys<double> &P = A.P;
    const int nx = P.nx, ny = P.ny, pitch = P.pitch;
    const long long ps = P.ps;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * ATY;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool live = x < nx && y < ny;
    const long long n = (long long)y * pitch + x;
    const double *sl = slot_base(A.seg, A.slot, A.stride);
    const double *fs = sl, *gs = sl + 9 * ps, *psi = sl + 27 * ps;

    for (int i = threadIdx.y * TX + threadIdx.x; i < (TX + 2) * (ATY + 2); i += TX * ATY) {
        const int lx = i % (TX + 2), ly = i / (TX + 2);
        const int gx = wrapx(x0 - 1 + lx, nx);
        const int gy = y0 - 1 + ly;
        const bool ghost = gy < 0 || gy >= ny;
        const long long m = (long long)mrow(gy, ny) * pitch + gx;
        const int xr = x0 - 1 + lx, gm = xr < 0 ? 0 : (xr >= nx ? nx - 1 : xr);
        const long long mp = OPEN ? (long long)mrow(gy, ny) * pitch + gm : m;
        const double p1 = A.phi1[mp], p2 = A.phi2[mp];
        s1[ly][lx] = p1;
        s2[ly][lx] = p2;
        sr[ly][lx] = P.rho[0] * cl01(p1) + P.rho[1] * cl01(p2) + P.rho[2] * cl01(1.0 - p1 - p2);
        const double q = psi[m];
        sp[ly][lx] = ghost ? -q : q;
    }
    __syncthreads();

    double pacc[NPB];
#pragma unroll
    for (int k = 0; k < NPB; k++) pacc[k] = 0.0;
    if (live) {
        const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
        NodeFwd<double> F;
        auto reduce = [&](const double (*s)[TX + 2], double &c, double &gx, double &gy, double *lp) {
            const double e = s[ly][lx + 1], w = s[ly][lx - 1], nn = s[ly + 1][lx], ss = s[ly - 1][lx];
            const double ne = s[ly + 1][lx + 1], nw = s[ly + 1][lx - 1], sw = s[ly - 1][lx - 1],
                         se = s[ly - 1][lx + 1];
            c = s[ly][lx];
            gx = (e - w) * (1.0 / 3.0) + ((ne - nw) + (se - sw)) * (1.0 / 12.0);
            gy = (nn - ss) * (1.0 / 3.0) + ((ne + nw) - (se + sw)) * (1.0 / 12.0);
            if (lp) *lp = (4.0 * ((e + w) + (nn + ss)) + ((ne + nw) + (se + sw)) - 20.0 * c) * (1.0 / 6.0);
        };
        reduce(s1, F.ph1, F.g1x, F.g1y, &F.l1);
        reduce(s2, F.ph2, F.g2x, F.g2y, &F.l2);
        reduce(sr, F.rho, F.grx, F.gry, nullptr);
        double pc;
        reduce(sp, pc, F.dpx, F.dpy, nullptr);
#pragma unroll
        for (int a = 0; a < 9; a++) F.f[a] = fs[a * ps + n];
#pragma unroll
        for (int q = 0; q < 18; q++) F.g[q] = gs[q * ps + n];
        node_forward(F, P);

        // adjoints of the outgoing populations: where the push put them
        const int dxp = (x == nx - 1) ? 1 - nx : 1, dxm = (x == 0) ? nx - 1 : -1;
        double fb[9], gb[18];
#pragma unroll
        for (int a = 0; a < 9; a++) {
            const bool walled = (cy(a) > 0 && y == ny - 1) || (cy(a) < 0 && y == 0);
            // dropped through an open end (a wall reflection takes precedence, as in the push)
            const bool leaves = OPEN && !walled && ((cx(a) > 0 && x == nx - 1) || (cx(a) < 0 && x == 0));
            const long long d = walled ? n : n + cy(a) * pitch + (cx(a) > 0 ? dxp : (cx(a) < 0 ? dxm : 0));
            const int q = walled ? opp(a) : a;
            fb[a] = leaves ? 0.0 : A.ab_src[q * ps + d];
            gb[a] = leaves ? 0.0 : A.ab_src[(9 + q) * ps + d];
            gb[9 + a] = leaves ? 0.0 : A.ab_src[(18 + q) * ps + d];
        }
        NodeBar B;
        node_reverse(F, P, fb, gb, B, pacc);
#pragma unroll
        for (int a = 0; a < 9; a++) A.ab_dst[a * ps + n] = B.f[a];
#pragma unroll
        for (int q = 0; q < 18; q++) A.ab_dst[(9 + q) * ps + n] = B.g[q];
        const double sv[13] = {B.ph1, B.g1x, B.g1y, B.l1, B.ph2, B.g2x, B.g2y, B.l2,
                               B.rho, B.grx, B.gry, B.dpx, B.dpy};
#pragma unroll
        for (int q = 0; q < 13; q++) A.sb[q * ps + n] = sv[q];
    }
    block_sum_add<NPB>(pacc, A.pacc);
}

// Transposed stencils: the node at m receives, from every node s whose stencil
// read it, the adjoint of that read. Rows: s = m - e_b, and at a wall row also
// the node whose ghost row mirrors onto m (negated for psi'). Columns: periodic,
// or in the open channel (OPEN) s = m - e_b inside and, at an end column, the
// node whose ghost column mirrors onto m (phi-like fields only; psi' stays
// periodic in x).
template <bool OPEN>
__global__ void __launch_bounds__(256) adj_gather_kernel(Phys<double> P, const double *sb, const double *phi1,
                                                         const double *phi2, double *pb, double *rhs,
                                                         unsigned long long *rmax) {
    const int nx = P.nx, ny = P.ny, pitch = P.pitch;
    const long long ps = P.ps;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    double ar = 0.0;
    if (x < nx && y < ny) {
        double b1 = 0.0, b2 = 0.0, br = 0.0, bp = 0.0;
        auto add_phi = [&](long long s, int b) {
            const double wx = wgx(b), wy = wgy(b), wl = wlp(b), wc = b == 0 ? 1.0 : 0.0;
            b1 += sb[0 * ps + s] * wc + sb[1 * ps + s] * wx + sb[2 * ps + s] * wy + sb[3 * ps + s] * wl;
            b2 += sb[4 * ps + s] * wc + sb[5 * ps + s] * wx + sb[6 * ps + s] * wy + sb[7 * ps + s] * wl;
            br += sb[8 * ps + s] * wc + sb[9 * ps + s] * wx + sb[10 * ps + s] * wy;
        };
        auto add_psi = [&](long long s, int b, double sign) {
            bp += sign * (sb[11 * ps + s] * wgx(b) + sb[12 * ps + s] * wgy(b));
        };
#pragma unroll
        for (int b = 0; b < 9; b++) {
            // source rows: the plain neighbour, and the mirror of a ghost row
            int ys[2], nys = 0;
            bool ghost_row[2];
            if (y - cy(b) >= 0 && y - cy(b) < ny) { ys[nys] = y - cy(b); ghost_row[nys++] = false; }
            if ((y == 0 && cy(b) < 0) || (y == ny - 1 && cy(b) > 0)) { ys[nys] = y; ghost_row[nys++] = true; }
            // source columns of the phi-like fields
            int xs[2], nxs = 0;
            if (OPEN) {
                if (x - cx(b) >= 0 && x - cx(b) < nx) xs[nxs++] = x - cx(b);
                if ((x == 0 && cx(b) < 0) || (x == nx - 1 && cx(b) > 0)) xs[nxs++] = x;
            } else {
                xs[nxs++] = wrapx(x - cx(b), nx);
            }
            const int xp = wrapx(x - cx(b), nx);  // psi' is periodic in x
            for (int j = 0; j < nys; j++) {
                for (int i = 0; i < nxs; i++) add_phi((long long)ys[j] * pitch + xs[i], b);
                add_psi((long long)ys[j] * pitch + xp, b, ghost_row[j] ? -1.0 : 1.0);
            }
        }
        const long long m = (long long)y * pitch + x;
        const double p1 = phi1[m], p2 = phi2[m], d3 = dcl01(1.0 - p1 - p2);
        pb[m] = b1 + br * (P.rho[0] * dcl01(p1) - P.rho[2] * d3);
        pb[ps + m] = b2 + br * (P.rho[1] * dcl01(p2) - P.rho[2] * d3);
        rhs[m] = bp;
        ar = fabs(bp);
        ar = ar == ar ? ar : INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) ar = fmax(ar, __shfl_xor_sync(0xffffffffu, ar, o));
    if (((threadIdx.y * blockDim.x + threadIdx.x) & 31) == 0 && ar > 0.0)
        atomicMax(rmax, (unsigned long long)__double_as_longlong(ar));
}

// Open channel: transpose of the boundary kernel that follows the collision
// (the Eq. 37 Zou-He inlet and the convective outlet, linear in the populations
// with constant coefficients, so no forward values are needed). In place on the
// adjoint after the step, one thread per row: the adjoints of the values the
// boundary overwrote go to the values they were computed from and become 0;
// the outlet's dependence on the state before the step goes to `keep`
// (27 values per row), added to the adjoint before the step by adj_open_add.
__global__ void adj_open_bc_kernel(Phys<double> P, double *ab, double *keep, double u_avg) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    if (y >= ny) return;
    const long long ps = P.ps, n = (long long)y * P.pitch, o = n + nx - 1, bn = o - 1;
    auto FA = [&](int a, long long m) -> double & { return ab[a * ps + m]; };
    auto GA = [&](int q, int a, long long m) -> double & { return ab[(9 + q * 9 + a) * ps + m]; };
    // inlet: reverse of the assignments (last first)
    double f1 = FA(1, n);
    FA(1, n) = 0.0;
    if (y == 0 || y == ny - 1) {  // f1 = u + f3 - f5 + f6 + f7 - f8
        FA(3, n) += f1;
        FA(5, n) -= f1;
        FA(6, n) += f1;
        FA(7, n) += f1;
        FA(8, n) -= f1;
    } else {  // f1 = f3 + 6 w1 u
        FA(3, n) += f1;
    }
    if (y == 0) {  // f8 = f2 - f4 + f5 + f6 - f7
        const double f8 = FA(8, n);
        FA(8, n) = 0.0;
        FA(2, n) += f8;
        FA(4, n) -= f8;
        FA(5, n) += f8;
        FA(6, n) += f8;
        FA(7, n) -= f8;
    } else if (y == ny - 1) {  // f5 = f4 - f2 - f6 + f7 + f8
        const double f5 = FA(5, n);
        FA(5, n) = 0.0;
        FA(4, n) += f5;
        FA(2, n) -= f5;
        FA(6, n) -= f5;
        FA(7, n) += f5;
        FA(8, n) += f5;
    } else {  // f5 = f7 + c - (f2 - f4)/2, f8 = f6 + c + (f2 - f4)/2
        const double f5 = FA(5, n), f8 = FA(8, n);
        FA(5, n) = 0.0;
        FA(8, n) = 0.0;
        FA(7, n) += f5;
        FA(6, n) += f8;
        FA(2, n) += 0.5 * (f8 - f5);
        FA(4, n) += 0.5 * (f5 - f8);
    }
    for (int q = 0; q < 2; q++) {  // inflowing phase-field populations are constants
        GA(q, 1, n) = 0.0;
        if (y != 0) GA(q, 5, n) = 0.0;
        if (y != ny - 1) GA(q, 8, n) = 0.0;
    }
    // outlet: chi_a = ((f_a - w_a p*)(t) + U (f_a - w_a p*)_{nx-2}(t+1)) / (1 + U)
    double *kf = keep + (long long)y * 27, *kg = kf + 9;
    for (int a = 0; a < 27; a++) kf[a] = 0.0;
    const double iu = 1.0 / (1.0 + u_avg);
    const int in3[3] = {3, 6, 7};
    for (int k = 0; k < 3; k++) {
        const int a = in3[k];
        if ((a == 6 && y == 0) || (a == 7 && y == ny - 1)) continue;  // from the wall
        const double s = FA(a, o) * iu;
        FA(a, o) = 0.0;
        kf[a] += s;
        FA(a, bn) += u_avg * s;
        const double w = wgt<double>(a);
        for (int c = 0; c < 9; c++) {
            kf[c] -= w * s;
            FA(c, bn) -= u_avg * w * s;
        }
        for (int q = 0; q < 2; q++) {
            const double sg = GA(q, a, o) * iu;
            GA(q, a, o) = 0.0;
            kg[q * 9 + a] += sg;
            GA(q, a, bn) += u_avg * sg;
        }
    }
}

// the outlet column's share of the adjoint before the step (see adj_open_bc)
__global__ void adj_open_add_kernel(Phys<double> P, const double *keep, double *ab) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= P.ny) return;
    const long long o = (long long)y * P.pitch + P.nx - 1;
    for (int q = 0; q < 27; q++) ab[q * P.ps + o] += keep[(long long)y * 27 + q];
}

// kb, the adjoint of H0 (cos, sin) through the right-hand side, and the
// phase-field adjoint added to every population of g_n.
__global__ void __launch_bounds__(256) adj_kbar_kernel(AdjKArgs A) {
    const Phys<double> &P = A.P;
    const int nx = P.nx, ny = P.ny, pitch = P.pitch;
    const long long ps = P.ps;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    double hacc[2] = {0.0, 0.0};
    if (x < nx && y < ny) {
        const long long m = (long long)y * pitch + x;
        double phb1 = A.pb[m], phb2 = A.pb[ps + m];
        if (A.ctl) {
            const double *lam = A.ctl->cur ? A.lamB : A.lamA;
            const double *psi = slot_base(A.seg, A.slot, A.stride) + 27 * ps;
            const double H0c = P.H0c, H0s = P.H0s;
            auto at = [&](const double *p, int xx, int yy) { return p[(long long)yy * pitch + wrapx(xx, nx)]; };
            const double psm = psi[m], lm = lam[m], km = A.k[m];
            double kb = 0.0, bx = 0.0, by = 0.0;
#pragma unroll
            for (int a = 1; a < 9; a++) {
                const double w3 = 3.0 * wgt<double>(a), eh = cx(a) * H0c + cy(a) * H0s;
                const int yy = y + cy(a);
                const bool gh = yy < 0 || yy >= ny;
                // this node's own residual
                const double pn = at(psi, x + cx(a), gh ? y : yy);
                kb += lm * w3 * (eh - (gh ? -pn : pn) + psm);
                const double kn = at(A.k, x + cx(a), gh ? y : yy);
                const double ca = w3 * (km + kn);
                bx += ca * cx(a);
                by += ca * cy(a);
                // the residual of the node n = m - e_a, whose link a reaches m
                const int sy = y - cy(a);
                if (sy >= 0 && sy < ny)
                    kb += at(lam, x - cx(a), sy) * w3 * (eh - psm + at(psi, x - cx(a), sy));
                // wall rows: the node whose ghost link a mirrors onto m
                if (gh) kb += at(lam, x - cx(a), y) * w3 * (eh + psm + at(psi, x - cx(a), y));
            }
            hacc[0] = lm * bx;
            hacc[1] = lm * by;
            const double p1 = A.phi1[m], p2 = A.phi2[m], d3 = dcl01(1.0 - p1 - p2);
            const double k2 = km * km;
            phb1 -= kb * k2 * (P.ik[0] * dcl01(p1) - P.ik[2] * d3);
            phb2 -= kb * k2 * (P.ik[1] * dcl01(p2) - P.ik[2] * d3);
        }
        double *gbn = A.ab + 9 * ps;
#pragma unroll
        for (int a = 0; a < 9; a++) {
            gbn[a * ps + m] += phb1;
            gbn[(9 + a) * ps + m] += phb2;
        }
    }
    block_sum_add<2>(hacc, A.hacc);
}

__global__ void set_slot_kernel(int *slot, int v) { *slot = v; }
__global__ void dec_slot_kernel(int *slot) { *slot -= 1; }

// ---------------------------------------------------------------- seeds
constexpr int SOB = 1024;

struct Cross {
    int first, last;
    double lo, hi;
    double alo, blo, ahi, bhi;  // the values either side of each crossing
};

__device__ __forceinline__ void cross_step(Cross &c, int i, double a, double b) {
    if (a < 0.5 && b >= 0.5 && c.first == -2) {
        c.first = i;
        c.lo = double(i) + (0.5 - a) / (b - a);
        c.alo = a;
        c.blo = b;
    }
    if (a >= 0.5 && b < 0.5) {
        c.last = i;
        c.hi = double(i) + (a - 0.5) / (a - b);
        c.ahi = a;
        c.bhi = b;
    }
}

// d lo / d(a, b) and d hi / d(a, b) of a crossing pair
__device__ __forceinline__ void cross_grad(const Cross &c, double *dlo, double *dhi) {
    const double r = c.blo - c.alo, q = c.ahi - c.bhi;
    dlo[0] = (0.5 - c.blo) / (r * r);
    dlo[1] = -(0.5 - c.alo) / (r * r);
    dhi[0] = (0.5 - c.bhi) / (q * q);
    dhi[1] = (c.ahi - 0.5) / (q * q);
}

__device__ __forceinline__ double indicator(const double *phi1, const double *phi2, long long n) {
    return cl01(phi1[n]) + cl01(phi2[n]);
}

// Adjoint of J = wT T_o + wO sum_nodes phi_1 phi_3 (unclamped) at the current
// state: T_o (Eq. 42) as the plain observables measure it (l_y the largest
// vertical 1/2-extent of phi^_1 + phi^_2, first column among equal maxima; l_x
// from the centre-line crossings in the frame that starts at column xcut).
// Writes the T_o part into pb (zeroed before); the overlap part is added by
// adj_seed_bcast.
__global__ void __launch_bounds__(SOB) adj_seed_obs_kernel(int nx, int ny, int pitch, long long ps,
                                                           const double *phi1, const double *phi2,
                                                           const ObsOut *prim, double wT, double *ext,
                                                           double *cl, double *pb, AdjOut *out) {
    __shared__ double sv[SOB];
    __shared__ int si[SOB];
    __shared__ double sred[SOB / 32];
    const int t = threadIdx.x;
    double ovl = 0.0;
    for (int x = t; x < nx; x += SOB) {
        Cross c{-2, -2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double a = 0.0, mid = 0.0;
        for (int i = -1; i < ny; i++) {
            double b = 0.0;
            if (i + 1 < ny) {
                const long long n = (long long)(i + 1) * pitch + x;
                b = indicator(phi1, phi2, n);
                const double p1 = phi1[n], p2 = phi2[n];
                ovl += p1 * (1.0 - p1 - p2);
                const int yy = i + 1;
                if ((ny & 1) ? yy == ny / 2 : (yy == ny / 2 - 1 || yy == ny / 2)) mid += b;
            }
            cross_step(c, i, a, b);
            a = b;
        }
        ext[x] = (c.first != -2 && c.last != -2) ? c.hi - c.lo : 0.0;
        cl[x] = (ny & 1) ? mid : 0.5 * mid;
    }
    __syncthreads();
    {
        double best = -1.0;
        int bi = INT_MAX;
        for (int x = t; x < nx; x += SOB)
            if (ext[x] > best) { best = ext[x]; bi = x; }
        sv[t] = best;
        si[t] = bi;
        __syncthreads();
        for (int s = SOB / 2; s > 0; s >>= 1) {
            if (t < s && (sv[t + s] > sv[t] || (sv[t + s] == sv[t] && si[t + s] < si[t]))) {
                sv[t] = sv[t + s];
                si[t] = si[t + s];
            }
            __syncthreads();
        }
    }
    for (int o = 16; o > 0; o >>= 1) ovl += __shfl_down_sync(0xffffffffu, ovl, o);
    if ((t & 31) == 0) sred[t / 32] = ovl;
    __syncthreads();
    if (t != 0) return;
    double tot = 0.0;
    for (int w = 0; w < SOB / 32; w++) tot += sred[w];
    // l_y again at the chosen column, keeping the crossing rows
    const int xs = si[0];
    Cross cy_{-2, -2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (xs < nx) {
        double a = 0.0;
        for (int i = -1; i < ny; i++) {
            const double b = i + 1 < ny ? indicator(phi1, phi2, (long long)(i + 1) * pitch + xs) : 0.0;
            cross_step(cy_, i, a, b);
            a = b;
        }
    }
    const bool hy = xs < nx && cy_.first != -2 && cy_.last != -2;
    const double ly = hy ? cy_.hi - cy_.lo : 0.0;
    // l_x along the centre line, unwrapped from column xcut
    const int xcut = prim->xcut;
    auto colx = [&](int j) { int xx = xcut + j; return xx >= nx ? xx - nx : xx; };
    Cross cx_{-2, -2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = -1; i < nx; i++) {
        const double a = i < 0 ? 0.0 : cl[colx(i)], b = i + 1 < nx ? cl[colx(i + 1)] : 0.0;
        cross_step(cx_, i, a, b);
    }
    const bool hx = cx_.first != -2 && cx_.last != -2;
    const double lx = hx ? cx_.hi - cx_.lo : 0.0;
    const double sum = lx + ly;
    const double To = sum > 0.0 ? (ly - lx) / sum : 0.0;
    out->T_o = To;
    out->overlap = tot;
    out->lx = lx;
    out->ly = ly;
    if (!(sum > 0.0) || wT == 0.0) return;
    const double lyb = wT * 2.0 * lx / (sum * sum), lxb = -wT * 2.0 * ly / (sum * sum);
    // seed the indicator adjoint at (column, row) onto phi_1, phi_2
    auto seed = [&](int xx, int yy, double v) {
        if (yy < 0 || yy >= ny || v == 0.0) return;
        const long long n = (long long)yy * pitch + xx;
        pb[n] += v * dcl01(phi1[n]);
        pb[ps + n] += v * dcl01(phi2[n]);
    };
    double dlo[2], dhi[2];
    if (hy) {
        cross_grad(cy_, dlo, dhi);
        seed(xs, cy_.first, -lyb * dlo[0]);
        seed(xs, cy_.first + 1, -lyb * dlo[1]);
        seed(xs, cy_.last, lyb * dhi[0]);
        seed(xs, cy_.last + 1, lyb * dhi[1]);
    }
    if (hx) {
        cross_grad(cx_, dlo, dhi);
        auto seed_cl = [&](int j, double v) {
            if (j < 0 || j >= nx) return;
            const int xx = colx(j);
            if (ny & 1) {
                seed(xx, ny / 2, v);
            } else {
                seed(xx, ny / 2 - 1, 0.5 * v);
                seed(xx, ny / 2, 0.5 * v);
            }
        };
        seed_cl(cx_.first, -lxb * dlo[0]);
        seed_cl(cx_.first + 1, -lxb * dlo[1]);
        seed_cl(cx_.last, lxb * dhi[0]);
        seed_cl(cx_.last + 1, lxb * dhi[1]);
    }
}

// adjoint state at the final step: fb = 0, gb^i_a = phib_i (+ the overlap part)
__global__ void __launch_bounds__(256) adj_seed_bcast_kernel(Phys<double> P, const double *phi1,
                                                             const double *phi2, const double *pb,
                                                             double wO, double *ab) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long ps = P.ps, m = (long long)y * P.pitch + x;
    const double p1 = phi1[m], p2 = phi2[m];
    const double b1 = pb[m] + wO * (1.0 - 2.0 * p1 - p2), b2 = pb[ps + m] - wO * p1;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        ab[a * ps + m] = 0.0;
        ab[(9 + a) * ps + m] = b1;
        ab[(18 + a) * ps + m] = b2;
    }
}

inline dim3 grid2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

}  // namespace

int adj_collide_blocks(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + ATY - 1) / ATY); }
int adj_kbar_blocks(int nx, int ny) { return ((nx + 31) / 32) * ((ny + 7) / 8); }
size_t adj_seed_scratch_bytes(int nx) { return 2ull * nx * sizeof(double); }

void launch_adj_phase(const Phys<double> &P, const double *seg, const int *slot, long long stride,
                      double *phi1, double *phi2, double *k, cudaStream_t s) {
    dim3 b(32, 8);
    adj_phase_kernel<<<grid2(P.nx, P.ny, b), b, 0, s>>>(P, seg, slot, stride, phi1, phi2, k);
}

void launch_adj_collide(const AdjArgs &a, int open_x, cudaStream_t s) {
    dim3 b(TX, ATY);
    if (open_x) adj_collide_kernel<true><<<grid2(a.P.nx, a.P.ny, b), b, 0, s>>>(a);
    else adj_collide_kernel<false><<<grid2(a.P.nx, a.P.ny, b), b, 0, s>>>(a);
}

void launch_adj_gather(const Phys<double> &P, const double *sb, const double *phi1, const double *phi2,
                       double *pb, double *rhs, unsigned long long *rmax, int open_x, cudaStream_t s) {
    dim3 b(32, 8);
    cudaMemsetAsync(rmax, 0, sizeof(unsigned long long), s);
    if (open_x) adj_gather_kernel<true><<<grid2(P.nx, P.ny, b), b, 0, s>>>(P, sb, phi1, phi2, pb, rhs, rmax);
    else adj_gather_kernel<false><<<grid2(P.nx, P.ny, b), b, 0, s>>>(P, sb, phi1, phi2, pb, rhs, rmax);
}

void launch_adj_open_bc(const Phys<double> &P, double *ab, double *keep, double u_avg, cudaStream_t s) {
    adj_open_bc_kernel<<<(P.ny + 63) / 64, 64, 0, s>>>(P, ab, keep, u_avg);
}

void launch_adj_open_add(const Phys<double> &P, const double *keep, double *ab, cudaStream_t s) {
    adj_open_add_kernel<<<(P.ny + 63) / 64, 64, 0, s>>>(P, keep, ab);
}

void launch_adj_kbar(const AdjKArgs &a, cudaStream_t s) {
    dim3 b(32, 8);
    adj_kbar_kernel<<<grid2(a.P.nx, a.P.ny, b), b, 0, s>>>(a);
}

void launch_set_slot(int *slot, int v, cudaStream_t s) { set_slot_kernel<<<1, 1, 0, s>>>(slot, v); }
void launch_dec_slot(int *slot, cudaStream_t s) { dec_slot_kernel<<<1, 1, 0, s>>>(slot); }

void launch_adj_seed(const Phys<double> &P, const double *phi1, const double *phi2, const ObsOut *prim,
                     double wT, double wO, void *scratch, double *pb, double *ab, AdjOut *out,
                     cudaStream_t s) {
    double *ext = static_cast<double *>(scratch), *cl = ext + P.nx;
    cudaMemsetAsync(pb, 0, 2 * P.ps * sizeof(double), s);
    adj_seed_obs_kernel<<<1, SOB, 0, s>>>(P.nx, P.ny, P.pitch, P.ps, phi1, phi2, prim, wT, ext, cl, pb, out);
    dim3 b(32, 8);
    adj_seed_bcast_kernel<<<grid2(P.nx, P.ny, b), b, 0, s>>>(P, phi1, phi2, pb, wO, ab);
}

}  // namespace fcd
