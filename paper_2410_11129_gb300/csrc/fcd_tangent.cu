// fcd_tangent.cu -- kernels of the tangent-linear (forward-mode) step that are
// not shared with the plain step: the derivative planes of Eq. 32, Eq. 8 and
// the derivatives of the shell deformation T_o (Eq. 42) and of the core-carrier
// overlap sum_nodes phi_1 phi_3 (a smooth proxy of breakup, which happens when
// the core touches the carrier; unclamped fields, so that the sum is a
// polynomial of the state: the clamped product has a kink at every bulk node
// where phi sits at 0 or 1 up to round-off).
//
// Layout: every field plane set of the tangent context holds the primal value
// followed by NT tangent copies; copy c of plane q of an np-plane set sits
// (np * c + q) planes from the base.
#include <climits>

#include "fcd_internal.cuh"

namespace fcd {

namespace {

__device__ __forceinline__ DualT ld_copies(const double *p, int q, int np, long long ps,
                                           long long n) {
    DualT r(p[q * ps + n]);
#pragma unroll
    for (int c = 0; c < NT; c++) r.d[c] = p[(np * (c + 1) + q) * ps + n];
    return r;
}

// phi_i = sum_a g^i_a and k = 1 / sum_i phi^_i / (1 + chi_i): derivative planes
// only (the primal planes come from the plain phase kernel).
__global__ void __launch_bounds__(256) tangent_phase_kernel(Phys<double> P, const double *g,
                                                            double *phi1, double *phi2, double *k) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long ps = P.ps, n = (long long)y * P.pitch + x;
    DualT p1(0.0), p2(0.0);
#pragma unroll
    for (int a = 0; a < 9; a++) {
        p1 += ld_copies(g, a, 18, ps, n);
        p2 += ld_copies(g, 9 + a, 18, ps, n);
    }
    const DualT kk = DualT(1.0) / (P.ik[0] * clamp01(p1) + P.ik[1] * clamp01(p2) +
                                   P.ik[2] * clamp01(DualT(1.0) - p1 - p2));
#pragma unroll
    for (int c = 0; c < NT; c++) {
        phi1[(c + 1) * ps + n] = p1.d[c];
        phi2[(c + 1) * ps + n] = p2.d[c];
        k[(c + 1) * ps + n] = kk.d[c];
    }
}

constexpr int TOB = 1024;

// First upward and last downward crossing of 1/2 (zero outside the range),
// with derivatives: lo = i + (1/2 - a)/(b - a), hi = i + (a - 1/2)/(a - b).
struct DCross {
    int first, last;
    DualT lo, hi;
};

__device__ __forceinline__ void cross_step(DCross &c, int i, const DualT &a, const DualT &b) {
    if (a < 0.5 && b >= 0.5 && c.first == -2) {
        c.first = i;
        c.lo = double(i) + (0.5 - a) / (b - a);
    }
    if (a >= 0.5 && b < 0.5) {
        c.last = i;
        c.hi = double(i) + (a - 0.5) / (a - b);
    }
}

__device__ __forceinline__ DualT node_phi(const double *g, int base, long long ps, long long n) {
    DualT p(0.0);
    for (int a = 0; a < 9; a++) p += ld_copies(g, base + a, 18, ps, n);
    return p;
}

// One block. Per column: the vertical 1/2-extent of the shell indicator
// phi^_1 + phi^_2 and its centre-line value; then l_y = the largest extent
// (first column among equal maxima), l_x from the centre-line crossings in the
// frame that starts at the emptiest column found by the plain observables, and
// T_o = (l_y - l_x) / (l_y + l_x).
__global__ void __launch_bounds__(TOB) tangent_obs_kernel(int nx, int ny, int pitch, long long ps,
                                                          const double *g, const ObsOut *prim,
                                                          DualT *ext, DualT *cl, TanOut *out) {
    __shared__ double sv[TOB];
    __shared__ int si[TOB];
    __shared__ DualT sred[TOB / 32];
    const int t = threadIdx.x;
    DualT ovl(0.0);
    for (int x = t; x < nx; x += TOB) {
        DCross c{-2, -2, DualT(0.0), DualT(0.0)};
        DualT a(0.0), mid(0.0);
        for (int i = -1; i < ny; i++) {
            DualT b(0.0);
            if (i + 1 < ny) {
                const long long n = (long long)(i + 1) * pitch + x;
                const DualT p1 = node_phi(g, 0, ps, n), p2 = node_phi(g, 9, ps, n);
                b = clamp01(p1) + clamp01(p2);
                ovl += p1 * (DualT(1.0) - p1 - p2);
                const int y = i + 1;
                if ((ny & 1) ? y == ny / 2 : (y == ny / 2 - 1 || y == ny / 2)) mid += b;
            }
            cross_step(c, i, a, b);
            a = b;
        }
        ext[x] = (c.first != -2 && c.last != -2) ? c.hi - c.lo : DualT(0.0);
        cl[x] = (ny & 1) ? mid : 0.5 * mid;
    }
    __syncthreads();
    // l_y: argmax over the columns
    {
        double best = -1.0;
        int bi = INT_MAX;
        for (int x = t; x < nx; x += TOB)
            if (ext[x].v > best) { best = ext[x].v; bi = x; }
        sv[t] = best;
        si[t] = bi;
        __syncthreads();
        for (int s = TOB / 2; s > 0; s >>= 1) {
            if (t < s && (sv[t + s] > sv[t] || (sv[t + s] == sv[t] && si[t + s] < si[t]))) {
                sv[t] = sv[t + s];
                si[t] = si[t + s];
            }
            __syncthreads();
        }
    }
    // overlap: fixed-order reduction (warp, then the warps in order)
    for (int o = 16; o > 0; o >>= 1) {
        DualT other;
        other.v = __shfl_down_sync(0xffffffffu, ovl.v, o);
#pragma unroll
        for (int c = 0; c < NT; c++) other.d[c] = __shfl_down_sync(0xffffffffu, ovl.d[c], o);
        ovl += other;
    }
    if ((t & 31) == 0) sred[t / 32] = ovl;
    __syncthreads();
    if (t == 0) {
        DualT tot(0.0);
        for (int w = 0; w < TOB / 32; w++) tot += sred[w];
        const DualT ly = si[0] < nx ? ext[si[0]] : DualT(0.0);
        // l_x along the centre line, unwrapped from the emptiest column
        const int xcut = prim->xcut;
        auto clv = [&](int j) {
            int x = xcut + j;
            x = x >= nx ? x - nx : x;
            return cl[x];
        };
        DCross c{-2, -2, DualT(0.0), DualT(0.0)};
        for (int i = -1; i < nx; i++) {
            const DualT a = i < 0 ? DualT(0.0) : clv(i), b = i + 1 < nx ? clv(i + 1) : DualT(0.0);
            cross_step(c, i, a, b);
        }
        const DualT lx = (c.first != -2 && c.last != -2) ? c.hi - c.lo : DualT(0.0);
        const DualT To = (lx.v + ly.v) > 0.0 ? (ly - lx) / (ly + lx) : DualT(0.0);
        out->T_o = To.v;
        out->overlap = tot.v;
        out->lx = lx.v;
        out->ly = ly.v;
        for (int q = 0; q < NT; q++) {
            out->dT_o[q] = To.d[q];
            out->doverlap[q] = tot.d[q];
            out->dlx[q] = lx.d[q];
            out->dly[q] = ly.d[q];
        }
    }
}

}  // namespace

void launch_tangent_phase(const Phys<double> &P, const double *g, double *phi1, double *phi2,
                          double *k, cudaStream_t s) {
    dim3 b(32, 8), gr((P.nx + 31) / 32, (P.ny + 7) / 8);
    tangent_phase_kernel<<<gr, b, 0, s>>>(P, g, phi1, phi2, k);
}

size_t tangent_obs_scratch_bytes(int nx) { return 2ull * nx * sizeof(DualT); }

void launch_tangent_obs(const Phys<double> &P, const double *g, const ObsOut *prim, void *scratch,
                        TanOut *out, cudaStream_t s) {
    DualT *ext = static_cast<DualT *>(scratch), *cl = ext + P.nx;
    tangent_obs_kernel<<<1, TOB, 0, s>>>(P.nx, P.ny, P.pitch, P.ps, g, prim, ext, cl, out);
}

}  // namespace fcd
