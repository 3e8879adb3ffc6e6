// fcd_obs.cu -- observables of the coupled step (arXiv 2410.11129, Sec. 2.5,
// Eqs. 38 and 42): phase masses, indicator-weighted centroids, extents of the
// 1/2 level sets of the shell (phi_1 + phi_2) and the core (phi_1), and the
// breakup test (the core touching the carrier). FP64 throughout; reductions
// run in a fixed order (per column, then one block over the columns) so that
// repeated calls give identical bits.
#include <climits>

#include "fcd_internal.cuh"

namespace fcd {

constexpr int COLS = OBS_COLS;  // per-column record: see obs_columns

template <int MODE>
struct StoreO { using type = float; };
template <>
struct StoreO<MODE_FP64> { using type = double; };

template <typename T, int MODE>
__global__ void obs_phi(Phys<T> P, const void *gv, double *phi1, double *phi2, ObsOut *out) {
    using S = typename StoreO<MODE>::type;
    const S *g = static_cast<const S *>(gv);
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long n = (long long)y * P.pitch + x, m = (long long)y * P.nx + x;
    T p1 = T(0), p2 = T(0);
    for (int a = 0; a < 9; a++) {
        p1 += T(g[a * P.ps + n]) - g_off<MODE, T>(a);
        p2 += T(g[(9 + a) * P.ps + n]) - g_off<MODE, T>(a);
    }
    phi1[m] = double(p1);
    phi2[m] = double(p2);
    if (!(fabs(double(p1)) < 1e300) || !(fabs(double(p2)) < 1e300)) out->nonfinite = 1;
}

__device__ __forceinline__ double c01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

// Core at a node with phi_1 >= 1/2 next to a carrier node (phi_3 >= 1/2)
// inside the channel; smallest y*nx + x wins.
__global__ void obs_touch(int nx, int ny, const double *phi1, const double *phi2, ObsOut *out,
                          int open) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    if (c01(phi1[(long long)y * nx + x]) < 0.5) return;
    for (int a = 1; a < 9; a++) {
        const int yy = y + cy(a);
        if (yy < 0 || yy >= ny) continue;
        int xx = x + cx(a);
        if (open && (xx < 0 || xx >= nx)) continue;  // outside an open channel
        xx = xx < 0 ? nx - 1 : (xx >= nx ? 0 : xx);
        const long long m = (long long)yy * nx + xx;
        if (c01(1.0 - phi1[m] - phi2[m]) >= 0.5) {
            atomicMin(&out->brk_now, (unsigned long long)((long long)y * nx + x));
            return;
        }
    }
}

// First upward and last downward crossing of 1/2 along v[0..n-1] (zero outside).
struct Cross {
    int first, last;
    double lo, hi;
};
template <typename F>
__device__ __forceinline__ Cross crossings(F v, int n) {
    Cross c{-2, -2, 0.0, 0.0};
    for (int i = -1; i < n; i++) {
        const double a = i < 0 ? 0.0 : v(i), b = i + 1 < n ? v(i + 1) : 0.0;
        if (a < 0.5 && b >= 0.5 && c.first == -2) { c.first = i; c.lo = i + (0.5 - a) / (b - a); }
        if (a >= 0.5 && b < 0.5) { c.last = i; c.hi = i + (a - 0.5) / (a - b); }
    }
    return c;
}

// Per column: masses (3), sum so, sum si, sum y*so, sum y*si, vertical extents
// of so and si, centre-line values of so and si.
__global__ void obs_columns(int nx, int ny, const double *phi1, const double *phi2, double *col) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    double m1 = 0, m2 = 0, m3 = 0, so = 0, si = 0, yso = 0, ysi = 0;
    for (int y = 0; y < ny; y++) {
        const double p1 = phi1[(long long)y * nx + x], p2 = phi2[(long long)y * nx + x];
        m1 += p1;
        m2 += p2;
        m3 += 1.0 - p1 - p2;
        const double i1 = c01(p1), o = i1 + c01(p2);
        so += o;
        si += i1;
        yso += y * o;
        ysi += y * i1;
    }
    auto vo = [&](int y) { return c01(phi1[(long long)y * nx + x]) + c01(phi2[(long long)y * nx + x]); };
    auto vi = [&](int y) { return c01(phi1[(long long)y * nx + x]); };
    const Cross co = crossings(vo, ny), ci = crossings(vi, ny);
    double *c = col + (long long)x * COLS;
    c[0] = m1; c[1] = m2; c[2] = m3; c[3] = so; c[4] = si; c[5] = yso; c[6] = ysi;
    c[7] = (co.first != -2 && co.last != -2) ? co.hi - co.lo : 0.0;
    c[8] = (ci.first != -2 && ci.last != -2) ? ci.hi - ci.lo : 0.0;
    if (ny & 1) {
        c[9] = vo(ny / 2);
        c[10] = vi(ny / 2);
    } else {
        c[9] = 0.5 * (vo(ny / 2 - 1) + vo(ny / 2));
        c[10] = 0.5 * (vi(ny / 2 - 1) + vi(ny / 2));
    }
}

constexpr int FIN = 1024;

// Fixed-order block sum of one value per thread.
__device__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = FIN / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}
__device__ double block_max(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = FIN / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// open: the frame starts at the inlet (no periodic seam to cut)
__global__ void __launch_bounds__(FIN) obs_final(int nx, const double *col, ObsOut *out, int open) {
    __shared__ double sh[FIN];
    __shared__ int ish[FIN];
    const int t = threadIdx.x;
    const int chunk = (nx + FIN - 1) / FIN, lo = t * chunk, hi = min(nx, lo + chunk);
    // masses
    for (int q = 0; q < 3; q++) {
        double s = 0;
        for (int x = lo; x < hi; x++) s += col[(long long)x * COLS + q];
        s = block_sum(s, sh);
        if (t == 0) out->mass[q] = s;
    }
    // emptiest column (first of the minima): the seam for the periodic frame
    {
        double best = INFINITY;
        int bi = nx;
        for (int x = lo; x < hi; x++) {
            const double v = col[(long long)x * COLS + 3];
            if (v < best) { best = v; bi = x; }
        }
        sh[t] = best;
        ish[t] = bi;
        __syncthreads();
        for (int s = FIN / 2; s > 0; s >>= 1) {
            if (t < s) {
                const double a = sh[t], b = sh[t + s];
                if (b < a || (b == a && ish[t + s] < ish[t])) { sh[t] = b; ish[t] = ish[t + s]; }
            }
            __syncthreads();
        }
    }
    const int xcut = open ? 0 : ish[0];
    __syncthreads();
    if (t == 0) out->xcut = xcut;
    for (int w = 0; w < 2; w++) {  // 0: shell indicator, 1: core indicator
        double m = 0, mx = 0, my = 0, ly = 0;
        for (int x = lo; x < hi; x++) {
            const double *c = col + (long long)x * COLS;
            const double xu = x >= xcut ? x : x + nx;
            m += c[3 + w];
            mx += xu * c[3 + w];
            my += c[5 + w];
            ly = fmax(ly, c[7 + w]);
        }
        m = block_sum(m, sh);
        mx = block_sum(mx, sh);
        my = block_sum(my, sh);
        ly = block_max(ly, sh);
        // centre-line crossings in the unwrapped frame j = 0..nx-1 (x = xcut + j)
        auto cl = [&](int j) {
            int x = xcut + j;
            x = x >= nx ? x - nx : x;
            return col[(long long)x * COLS + 9 + w];
        };
        int first = INT_MAX, last = -3;
        double flo = 0, lhi = 0;
        const int jhi = min(nx, (t + 1) * chunk);
        for (int i = (t == 0 ? -1 : t * chunk); i < jhi; i++) {
            const double a = i < 0 ? 0.0 : cl(i), b = i + 1 < nx ? cl(i + 1) : 0.0;
            if (a < 0.5 && b >= 0.5 && first == INT_MAX) { first = i; flo = i + (0.5 - a) / (b - a); }
            if (a >= 0.5 && b < 0.5) { last = i; lhi = i + (a - 0.5) / (a - b); }
        }
        // smallest first crossing and largest last crossing over the threads
        ish[t] = first;
        sh[t] = flo;
        __syncthreads();
        for (int s = FIN / 2; s > 0; s >>= 1) {
            if (t < s && ish[t + s] < ish[t]) { ish[t] = ish[t + s]; sh[t] = sh[t + s]; }
            __syncthreads();
        }
        const int gfirst = ish[0];
        const double glo = sh[0];
        __syncthreads();
        ish[t] = last;
        sh[t] = lhi;
        __syncthreads();
        for (int s = FIN / 2; s > 0; s >>= 1) {
            if (t < s && ish[t + s] > ish[t]) { ish[t] = ish[t + s]; sh[t] = sh[t + s]; }
            __syncthreads();
        }
        const int glast = ish[0];
        const double ghi = sh[0];
        __syncthreads();
        if (t == 0) {
            const double lx = (gfirst != INT_MAX && glast != -3) ? ghi - glo : 0.0;
            const double cxv = m > 0.0 ? fmod(mx / m, (double)nx) : 0.0;
            const double cyv = m > 0.0 ? my / m : 0.0;
            if (w == 0) { out->xc_shell = cxv; out->yc_shell = cyv; out->lx_o = lx; out->ly_o = ly; }
            else { out->xc_core = cxv; out->yc_core = cyv; out->lx_i = lx; out->ly_i = ly; }
        }
    }
}

template <typename T>
void launch_observe(int mode, const Phys<T> &P, const void *g, double *scratch, ObsOut *out,
                    cudaStream_t s, int open_x) {
    const long long N = (long long)P.nx * P.ny;
    double *phi1 = scratch, *phi2 = scratch + N, *col = scratch + 2 * N;
    cudaMemsetAsync(out, 0, sizeof(ObsOut), s);
    cudaMemsetAsync(&out->brk_now, 0xff, sizeof(unsigned long long), s);
    dim3 b(32, 8), gr((P.nx + 31) / 32, (P.ny + 7) / 8);
    if constexpr (sizeof(T) == 8) {
        obs_phi<T, MODE_FP64><<<gr, b, 0, s>>>(P, g, phi1, phi2, out);
    } else {
        if (mode == MODE_FP32) obs_phi<T, MODE_FP32><<<gr, b, 0, s>>>(P, g, phi1, phi2, out);
        else obs_phi<T, MODE_FP32_OFFSET><<<gr, b, 0, s>>>(P, g, phi1, phi2, out);
    }
    obs_touch<<<gr, b, 0, s>>>(P.nx, P.ny, phi1, phi2, out, open_x);
    obs_columns<<<(P.nx + 127) / 128, 128, 0, s>>>(P.nx, P.ny, phi1, phi2, col);
    obs_final<<<1, FIN, 0, s>>>(P.nx, col, out, open_x);
}

size_t observe_scratch_doubles(int nx, int ny) { return observe_scratch_doubles_of(nx, ny); }

template void launch_observe<float>(int, const Phys<float> &, const void *, double *, ObsOut *,
                                    cudaStream_t, int);
template void launch_observe<double>(int, const Phys<double> &, const void *, double *,
                                     ObsOut *, cudaStream_t, int);

}  // namespace fcd
