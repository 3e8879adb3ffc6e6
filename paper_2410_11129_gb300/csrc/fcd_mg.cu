// fcd_mg.cu -- multigrid solve of the magnetic scalar potential (arXiv 2410.11129,
// Sec. 2.1, Eqs. 5-8): div[(1 + chi) grad psi] = 0, psi = psi0 + psi',
// psi0 = -H0 (x cos(alpha) + y sin(alpha)), periodic in x, psi' = 0 on the
// half-way wall faces.
//
// Level 0 is the lattice itself with the isotropic 9-point link operator
//   (L psi)_0 = 6 sum_a w_a (k_0 + k_a)/2 (psi_a - psi_0)
// (for uniform k it is k times the Laplacian of Eq. 35). The right-hand side
// -L psi0 = 6 H0 sum_a w_a k_0a (e_a . e_alpha) is formed on the fly from k.
// Coarser levels merge cells in pairs (the last three when a count is odd),
// giving tensor grids of any size, and carry a 5-point finite-volume operator
// with arithmetic face permeabilities. Cycles are V(0, 2) on level 0 and V(2, 2)
// below; residuals are summed onto the coarse cells and corrections are
// interpolated bilinearly between cell centres (zero on the walls).
//
// Level 0 is smoothed by block Gauss-Seidel: each 32 x 8 tile loads its cells
// with a one-cell frozen halo into shared memory, adds the interpolated coarse
// correction, runs four-colour sweeps and writes the other buffer. Coarse levels
// above a size threshold run colour passes over the whole grid; the remaining
// small levels run inside one 1024-thread block. Every kernel reads the control
// block and returns at once when the cycle is not needed, so the cycle loop can
// live in a CUDA-graph while node (the last kernel sets the loop condition) or
// be driven from the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fcd_internal.cuh"

namespace fcd {

constexpr int SX = 32, SY = 8;     // level-0 smoothing tile
constexpr int CTA_THREADS = 1024;
constexpr int NU_PRE = 2, NU_POST = 2, NU_FINE = 2, NU_COARSEST = 24;

__device__ __forceinline__ double norm_of(const MgCtl *c) {
    return __longlong_as_double((long long)c->norm_bits);
}
// The rest of a cycle is skipped once the solve is done, the residual of
// this cycle met the tolerance, or the cycle cap was reached.
__device__ __forceinline__ bool cycle_skip(const MgCtl *c) {
    return c->done || norm_of(c) <= c->tolH0 || c->iter >= c->max_iter;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// ------------------------------------------------------------------ level 0
// Coefficients of the 9-point operator at lattice node (x, y); neighbours in
// ghost rows mirror k and negate psi'.
template <typename T>
struct Node9 {
    T c[9];       // c_a = 6 w_a (k_0 + k_a)/2, a = 1..8
    T diag;       // sum_a c_a + the coefficient whose ghost mirrors the node itself
    T b;          // right-hand side -L psi0
};

template <typename T, typename KF>
__device__ __forceinline__ Node9<T> node9(KF kat, int y, int ny, T H0c, T H0s) {
    Node9<T> n;
    const T k0 = kat(0, 0);
    n.diag = T(0);
    n.b = T(0);
#pragma unroll
    for (int a = 1; a < 9; a++) {
        const T ca = T(6) * wgt<T>(a) * T(0.5) * (k0 + kat(cx(a), cy(a)));
        n.c[a] = ca;
        n.diag += ca;
        n.b += ca * (T(cx(a)) * H0c + T(cy(a)) * H0s);
        const int yy = y + cy(a);
        if ((yy < 0 || yy >= ny) && cx(a) == 0) n.diag += ca;  // psi'(ghost) = -psi'(node)
    }
    return n;
}

// sum of c_a * psi~_a over neighbours that are not the node itself
template <typename T, typename PF>
__device__ __forceinline__ T off9(const Node9<T> &n, PF pat, int y, int ny) {
    T s = T(0);
#pragma unroll
    for (int a = 1; a < 9; a++) {
        const int yy = y + cy(a);
        if (yy < 0 || yy >= ny) {
            if (cx(a) != 0) s -= n.c[a] * pat(cx(a), 0);  // mirror of a diagonal ghost
        } else {
            s += n.c[a] * pat(cx(a), cy(a));
        }
    }
    return s;
}

template <typename T>
__device__ __forceinline__ T interp_coarse(const Level<T> &F, const Level<T> &C, int i, int j) {
    const int x0 = F.px0[i], x1 = F.px1[i];
    const T wx = F.pwx[i];
    const int y0 = F.py0[j], y1 = F.py1[j];
    const T wy = F.pwy[j];
    T a = T(0), b = T(0);
    if (y0 >= 0) a = (T(1) - wx) * C.e[(long long)y0 * C.pitch + x0] + wx * C.e[(long long)y0 * C.pitch + x1];
    if (y1 >= 0) b = (T(1) - wx) * C.e[(long long)y1 * C.pitch + x0] + wx * C.e[(long long)y1 * C.pitch + x1];
    return (T(1) - wy) * a + wy * b;
}

// Residual of level 0 on the children of each level-1 cell, summed onto it;
// the max-norm over the lattice goes to the control block. Also clears e_1.
template <typename T>
__global__ void __launch_bounds__(256) resid0_restrict(Level<T> L0, Level<T> L1, T H0c, T H0s,
                                                       MgCtl *ctl) {
    if (ctl->done) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    double mx = 0.0;
    if (I < L1.nx && J < L1.ny) {
        const T *psi = ctl->cur ? L0.r : L0.e;
        const int nx = L0.nx, ny = L0.ny, pitch = L0.pitch;
        T sum = T(0);
        for (int j = L1.cy0[J]; j < L1.cy0[J + 1]; j++) {
            for (int i = L1.cx0[I]; i < L1.cx0[I + 1]; i++) {
                auto kat = [&](int dx, int dy) {
                    int xx = i + dx;
                    xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
                    int yy = j + dy;
                    yy = yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy);
                    return L0.k[(long long)yy * pitch + xx];
                };
                auto pat = [&](int dx, int dy) {
                    int xx = i + dx;
                    xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
                    return psi[(long long)(j + dy) * pitch + xx];
                };
                const Node9<T> nd = node9<T>(kat, j, ny, H0c, H0s);
                const T p0 = psi[(long long)j * pitch + i];
                const T r = nd.b - (off9<T>(nd, pat, j, ny) - nd.diag * p0);
                sum += r;
                const double ar = fabs((double)r);
                mx = ar <= mx ? mx : (ar == ar ? ar : INFINITY);  // NaN counts as infinite
            }
        }
        L1.b[(long long)J * L1.pitch + I] = sum;
        L1.e[(long long)J * L1.pitch + I] = T(0);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0) atomic_max_nonneg(&ctl->norm_bits, mx);
}

// Level-0 block Gauss-Seidel (optionally after adding the coarse correction).
template <typename T>
__global__ void __launch_bounds__(SX *SY) smooth0(Level<T> L0, Level<T> L1, int add_coarse,
                                                  int sweeps, T H0c, T H0s, MgCtl *ctl) {
    if (cycle_skip(ctl)) return;
    __shared__ T sp[SY + 2][SX + 2];
    __shared__ T sk[SY + 2][SX + 2];
    const int nx = L0.nx, ny = L0.ny, pitch = L0.pitch;
    const int x0 = blockIdx.x * SX, y0 = blockIdx.y * SY;
    const T *src = ctl->cur ? L0.r : L0.e;
    T *dst = ctl->cur ? L0.e : L0.r;
    for (int t = threadIdx.y * SX + threadIdx.x; t < (SX + 2) * (SY + 2); t += SX * SY) {
        const int lx = t % (SX + 2), ly = t / (SX + 2);
        int gx = x0 - 1 + lx;
        gx = ((gx % nx) + nx) % nx;
        const int gy = y0 - 1 + ly;
        const int my = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
        sk[ly][lx] = L0.k[(long long)my * pitch + gx];
        T v = T(0);
        if (gy >= 0 && gy < ny) {
            v = src[(long long)gy * pitch + gx];
            if (add_coarse) v += interp_coarse(L0, L1, gx, gy);
        }
        sp[ly][lx] = v;  // ghost rows are never read: the mirror is used instead
    }
    __syncthreads();
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool own = x < nx && y < ny;
    Node9<T> nd;
    if (own) {
        auto kat = [&](int dx, int dy) { return sk[ly + dy][lx + dx]; };
        nd = node9<T>(kat, y, ny, H0c, H0s);
    }
    const int colour = (x & 1) + 2 * (y & 1);
    auto pat = [&](int dx, int dy) { return sp[ly + dy][lx + dx]; };
    for (int s = 0; s < sweeps; s++) {
        for (int c = 0; c < 4; c++) {
            if (own && colour == c) sp[ly][lx] = (off9<T>(nd, pat, y, ny) - nd.b) / nd.diag;
            __syncthreads();
        }
    }
    if (own) dst[(long long)y * pitch + x] = sp[ly][lx];
}

// ------------------------------------------------------------- coarse levels
template <typename T>
struct FV {
    T te, tw, tn, ts;     // face transmissibilities (tn/ts to the wall when at the edge)
    int ie, iw;           // periodic neighbours
    bool hasn, hass;      // neighbour inside (false: wall with value 0)
};

template <typename T>
__device__ __forceinline__ FV<T> fv_coef(const Level<T> &L, int I, int J) {
    FV<T> f;
    const int nx = L.nx, ny = L.ny, p = L.pitch;
    const T k0 = L.k[(long long)J * p + I];
    f.ie = I + 1 == nx ? 0 : I + 1;
    f.iw = I == 0 ? nx - 1 : I - 1;
    const T dxe = I + 1 == nx ? L.xc[0] + L.Lx - L.xc[I] : L.xc[I + 1] - L.xc[I];
    const T dxw = I == 0 ? L.xc[0] + L.Lx - L.xc[nx - 1] : L.xc[I] - L.xc[I - 1];
    f.te = T(0.5) * (k0 + L.k[(long long)J * p + f.ie]) * L.wy[J] / dxe;
    f.tw = T(0.5) * (k0 + L.k[(long long)J * p + f.iw]) * L.wy[J] / dxw;
    f.hasn = J + 1 < ny;
    f.hass = J > 0;
    f.tn = f.hasn ? T(0.5) * (k0 + L.k[(long long)(J + 1) * p + I]) * L.wx[I] / (L.yc[J + 1] - L.yc[J])
                  : k0 * L.wx[I] / (L.yhi - L.yc[J]);
    f.ts = f.hass ? T(0.5) * (k0 + L.k[(long long)(J - 1) * p + I]) * L.wx[I] / (L.yc[J] - L.yc[J - 1])
                  : k0 * L.wx[I] / (L.yc[J] - L.ylo);
    return f;
}

template <typename T>
__device__ __forceinline__ T fv_nb(const Level<T> &L, const FV<T> &f, int I, int J) {
    const int p = L.pitch;
    T s = f.te * L.e[(long long)J * p + f.ie] + f.tw * L.e[(long long)J * p + f.iw];
    if (f.hasn) s += f.tn * L.e[(long long)(J + 1) * p + I];
    if (f.hass) s += f.ts * L.e[(long long)(J - 1) * p + I];
    return s;
}

__device__ __forceinline__ int fv_colour(int I, int J, int nx) {
    return ((nx & 1) && I == nx - 1) ? 2 + (J & 1) : ((I + J) & 1);
}

template <typename T>
__device__ __forceinline__ void fv_gs_cell(const Level<T> &L, int I, int J) {
    const FV<T> f = fv_coef(L, I, J);
    const T d = f.te + f.tw + f.tn + f.ts;
    L.e[(long long)J * L.pitch + I] = (fv_nb(L, f, I, J) - L.b[(long long)J * L.pitch + I]) / d;
}

template <typename T>
__device__ __forceinline__ T fv_resid(const Level<T> &L, int I, int J) {
    const FV<T> f = fv_coef(L, I, J);
    const T d = f.te + f.tw + f.tn + f.ts;
    const T e0 = L.e[(long long)J * L.pitch + I];
    return L.b[(long long)J * L.pitch + I] - (fv_nb(L, f, I, J) - d * e0);
}

template <typename T>
__device__ __forceinline__ void k_restrict_cell(const Level<T> &C, const Level<T> &F, int I, int J) {
    T s = T(0);
    for (int j = C.cy0[J]; j < C.cy0[J + 1]; j++)
        for (int i = C.cx0[I]; i < C.cx0[I + 1]; i++)
            s += F.k[(long long)j * F.pitch + i] * F.wx[i] * F.wy[j];
    C.k[(long long)J * C.pitch + I] = s / (C.wx[I] * C.wy[J]);
}

template <typename T>
__device__ __forceinline__ void resid_restrict_cell(const Level<T> &F, const Level<T> &C, int I, int J) {
    T s = T(0);
    for (int j = C.cy0[J]; j < C.cy0[J + 1]; j++)
        for (int i = C.cx0[I]; i < C.cx0[I + 1]; i++) s += fv_resid(F, i, j);
    C.b[(long long)J * C.pitch + I] = s;
    C.e[(long long)J * C.pitch + I] = T(0);
}

template <typename T>
__global__ void k_restrict(Level<T> C, Level<T> F) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I < C.nx && J < C.ny) k_restrict_cell(C, F, I, J);
}

template <typename T>
__global__ void fv_smooth_colour(Level<T> L, int colour, MgCtl *ctl) {
    if (cycle_skip(ctl)) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I < L.nx && J < L.ny && fv_colour(I, J, L.nx) == colour) fv_gs_cell(L, I, J);
}

template <typename T>
__global__ void fv_resid_restrict(Level<T> F, Level<T> C, MgCtl *ctl) {
    if (cycle_skip(ctl)) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I < C.nx && J < C.ny) resid_restrict_cell(F, C, I, J);
}

template <typename T>
__global__ void fv_prolong(Level<T> F, Level<T> C, MgCtl *ctl) {
    if (cycle_skip(ctl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i < F.nx && j < F.ny) F.e[(long long)j * F.pitch + i] += interp_coarse(F, C, i, j);
}

// Levels lc .. nl-1 inside one block.
template <typename T>
__device__ void cta_smooth(const Level<T> &L, int sweeps) {
    const int n = L.nx * L.ny, ncol = (L.nx & 1) ? 4 : 2;
    for (int s = 0; s < sweeps; s++)
        for (int c = 0; c < ncol; c++) {
            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                const int I = t % L.nx, J = t / L.nx;
                if (fv_colour(I, J, L.nx) == c) fv_gs_cell(L, I, J);
            }
            __syncthreads();
        }
}

template <typename T>
__global__ void __launch_bounds__(CTA_THREADS) coarse_cta(const Level<T> *lv, int lc, int nl,
                                                         MgCtl *ctl) {
    if (cycle_skip(ctl)) return;
    for (int l = lc; l < nl - 1; l++) {
        const Level<T> F = lv[l], C = lv[l + 1];
        cta_smooth(F, NU_PRE);
        for (int t = threadIdx.x; t < C.nx * C.ny; t += blockDim.x)
            resid_restrict_cell(F, C, t % C.nx, t / C.nx);
        __syncthreads();
    }
    cta_smooth(lv[nl - 1], NU_COARSEST);
    for (int l = nl - 2; l >= lc; l--) {
        const Level<T> F = lv[l], C = lv[l + 1];
        for (int t = threadIdx.x; t < F.nx * F.ny; t += blockDim.x) {
            const int i = t % F.nx, j = t / F.nx;
            F.e[(long long)j * F.pitch + i] += interp_coarse(F, C, i, j);
        }
        __syncthreads();
        cta_smooth(F, NU_POST);
    }
}

template <typename T>
__global__ void __launch_bounds__(CTA_THREADS) k_restrict_cta(const Level<T> *lv, int lc, int nl) {
    for (int l = lc; l < nl; l++) {
        const Level<T> C = lv[l], F = lv[l - 1];
        for (int t = threadIdx.x; t < C.nx * C.ny; t += blockDim.x) k_restrict_cell(C, F, t % C.nx, t / C.nx);
        __syncthreads();
    }
}

__global__ void mg_begin_kernel(MgCtl *ctl, double tolH0, int max_iter) {
    ctl->norm_bits = 0ull;
    ctl->iter = 0;
    ctl->done = 0;
    ctl->converged = 0;
    ctl->tolH0 = tolH0;
    ctl->max_iter = max_iter;
    ctl->keep_going = 1;
}

__global__ void mg_cycle_end(MgCtl *ctl, cudaGraphConditionalHandle h, int in_graph) {
    ctl->cycles_launched++;
    if (!ctl->done) {
        const double nrm = norm_of(ctl);
        if (nrm <= ctl->tolH0 || ctl->iter >= ctl->max_iter || !(nrm < INFINITY)) {
            ctl->done = 1;
            ctl->converged = nrm <= ctl->tolH0;
            if (!ctl->converged) ctl->nonconv_count++;
            ctl->last_resid = ctl->H0 > 0.0 ? nrm / ctl->H0 : 0.0;
            ctl->last_iters = ctl->iter;
        } else {
            ctl->iter++;
            ctl->total_cycles++;
            ctl->cur ^= 1;
            ctl->norm_bits = 0ull;
        }
    }
    ctl->keep_going = !ctl->done;
    if (in_graph) cudaGraphSetConditional(h, ctl->keep_going ? 1u : 0u);
}

// ------------------------------------------------------------------ host side
template <typename T>
struct MgHost {
    int nl = 0, lc = 1;
    std::vector<Level<T>> lv;
    Level<T> *d_lv = nullptr;
    MgCtl *ctl = nullptr;
    std::vector<void *> mem;
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *user = nullptr;
    int ncolours_sum = 0;  // grid-wide coarse colour launches per cycle
};

static std::vector<int> merge_faces(int n) {
    // pairs of cells; when n is odd the last three cells form one
    std::vector<int> f(1, 0);
    const int nc = n / 2;
    int i = 0;
    for (int c = 0; c < nc; c++) {
        i += (c == nc - 1 && (n & 1)) ? 3 : 2;
        f.push_back(i);
    }
    return f;
}

struct Uploader {
    void *(*alloc)(size_t, void *);
    void *user;
    std::vector<void *> *mem;
    bool ok = true;
    template <typename U>
    U *put(const void *src, size_t bytes) {
        void *p = alloc(bytes, user);
        if (!p) { ok = false; return nullptr; }
        mem->push_back(p);
        if (src && cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
        return static_cast<U *>(p);
    }
};

// 1D linear interpolation from coarse centres onto fine centres; periodic
// when period > 0, else walls (index -1) at lo and hi.
template <typename T>
static void interp_table(const std::vector<double> &fine, const std::vector<double> &coarse,
                         double period, double lo, double hi, std::vector<int> &i0,
                         std::vector<int> &i1, std::vector<T> &w) {
    const int n = (int)coarse.size();
    for (double xf : fine) {
        int j = int(std::upper_bound(coarse.begin(), coarse.end(), xf) - coarse.begin()) - 1;
        int a, b;
        double xa, xb;
        if (period > 0) {
            if (j < 0) { a = n - 1; b = 0; xa = coarse[n - 1] - period; xb = coarse[0]; }
            else if (j >= n - 1) { a = n - 1; b = 0; xa = coarse[n - 1]; xb = coarse[0] + period; }
            else { a = j; b = j + 1; xa = coarse[j]; xb = coarse[j + 1]; }
        } else {
            if (j < 0) { a = -1; b = 0; xa = lo; xb = coarse[0]; }
            else if (j >= n - 1) { a = n - 1; b = -1; xa = coarse[n - 1]; xb = hi; }
            else { a = j; b = j + 1; xa = coarse[j]; xb = coarse[j + 1]; }
        }
        i0.push_back(a);
        i1.push_back(b);
        w.push_back(T((xf - xa) / (xb - xa)));
    }
}

template <typename T>
MgHost<T> *mg_create(int nx, int ny, int pitch, T *k0, T *psiA, T *psiB, MgCtl *ctl,
                     void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *user,
                     char *err, size_t errlen) {
    MgHost<T> *m = new MgHost<T>();
    m->alloc = alloc;
    m->release = release;
    m->user = user;
    m->ctl = ctl;
    Uploader up{alloc, user, &m->mem};
    // geometry of every level: faces in lattice units
    std::vector<std::vector<int>> fx(1), fy(1), cx0(1), cy0(1);
    for (int i = 0; i <= nx; i++) fx[0].push_back(i);
    for (int j = 0; j <= ny; j++) fy[0].push_back(j);
    const int minc = 3;
    while (true) {
        const int px = (int)fx.back().size() - 1, py = (int)fy.back().size() - 1;
        const bool cxo = px > minc, cyo = py > minc;
        if (!cxo && !cyo) break;
        std::vector<int> mx, my;
        if (cxo) mx = merge_faces(px); else for (int i = 0; i <= px; i++) mx.push_back(i);
        if (cyo) my = merge_faces(py); else for (int j = 0; j <= py; j++) my.push_back(j);
        std::vector<int> nfx, nfy;
        for (int v : mx) nfx.push_back(fx.back()[v]);
        for (int v : my) nfy.push_back(fy.back()[v]);
        fx.push_back(nfx);
        fy.push_back(nfy);
        cx0.push_back(mx);
        cy0.push_back(my);
    }
    m->nl = (int)fx.size();
    m->lv.resize(m->nl);
    std::vector<std::vector<double>> xcs(m->nl), ycs(m->nl);
    for (int l = 0; l < m->nl; l++) {
        for (size_t i = 0; i + 1 < fx[l].size(); i++) xcs[l].push_back(0.5 * (fx[l][i] + fx[l][i + 1]));
        for (size_t j = 0; j + 1 < fy[l].size(); j++) ycs[l].push_back(0.5 * (fy[l][j] + fy[l][j + 1]));
    }
    // first level small enough for the single-block kernel
    const long long cta_cells = 4096;
    m->lc = m->nl;
    for (int l = 1; l < m->nl; l++) {
        if ((long long)xcs[l].size() * ycs[l].size() <= cta_cells) { m->lc = l; break; }
    }
    if (m->lc >= m->nl) m->lc = m->nl - 1;  // the coarsest level always runs in the block
    for (int l = 0; l < m->nl; l++) {
        Level<T> &L = m->lv[l];
        std::memset(&L, 0, sizeof(L));
        L.nx = (int)xcs[l].size();
        L.ny = (int)ycs[l].size();
        L.Lx = T(nx);
        L.ylo = T(0);
        L.yhi = T(ny);
        if (l == 0) {
            L.pitch = pitch;
            L.k = k0;
            L.e = psiA;
            L.r = psiB;
        } else {
            L.pitch = L.nx;
            size_t cells = (size_t)L.nx * L.ny;
            L.e = up.put<T>(nullptr, cells * sizeof(T));
            L.b = up.put<T>(nullptr, cells * sizeof(T));
            L.k = up.put<T>(nullptr, cells * sizeof(T));
            L.cx0 = up.put<int>(cx0[l].data(), cx0[l].size() * sizeof(int));
            L.cy0 = up.put<int>(cy0[l].data(), cy0[l].size() * sizeof(int));
        }
        std::vector<T> xc(L.nx), wx(L.nx), yc(L.ny), wy(L.ny);
        for (int i = 0; i < L.nx; i++) { xc[i] = T(xcs[l][i]); wx[i] = T(fx[l][i + 1] - fx[l][i]); }
        for (int j = 0; j < L.ny; j++) { yc[j] = T(ycs[l][j]); wy[j] = T(fy[l][j + 1] - fy[l][j]); }
        L.xc = up.put<T>(xc.data(), xc.size() * sizeof(T));
        L.wx = up.put<T>(wx.data(), wx.size() * sizeof(T));
        L.yc = up.put<T>(yc.data(), yc.size() * sizeof(T));
        L.wy = up.put<T>(wy.data(), wy.size() * sizeof(T));
        if (l + 1 < m->nl) {
            std::vector<int> a0, a1, b0, b1;
            std::vector<T> wa, wb;
            interp_table<T>(xcs[l], xcs[l + 1], double(nx), 0, 0, a0, a1, wa);
            interp_table<T>(ycs[l], ycs[l + 1], -1.0, 0.0, double(ny), b0, b1, wb);
            L.px0 = up.put<int>(a0.data(), a0.size() * sizeof(int));
            L.px1 = up.put<int>(a1.data(), a1.size() * sizeof(int));
            L.pwx = up.put<T>(wa.data(), wa.size() * sizeof(T));
            L.py0 = up.put<int>(b0.data(), b0.size() * sizeof(int));
            L.py1 = up.put<int>(b1.data(), b1.size() * sizeof(int));
            L.pwy = up.put<T>(wb.data(), wb.size() * sizeof(T));
        }
    }
    m->d_lv = up.put<Level<T>>(m->lv.data(), m->lv.size() * sizeof(Level<T>));
    for (int l = 1; l < m->lc; l++) m->ncolours_sum += (m->lv[l].nx & 1) ? 4 : 2;
    if (!up.ok) {
        snprintf(err, errlen, "multigrid: device allocation or upload failed");
        mg_destroy(m);
        return nullptr;
    }
    return m;
}

template <typename T>
void mg_destroy(MgHost<T> *m) {
    if (!m) return;
    for (void *p : m->mem) m->release(p, m->user);
    delete m;
}

static dim3 g2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

template <typename T>
void mg_prepare(MgHost<T> *m, cudaStream_t s) {
    dim3 b(32, 8);
    for (int l = 1; l < m->lc; l++)
        k_restrict<T><<<g2(m->lv[l].nx, m->lv[l].ny, b), b, 0, s>>>(m->lv[l], m->lv[l - 1]);
    if (m->lc < m->nl) k_restrict_cta<T><<<1, CTA_THREADS, 0, s>>>(m->d_lv, m->lc, m->nl);
}

template <typename T>
void mg_begin(MgHost<T> *m, double tolH0, int max_iter, cudaStream_t s) {
    mg_begin_kernel<<<1, 1, 0, s>>>(m->ctl, tolH0, max_iter);
}

template <typename T>
void mg_cycle(MgHost<T> *m, T H0c, T H0s, cudaGraphConditionalHandle h, int in_graph,
              cudaStream_t s) {
    dim3 b(32, 8);
    const std::vector<Level<T>> &lv = m->lv;
    resid0_restrict<T><<<g2(lv[1].nx, lv[1].ny, b), b, 0, s>>>(lv[0], lv[1], H0c, H0s, m->ctl);
    for (int l = 1; l < m->lc; l++) {
        const int nc = (lv[l].nx & 1) ? 4 : 2;
        for (int sw = 0; sw < NU_PRE; sw++)
            for (int c = 0; c < nc; c++)
                fv_smooth_colour<T><<<g2(lv[l].nx, lv[l].ny, b), b, 0, s>>>(lv[l], c, m->ctl);
        fv_resid_restrict<T><<<g2(lv[l + 1].nx, lv[l + 1].ny, b), b, 0, s>>>(lv[l], lv[l + 1], m->ctl);
    }
    coarse_cta<T><<<1, CTA_THREADS, 0, s>>>(m->d_lv, m->lc, m->nl, m->ctl);
    for (int l = m->lc - 1; l >= 1; l--) {
        const int nc = (lv[l].nx & 1) ? 4 : 2;
        fv_prolong<T><<<g2(lv[l].nx, lv[l].ny, b), b, 0, s>>>(lv[l], lv[l + 1], m->ctl);
        for (int sw = 0; sw < NU_POST; sw++)
            for (int c = 0; c < nc; c++)
                fv_smooth_colour<T><<<g2(lv[l].nx, lv[l].ny, b), b, 0, s>>>(lv[l], c, m->ctl);
    }
    dim3 bs(SX, SY);
    smooth0<T><<<g2(lv[0].nx, lv[0].ny, bs), bs, 0, s>>>(lv[0], lv[1], 1, NU_FINE, H0c, H0s, m->ctl);
    mg_cycle_end<<<1, 1, 0, s>>>(m->ctl, h, in_graph);
}

template <typename T>
int mg_kernels_per_cycle(const MgHost<T> *m) {
    int n = 4;  // resid0_restrict, coarse_cta, smooth0, cycle_end
    for (int l = 1; l < m->lc; l++) n += 2 + ((m->lv[l].nx & 1) ? 4 : 2) * (NU_PRE + NU_POST);
    return n;
}

template <typename T>
int mg_levels(const MgHost<T> *m) { return m->nl; }

template <typename T>
int mg_pre_kernels(const MgHost<T> *m) {
    return (m->lc - 1) + (m->lc < m->nl ? 1 : 0) + 1;
}

#define FCD_MG_INST(T)                                                                          \
    template MgHost<T> *mg_create<T>(int, int, int, T *, T *, T *, MgCtl *,                     \
                                     void *(*)(size_t, void *), void (*)(void *, void *), void *, \
                                     char *, size_t);                                           \
    template void mg_destroy<T>(MgHost<T> *);                                                   \
    template void mg_prepare<T>(MgHost<T> *, cudaStream_t);                                     \
    template void mg_begin<T>(MgHost<T> *, double, int, cudaStream_t);                          \
    template void mg_cycle<T>(MgHost<T> *, T, T, cudaGraphConditionalHandle, int, cudaStream_t); \
    template int mg_kernels_per_cycle<T>(const MgHost<T> *);                                    \
    template int mg_levels<T>(const MgHost<T> *);                                               \
    template int mg_pre_kernels<T>(const MgHost<T> *);
FCD_MG_INST(float)
FCD_MG_INST(double)

}  // namespace fcd
