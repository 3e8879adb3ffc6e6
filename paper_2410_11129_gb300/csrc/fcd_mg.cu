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
// with arithmetic face permeabilities. The coarse levels run in FP32 for both
// storage types (mixed-precision defect correction): level 0 keeps the compute
// type, forms the residual that is restricted and adds the interpolated
// correction, so the coarse precision only perturbs each cycle's contraction,
// not the converged potential; on this GPU FP64 arithmetic is 1/58 of FP32, and
// the single-block coarse levels are bound by one SM's arithmetic. Cycles are V(0, 2) on level 0 and V(2, 2)
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
#include <type_traits>
#include <vector>

#include "fcd_internal.cuh"

namespace fcd {

constexpr int SX = 32, SY = 8;     // level-0 smoothing tile
constexpr int CTA_THREADS = 1024;
constexpr int NU_PRE = 2, NU_POST = 2, NU_FINE = 2;  // grid-wide levels: V(2,2); lattice: V(0,2)
constexpr int NU_CTA = 1, NU_COARSEST = 8;           // single-block levels: V(1,1)
constexpr int MIN_COARSE = 100;                      // coarsening stops at this many cells
// Every solve opens with NU_SMOOTH_ONLY lattice sweeps (no residual check
// before them). One: block Gauss-Seidel with a frozen halo leaves the residual
// it cannot remove on the tile borders, and further sweeps in the same launch
// only sharpen it there. Cheaper cycles tried before a V-cycle: lattice sweeps
// when the starting residual is within SMOOTH_RATIO of the tolerance (once per
// solve), else a two-grid cycle (NU_TWOGRID sweeps on level 1, at most twice
// per solve). The residual changes between time steps are local, so both
// usually suffice after the extrapolated initial guess (numpy prototype: the
// two-grid cycle reduces such residuals as much as a V-cycle). Measured on the
// 1600 x 200, 2400 x 300 and 9600 x 1200 FP32 channels (4000-10000 steps): one
// opening sweep and two level-1 sweeps leave 1.00-1.01 residual evaluations
// per step, three and four 1.19-1.2; the count depends on rounding-level
// details near the tolerance, and this pair was the best on all three.
constexpr double SMOOTH_RATIO = 2.5;
constexpr int NU_SMOOTH_ONLY = 1, NU_TWOGRID = 2;
constexpr size_t CTA_SMEM_MAX = 200 * 1024;  // shared memory of the single-block levels
constexpr size_t CTA_CELLS = 2048;            // cells of the single-block levels
using TC = float;                             // type of the coarse levels (>= 1)

__device__ __forceinline__ double norm_of(const MgCtl *c) {
    return __longlong_as_double((long long)c->norm_bits);
}
// The rest of a cycle is skipped once the solve is done, the residual of
// this cycle met the tolerance, or the cycle cap was reached.
__device__ __forceinline__ bool cycle_skip(const MgCtl *c) {
    return c->done || norm_of(c) <= c->tolH0 || c->iter >= c->max_iter;
}

// cycle_skip evaluated once per block (the FP64 compare is costly on this GPU).
__device__ __forceinline__ bool block_skip(const MgCtl *c, bool first = false) {
    __shared__ int flag;
    if (threadIdx.x == 0 && threadIdx.y == 0)
        flag = first ? (c->done || c->iter >= c->max_iter) : cycle_skip(c);
    __syncthreads();
    return flag != 0;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// Thread 0 of a level-0 tile, after the tile's writes: true for the last of the
// launch's nblocks tiles to finish (lin: the tile's index in the launch).
// mx_bits (the tile's max |r| as double bits, 0 for none) goes to
// ctl->norm_bits on the way. Updates of one counter serialise (about 0.9 ns each
// on this GPU, measured with a grid barrier), so a launch of GROUPED_TILES tiles
// or more reports through MG_GROUPS group counters in separate lines: no counter
// takes more than ceil(nblocks / MG_GROUPS) or MG_GROUPS updates. Smaller
// launches keep one counter, whose chain is shorter than the second level's
// latency (measured on the 1600 x 200 channel: 4 us per step slower grouped).
// The group counters are back at zero when the launch ends.
constexpr unsigned GROUPED_TILES = 8192;
__device__ __forceinline__ bool tile_done(MgCtl *ctl, MgGroup *grp, unsigned lin, unsigned nblocks,
                                          unsigned long long mx_bits) {
    __threadfence();
    unsigned arrivals = nblocks;
    if (grp && nblocks >= GROUPED_TILES) {
        const unsigned g = lin % MG_GROUPS;
        MgGroup &G = grp[g];
        const unsigned gsize = nblocks / MG_GROUPS + (g < nblocks % MG_GROUPS ? 1u : 0u);
        if (mx_bits) atomicMax(&G.max_bits, mx_bits);
        __threadfence();
        if (atomicAdd(&G.count, 1u) != gsize - 1) return false;
        __threadfence();
        G.count = 0;
        mx_bits = atomicExch(&G.max_bits, 0ull);
        arrivals = MG_GROUPS;
    }
    if (mx_bits) atomicMax(&ctl->norm_bits, mx_bits);
    __threadfence();
    if (atomicAdd(&ctl->blocks_done, 1u) != arrivals - 1) return false;
    __threadfence();
    ctl->blocks_done = 0;
    return true;
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

// W: the node may lie on a wall row (y = 0 or ny - 1), whose ghost neighbours
// follow the mirror rules; W = false (a tile without wall rows) drops the test.
template <typename T, bool W = true, typename KF>
__device__ __forceinline__ Node9<T> node9(KF kat, int y, int ny, T H0c, T H0s) {
    Node9<T> n;
    const T k0 = kat(0, 0);
    if constexpr (!W) {
        // The same operator with its sums regrouped: pairwise for the diagonal,
        // and since sum_a w_a e_a = 0 the k_0 part of -L psi0 cancels exactly,
        // b = 3 sum_a w_a k_a (e_a . H0 e_alpha), formed from opposite
        // differences of k (zero in a uniform medium).
        T kv[9];
#pragma unroll
        for (int a = 1; a < 9; a++) {
            kv[a] = kat(cx(a), cy(a));
            n.c[a] = T(6) * wgt<T>(a) * T(0.5) * (k0 + kv[a]);
        }
        n.diag = ((n.c[1] + n.c[2]) + (n.c[3] + n.c[4])) + ((n.c[5] + n.c[6]) + (n.c[7] + n.c[8]));
        n.b = T(1.0 / 3.0) * ((kv[1] - kv[3]) * H0c + (kv[2] - kv[4]) * H0s) +
              T(1.0 / 12.0) * ((kv[5] - kv[7]) * (H0c + H0s) + (kv[6] - kv[8]) * (H0s - H0c));
        (void)y;
        (void)ny;
        return n;
    }
    n.diag = T(0);
    n.b = T(0);
#pragma unroll
    for (int a = 1; a < 9; a++) {
        const T ca = T(6) * wgt<T>(a) * T(0.5) * (k0 + kat(cx(a), cy(a)));
        n.c[a] = ca;
        n.diag += ca;
        n.b += ca * (T(cx(a)) * H0c + T(cy(a)) * H0s);
        if constexpr (W) {
            const int yy = y + cy(a);
            if ((yy < 0 || yy >= ny) && cx(a) == 0) n.diag += ca;  // psi'(ghost) = -psi'(node)
        }
    }
    return n;
}

// sum of c_a * psi~_a over neighbours that are not the node itself
template <typename T, bool W = true, typename PF>
__device__ __forceinline__ T off9(const Node9<T> &n, PF pat, int y, int ny) {
    T s = T(0);
#pragma unroll
    for (int a = 1; a < 9; a++) {
        if constexpr (W) {
            const int yy = y + cy(a);
            if (yy < 0 || yy >= ny) {
                if (cx(a) != 0) s -= n.c[a] * pat(cx(a), 0);  // mirror of a diagonal ghost
                continue;
            }
        }
        s += n.c[a] * pat(cx(a), cy(a));
    }
    return s;
}

// FP32 level 0 with psi' = hi + lo (see psi_planes): the right-hand side and
// the residual written per opposite link pair (a, opp a), a in {1, 2, 5, 6}:
//   b = sum_pairs (c_a - c_opp)(e_a . H0 e_alpha)
//   sum_a c_a d_a = sum_pairs [c_a (d_a + d_opp) + (c_opp - c_a) d_opp]
// with d_a = psi'~_a - psi'_0 formed from the hi and lo parts separately.
// Neighbouring values of psi' differ little, so the hi differences are exact
// (Sterbenz) and every term scales with the local variation of psi' and k,
// not with |psi'|; in a uniform medium c_opp - c_a and b are exactly 0. The
// rounding of the residual is then ~1e-7 H0 instead of ~1e-5 H0.
// first link of each opposite pair: 1, 2, 5, 6 for q = 0..3
__host__ __device__ constexpr int pair_a(int q) { return q < 2 ? q + 1 : q + 3; }

template <bool W = true, typename KF>
__device__ __forceinline__ Node9<float> node9_pairs(KF kat, int y, int ny, float H0c, float H0s) {
    Node9<float> n;
    const float k0 = kat(0, 0);
    n.diag = 0.f;
#pragma unroll
    for (int a = 1; a < 9; a++) {
        const float ca = 3.f * wgt<float>(a) * (k0 + kat(cx(a), cy(a)));
        n.c[a] = ca;
        n.diag += ca;
        if constexpr (W) {
            const int yy = y + cy(a);
            if ((yy < 0 || yy >= ny) && cx(a) == 0) n.diag += ca;  // psi'(ghost) = -psi'(node)
        }
    }
    n.b = 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int a = pair_a(q);
        n.b += (n.c[a] - n.c[opp(a)]) * (float(cx(a)) * H0c + float(cy(a)) * H0s);
    }
    return n;
}

// b - L psi' at the node, psi' = hat + lat (accessors relative to the node).
template <bool W = true, typename HF, typename LF>
__device__ __forceinline__ float resid_pairs(const Node9<float> &n, HF hat, LF lat, int y, int ny) {
    const float h0 = hat(0, 0), l0 = lat(0, 0);
    auto dl = [&](int a) -> float {
        if constexpr (W) {
            const int yy = y + cy(a);
            if (yy < 0 || yy >= ny) {  // mirrored ghost: psi'~ = -psi'(x + cx, y)
                if (cx(a) == 0) return -(h0 + h0) - (l0 + l0);
                return -(hat(cx(a), 0) + h0) - (lat(cx(a), 0) + l0);
            }
        }
        return (hat(cx(a), cy(a)) - h0) + (lat(cx(a), cy(a)) - l0);
    };
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int a = pair_a(q), o = opp(a);
        const float da = dl(a), dop = dl(o);
        sum += n.c[a] * (da + dop) + (n.c[o] - n.c[a]) * dop;
    }
    return n.b - sum;
}

// (hi, lo) += v, renormalised.
__device__ __forceinline__ void comp_add(float &hi, float &lo, float v) {
    float s, e;
    two_sum(hi, __fadd_rn(lo, v), s, e);
    hi = s;
    lo = e;
}

// FP64 hierarchies keep the lattice level's node coefficients in COEF planes,
// formed once per solve by coef0_kernel (k does not change within a solve):
// the FP64 arithmetic of node9 and its division cost more than the loads on
// this GPU (FP64 is 1/58 of FP32). FP32 hierarchies form them on the fly.
constexpr int COEF = 11;  // c_1..c_8, diag, 1/diag, b
template <typename T>
__host__ __device__ constexpr bool keeps_coef() { return sizeof(T) == 8; }

template <typename T>
__device__ __forceinline__ void coef_load(const Level<T> &L0, long long n, Node9<T> &nd, T &inv) {
    const long long ps = (long long)L0.pitch * L0.ny;
#pragma unroll
    for (int a = 1; a < 9; a++) nd.c[a] = L0.coef[(a - 1) * ps + n];
    nd.diag = L0.coef[8 * ps + n];
    inv = L0.coef[9 * ps + n];
    nd.b = L0.coef[10 * ps + n];
}

template <typename T>
__global__ void __launch_bounds__(256) coef0_kernel(Level<T> L0, T H0c, T H0s) {
    const int nx = L0.nx, ny = L0.ny, pitch = L0.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    auto kat = [&](int dx, int dy) {
        int xx = x + dx;
        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        const int yy = y + dy < 0 ? 0 : (y + dy >= ny ? ny - 1 : y + dy);  // mirrored ghost rows
        return L0.k[(long long)yy * pitch + xx];
    };
    const Node9<T> nd = node9<T>(kat, y, ny, H0c, H0s);
    const long long ps = (long long)pitch * ny, n = (long long)y * pitch + x;
#pragma unroll
    for (int a = 1; a < 9; a++) L0.coef[(a - 1) * ps + n] = nd.c[a];
    L0.coef[8 * ps + n] = nd.diag;
    L0.coef[9 * ps + n] = T(1) / nd.diag;
    L0.coef[10 * ps + n] = nd.b;
}

// Interpolation weights of a tile's columns and rows, staged in shared memory.
template <typename T, int NXT, int NYT>
struct ProlongTile {
    int x0[NXT], x1[NXT], y0[NYT], y1[NYT];
    T wx[NXT], wy[NYT];
};

template <typename T, int NXT, int NYT>
__device__ __forceinline__ void prolong_tile_load(ProlongTile<T, NXT, NYT> &pt, const Level<T> &F,
                                                  int gx_first, int gy_first) {
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if (t < NXT) {
        int gx = gx_first + t;
        if (gx < 0) gx += F.nx;
        while (gx >= F.nx) gx -= F.nx;
        pt.x0[t] = F.px0[gx];
        pt.x1[t] = F.px1[gx];
        pt.wx[t] = F.pwx[gx];
    } else if (t < NXT + NYT) {
        const int q = t - NXT, gy = gy_first + q;
        if (gy >= 0 && gy < F.ny) {
            pt.y0[q] = F.py0[gy];
            pt.y1[q] = F.py1[gy];
            pt.wy[q] = F.pwy[gy];
        } else {
            pt.y0[q] = -1;
            pt.y1[q] = -1;
            pt.wy[q] = T(0);
        }
    }
}

template <typename T, typename U, int NXT, int NYT>
__device__ __forceinline__ T prolong_at(const ProlongTile<T, NXT, NYT> &pt, const Level<U> &C,
                                        int lx, int ly) {
    const int x0 = pt.x0[lx], x1 = pt.x1[lx], y0 = pt.y0[ly], y1 = pt.y1[ly];
    const T wx = pt.wx[lx], wy = pt.wy[ly];
    T a = T(0), b = T(0);
    if (y0 >= 0)
        a = (T(1) - wx) * T(C.e[(long long)y0 * C.pitch + x0]) + wx * T(C.e[(long long)y0 * C.pitch + x1]);
    if (y1 >= 0)
        b = (T(1) - wx) * T(C.e[(long long)y1 * C.pitch + x0]) + wx * T(C.e[(long long)y1 * C.pitch + x1]);
    return (T(1) - wy) * a + wy * b;
}

__device__ void cycle_decide(MgCtl *ctl, cudaGraphConditionalHandle hw,
                             cudaGraphConditionalHandle hi, int in_graph);

// Residual of level 0 on the children of each level-1 cell, summed onto it,
// and the level-1 permeability (mean of the children); the max-norm over the
// lattice goes to the control block. A 32 x 8 block of level-1 cells stages
// its lattice footprint (at most 65 x 17 cells plus a one-cell ring) of k and
// psi' in shared memory.
constexpr int RX = 2 * 32 + 1 + 2, RY = 2 * 8 + 1 + 2;

// One 32 x 8 block of level-1 cells (bx, by) of a grid of nblocks blocks;
// grid_lead: the block that reports a solve that is already done. SPLIT as
// for the smoothing tiles.
template <typename T, bool COMP, bool SPLIT = true>
__device__ __forceinline__ void resid0_tile(const Level<T> &L0, const Level<TC> &L1, T H0c, T H0s,
                                            MgCtl *ctl, cudaGraphConditionalHandle hw,
                                            cudaGraphConditionalHandle hi, int in_graph, int bx,
                                            int by, unsigned nblocks, bool grid_lead) {
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    if (ctl->done) {
        if (lead && grid_lead) cycle_decide(ctl, hw, hi, in_graph);
        return;
    }
    static_assert(!COMP || sizeof(T) == 4, "the hi + lo pair is an FP32 form");
    __shared__ T sk[RY][RX], sp[RY][RX];
    __shared__ T sl[COMP ? RY : 1][COMP ? RX : 1];  // lo part of psi' (FP32 level 0)
    const int nx = L0.nx, ny = L0.ny, pitch = L0.pitch;
    const long long lo_off = (long long)pitch * ny;
    const int I0 = bx * 32, J0 = by * 8;
    const int I1 = min(I0 + 32, L1.nx), J1 = min(J0 + 8, L1.ny);
    const int fx0 = L1.cx0[I0], fx1 = L1.cx0[I1], fy0 = L1.cy0[J0], fy1 = L1.cy0[J1];
    const int wx = fx1 - fx0 + 2, wy = fy1 - fy0 + 2;
    const T *psi = ctl->cur ? L0.r : L0.e;
    {  // all loads issued before the shared-memory stores: warp w takes footprint
       // rows w, w + 8, w + 16, lane l columns l, l + 32, l + 64
        constexpr int NR = (RY + 7) / 8, NC = (RX + 31) / 32;
        const int lane = threadIdx.x, warp = threadIdx.y;
        int gxs[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) {
            int gx = fx0 - 1 + lane + 32 * c;
            gx = gx < 0 ? gx + nx : gx;
            while (gx >= nx) gx -= nx;
            gxs[c] = gx;
        }
        T kv[NR][NC], pv[NR][NC], lv[COMP ? NR : 1][COMP ? NC : 1];
#pragma unroll
        for (int r = 0; r < NR; r++) {
            const int ly = warp + 8 * r, gy = fy0 - 1 + ly;
            const int my = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
#pragma unroll
            for (int c = 0; c < NC; c++) {
                kv[r][c] = T(0);
                pv[r][c] = T(0);
                if constexpr (COMP) lv[r][c] = T(0);
                if (ly < wy && lane + 32 * c < wx) {
                    const long long m = (long long)my * pitch + gxs[c];
                    kv[r][c] = L0.k[m];  // mirrored ghost rows
                    pv[r][c] = psi[m];   // ghost rows never read
                    if constexpr (COMP) lv[r][c] = psi[lo_off + m];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < NR; r++)
#pragma unroll
            for (int c = 0; c < NC; c++) {
                const int ly = warp + 8 * r, lx = lane + 32 * c;
                if (ly < wy && lx < wx) {
                    sk[ly][lx] = kv[r][c];
                    sp[ly][lx] = pv[r][c];
                    if constexpr (COMP) sl[ly][lx] = lv[r][c];
                }
            }
    }
    __syncthreads();
    const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
    T mxt = T(0);  // a max is exact in the compute type; only the reduction is FP64
    // W: the footprint holds a wall row, whose nodes take the ghost rules
    auto cells = [&](auto wall) {
        constexpr bool W = decltype(wall)::value;
        if (!(I < L1.nx && J < L1.ny)) return;
        T sum = T(0), ksum = T(0);
        auto child = [&](int i, int j) {
            const int lx = i - fx0 + 1, ly = j - fy0 + 1;
            auto kat = [&](int dx, int dy) { return sk[ly + dy][lx + dx]; };
            auto pat = [&](int dx, int dy) { return sp[ly + dy][lx + dx]; };
            T r;
            if constexpr (COMP) {
                auto lat = [&](int dx, int dy) { return sl[ly + dy][lx + dx]; };
                Node9<float> nd = node9_pairs<W>(kat, j, ny, H0c, H0s);
                if (L0.rhs) nd.b = L0.rhs[(long long)j * pitch + i];
                r = resid_pairs<W>(nd, pat, lat, j, ny);
            } else {
                Node9<T> nd;
                if constexpr (keeps_coef<T>()) {
                    T inv;
                    coef_load(L0, (long long)j * pitch + i, nd, inv);
                    (void)kat;
                } else {
                    nd = node9<T, W>(kat, j, ny, H0c, H0s);
                }
                const T bb = L0.rhs ? L0.rhs[(long long)j * pitch + i] : nd.b;
                r = bb - (off9<T, W>(nd, pat, j, ny) - nd.diag * sp[ly][lx]);
            }
            sum += r;
            ksum += sk[ly][lx];
            const T ar = fabs(r);
            mxt = ar <= mxt ? mxt : (ar == ar ? ar : T(INFINITY));  // NaN counts as infinite
        };
        const int ia = L1.cx0[I], ib = L1.cx0[I + 1], ja = L1.cy0[J], jb = L1.cy0[J + 1];
        if (ib - ia == 2 && jb - ja == 2) {  // the common 2 x 2 merge, unrolled
            child(ia, ja);
            child(ia + 1, ja);
            child(ia, ja + 1);
            child(ia + 1, ja + 1);
        } else {
            for (int j = ja; j < jb; j++)
                for (int i = ia; i < ib; i++) child(i, j);
        }
        L1.b[(long long)J * L1.pitch + I] = TC(sum);
        L1.k[(long long)J * L1.pitch + I] = TC(ksum / (T(L1.wx[I]) * T(L1.wy[J])));  // unit lattice cells
    };
    if (!SPLIT || fy0 == 0 || fy1 >= ny) cells(std::true_type{});
    else cells(std::false_type{});
    for (int o = 16; o > 0; o >>= 1) mxt = fmax(mxt, __shfl_xor_sync(0xffffffffu, mxt, o));
    __shared__ T wmax[8];  // one per warp (blockDim 32 x 8)
    if (threadIdx.x == 0) wmax[threadIdx.y] = mxt;
    __syncthreads();
    if (lead) {  // the last block to finish sees the whole norm and decides the cycle
        T m = wmax[0];
#pragma unroll
        for (int w = 1; w < 8; w++) m = fmax(m, wmax[w]);
        const double mx = (double)m;
        const unsigned long long bits = mx > 0.0 ? (unsigned long long)__double_as_longlong(mx) : 0ull;
        const unsigned lin = (unsigned)(by * ((L1.nx + 31) / 32) + bx);
        if (tile_done(ctl, L0.grp, lin, nblocks, bits)) cycle_decide(ctl, hw, hi, in_graph);
    }
}

template <typename T, bool COMP>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 4) resid0_restrict(Level<T> L0, Level<TC> L1, T H0c, T H0s,
                                                       MgCtl *ctl, cudaGraphConditionalHandle hw,
                                                       cudaGraphConditionalHandle hi, int in_graph) {
    resid0_tile<T, COMP>(L0, L1, H0c, H0s, ctl, hw, hi, in_graph, blockIdx.x, blockIdx.y,
                         gridDim.x * gridDim.y, blockIdx.x == 0 && blockIdx.y == 0);
}

__device__ void cycle_close(MgCtl *ctl);

// Level-0 block Gauss-Seidel after adding the coarse correction; the last
// block to finish closes the cycle. A 32 x 8 tile runs on 64 threads, each
// owning one 2 x 2 quad: the quad holds one node of each colour (x0 and y0
// are even), so in every colour phase every thread updates exactly one node.
// Same-colour nodes are not 9-point neighbours, so the result does not depend
// on the order within a phase.
constexpr int QT = (SX / 2) * (SY / 2);  // threads of a smoothing tile
static_assert(QT % 32 == 0 && 2 * (SY + 2) <= QT, "tile load layout");
constexpr int TILE_ROWS = (SY + 2 + QT / 32 - 1) / (QT / 32);  // ring rows per warp

// One 32 x 8 tile (bx, by) of a grid of nblocks tiles. SPLIT: tiles without a
// wall row take a second copy of the sweeps that skips the ghost tests (fewer
// instructions; the batched kernels keep one copy to bound their registers).
template <typename T, bool COMP, bool SPLIT = true>
__device__ __forceinline__ void smooth0_tile(const Level<T> &L0, const Level<TC> &L1,
                                             int add_coarse, int sweeps, T H0c, T H0s, MgCtl *ctl,
                                             int first, int bx, int by, unsigned nblocks) {
    const int tid = threadIdx.x;
    // first: the sweeps that open a solve (no residual known yet)
    if (block_skip(ctl, first != 0)) return;
    static_assert(!COMP || sizeof(T) == 4, "the hi + lo pair is an FP32 form");
    __shared__ T sp[SY + 2][SX + 2];
    __shared__ T sl[COMP ? SY + 2 : 1][COMP ? SX + 2 : 1];  // lo part of psi' (FP32)
    __shared__ T sk[SY + 2][SX + 2];
    const int nx = L0.nx, ny = L0.ny, pitch = L0.pitch;
    const long long lo_off = (long long)pitch * ny;
    const int x0 = bx * SX, y0 = by * SY;
    const T *src = ctl->cur ? L0.r : L0.e;
    T *dst = ctl->cur ? L0.e : L0.r;
    __shared__ ProlongTile<T, SX + 2, SY + 2> pt;
    if (add_coarse) prolong_tile_load(pt, L0, x0 - 1, y0 - 1);
    {  // tile with its frozen one-cell ring, all loads issued before the stores: warp w
       // takes ring rows w, w + QT/32, ..., lane l column l; the two last columns
       // (2 (SY + 2) values) go to threads 0 .. 2 SY + 3
        const int lane = tid & 31, warp = tid >> 5;
        auto wrap = [&](int gx) {
            if (gx < 0) gx += nx;
            while (gx >= nx) gx -= nx;
            return gx;
        };
        const int gxa = wrap(x0 - 1 + lane);
        const bool extra = tid < 2 * (SY + 2);
        const int ey = tid >> 1, ex = SX + (tid & 1), gxe = wrap(x0 - 1 + ex);
        T kv[TILE_ROWS + 1], pv[TILE_ROWS + 1], lv[COMP ? TILE_ROWS + 1 : 1];
#pragma unroll
        for (int q = 0; q <= TILE_ROWS; q++) {
            const int ly = q < TILE_ROWS ? warp + q * (QT / 32) : ey;
            const int gx = q < TILE_ROWS ? gxa : gxe;
            const bool act = q < TILE_ROWS ? ly < SY + 2 : extra;
            kv[q] = T(0);
            pv[q] = T(0);
            if constexpr (COMP) lv[q] = T(0);
            if (act) {
                const int gy = y0 - 1 + ly;
                const int my = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
                kv[q] = L0.k[(long long)my * pitch + gx];
                if (gy >= 0 && gy < ny) {
                    pv[q] = src[(long long)gy * pitch + gx];
                    if constexpr (COMP) lv[q] = src[lo_off + (long long)gy * pitch + gx];
                }
            }
        }
#pragma unroll
        for (int q = 0; q <= TILE_ROWS; q++) {
            const int ly = q < TILE_ROWS ? warp + q * (QT / 32) : ey;
            const int lx = q < TILE_ROWS ? lane : ex;
            if (q < TILE_ROWS ? ly < SY + 2 : extra) {
                sk[ly][lx] = kv[q];
                sp[ly][lx] = pv[q];
                if constexpr (COMP) sl[ly][lx] = lv[q];
            }
        }
    }
    __syncthreads();
    if (add_coarse) {  // ghost rows are never read: the mirror is used instead
        for (int t = tid; t < (SX + 2) * (SY + 2); t += QT) {
            const int lx = t % (SX + 2), ly = t / (SX + 2), gy = y0 - 1 + ly;
            if (gy >= 0 && gy < ny) {
                if constexpr (COMP) comp_add(sp[ly][lx], sl[ly][lx], prolong_at(pt, L1, lx, ly));
                else sp[ly][lx] += prolong_at(pt, L1, lx, ly);
            }
        }
        __syncthreads();
    }
    const int qx = 2 * (tid % (SX / 2)), qy = 2 * (tid / (SX / 2));
    // W: the tile holds a wall row, whose nodes take the ghost rules
    auto sweep_tile = [&](auto wall) {
        constexpr bool W = decltype(wall)::value;
        Node9<T> nd[4];
        T inv_diag[4];
        bool own[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {  // colour c = (x & 1) + 2 (y & 1) is quad node (c & 1, c >> 1)
            const int lx = qx + (c & 1) + 1, ly = qy + (c >> 1) + 1;
            const int x = x0 + lx - 1, y = y0 + ly - 1;
            own[c] = x < nx && y < ny;
            inv_diag[c] = T(0);
            if (own[c]) {
                if constexpr (keeps_coef<T>()) {
                    coef_load(L0, (long long)y * pitch + x, nd[c], inv_diag[c]);
                } else {
                    auto kat = [&](int dx, int dy) { return sk[ly + dy][lx + dx]; };
                    if constexpr (COMP) nd[c] = node9_pairs<W>(kat, y, ny, H0c, H0s);
                    else nd[c] = node9<T, W>(kat, y, ny, H0c, H0s);
                    inv_diag[c] = T(1) / nd[c].diag;
                }
                if (L0.rhs) nd[c].b = L0.rhs[(long long)y * pitch + x];
            }
        }
        for (int s = 0; s < sweeps; s++) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int lx = qx + (c & 1) + 1, ly = qy + (c >> 1) + 1, y = y0 + ly - 1;
                auto pat = [&](int dx, int dy) { return sp[ly + dy][lx + dx]; };
                if (own[c]) {
                    if constexpr (COMP) {  // correction form: dr/dpsi'_0 = diag, so psi'_0 -= r_0 / diag
                        auto lat = [&](int dx, int dy) { return sl[ly + dy][lx + dx]; };
                        const float r = resid_pairs<W>(nd[c], pat, lat, y, ny);
                        comp_add(sp[ly][lx], sl[ly][lx], -r * inv_diag[c]);
                    } else {
                        sp[ly][lx] = (off9<T, W>(nd[c], pat, y, ny) - nd[c].b) * inv_diag[c];
                    }
                }
                __syncthreads();
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int lx = qx + (c & 1) + 1, ly = qy + (c >> 1) + 1;
            if (own[c]) {
                const long long n = (long long)(y0 + ly - 1) * pitch + (x0 + lx - 1);
                dst[n] = sp[ly][lx];
                if constexpr (COMP) dst[lo_off + n] = sl[ly][lx];
            }
        }
    };
    if (!SPLIT || y0 == 0 || y0 + SY >= ny) sweep_tile(std::true_type{});
    else sweep_tile(std::false_type{});
    __syncthreads();
    if (tid == 0) {
        const unsigned lin = (unsigned)(by * ((nx + SX - 1) / SX) + bx);
        if (tile_done(ctl, L0.grp, lin, nblocks, 0ull)) cycle_close(ctl);
    }
}

template <typename T, bool COMP>
__global__ void __launch_bounds__(QT) smooth0(Level<T> L0, Level<TC> L1, int add_coarse,
                                              int sweeps, T H0c, T H0s, MgCtl *ctl, int first) {
    smooth0_tile<T, COMP>(L0, L1, add_coarse, sweeps, H0c, H0s, ctl, first, blockIdx.x, blockIdx.y,
                          gridDim.x * gridDim.y);
}

// Host-side dispatch on the lattice level's form (FP32: one plane or the pair).
template <typename T>
static void launch_smooth0(const Level<T> &L0, const Level<TC> &L1, int add, int sweeps, T H0c,
                           T H0s, MgCtl *ctl, int first, cudaStream_t s) {
    const dim3 g((L0.nx + SX - 1) / SX, (L0.ny + SY - 1) / SY);
    if constexpr (sizeof(T) == 4) {
        if (L0.comp) {
            smooth0<T, true><<<g, QT, 0, s>>>(L0, L1, add, sweeps, H0c, H0s, ctl, first);
            return;
        }
    }
    smooth0<T, false><<<g, QT, 0, s>>>(L0, L1, add, sweeps, H0c, H0s, ctl, first);
}

template <typename T>
static void launch_resid0(const Level<T> &L0, const Level<TC> &L1, T H0c, T H0s, MgCtl *ctl,
                          cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hi, int in_graph,
                          cudaStream_t s) {
    const dim3 b(32, 8), g((L1.nx + 31) / 32, (L1.ny + 7) / 8);
    if constexpr (sizeof(T) == 4) {
        if (L0.comp) {
            resid0_restrict<T, true><<<g, b, 0, s>>>(L0, L1, H0c, H0s, ctl, hw, hi, in_graph);
            return;
        }
    }
    resid0_restrict<T, false><<<g, b, 0, s>>>(L0, L1, H0c, H0s, ctl, hw, hi, in_graph);
}

// ------------------------------------------------------------- coarse levels
template <typename T>
struct FV {
    T te, tw, tn, ts;     // face transmissibilities (tn/ts to the wall when at the edge)
    int ie, iw;           // periodic neighbours
    bool hasn, hass;      // neighbour inside (false: wall with value 0)
};

template <typename T, typename KF>
__device__ __forceinline__ FV<T> fv_coef(const Level<T> &L, int I, int J, KF kat) {
    FV<T> f;
    const int nx = L.nx, ny = L.ny;
    const T k0 = kat(0, 0);
    f.ie = I + 1 == nx ? 0 : I + 1;
    f.iw = I == 0 ? nx - 1 : I - 1;
    f.te = T(0.5) * (k0 + kat(1, 0)) * L.wy[J] * L.ixe[I];
    f.tw = T(0.5) * (k0 + kat(-1, 0)) * L.wy[J] * L.ixe[f.iw];
    f.hasn = J + 1 < ny;
    f.hass = J > 0;
    f.tn = (f.hasn ? T(0.5) * (k0 + kat(0, 1)) : k0) * L.wx[I] * L.iyn[J];
    f.ts = (f.hass ? T(0.5) * (k0 + kat(0, -1)) : k0) * L.wx[I] * L.iys[J];
    return f;
}

__device__ __forceinline__ int fv_colour(int I, int J, int nx) {
    return ((nx & 1) && I == nx - 1) ? 2 + (J & 1) : ((I + J) & 1);
}

// Residual b - A e of a coarse level held in global memory (e given).
template <typename T>
__device__ __forceinline__ T fv_resid_global(const Level<T> &L, const T *e, int I, int J) {
    const int p = L.pitch, ny = L.ny;
    auto kat = [&](int dx, int dy) {
        int ii = I + dx;
        ii = ii < 0 ? L.nx - 1 : (ii >= L.nx ? 0 : ii);
        return L.k[(long long)(J + dy) * p + ii];
    };
    const FV<T> f = fv_coef(L, I, J, kat);
    const T e0 = e[(long long)J * p + I];
    T s = f.te * e[(long long)J * p + f.ie] + f.tw * e[(long long)J * p + f.iw];
    if (f.hasn) s += f.tn * e[(long long)(J + 1) * p + I];
    if (f.hass) s += f.ts * e[(long long)(J - 1) * p + I];
    (void)ny;
    return L.b[(long long)J * p + I] - (s - (f.te + f.tw + f.tn + f.ts) * e0);
}

// Tiled block Gauss-Seidel on a grid-wide coarse level. KIND 0 (pre-smoothing):
// zero initial guess, output to L.r. KIND 1 (post-smoothing): L.r plus the
// coarse correction, output to L.e. KIND 2 (two-grid solve): zero initial
// guess, output to L.e.
template <typename T, int KIND>
__device__ __forceinline__ void fv_smooth_tile(const Level<T> &L, const Level<T> &C, int sweeps,
                                               MgCtl *ctl, int bx, int by) {
    constexpr bool POST = KIND == 1;
    if (block_skip(ctl)) return;
    __shared__ T se[SY + 2][SX + 2];
    __shared__ T sk[SY + 2][SX + 2];
    const int nx = L.nx, ny = L.ny, p = L.pitch;
    const int x0 = bx * SX, y0 = by * SY;
    __shared__ ProlongTile<T, SX + 2, SY + 2> pt;
    if (POST) prolong_tile_load(pt, L, x0 - 1, y0 - 1);
    for (int t = threadIdx.y * SX + threadIdx.x; t < (SX + 2) * (SY + 2); t += SX * SY) {
        const int lx = t % (SX + 2), ly = t / (SX + 2);
        int gx = x0 - 1 + lx;
        if (gx < 0) gx += nx;
        while (gx >= nx) gx -= nx;
        const int gy = y0 - 1 + ly;
        T kv = T(0), ev = T(0);
        if (gy >= 0 && gy < ny) {
            kv = L.k[(long long)gy * p + gx];
            if (POST) ev = L.r[(long long)gy * p + gx];
        }
        sk[ly][lx] = kv;
        se[ly][lx] = ev;
    }
    __syncthreads();
    if (POST) {
        for (int t = threadIdx.y * SX + threadIdx.x; t < (SX + 2) * (SY + 2); t += SX * SY) {
            const int lx = t % (SX + 2), ly = t / (SX + 2), gy = y0 - 1 + ly;
            if (gy >= 0 && gy < ny) se[ly][lx] += prolong_at(pt, C, lx, ly);
        }
        __syncthreads();
    }
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
    const int I = x0 + threadIdx.x, J = y0 + threadIdx.y;
    const bool own = I < nx && J < ny;
    FV<T> f;
    T idg = T(0), b = T(0);
    if (own) {
        auto kat = [&](int dx, int dy) { return sk[ly + dy][lx + dx]; };
        f = fv_coef(L, I, J, kat);
        idg = T(1) / (f.te + f.tw + f.tn + f.ts);
        b = L.b[(long long)J * p + I];
    }
    const int colour = own ? fv_colour(I, J, nx) : -1;
    const int ncol = (nx & 1) ? 4 : 2;
    for (int s = 0; s < sweeps; s++)
        for (int c = 0; c < ncol; c++) {
            if (colour == c) {
                T v = f.te * se[ly][lx + 1] + f.tw * se[ly][lx - 1];
                if (f.hasn) v += f.tn * se[ly + 1][lx];
                if (f.hass) v += f.ts * se[ly - 1][lx];
                se[ly][lx] = (v - b) * idg;
            }
            __syncthreads();
        }
    if (own) (KIND == 0 ? L.r : L.e)[(long long)J * p + I] = se[ly][lx];
}

template <typename T, int KIND>
__global__ void __launch_bounds__(SX *SY) fv_smooth(Level<T> L, Level<T> C, int sweeps,
                                                    MgCtl *ctl) {
    fv_smooth_tile<T, KIND>(L, C, sweeps, ctl, blockIdx.x, blockIdx.y);
}

// Residual of a grid-wide level (pre-smoothed iterate in F.r) summed onto the
// next level, and the next level's permeability (area-weighted mean).
template <typename T>
__device__ __forceinline__ void fv_resid_tile(const Level<T> &F, const Level<T> &C, MgCtl *ctl,
                                              int bx, int by) {
    if (cycle_skip(ctl)) return;
    const int I = bx * 32 + threadIdx.x, J = by * 8 + threadIdx.y;
    if (I >= C.nx || J >= C.ny) return;
    T sr = T(0), sk = T(0);
    for (int j = C.cy0[J]; j < C.cy0[J + 1]; j++)
        for (int i = C.cx0[I]; i < C.cx0[I + 1]; i++) {
            sr += fv_resid_global(F, F.r, i, j);
            sk += F.k[(long long)j * F.pitch + i] * F.wx[i] * F.wy[j];
        }
    C.b[(long long)J * C.pitch + I] = sr;
    C.k[(long long)J * C.pitch + I] = sk / (C.wx[I] * C.wy[J]);
}

template <typename T>
__global__ void __launch_bounds__(256) fv_resid_restrict(Level<T> F, Level<T> C, MgCtl *ctl) {
    fv_resid_tile<T>(F, C, ctl, blockIdx.x, blockIdx.y);
}

// ---- levels lc .. nl-1 inside one block, resident in shared memory.
// Per level: e, b, k, te (east face), tn (north face, wall at the top), and dg,
// the reciprocal of the diagonal.
constexpr int MAX_LEVELS = 24;
constexpr int CTA_ARRAYS = 6;

template <typename T>
struct CtaView {
    T *e, *b, *k, *te, *tn, *dg;
};

template <typename T>
__device__ __forceinline__ CtaView<T> cta_view(T *sm, const int *off, const Level<T> *L, int l) {
    const int n = L[l].nx * L[l].ny;
    T *base = sm + off[l];
    return CtaView<T>{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n};
}

template <typename T>
__device__ __forceinline__ void cta_gs(const Level<T> &L, const CtaView<T> &V, int sweeps,
                                       int tid, int nthr, bool warp_only) {
    const int nx = L.nx, ny = L.ny, n = nx * ny, ncol = (nx & 1) ? 4 : 2;
    for (int s = 0; s < sweeps; s++)
        for (int c = 0; c < ncol; c++) {
            for (int t = tid; t < n; t += nthr) {
                const int I = t % nx, J = t / nx;
                if (fv_colour(I, J, nx) != c) continue;
                const int iw = I == 0 ? nx - 1 : I - 1, ie = I + 1 == nx ? 0 : I + 1;
                T v = V.te[t] * V.e[J * nx + ie] + V.te[J * nx + iw] * V.e[J * nx + iw];
                if (J + 1 < ny) v += V.tn[t] * V.e[t + nx];
                if (J > 0) v += V.tn[t - nx] * V.e[t - nx];
                V.e[t] = (v - V.b[t]) * V.dg[t];
            }
            if (warp_only) __syncwarp();
            else __syncthreads();
        }
}

template <typename T>
__device__ __forceinline__ void coarse_cta_block(const Level<T> *lv, int lc, int nl, MgCtl *ctl) {
    if (cycle_skip(ctl)) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ Level<T> L[MAX_LEVELS];
    __shared__ int off[MAX_LEVELS];
    T *sm = reinterpret_cast<T *>(smraw);
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid < nl) L[tid] = lv[tid];
    __syncthreads();
    if (tid == 0) {
        int o = 0;
        for (int l = lc; l < nl; l++) { off[l] = o; o += CTA_ARRAYS * L[l].nx * L[l].ny; }
    }
    __syncthreads();
    // inputs of level lc; permeabilities of the deeper levels
    {
        const CtaView<T> V = cta_view(sm, off, L, lc);
        const int nx = L[lc].nx, n = nx * L[lc].ny;
        for (int t = tid; t < n; t += nthr) {
            const long long g = (long long)(t / nx) * L[lc].pitch + t % nx;
            V.b[t] = L[lc].b[g];
            V.k[t] = L[lc].k[g];
            V.e[t] = T(0);
        }
        __syncthreads();
    }
    for (int l = lc + 1; l < nl; l++) {
        const CtaView<T> F = cta_view(sm, off, L, l - 1), V = cta_view(sm, off, L, l);
        const Level<T> &C = L[l], &Fl = L[l - 1];
        for (int t = tid; t < C.nx * C.ny; t += nthr) {
            const int I = t % C.nx, J = t / C.nx;
            T s = T(0);
            for (int j = C.cy0[J]; j < C.cy0[J + 1]; j++)
                for (int i = C.cx0[I]; i < C.cx0[I + 1]; i++) s += F.k[j * Fl.nx + i] * Fl.wx[i] * Fl.wy[j];
            V.k[t] = s / (C.wx[I] * C.wy[J]);
        }
        __syncthreads();
    }
    for (int l = lc; l < nl; l++) {  // face coefficients and diagonals
        const CtaView<T> V = cta_view(sm, off, L, l);
        const Level<T> &C = L[l];
        const int nx = C.nx;
        for (int t = tid; t < nx * C.ny; t += nthr) {
            const int I = t % nx, J = t / nx;
            auto kat = [&](int dx, int dy) {
                int ii = I + dx;
                ii = ii < 0 ? nx - 1 : (ii >= nx ? 0 : ii);
                return V.k[(J + dy) * nx + ii];
            };
            const FV<T> f = fv_coef(C, I, J, kat);
            V.te[t] = f.te;
            V.tn[t] = f.tn;
            V.dg[t] = T(1) / (f.te + f.tw + f.tn + f.ts);  // reciprocal of the diagonal
        }
    }
    __syncthreads();
    // V-cycle: down
    for (int l = lc; l < nl - 1; l++) {
        const CtaView<T> F = cta_view(sm, off, L, l), V = cta_view(sm, off, L, l + 1);
        cta_gs(L[l], F, NU_CTA, tid, nthr, false);
        const Level<T> &C = L[l + 1];
        const int fnx = L[l].nx, fny = L[l].ny;
        for (int t = tid; t < C.nx * C.ny; t += nthr) {
            const int I = t % C.nx, J = t / C.nx;
            T s = T(0);
            for (int j = C.cy0[J]; j < C.cy0[J + 1]; j++)
                for (int i = C.cx0[I]; i < C.cx0[I + 1]; i++) {
                    const int q = j * fnx + i;
                    const int iw = i == 0 ? fnx - 1 : i - 1, ie = i + 1 == fnx ? 0 : i + 1;
                    T v = F.te[q] * F.e[j * fnx + ie] + F.te[j * fnx + iw] * F.e[j * fnx + iw];
                    if (j + 1 < fny) v += F.tn[q] * F.e[q + fnx];
                    if (j > 0) v += F.tn[q - fnx] * F.e[q - fnx];
                    s += F.b[q] - (v - F.e[q] / F.dg[q]);
                }
            V.b[t] = s;
            V.e[t] = T(0);
        }
        __syncthreads();
    }
    {  // coarsest (<= 100 cells, walls at most a few cells away: GS converges fast)
        const CtaView<T> V = cta_view(sm, off, L, nl - 1);
        cta_gs(L[nl - 1], V, NU_COARSEST, tid, nthr, false);
    }
    // up
    for (int l = nl - 2; l >= lc; l--) {
        const CtaView<T> F = cta_view(sm, off, L, l), V = cta_view(sm, off, L, l + 1);
        const Level<T> &Fl = L[l];
        for (int t = tid; t < Fl.nx * Fl.ny; t += nthr) {
            const int i = t % Fl.nx, j = t / Fl.nx;
            const int x0 = Fl.px0[i], x1 = Fl.px1[i], y0 = Fl.py0[j], y1 = Fl.py1[j];
            const T wx = Fl.pwx[i], wy = Fl.pwy[j];
            const int cnx = L[l + 1].nx;
            T a = T(0), b = T(0);
            if (y0 >= 0) a = (T(1) - wx) * V.e[y0 * cnx + x0] + wx * V.e[y0 * cnx + x1];
            if (y1 >= 0) b = (T(1) - wx) * V.e[y1 * cnx + x0] + wx * V.e[y1 * cnx + x1];
            F.e[t] += (T(1) - wy) * a + wy * b;
        }
        __syncthreads();
        cta_gs(L[l], F, NU_CTA, tid, nthr, false);
    }
    {
        const CtaView<T> V = cta_view(sm, off, L, lc);
        const int nx = L[lc].nx, n = nx * L[lc].ny;
        for (int t = tid; t < n; t += nthr) L[lc].e[(long long)(t / nx) * L[lc].pitch + t % nx] = V.e[t];
    }
}

template <typename T>
__global__ void __launch_bounds__(CTA_THREADS) coarse_cta(const Level<T> *lv, int lc, int nl,
                                                         MgCtl *ctl) {
    coarse_cta_block<T>(lv, lc, nl, ctl);
}

// Start of a cycle (one thread, after the lattice residual is complete):
// converged, capped or non-finite -> record the result and stop; otherwise run
// a V-cycle, or only lattice sweeps when the residual is already close to the
// tolerance. In a graph it sets the loop and switch conditions (in_graph 1),
// or the loop condition only (in_graph 3: the loop body's dispatch kernel sets
// the switch from ctl->mode).
__device__ void cycle_decide(MgCtl *ctl, cudaGraphConditionalHandle hw,
                             cudaGraphConditionalHandle hi, int in_graph) {
    ctl->cycles_launched++;
    if (!ctl->done) {
        const double nrm = norm_of(ctl);
        if (nrm <= ctl->tolH0 || ctl->iter >= ctl->max_iter || !(nrm < INFINITY)) {
            ctl->done = 1;
            ctl->converged = nrm <= ctl->tolH0;
            if (!ctl->converged) ctl->nonconv_count++;
            ctl->last_resid = ctl->H0 > 0.0 ? nrm / ctl->H0 : 0.0;
            ctl->last_iters = ctl->iter;
        }
    }
    ctl->keep_going = !ctl->done;
    if (ctl->done) {
        ctl->mode = 3;
    } else if (ctl->smooth_left > 0 && norm_of(ctl) <= SMOOTH_RATIO * ctl->tolH0) {
        ctl->mode = 1;  // close to the tolerance: lattice sweeps only
        ctl->smooth_left--;
    } else if (ctl->twogrid_left > 0) {
        ctl->mode = 2;  // two-grid cycle
        ctl->twogrid_left--;
        ctl->smooth_left = 0;
    } else {
        ctl->mode = 0;  // full V-cycle
    }
    if (in_graph == 1) {
        // switch node: 0 V-cycle, 1 lattice sweeps, 2 two-grid, 3 no body
        cudaGraphSetConditional(hi, (unsigned)ctl->mode);
        cudaGraphSetConditional(hw, ctl->keep_going ? 1u : 0u);
    } else if (in_graph == 3) {  // the loop condition only (the body dispatches the mode)
        cudaGraphSetConditional(hw, ctl->keep_going ? 1u : 0u);
    }
}

__global__ void cycle_dispatch_kernel(MgCtl *ctl, cudaGraphConditionalHandle hs) {
    if (threadIdx.x == 0) {
        ctl->dispatches++;
        cudaGraphSetConditional(hs, (unsigned)ctl->mode);
    }
}



// End of a full cycle (one thread): count it, flip the lattice buffer, clear
// the norm for the next residual.
__device__ void cycle_close(MgCtl *ctl) {
    ctl->iter++;
    if (ctl->mode == 1) ctl->smooth_cycles++;
    else if (ctl->mode == 2) ctl->twogrid_cycles++;
    else ctl->total_cycles++;
    ctl->cur ^= 1;
    ctl->norm_bits = 0ull;
}

// ------------------------------------------------------------------ host side
template <typename T>
struct MgHost {
    int nl = 0, lc = 1;
    bool coef_shared = false;   // level-0 coefficient planes are another hierarchy's
    Level<T> L0;                // the lattice level
    std::vector<Level<TC>> lv;  // levels 1 .. nl-1 (entry 0 unused)
    Level<TC> *d_lv = nullptr;
    MgCtl *ctl = nullptr;
    std::vector<void *> mem;
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *user = nullptr;
    size_t cta_smem = 0;
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
                     char *err, size_t errlen, int comp, const MgHost<T> *share_coef) {
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
        if ((!cxo && !cyo) || (fx.size() > 1 && (long long)px * py <= MIN_COARSE)) break;
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
    // levels lc..nl-1 run in one block with their arrays in shared memory:
    // the first level from which the rest fits the budget
    // (one SM's issue rate bounds that block, so it only takes the small levels)
    m->lc = m->nl - 1;
    for (int l = 1; l < m->nl; l++) {
        size_t bytes = 0, cells = 0;
        for (int q = l; q < m->nl; q++) {
            cells += xcs[q].size() * ycs[q].size();
            bytes += (size_t)CTA_ARRAYS * xcs[q].size() * ycs[q].size() * sizeof(TC);
        }
        if (bytes <= CTA_SMEM_MAX && cells <= CTA_CELLS) { m->lc = l; break; }
    }
    m->cta_smem = 0;
    for (int q = m->lc; q < m->nl; q++) m->cta_smem += (size_t)CTA_ARRAYS * xcs[q].size() * ycs[q].size() * sizeof(TC);
    if (m->nl > MAX_LEVELS || m->cta_smem > CTA_SMEM_MAX) {
        snprintf(err, errlen, "multigrid: hierarchy too deep or coarse levels too large");
        mg_destroy(m);
        return nullptr;
    }
    // The limit is a property of the kernel, shared by every context in the
    // process: set it to the fixed budget, not to this hierarchy's need.
    if (cudaFuncSetAttribute(coarse_cta<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CTA_SMEM_MAX) != cudaSuccess) {
        snprintf(err, errlen, "multigrid: cannot reserve %zu bytes of shared memory", m->cta_smem);
        mg_destroy(m);
        return nullptr;
    }
    // geometry of level l in the level's own type U
    auto geometry = [&](auto &L, int l) {
        using U = typename std::remove_reference_t<decltype(L)>::value_type;
        L.nx = (int)xcs[l].size();
        L.ny = (int)ycs[l].size();
        L.Lx = U(nx);
        L.ylo = U(0);
        L.yhi = U(ny);
        std::vector<U> xc(L.nx), wx(L.nx), yc(L.ny), wy(L.ny);
        for (int i = 0; i < L.nx; i++) { xc[i] = U(xcs[l][i]); wx[i] = U(fx[l][i + 1] - fx[l][i]); }
        for (int j = 0; j < L.ny; j++) { yc[j] = U(ycs[l][j]); wy[j] = U(fy[l][j + 1] - fy[l][j]); }
        L.xc = up.put<U>(xc.data(), xc.size() * sizeof(U));
        L.wx = up.put<U>(wx.data(), wx.size() * sizeof(U));
        L.yc = up.put<U>(yc.data(), yc.size() * sizeof(U));
        L.wy = up.put<U>(wy.data(), wy.size() * sizeof(U));
        {  // inverse centre distances (periodic in x; walls at 0 and ny in y)
            std::vector<U> ixe(L.nx), iyn(L.ny), iys(L.ny);
            for (int i = 0; i < L.nx; i++) {
                const double d = i + 1 == L.nx ? xcs[l][0] + nx - xcs[l][i] : xcs[l][i + 1] - xcs[l][i];
                ixe[i] = U(1.0 / d);
            }
            for (int j = 0; j < L.ny; j++) {
                const double dn = j + 1 < L.ny ? ycs[l][j + 1] - ycs[l][j] : double(ny) - ycs[l][j];
                const double ds = j > 0 ? ycs[l][j] - ycs[l][j - 1] : ycs[l][j];
                iyn[j] = U(1.0 / dn);
                iys[j] = U(1.0 / ds);
            }
            L.ixe = up.put<U>(ixe.data(), ixe.size() * sizeof(U));
            L.iyn = up.put<U>(iyn.data(), iyn.size() * sizeof(U));
            L.iys = up.put<U>(iys.data(), iys.size() * sizeof(U));
        }
        if (l + 1 < m->nl) {  // interpolation from level l + 1 onto level l
            std::vector<int> a0, a1, b0, b1;
            std::vector<U> wa, wb;
            interp_table<U>(xcs[l], xcs[l + 1], double(nx), 0, 0, a0, a1, wa);
            interp_table<U>(ycs[l], ycs[l + 1], -1.0, 0.0, double(ny), b0, b1, wb);
            L.px0 = up.put<int>(a0.data(), a0.size() * sizeof(int));
            L.px1 = up.put<int>(a1.data(), a1.size() * sizeof(int));
            L.pwx = up.put<U>(wa.data(), wa.size() * sizeof(U));
            L.py0 = up.put<int>(b0.data(), b0.size() * sizeof(int));
            L.py1 = up.put<int>(b1.data(), b1.size() * sizeof(int));
            L.pwy = up.put<U>(wb.data(), wb.size() * sizeof(U));
        }
    };
    {
        Level<T> &L = m->L0;
        std::memset(&L, 0, sizeof(L));
        geometry(L, 0);
        L.pitch = pitch;
        L.k = k0;
        L.e = psiA;
        L.r = psiB;
        L.comp = sizeof(T) == 4 && comp ? 1 : 0;
        {
            const std::vector<MgGroup> zero(MG_GROUPS, MgGroup{});
            L.grp = up.put<MgGroup>(zero.data(), MG_GROUPS * sizeof(MgGroup));
        }
        if (keeps_coef<T>()) {
            if (share_coef) {  // same lattice and k: the other hierarchy forms them
                L.coef = share_coef->L0.coef;
                m->coef_shared = true;
            } else {
                L.coef = up.put<T>(nullptr, (size_t)COEF * pitch * ny * sizeof(T));
            }
        }
    }
    for (int l = 0; l < m->nl; l++) {
        Level<TC> &L = m->lv[l];
        std::memset(&L, 0, sizeof(L));
        if (l == 0) continue;  // the lattice level is m->L0
        geometry(L, l);
        L.pitch = L.nx;
        const size_t cells = (size_t)L.nx * L.ny;
        L.e = up.put<TC>(nullptr, cells * sizeof(TC));
        L.r = up.put<TC>(nullptr, cells * sizeof(TC));
        L.b = up.put<TC>(nullptr, cells * sizeof(TC));
        L.k = up.put<TC>(nullptr, cells * sizeof(TC));
        L.cx0 = up.put<int>(cx0[l].data(), cx0[l].size() * sizeof(int));
        L.cy0 = up.put<int>(cy0[l].data(), cy0[l].size() * sizeof(int));
    }
    m->d_lv = up.put<Level<TC>>(m->lv.data(), m->lv.size() * sizeof(Level<TC>));
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
void mg_cycle_dispatch(MgHost<T> *m, cudaGraphConditionalHandle hs, cudaStream_t s) {
    cycle_dispatch_kernel<<<1, 32, 0, s>>>(m->ctl, hs);
}

template <typename T>
void mg_cycle_head(MgHost<T> *m, T H0c, T H0s, cudaGraphConditionalHandle hw,
                   cudaGraphConditionalHandle hi, int in_graph, cudaStream_t s) {
    const std::vector<Level<TC>> &lv = m->lv;
    launch_resid0<T>(m->L0, lv[1], H0c, H0s, m->ctl, hw, hi, in_graph, s);
}

template <typename T>
void mg_cycle_rest(MgHost<T> *m, T H0c, T H0s, cudaStream_t s) {
    dim3 b(32, 8), bs(SX, SY);
    const std::vector<Level<TC>> &lv = m->lv;
    for (int l = 1; l < m->lc; l++) {
        fv_smooth<TC, 0><<<g2(lv[l].nx, lv[l].ny, bs), bs, 0, s>>>(lv[l], lv[l + 1], NU_PRE, m->ctl);
        fv_resid_restrict<TC><<<g2(lv[l + 1].nx, lv[l + 1].ny, b), b, 0, s>>>(lv[l], lv[l + 1], m->ctl);
    }
    coarse_cta<TC><<<1, CTA_THREADS, m->cta_smem, s>>>(m->d_lv, m->lc, m->nl, m->ctl);
    for (int l = m->lc - 1; l >= 1; l--)
        fv_smooth<TC, 1><<<g2(lv[l].nx, lv[l].ny, bs), bs, 0, s>>>(lv[l], lv[l + 1], NU_POST, m->ctl);
    launch_smooth0<T>(m->L0, lv[1], 1, NU_FINE, H0c, H0s, m->ctl, 0, s);
}

template <typename T>
void mg_cycle_smooth(MgHost<T> *m, T H0c, T H0s, cudaStream_t s) {
    const std::vector<Level<TC>> &lv = m->lv;
    launch_smooth0<T>(m->L0, lv[1], 0, NU_SMOOTH_ONLY, H0c, H0s, m->ctl, 0, s);
}

template <typename T>
void mg_presmooth(MgHost<T> *m, T H0c, T H0s, cudaStream_t s) {
    const std::vector<Level<TC>> &lv = m->lv;
    if (keeps_coef<T>() && !m->coef_shared) {  // the solve's node coefficients, before its first sweep
        dim3 b(32, 8);
        coef0_kernel<T><<<g2(m->L0.nx, m->L0.ny, b), b, 0, s>>>(m->L0, H0c, H0s);
    }
    launch_smooth0<T>(m->L0, lv[1], 0, NU_SMOOTH_ONLY, H0c, H0s, m->ctl, 1, s);
}

template <typename T>
void mg_cycle_twogrid(MgHost<T> *m, T H0c, T H0s, cudaStream_t s) {
    dim3 bs(SX, SY);
    const std::vector<Level<TC>> &lv = m->lv;
    fv_smooth<TC, 2><<<g2(lv[1].nx, lv[1].ny, bs), bs, 0, s>>>(lv[1], lv[1], NU_TWOGRID, m->ctl);
    launch_smooth0<T>(m->L0, lv[1], 1, NU_FINE, H0c, H0s, m->ctl, 0, s);
}

template <typename T>
int mg_kernels_per_cycle(const MgHost<T> *m) { return 2 + 3 * (m->lc - 1); }  // after the head

template <typename T>
int mg_levels(const MgHost<T> *m) { return m->nl; }

// ------------------------------------------------------------ batched solves
// The potential solves of many FP32 channels driven by one fixed set of
// kernels: each kernel runs over a work list of (instance, tile) entries that
// spans every instance, and each block does its instance's part of the cycle
// its instance's control block chose (blocks of instances in another mode, or
// already converged, return at once). Per-instance completion is counted per
// control block against the instance's own tile count; the last block of the
// whole residual launch keeps the batch's loop going while any solve is.
struct MgBatchInst {
    Level<float> L0;
    const Level<TC> *lv;  // the instance's device level table (entry 0 unused)
    int nl, lc;
    MgCtl *ctl;
    float H0c, H0s;
    unsigned n0;  // level-0 smoothing tiles
    unsigned n1;  // residual blocks (32 x 8 level-1 cells)
    int gx0, gx1; // tiles per row of the two
};
// A work-list entry: cnt consecutive tiles (row-major from (bx, by)) of one
// instance at level lvl. The lists hold CHUNK tiles per entry (measured on the
// 96-channel sweep: 8 tiles per block made the batched step 10% slower than 1).
struct MgBatchTile {
    int inst, bx, by, lvl, cnt;
};
constexpr int CHUNK = 1;
struct MgBatchCtl {
    unsigned blocks_done;  // instances whose residual blocks have all run
    unsigned any;   // after a residual launch: 1 while some solve goes on
    unsigned any_v; // ... some instance runs a V-cycle in this pass
    unsigned any_t; // ... some instance runs a two-grid cycle in this pass
};

constexpr int BS_FIRST = 0;  // the sweeps that open every solve
constexpr int BS_CYCLE = 1;  // the lattice part that ends every cycle

template <bool COMP>
__global__ void __launch_bounds__(QT) smooth0_batch(const MgBatchInst *tab, const MgBatchTile *tiles,
                                                    int kind) {
    const MgBatchTile t = tiles[blockIdx.x];
    const MgBatchInst &I = tab[t.inst];
    int add = 0, sweeps = NU_SMOOTH_ONLY;
    if (kind == BS_CYCLE) {  // V-cycle and two-grid cycle: coarse correction; else sweeps only
        const int m = I.ctl->mode;
        if (m == 3) return;  // this solve is over (uniform across the block)
        add = m == 0 || m == 2;
        sweeps = add ? NU_FINE : NU_SMOOTH_ONLY;
    }
    const int q0 = t.by * I.gx0 + t.bx;
    for (int q = q0; q < q0 + t.cnt; q++) {
        smooth0_tile<float, COMP>(I.L0, I.lv[1], add, sweeps, I.H0c, I.H0s, I.ctl, kind == BS_FIRST,
                                  q % I.gx0, q / I.gx0, I.n0);
        __syncthreads();  // the tile's shared arrays are reused by the next one
    }
}

template <bool COMP>
__global__ void __launch_bounds__(256) resid0_batch(const MgBatchInst *tab, const MgBatchTile *tiles,
                                                    MgBatchCtl *bc, int ninst,
                                                    cudaGraphConditionalHandle hw,
                                                    cudaGraphConditionalHandle hv,
                                                    cudaGraphConditionalHandle ht, int in_graph) {
    const MgBatchTile t = tiles[blockIdx.x];
    const MgBatchInst &I = tab[t.inst];
    if (!I.ctl->done) {  // uniform across the block
        const int q0 = t.by * I.gx1 + t.bx;
        for (int q = q0; q < q0 + t.cnt; q++) {
            resid0_tile<float, COMP>(I.L0, I.lv[1], I.H0c, I.H0s, I.ctl, 0, 0, 0, q % I.gx1, q / I.gx1,
                                     I.n1, false);
            __syncthreads();  // the tile's shared arrays are reused by the next one
        }
    }
    // Completion is counted per instance (its control block), and the last block
    // of each instance counts the instance on the batch: one contended counter
    // update per instance, not per block.
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();
        if (atomicAdd(&I.ctl->batch_visits, (unsigned)t.cnt) + (unsigned)t.cnt != I.n1) return;
        I.ctl->batch_visits = 0;
        __threadfence();
        if (atomicAdd(&bc->blocks_done, 1u) == (unsigned)ninst - 1) {
            __threadfence();
            bc->blocks_done = 0;
            unsigned any = 0, any_v = 0, any_t = 0;
            for (int i = 0; i < ninst; i++) {
                const volatile MgCtl *c = tab[i].ctl;
                if (c->done) continue;
                any = 1u;
                any_v |= c->mode == 0 ? 1u : 0u;
                any_t |= c->mode == 2 ? 1u : 0u;
            }
            bc->any = any;
            bc->any_v = any_v;
            bc->any_t = any_t;
            if (in_graph) cudaGraphSetConditional(hw, any);  // the batch's loop
            if (in_graph == 1) {  // IF nodes around the V-cycle and two-grid kernels
                cudaGraphSetConditional(hv, any_v);
                cudaGraphSetConditional(ht, any_t);
            }
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(SX *SY) fv_smooth_batch(const MgBatchInst *tab,
                                                          const MgBatchTile *tiles, int sweeps) {
    const MgBatchTile t = tiles[blockIdx.x];
    const MgBatchInst &I = tab[t.inst];
    if (I.ctl->mode != (KIND == 2 ? 2 : 0)) return;
    const Level<TC> &L = I.lv[t.lvl];
    fv_smooth_tile<TC, KIND>(L, KIND == 2 ? L : I.lv[t.lvl + 1], sweeps, I.ctl, t.bx, t.by);
}

__global__ void __launch_bounds__(256) fv_resid_batch(const MgBatchInst *tab, const MgBatchTile *tiles) {
    const MgBatchTile t = tiles[blockIdx.x];
    const MgBatchInst &I = tab[t.inst];
    if (I.ctl->mode != 0) return;
    fv_resid_tile<TC>(I.lv[t.lvl], I.lv[t.lvl + 1], I.ctl, t.bx, t.by);
}

__global__ void __launch_bounds__(CTA_THREADS) coarse_batch(const MgBatchInst *tab, const int *inst) {
    const MgBatchInst &I = tab[inst[blockIdx.x]];
    if (I.ctl->mode != 0) return;
    coarse_cta_block<TC>(I.lv, I.lc, I.nl, I.ctl);
}

struct MgBatch {
    int ninst = 0, maxlc = 1;
    int comp = 0;  // the instances' level-0 form (one for the whole batch)
    MgBatchInst *d_tab = nullptr;
    MgBatchCtl *d_ctl = nullptr;
    int *d_inst = nullptr;                     // every instance (coarse blocks)
    MgBatchTile *d_t0 = nullptr, *d_t1 = nullptr, *d_tl1 = nullptr;
    int n_t0 = 0, n_t1 = 0, n_tl1 = 0;         // level-0 tiles, residual blocks, level-1 fv tiles
    std::vector<MgBatchTile *> d_fvs, d_fvr;   // per level l >= 1: fv tiles of l, restriction to l + 1
    std::vector<int> n_fvs, n_fvr;
    size_t cta_smem = 0;
    std::vector<void *> mem;
    void (*release)(void *, void *) = nullptr;
    void *user = nullptr;
};

MgBatch *mg_batch_create(const std::vector<MgHost<float> *> &ms, const std::vector<float> &H0c,
                         const std::vector<float> &H0s, void *(*alloc)(size_t, void *),
                         void (*release)(void *, void *), void *user, char *err, size_t errlen) {
    MgBatch *b = new MgBatch();
    b->release = release;
    b->user = user;
    b->ninst = (int)ms.size();
    b->comp = ms.empty() ? 0 : ms[0]->L0.comp;
    for (const MgHost<float> *m : ms)
        if (m->L0.comp != b->comp) {
            snprintf(err, errlen, "multigrid batch: instances of both level-0 forms");
            delete b;
            return nullptr;
        }
    Uploader up{alloc, user, &b->mem};
    std::vector<MgBatchInst> tab;
    std::vector<MgBatchTile> t0, t1, tl1;
    std::vector<int> ids;
    for (int i = 0; i < b->ninst; i++) {
        const MgHost<float> *m = ms[i];
        MgBatchInst I;
        std::memset(&I, 0, sizeof I);
        I.L0 = m->L0;
        I.lv = m->d_lv;
        I.nl = m->nl;
        I.lc = m->lc;
        I.ctl = m->ctl;
        I.H0c = H0c[i];
        I.H0s = H0s[i];
        const int gx0 = (m->L0.nx + SX - 1) / SX, gy0 = (m->L0.ny + SY - 1) / SY;
        const int gx1 = (m->lv[1].nx + 31) / 32, gy1 = (m->lv[1].ny + 7) / 8;
        const int gxl = (m->lv[1].nx + SX - 1) / SX, gyl = (m->lv[1].ny + SY - 1) / SY;
        I.n0 = (unsigned)(gx0 * gy0);
        I.n1 = (unsigned)(gx1 * gy1);
        I.gx0 = gx0;
        I.gx1 = gx1;
        tab.push_back(I);
        ids.push_back(i);
        for (int q = 0; q < gx0 * gy0; q += CHUNK)
            t0.push_back({i, q % gx0, q / gx0, 0, std::min(CHUNK, gx0 * gy0 - q)});
        for (int q = 0; q < gx1 * gy1; q += CHUNK)
            t1.push_back({i, q % gx1, q / gx1, 1, std::min(CHUNK, gx1 * gy1 - q)});
        for (int y = 0; y < gyl; y++)
            for (int x = 0; x < gxl; x++) tl1.push_back({i, x, y, 1, 1});
        b->maxlc = std::max(b->maxlc, m->lc);
        b->cta_smem = std::max(b->cta_smem, m->cta_smem);
    }
    b->d_fvs.assign(b->maxlc, nullptr);
    b->d_fvr.assign(b->maxlc, nullptr);
    b->n_fvs.assign(b->maxlc, 0);
    b->n_fvr.assign(b->maxlc, 0);
    for (int l = 1; l < b->maxlc; l++) {
        std::vector<MgBatchTile> fs, fr;
        for (int i = 0; i < b->ninst; i++) {
            const MgHost<float> *m = ms[i];
            if (m->lc <= l) continue;  // level l runs inside this instance's coarse block
            const Level<TC> &L = m->lv[l], &C = m->lv[l + 1];
            for (int y = 0; y < (L.ny + SY - 1) / SY; y++)
                for (int x = 0; x < (L.nx + SX - 1) / SX; x++) fs.push_back({i, x, y, l, 1});
            for (int y = 0; y < (C.ny + 7) / 8; y++)
                for (int x = 0; x < (C.nx + 31) / 32; x++) fr.push_back({i, x, y, l, 1});
        }
        b->n_fvs[l] = (int)fs.size();
        b->n_fvr[l] = (int)fr.size();
        b->d_fvs[l] = up.put<MgBatchTile>(fs.data(), fs.size() * sizeof(MgBatchTile));
        b->d_fvr[l] = up.put<MgBatchTile>(fr.data(), fr.size() * sizeof(MgBatchTile));
    }
    b->d_tab = up.put<MgBatchInst>(tab.data(), tab.size() * sizeof(MgBatchInst));
    b->d_inst = up.put<int>(ids.data(), ids.size() * sizeof(int));
    b->d_t0 = up.put<MgBatchTile>(t0.data(), t0.size() * sizeof(MgBatchTile));
    b->d_t1 = up.put<MgBatchTile>(t1.data(), t1.size() * sizeof(MgBatchTile));
    b->d_tl1 = up.put<MgBatchTile>(tl1.data(), tl1.size() * sizeof(MgBatchTile));
    MgBatchCtl zero{0u, 0u, 0u, 0u};
    b->d_ctl = up.put<MgBatchCtl>(&zero, sizeof zero);
    b->n_t0 = (int)t0.size();
    b->n_t1 = (int)t1.size();
    b->n_tl1 = (int)tl1.size();
    if (cudaFuncSetAttribute(coarse_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CTA_SMEM_MAX) != cudaSuccess) {
        snprintf(err, errlen, "batched multigrid: cannot reserve the coarse levels' shared memory");
        mg_batch_destroy(b);
        return nullptr;
    }
    if (!up.ok) {
        snprintf(err, errlen, "batched multigrid: device allocation or upload failed");
        mg_batch_destroy(b);
        return nullptr;
    }
    return b;
}

void mg_batch_destroy(MgBatch *b) {
    if (!b) return;
    for (void *p : b->mem) b->release(p, b->user);
    delete b;
}

void mg_batch_presmooth(MgBatch *b, cudaStream_t s) {
    if (b->comp) smooth0_batch<true><<<b->n_t0, QT, 0, s>>>(b->d_tab, b->d_t0, BS_FIRST);
    else smooth0_batch<false><<<b->n_t0, QT, 0, s>>>(b->d_tab, b->d_t0, BS_FIRST);
}

// One pass of the loop body, in three parts: every instance's cycle head
// (mg_batch_head); the coarse-level kernels of the V-cycle (mg_batch_vcycle)
// and of the two-grid cycle (mg_batch_twogrid), each acting only for the
// instances whose head chose it; and the lattice part that ends every cycle
// (mg_batch_close). In a graph the middle two sit in IF nodes whose conditions
// the head sets (hv, ht): a pass in which no instance chose that cycle skips
// their launches.
void mg_batch_head(MgBatch *b, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hv,
                   cudaGraphConditionalHandle ht, int in_graph, cudaStream_t s) {
    if (b->comp)
        resid0_batch<true><<<b->n_t1, dim3(32, 8), 0, s>>>(b->d_tab, b->d_t1, b->d_ctl, b->ninst, hw,
                                                           hv, ht, in_graph);
    else
        resid0_batch<false><<<b->n_t1, dim3(32, 8), 0, s>>>(b->d_tab, b->d_t1, b->d_ctl, b->ninst, hw,
                                                            hv, ht, in_graph);
}

void mg_batch_vcycle(MgBatch *b, cudaStream_t s) {
    for (int l = 1; l < b->maxlc; l++) {
        fv_smooth_batch<0><<<b->n_fvs[l], dim3(SX, SY), 0, s>>>(b->d_tab, b->d_fvs[l], NU_PRE);
        fv_resid_batch<<<b->n_fvr[l], dim3(32, 8), 0, s>>>(b->d_tab, b->d_fvr[l]);
    }
    coarse_batch<<<b->ninst, CTA_THREADS, b->cta_smem, s>>>(b->d_tab, b->d_inst);
    for (int l = b->maxlc - 1; l >= 1; l--)
        fv_smooth_batch<1><<<b->n_fvs[l], dim3(SX, SY), 0, s>>>(b->d_tab, b->d_fvs[l], NU_POST);
}

void mg_batch_twogrid(MgBatch *b, cudaStream_t s) {
    fv_smooth_batch<2><<<b->n_tl1, dim3(SX, SY), 0, s>>>(b->d_tab, b->d_tl1, NU_TWOGRID);
}

void mg_batch_close(MgBatch *b, cudaStream_t s) {
    if (b->comp) smooth0_batch<true><<<b->n_t0, QT, 0, s>>>(b->d_tab, b->d_t0, BS_CYCLE);
    else smooth0_batch<false><<<b->n_t0, QT, 0, s>>>(b->d_tab, b->d_t0, BS_CYCLE);
}

void mg_batch_body(MgBatch *b, cudaStream_t s) {
    mg_batch_head(b, 0, 0, 0, 0, s);
    mg_batch_vcycle(b, s);
    mg_batch_twogrid(b, s);
    mg_batch_close(b, s);
}

int mg_batch_body_kernels(const MgBatch *b) { return 4 + 3 * (b->maxlc - 1); }

int mg_batch_any(MgBatch *b, cudaStream_t s) {
    MgBatchCtl c;
    if (cudaMemcpyAsync(&c, b->d_ctl, sizeof c, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    return c.any ? 1 : 0;
}

// ------------------------------------------------------------ tangent solves
template <typename T>
void mg_set_rhs(MgHost<T> *m, const T *rhs) { m->L0.rhs = rhs; }

// The reset the phase kernel performs at the start of a solve, with the
// tolerance scaled by max |rhs| of the tangent right-hand side (the first
// residual check ends a solve whose right-hand side is zero).
__global__ void mg_reset_kernel(MgCtl *c, const unsigned long long *scale_bits, double tol,
                                int max_iter) {
    c->norm_bits = 0ull;
    c->iter = 0;
    c->done = 0;
    c->converged = 0;
    // a zero right-hand side: the solution is zero and the guess is kept
    const double scale = __longlong_as_double((long long)*scale_bits);
    c->tolH0 = scale > 0.0 ? tol * scale : INFINITY;
    c->max_iter = max_iter;
    c->keep_going = 1;
    c->blocks_done = 0u;
    c->mode = 1;
    c->smooth_left = 0;
    c->twogrid_left = 2;
}

void mg_reset_scaled(MgCtl *ctl, const unsigned long long *scale_bits, double tol, int max_iter,
                     cudaStream_t s) {
    mg_reset_kernel<<<1, 1, 0, s>>>(ctl, scale_bits, tol, max_iter);
}

// Differentiating L(k)(psi0 + psi') = 0 along one parameter direction:
// L(k) dpsi' = b(k, dH0) + b(dk, H0) - L(dk) psi', where b(k, H0) = -L(k) psi0
// is bilinear and L is linear in k, boundary rows included.
__global__ void __launch_bounds__(256) tangent_rhs_kernel(Level<double> L0, const double *dk,
                                                          double H0c, double H0s, double dH0c,
                                                          double dH0s, const MgCtl *ctl, double *rhs,
                                                          unsigned long long *rmax_bits) {
    const int nx = L0.nx, ny = L0.ny, pitch = L0.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    double ar = 0.0;
    if (x < nx && y < ny) {
        const double *psi = ctl->cur ? L0.r : L0.e;
        auto col = [&](int dx) {
            int xx = x + dx;
            return xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        };
        auto row = [&](int dy) {
            const int yy = y + dy;
            return yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy);  // mirrored ghost rows
        };
        auto kat = [&](int dx, int dy) { return L0.k[(long long)row(dy) * pitch + col(dx)]; };
        auto dkat = [&](int dx, int dy) { return dk[(long long)row(dy) * pitch + col(dx)]; };
        auto pat = [&](int dx, int dy) { return psi[(long long)(y + dy) * pitch + col(dx)]; };
        const Node9<double> nk = node9<double>(kat, y, ny, dH0c, dH0s);
        const Node9<double> nd = node9<double>(dkat, y, ny, H0c, H0s);
        const long long n = (long long)y * pitch + x;
        const double Ldk = off9<double>(nd, pat, y, ny) - nd.diag * psi[n];
        const double r = nk.b + nd.b - Ldk;
        rhs[n] = r;
        ar = fabs(r);
        ar = ar == ar ? ar : INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) ar = fmax(ar, __shfl_xor_sync(0xffffffffu, ar, o));
    if ((threadIdx.x & 31) == 0 && ar > 0.0) atomic_max_nonneg(rmax_bits, ar);
}

void mg_tangent_rhs(MgHost<double> *m, const double *dk, double H0c, double H0s, double dH0c,
                    double dH0s, double *rhs, unsigned long long *rmax_bits, cudaStream_t s) {
    dim3 b(32, 8);
    const Level<double> &L0 = m->L0;
    cudaMemsetAsync(rmax_bits, 0, sizeof(unsigned long long), s);
    tangent_rhs_kernel<<<g2(L0.nx, L0.ny, b), b, 0, s>>>(L0, dk, H0c, H0s, dH0c, dH0s, m->ctl, rhs,
                                                          rmax_bits);
}

__global__ void psi_io_kernel(const MgCtl *ctl, double *A, double *B, int op, double *plane,
                              double *prev, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *cur = ctl->cur ? B : A;
    if (op == 0) {
        plane[i] = cur[i];
    } else if (op == 1) {
        cur[i] = plane[i];
    } else {
        const double v = plane[i];
        cur[i] = 2.0 * v - prev[i];
        prev[i] = v;
    }
}

void mg_psi_io(MgHost<double> *m, int op, double *plane, double *prev, cudaStream_t s) {
    const Level<double> &L0 = m->L0;
    const long long n = (long long)L0.pitch * L0.ny;
    psi_io_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m->ctl, L0.e, L0.r, op, plane, prev, n);
}

#define FCD_MG_INST(T)                                                                          \
    template MgHost<T> *mg_create<T>(int, int, int, T *, T *, T *, MgCtl *,                     \
                                     void *(*)(size_t, void *), void (*)(void *, void *), void *, \
                                     char *, size_t, int, const MgHost<T> *);                   \
    template void mg_destroy<T>(MgHost<T> *);                                                   \
    template void mg_cycle_head<T>(MgHost<T> *, T, T, cudaGraphConditionalHandle,                \
                                   cudaGraphConditionalHandle, int, cudaStream_t);              \
    template void mg_cycle_rest<T>(MgHost<T> *, T, T, cudaStream_t);                             \
    template void mg_cycle_smooth<T>(MgHost<T> *, T, T, cudaStream_t);                           \
    template void mg_cycle_twogrid<T>(MgHost<T> *, T, T, cudaStream_t);                          \
    template void mg_presmooth<T>(MgHost<T> *, T, T, cudaStream_t);                              \
    template int mg_kernels_per_cycle<T>(const MgHost<T> *);                                    \
    template void mg_cycle_dispatch<T>(MgHost<T> *, cudaGraphConditionalHandle, cudaStream_t);    \
    template int mg_levels<T>(const MgHost<T> *);                                               \
    template void mg_set_rhs<T>(MgHost<T> *, const T *);
FCD_MG_INST(float)
FCD_MG_INST(double)

}  // namespace fcd
