// fcd_lbm.cu -- lattice Boltzmann kernels of the coupled step (arXiv 2410.11129).
//
// phase_kernel   : Eq. 32 (phi_i = sum_a g^i_a), Eq. 24, Eq. 8 (k = 1 + chi)
// collide_kernel : one fused pass per node: isotropic gradients and Laplacians
//                  (Eqs. 34-35) from shared-memory tiles with a one-node halo,
//                  chemical potentials and surface tension (Eqs. 25-28, 36),
//                  Kelvin force (Eqs. 5, 7, 9), pressure, viscous and driving
//                  forces (Eq. 19), velocity (Eq. 22), MRT collision of f
//                  (Eqs. 12-18), BGK collision of g^1, g^2 (Eqs. 29-31), push
//                  streaming with half-way bounce-back.
// The MRT collision is evaluated in closed form: with every rate 1 except the
// two stress moments (Eq. 13), the post-collision populations are
// f^eq + F/2 + (1 - s_nu)/4 [dpxx (row pxx) + dpxy (row pxy)].
#include "fcd_internal.cuh"

namespace fcd {

template <int MODE>
struct StoreT { using type = float; };
template <>
struct StoreT<MODE_FP64> { using type = double; };
template <>
struct StoreT<MODE_TANGENT> { using type = double; };

// ---------------------------------------------------------------- phase
// One 32 x (8 ROWS) tile of nodes starting at (x0, y0), run by 32 x 8 threads,
// each taking ROWS nodes 8 rows apart with all their loads issued first; the
// lead block of the grid also resets the control block and advances the step
// counter.
template <typename T, int MODE, int ROWS = 1>
__device__ __forceinline__ void phase_tile(const Phys<T> &P, const void *gv, T *phi1, T *phi2,
                                           T *k, const PhaseCtl &pc, int x0, int y0, bool lead) {
    using S = typename StoreT<MODE>::type;
    if (pc.ctl && lead && threadIdx.x == 0 && threadIdx.y == 0) {
        MgCtl *c = pc.ctl;
        if (pc.reset) {  // start of a potential solve
            c->norm_bits = 0ull;
            c->iter = 0;
            c->done = 0;
            c->converged = 0;
            c->tolH0 = pc.tolH0;
            c->max_iter = pc.max_iter;
            c->keep_going = 1;
            c->blocks_done = 0u;
            c->mode = 1;         // the opening sweeps count as a lattice-sweep cycle
            c->smooth_left = 0;  // ... and use up the sweep allowance
            c->twogrid_left = 2;
        }
        if (pc.step) {
            c->step_cur = *pc.step;
            *pc.step += 1;
        }
    }
    const S *g = static_cast<const S *>(gv);
    const int x = x0 + threadIdx.x;
    constexpr bool PAIR = psi_planes<T>() == 2;
    T *psi = pc.extrap ? static_cast<T *>(pc.ctl->cur ? pc.psiB : pc.psiA) : nullptr;
    T *prev = static_cast<T *>(pc.psi_prev);
    const long long L = P.ps;  // the lo plane of a pair, one plane on
    const bool pair = PAIR && pc.comp;
    bool ok[ROWS];
    long long n[ROWS];
    S gv_[ROWS][18];
    T ps_[ROWS][2], pp_[ROWS][2];
#pragma unroll
    for (int r = 0; r < ROWS; r++) {
        const int y = y0 + threadIdx.y + 8 * r;
        ok[r] = x < P.nx && y < P.ny;
        n[r] = (long long)y * P.pitch + x;
        if (!ok[r]) continue;
#pragma unroll
        for (int a = 0; a < 18; a++) gv_[r][a] = g[a * P.ps + n[r]];
        if (psi) {
            ps_[r][0] = psi[n[r]];
            pp_[r][0] = prev[n[r]];
            if (pair) {
                ps_[r][1] = psi[L + n[r]];
                pp_[r][1] = prev[L + n[r]];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < ROWS; r++) {
        if (!ok[r]) continue;
        const long long m = n[r];
        T p1 = T(0), p2 = T(0);
#pragma unroll
        for (int a = 0; a < 9; a++) {
            p1 += T(gv_[r][a]) - g_off<MODE, T>(a);
            p2 += T(gv_[r][9 + a]) - g_off<MODE, T>(a);
        }
        phi1[m] = p1;
        phi2[m] = p2;
        if (psi) {  // second-order extrapolation in time of the potential
            if (pair) {  // psi' = hi + lo
                const float h = ps_[r][0], l = ps_[r][1], ph = pp_[r][0], pl = pp_[r][1];
                prev[m] = h;
                prev[L + m] = l;
                float a, e, hh, ll;
                two_sum(2.f * h, -ph, a, e);
                two_sum(a, __fadd_rn(__fsub_rn(2.f * l, pl), e), hh, ll);
                psi[m] = hh;
                psi[L + m] = ll;
            } else {
                const T now = ps_[r][0], before = pp_[r][0];
                prev[m] = now;
                psi[m] = T(2) * now - before;
            }
        }
        if (k) {
            T h1 = clamp01(p1), h2 = clamp01(p2), h3 = clamp01(T(1) - p1 - p2);
            k[m] = T(1) / (P.ik[0] * h1 + P.ik[1] * h2 + P.ik[2] * h3);
        }
    }
}

// Two rows per thread, all 36 population loads in flight before the sums
// (measured: the phase recovery of the 9600 x 1200 channel 202 -> 179 us, of
// 2400 x 300 22.5 -> 20.3 us).
template <typename T, int MODE>
__global__ void __launch_bounds__(256) phase_kernel(Phys<T> P, const void *gv, T *phi1, T *phi2,
                                                    T *k, PhaseCtl pc) {
    phase_tile<T, MODE, 2>(P, gv, phi1, phi2, k, pc, blockIdx.x * 32, blockIdx.y * 16,
                           blockIdx.x == 0 && blockIdx.y == 0);
}

// ---------------------------------------------------------------- collide
// Division inside the collide kernel: IEEE for FP64; the FP32 forms use the
// fast single-precision divide (about 2 ulp), well inside their 1e-4 budget.
template <typename T>
__device__ __forceinline__ T cdiv(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float cdiv<float>(float a, float b) { return __fdividef(a, b); }

// Error-free running sum in FP32 (Knuth's TwoSum): hi + lo equals the exact sum
// of the added values as long as lo stays far from rounding (a few dozen terms).
struct FSum {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float b) {
        const float s = __fadd_rn(hi, b);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    // (this - o) rounded once
    __device__ __forceinline__ float minus(const FSum &o) const {
        FSum d;
        d.hi = hi;
        d.add(-o.hi);
        return __fadd_rn(d.hi, __fadd_rn(d.lo, __fsub_rn(lo, o.lo)));
    }
    // (this - o) rounded to FP32 without bias: rounded to the nearest value v
    // with its exact error e, then moved one unit toward e with probability
    // |e| / unit (u01: a uniform number in [0, 1)), so that the stored value's
    // expectation is the difference itself. Round-to-nearest alone repeats the
    // same rounding at a node whose remainder changes little between steps.
    __device__ __forceinline__ float minus_unbiased(const FSum &o, float u01) const {
        FSum d;
        d.hi = hi;
        d.add(-o.hi);
        float v, e;
        two_sum(d.hi, __fadd_rn(d.lo, __fsub_rn(lo, o.lo)), v, e);
        if (e != 0.0f) {
            const float next = nextafterf(v, e > 0.0f ? INFINITY : -INFINITY);
            if (u01 * fabsf(__fsub_rn(next, v)) < fabsf(e)) v = next;
        }
        return v;
    }
};

// Uniform number in [0, 1) from a 32-bit key: a multiply-xorshift integer
// hash (the constants of the "lowbias32" mixer), top 24 bits.
__device__ __forceinline__ float hash_u01(unsigned h) {
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return float(h >> 8) * (1.0f / 16777216.0f);
}

// e_a . (vx, vy) for the D2Q9 velocity e_a, written without the products by a
// zero component (IEEE arithmetic keeps 0 * v, which is not 0 for every v).
template <typename R>
__device__ __forceinline__ R edot(int a, const R &vx, const R &vy) {
    const int ex = cx(a), ey = cy(a);
    if (ex == 0 && ey == 0) return R(0);
    if (ex == 0) return ey > 0 ? vy : -vy;
    if (ey == 0) return ex > 0 ? vx : -vx;
    return (ex > 0 ? vx : -vx) + (ey > 0 ? vy : -vy);
}

template <typename R, typename B>
struct Stencil {
    R c, e, w, n, s, ne, nw, sw, se;
    template <int W>
    __device__ __forceinline__ void load(const R (*a)[W], int lx, int ly) {
        c = a[ly][lx];
        e = a[ly][lx + 1];
        w = a[ly][lx - 1];
        n = a[ly + 1][lx];
        s = a[ly - 1][lx];
        ne = a[ly + 1][lx + 1];
        nw = a[ly + 1][lx - 1];
        sw = a[ly - 1][lx - 1];
        se = a[ly - 1][lx + 1];
    }
    // Eq. 34 with c_s^2 = 1/3: 3 sum_a w_a e_a phi_a
    __device__ __forceinline__ R gx() const {
        return (e - w) * B(1.0 / 3.0) + ((ne - nw) + (se - sw)) * B(1.0 / 12.0);
    }
    __device__ __forceinline__ R gy() const {
        return (n - s) * B(1.0 / 3.0) + ((ne + nw) - (se + sw)) * B(1.0 / 12.0);
    }
    // Eq. 35: 6 sum_a w_a (phi_a - phi_0)
    __device__ __forceinline__ R lap() const {
        return (B(4) * ((e + w) + (n + s)) + ((ne + nw) + (se + sw)) - B(20) * c) *
               B(1.0 / 6.0);
    }
};

// Field and population access. Plain modes: one plane per quantity. Tangent
// mode: the primal plane set is followed by NT tangent copies, copy c of plane
// q of an np-plane set at (np * c + q) planes from the base.
template <typename R, typename T>
__device__ __forceinline__ R ld_field(const T *p, long long i, long long ps) {
    if constexpr (sizeof(R) == sizeof(T)) {
        (void)ps;
        return R(p[i]);
    } else {
        R r(p[i]);
#pragma unroll
        for (int c = 0; c < NT; c++) r.d[c] = p[i + (c + 1) * ps];
        return r;
    }
}
template <typename R, typename S>
__device__ __forceinline__ R ld_pop(const S *p, int q, int np, int ps, int n) {
    if constexpr (sizeof(R) == sizeof(S)) {
        (void)np;
        return R(p[q * ps + n]);
    } else {
        R r(p[q * ps + n]);
#pragma unroll
        for (int c = 0; c < NT; c++) r.d[c] = p[(np * (c + 1) + q) * ps + n];
        return r;
    }
}
template <typename S, typename R>
__device__ __forceinline__ void st_pop(S *p, int q, int np, int ps, int n, const R &v) {
    if constexpr (sizeof(R) == sizeof(S)) {
        (void)np;
        p[q * ps + n] = S(v);
    } else {
        p[q * ps + n] = v.v;
#pragma unroll
        for (int c = 0; c < NT; c++) p[(np * (c + 1) + q) * ps + n] = v.d[c];
    }
}

// Tile height: the dual tiles of the tangent step are five times larger.
template <int MODE>
__host__ __device__ constexpr int tile_y() { return MODE == MODE_TANGENT ? 4 : TY; }
template <int MODE>
__host__ __device__ constexpr int collide_min_blocks() { return MODE == MODE_FP32 || MODE == MODE_FP32_OFFSET ? 4 : 1; }

// OPEN: the channel's x ends are an inlet and an outlet (phi-like fields
// mirrored there, populations leaving through them dropped; psi' stays
// periodic); otherwise x is periodic.
// One TX x TYM tile of nodes starting at (x0, y0), run by TX x TYM threads.
template <typename T, int MODE, bool OPEN, int TYM = tile_y<MODE>()>
__device__ __forceinline__ void collide_tile(const LbmArgs<T, typename Compute<T, MODE>::type> &A,
                                             int x0, int y0) {
    using S = typename StoreT<MODE>::type;
    using R = typename Compute<T, MODE>::type;  // arithmetic type
    using B = T;                                // type of the constants
    __shared__ R s1[TYM + 2][TX + 2], s2[TYM + 2][TX + 2], sr[TYM + 2][TX + 2], sp[TYM + 2][TX + 2];
    const Phys<R> &P = A.P;
    const int nx = P.nx, ny = P.ny, pitch = P.pitch;
    const long long ps = P.ps;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool live = x < nx && y < ny;
    const long long n = (long long)y * pitch + x;

    // FP32 forms: issue the 27 population loads first so that their latency
    // overlaps the halo fill and the force evaluation (FP64 keeps them late:
    // its register budget is already large).
    constexpr bool EARLY = MODE == MODE_FP32 || MODE == MODE_FP32_OFFSET;
    const S *fs = static_cast<const S *>(A.f_src);
    const S *gs = static_cast<const S *>(A.g_src);
    S fpre[EARLY ? 9 : 1], gpre[EARLY ? 18 : 1];
    if constexpr (EARLY) {
        if (live) {
#pragma unroll
            for (int a = 0; a < 9; a++) fpre[a] = __ldg(fs + (a * (int)ps + (int)n));
#pragma unroll
            for (int a = 0; a < 18; a++) gpre[a] = __ldg(gs + (a * (int)ps + (int)n));
        }
    }
    const T *psi = A.ctl->cur ? A.psi1 : A.psi0;

    for (int i = threadIdx.y * TX + threadIdx.x; i < (TX + 2) * (TYM + 2); i += TX * TYM) {
        int lx = i % (TX + 2), ly = i / (TX + 2);
        int gx = x0 - 1 + lx;
        const int gm = gx < 0 ? 0 : (gx >= nx ? nx - 1 : gx);  // mirrored column (open ends)
        if (gx < 0) gx += nx;
        while (gx >= nx) gx -= nx;
        int gy = y0 - 1 + ly;
        bool ghost = gy < 0 || gy >= ny;
        int my = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
        long long m = (long long)my * pitch + gx;
        const long long mp = OPEN ? (long long)my * pitch + gm : m;
        const R p1 = ld_field<R>(A.phi1, mp, ps), p2 = ld_field<R>(A.phi2, mp, ps);
        s1[ly][lx] = p1;  // mirrored ghost rows: zero normal gradient
        s2[ly][lx] = p2;
        sr[ly][lx] = P.rho[0] * clamp01(p1) + P.rho[1] * clamp01(p2) +
                     P.rho[2] * clamp01(B(1) - p1 - p2);
        const R q = ld_field<R>(psi, m, ps);
        sp[ly][lx] = ghost ? -q : q;  // psi' = 0 on the wall faces
    }
    __syncthreads();

    if (!live) return;
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;

    Stencil<R, B> st;
    st.load(s1, lx, ly);
    const R ph1 = st.c, g1x = st.gx(), g1y = st.gy(), l1 = st.lap();
    st.load(s2, lx, ly);
    const R ph2 = st.c, g2x = st.gx(), g2y = st.gy(), l2 = st.lap();
    const R ph3 = B(1) - ph1 - ph2;
    const R g3x = -(g1x + g2x), g3y = -(g1y + g2y), l3 = -(l1 + l2);
    st.load(sr, lx, ly);
    const R rho = st.c, grx = st.gx(), gry = st.gy();
    st.load(sp, lx, ly);
    const R dpx = st.gx(), dpy = st.gy();

    const R h1 = clamp01(ph1), h2 = clamp01(ph2), h3 = clamp01(ph3);

    // Surface tension (Eqs. 25, 28, 36). With phi_3 = 1 - phi_1 - phi_2 the
    // gradients sum to zero, so the part of mu_i common to all phases drops out:
    // F_s = sum_i [ (12/xi) dH/dphi_i - (3/4) xi gamma_i lap phi_i ] grad phi_i.
    R Fx, Fy;
    {
        const R gp = P.gam[0] * ph1 + P.gam[1] * ph2 + P.gam[2] * ph3;
        const R q3 = ph1 * ph2 * ph3;
        const R a1 = ph1 * ph1, a2 = ph2 * ph2, a3 = ph3 * ph3;
        const R d1 = B(2) * ph1 * (P.s12 * a2 + P.s13 * a3) + ph2 * ph3 * gp + P.gam[0] * q3 +
                     B(2) * P.eta * ph1 * a2 * a3;
        const R d2 = B(2) * ph2 * (P.s12 * a1 + P.s23 * a3) + ph1 * ph3 * gp + P.gam[1] * q3 +
                     B(2) * P.eta * a1 * ph2 * a3;
        const R d3 = B(2) * ph3 * (P.s13 * a1 + P.s23 * a2) + ph1 * ph2 * gp + P.gam[2] * q3 +
                     B(2) * P.eta * a1 * a2 * ph3;
        const R m1 = P.twelve_over_xi * d1 - P.lap_coef[0] * l1;
        const R m2 = P.twelve_over_xi * d2 - P.lap_coef[1] * l2;
        const R m3 = P.twelve_over_xi * d3 - P.lap_coef[2] * l3;
        Fx = m1 * g1x + m2 * g2x + m3 * g3x;
        Fy = m1 * g1y + m2 * g2y + m3 * g3y;
    }
    // Kelvin force F_m = -(1/2) |H|^2 grad chi (Eq. 7); grad chi by Eq. 9 with
    // grad phi_3 = -(grad phi_1 + grad phi_2); H = H0 e_alpha - grad psi' (Eq. 5).
    {
        const R kk = cdiv(R(B(1)), P.ik[0] * h1 + P.ik[1] * h2 + P.ik[2] * h3);
        const R gcx = -kk * kk * (P.dk1 * g1x + P.dk2 * g2x);
        const R gcy = -kk * kk * (P.dk1 * g1y + P.dk2 * g2y);
        const R Hx = P.H0c - dpx, Hy = P.H0s - dpy;
        const R hh = B(0.5) * (Hx * Hx + Hy * Hy);
        Fx -= hh * gcx;
        Fy -= hh * gcy;
    }

    // Populations.
    R f[9];
#pragma unroll
    for (int a = 0; a < 9; a++) {
        if constexpr (EARLY) f[a] = R(fpre[a]) - f_off<MODE, B>(a);
        else f[a] = ld_pop<R>(fs, a, 9, (int)ps, (int)n) - f_off<MODE, B>(a);
    }
    const R pst = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const R jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const R jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const R mpxx = (f[1] + f[3]) - (f[2] + f[4]);
    const R mpxy = (f[5] + f[7]) - (f[6] + f[8]);
    const R me = B(2) * ((f[5] + f[6]) + (f[7] + f[8])) - ((f[1] + f[2]) + (f[3] + f[4])) -
                 B(4) * f[0];

    // Pressure (F_p = -(p/rho) grad rho with p = rho c_s^2 p*) and driving force.
    Fx += -pst * B(1.0 / 3.0) * grx + P.G;
    Fy += -pst * B(1.0 / 3.0) * gry;
    const R inv_rho = cdiv(R(B(1)), rho), half_inv_rho = B(0.5) * inv_rho;
    const R upx = jx + Fx * half_inv_rho, upy = jy + Fy * half_inv_rho;
    const R tau = P.tau[0] * h1 + P.tau[1] * h2 + P.tau[2] * h3;
    const R snu = cdiv(R(B(1)), B(0.5) + tau);
    // Viscous force from the non-equilibrium stress (moments of f - f^eq(p*, u')):
    // Pi = (1/6) m_e + (1/2) s_nu m_pxx on the diagonal, s_nu m_pxy off it.
    {
        const R he = me - (B(3) * (upx * upx + upy * upy) - B(2) * pst);
        const R hxx = mpxx - (upx * upx - upy * upy);
        const R hxy = mpxy - upx * upy;
        const R Pxx = he * B(1.0 / 6.0) + B(0.5) * snu * hxx;
        const R Pyy = he * B(1.0 / 6.0) - B(0.5) * snu * hxx;
        const R Pxy = snu * hxy;
        const R Fmx = -tau * (Pxx * grx + Pxy * gry);
        const R Fmy = -tau * (Pxy * grx + Pyy * gry);
        Fx += Fmx;
        Fy += Fmy;
    }
    const R ux = jx + Fx * half_inv_rho, uy = jy + Fy * half_inv_rho;
    const R uu = B(1.5) * (ux * ux + uy * uy);

    if (A.macro) {
        A.macro[n] = value(ux);
        A.macro[ps + n] = value(uy);
        A.macro[2 * ps + n] = value(pst);
    }
    // Instability record: a non-finite velocity or pressure (NaN fails the
    // compare) marks the step in flight; the host reads it at its next
    // synchronising call. No trap: the step completes.
    if (A.unst && !(fabs(value(ux) + value(uy) + value(pst)) < B(1e30)))
        atomicMin(A.unst, (unsigned long long)(*A.step));

    // Breakup: the core (phi_1 >= 1/2) touches the carrier (phi_3 >= 1/2) at a
    // D2Q9 neighbour inside the channel; keep the first (step, y, x).
    if (A.brk && h1 >= B(0.5) && *((volatile unsigned long long *)A.brk) == ~0ull) {
        bool touch = false;
#pragma unroll
        for (int a = 1; a < 9; a++) {
            int yy = y + cy(a);
            if (yy < 0 || yy >= ny) continue;
            if (OPEN && (x + cx(a) < 0 || x + cx(a) >= nx)) continue;
            const R q1 = s1[ly + cy(a)][lx + cx(a)], q2 = s2[ly + cy(a)][lx + cx(a)];
            touch |= clamp01(B(1) - q1 - q2) >= B(0.5);
        }
        if (touch) {
            unsigned long long key = ((unsigned long long)(*A.step) << 32) |
                                     (unsigned long long)((long long)y * nx + x);
            atomicMin(A.brk, key);
        }
    }

    // Push streaming: 32-bit offsets (every plane fits in 2^31 elements, checked
    // at create), x-neighbour deltas with the periodic seam folded in, and wall
    // flags that are uniform across a warp (a warp is one tile row).
    const int n32 = y * pitch + x, ps32 = (int)ps;
    const int dxp = (x == nx - 1) ? 1 - nx : 1, dxm = (x == 0) ? nx - 1 : -1;
    const bool top = y == ny - 1, bot = y == 0;
    auto dest = [&](int a) {
        return n32 + cy(a) * pitch + (cx(a) > 0 ? dxp : (cx(a) < 0 ? dxm : 0));
    };
    auto walled = [&](int a) { return (cy(a) > 0 && top) || (cy(a) < 0 && bot); };
    // open channel: populations leaving through the inlet or the outlet
    auto leaves = [&](int a) {
        return OPEN && ((cx(a) > 0 && x == nx - 1) || (cx(a) < 0 && x == 0));
    };

    // Deviation of the equilibria from rest, D_a = 3 e.u + 4.5 (e.u)^2 - 1.5 u.u:
    // f^eq = w (p* + D) (Eq. 16), Gamma = w (1 + D) (Eq. 18).
    R dev[9];
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const R eu = edot(a, ux, uy);
        dev[a] = B(3) * eu + B(4.5) * eu * eu - uu;
    }

    // MRT collision in closed form and push streaming of f.
    S *fd = static_cast<S *>(A.f_dst);
    const R dxx = mpxx - (ux * ux - uy * uy);
    const R dxy = mpxy - ux * uy;
    const R rel = (B(1) - snu) * B(0.25);
    const R fr = B(3) * inv_rho;
    const R Ftx = B(0.5) * Fx * fr, Fty = B(0.5) * Fy * fr;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const B w = wgt<B>(a);
        R v = w * (a == 0 ? pst + dev[a] : (pst + dev[a]) + edot(a, Ftx, Fty));
        // rows of p_xx (+1 on 1, 3; -1 on 2, 4) and p_xy (+1 on 5, 7; -1 on 6, 8)
        if (a == 1 || a == 3) v += rel * dxx;
        else if (a == 2 || a == 4) v += rel * -dxx;
        else if (a == 5 || a == 7) v += rel * dxy;
        else if (a == 6 || a == 8) v += rel * -dxy;
        if (walled(a)) st_pop(fd, opp(a), 9, ps32, n32, v + f_off<MODE, B>(opp(a)));
        else if (!leaves(a)) st_pop(fd, a, 9, ps32, dest(a), v + f_off<MODE, B>(a));
    }

    // Phase fields (Eqs. 29-31): g* = (1 - om) g + om phi Gamma + (1 - om/2) F^phi,
    // F^phi_a = w_a e_a . q_i, q_i = theta_i n_i - (1/3) sum_j theta_j n_j.
    R qx[2], qy[2];
    {
        const R t1 = P.four_over_xi * h1 * (B(1) - h1);
        const R t2 = P.four_over_xi * h2 * (B(1) - h2);
        const R t3 = P.four_over_xi * h3 * (B(1) - h3);
        const R i1 = cdiv(t1, sqrt(g1x * g1x + g1y * g1y) + P.eps_n);
        const R i2 = cdiv(t2, sqrt(g2x * g2x + g2y * g2y) + P.eps_n);
        const R i3 = cdiv(t3, sqrt(g3x * g3x + g3y * g3y) + P.eps_n);
        const R mx = (i1 * g1x + i2 * g2x + i3 * g3x) * B(1.0 / 3.0);
        const R my = (i1 * g1y + i2 * g2y + i3 * g3y) * B(1.0 / 3.0);
        qx[0] = i1 * g1x - mx;
        qy[0] = i1 * g1y - my;
        qx[1] = i2 * g2x - mx;
        qy[1] = i2 * g2y - my;
    }
    S *gd = static_cast<S *>(A.g_dst);
    // FP32 offset form: the rest population takes the exact remainder of the
    // node's pre-collision sum minus its eight stored outgoing populations
    // (error-free sums), so that the collision conserves each phase's mass up
    // to one rounding per node; the stored values are offsets by a constant,
    // so conserving their sum conserves sum_a g.
    constexpr bool CONSERVE = MODE == MODE_FP32_OFFSET;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const R phi = i == 0 ? ph1 : ph2;
        const R ophi = P.om_phi * phi;
        const R sqx = P.src_phi * qx[i], sqy = P.src_phi * qy[i];
        FSum pre, post;
        if constexpr (CONSERVE) {
#pragma unroll
            for (int a = 0; a < 9; a++) pre.add(float(gpre[i * 9 + a]));
        }
#pragma unroll
        for (int a = CONSERVE ? 1 : 0; a < 9; a++) {
            const B w = wgt<B>(a);
            R gv;
            if constexpr (EARLY) gv = R(gpre[i * 9 + a]) - g_off<MODE, B>(a);
            else gv = ld_pop<R>(gs, i * 9 + a, 18, ps32, n32) - g_off<MODE, B>(a);
            const R v = P.keep_phi * gv +
                        w * (a == 0 ? ophi * (B(1) + dev[a]) : ophi * (B(1) + dev[a]) + edot(a, sqx, sqy));
            const R out = v + g_off<MODE, B>(walled(a) ? opp(a) : a);
            if constexpr (CONSERVE) {
                const S sv = S(out);
                post.add(float(sv));
                if (walled(a)) gd[(i * 9 + opp(a)) * ps32 + n32] = sv;
                else if (!leaves(a)) gd[(i * 9 + a) * ps32 + dest(a)] = sv;
            } else {
                if (walled(a)) st_pop(gd, i * 9 + opp(a), 18, ps32, n32, out);
                else if (!leaves(a)) st_pop(gd, i * 9 + a, 18, ps32, dest(a), out);
            }
        }
        if constexpr (CONSERVE) {  // key: node, step, phase (reproducible)
            const unsigned key = (unsigned)n32 * 0x9E3779B1u ^ (unsigned)(*A.step) * 0x85EBCA77u ^
                                 (unsigned)(i + 1) * 0xC2B2AE3Du;
            gd[(i * 9) * ps32 + n32] = S(pre.minus_unbiased(post, hash_u01(key)));
        }
    }
}

// TYM rows per tile; MINB resident blocks per SM bound the registers (FP32:
// 64 per thread at either height).
template <typename T, int MODE, bool OPEN, int TYM = tile_y<MODE>(), int MINB = collide_min_blocks<MODE>()>
__global__ void __launch_bounds__(TX *TYM, MINB)
    collide_kernel(LbmArgs<T, typename Compute<T, MODE>::type> A) {
    collide_tile<T, MODE, OPEN, TYM>(A, blockIdx.x * TX, blockIdx.y * TYM);
}

// ---------------------------------------------------------------- batched
// Many periodic channels in one launch: block b takes tile tiles[b] (instance,
// tile origin) and that instance's arguments from tab. The collide's
// arguments are staged in shared memory (read by every thread many times).
template <typename T, int MODE>
__global__ void __launch_bounds__(256) phase_batch_kernel(const BatchLbm<T> *tab,
                                                          const BatchTile *tiles) {
    const BatchTile t = tiles[blockIdx.x];
    const BatchLbm<T> &b = tab[t.inst];
    phase_tile<T, MODE>(b.lbm.P, b.lbm.g_src, b.phi1, b.phi2, b.k, b.pc, t.x0, t.y0, t.lead != 0);
}

template <typename T, int MODE, int TYM, int MINB>
__global__ void __launch_bounds__(TX *TYM, MINB) collide_batch_kernel(const BatchLbm<T> *tab,
                                                                      const BatchTile *tiles) {
    static_assert(sizeof(LbmArgs<T>) % sizeof(int) == 0, "argument block copied as words");
    __shared__ __align__(16) int raw[sizeof(LbmArgs<T>) / sizeof(int)];
    const BatchTile t = tiles[blockIdx.x];
    const int *src = reinterpret_cast<const int *>(&tab[t.inst].lbm);
    for (int i = threadIdx.y * TX + threadIdx.x; i < (int)(sizeof(LbmArgs<T>) / sizeof(int)); i += TX * TYM)
        raw[i] = src[i];
    __syncthreads();
    collide_tile<T, MODE, false, TYM>(*reinterpret_cast<const LbmArgs<T> *>(raw), t.x0, t.y0);
}

// ---------------------------------------------------------------- open ends
// Inlet (x = 0), Eq. 37: the Poiseuille parabola with centre-line speed u_max
// between the half-way walls. Zou-He in the velocity-based form: the unknown
// populations 1, 5, 8 reflect the non-equilibrium part of their opposites,
// f_a = f_opp(a) + 6 w_a e_a.u, with -/+ (f2 - f4)/2 on 5 and 8 zeroing the
// wall-normal momentum; at the two corner nodes the wall supplies one of 5, 8
// and the two unknowns follow from both momentum components. The inflow is pure
// carrier: its phase-field populations are zero.
// Outlet (x = nx - 1): convective condition chi(t+1) = (chi(t) + U chi_{nx-2}(t+1))
// / (1 + U), U = u_avg, on f_a - w_a p* with the outlet holding the reference
// p* = 0, and on g as it is.
template <typename T, int MODE>
__global__ void open_bc_kernel(Phys<T> P, const void *fsv, const void *gsv, void *fdv, void *gdv,
                               T u_max, T u_avg) {
    using S = typename StoreT<MODE>::type;
    using R = typename Compute<T, MODE>::type;  // dual numbers in the tangent step
    using B = T;
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    if (y >= ny) return;
    const int ps = (int)P.ps, n = y * P.pitch, o = n + nx - 1, b = o - 1;
    const S *fs = static_cast<const S *>(fsv);
    const S *gs = static_cast<const S *>(gsv);
    S *fd = static_cast<S *>(fdv);
    S *gd = static_cast<S *>(gdv);
    auto F = [&](const S *p, int a, int m) { return ld_pop<R>(p, a, 9, ps, m) - f_off<MODE, B>(a); };
    auto G = [&](const S *p, int q, int a, int m) {
        return ld_pop<R>(p, q * 9 + a, 18, ps, m) - g_off<MODE, B>(a);
    };
    // inlet (the profile is data: no derivative)
    const B u = u_max * B(4) * (B(y) + B(0.5)) * (B(ny) - B(0.5) - B(y)) / (B(ny) * B(ny));
    R fl[9];
#pragma unroll
    for (int a = 0; a < 9; a++) fl[a] = F(fd, a, n);
    if (y == 0) {
        fl[8] = fl[2] - fl[4] + fl[5] + fl[6] - fl[7];
    } else if (y == ny - 1) {
        fl[5] = fl[4] - fl[2] - fl[6] + fl[7] + fl[8];
    } else {
        fl[5] = fl[7] + B(6) * wgt<B>(5) * u - B(0.5) * (fl[2] - fl[4]);
        fl[8] = fl[6] + B(6) * wgt<B>(8) * u + B(0.5) * (fl[2] - fl[4]);
    }
    if (y == 0 || y == ny - 1) fl[1] = u + fl[3] - fl[5] + fl[6] + fl[7] - fl[8];
    else fl[1] = fl[3] + B(6) * wgt<B>(1) * u;
    st_pop(fd, 1, 9, ps, n, fl[1] + f_off<MODE, B>(1));
    st_pop(fd, 5, 9, ps, n, fl[5] + f_off<MODE, B>(5));
    st_pop(fd, 8, 9, ps, n, fl[8] + f_off<MODE, B>(8));
    for (int q = 0; q < 2; q++) {
        st_pop(gd, q * 9 + 1, 18, ps, n, R(g_off<MODE, B>(1)));
        if (y != 0) st_pop(gd, q * 9 + 5, 18, ps, n, R(g_off<MODE, B>(5)));
        if (y != ny - 1) st_pop(gd, q * 9 + 8, 18, ps, n, R(g_off<MODE, B>(8)));
    }
    // outlet
    R pb = R(B(0)), po = R(B(0));
    for (int a = 0; a < 9; a++) {
        pb += F(fd, a, b);
        po += F(fs, a, o);
    }
    const B pout = B(0);
    const int in3[3] = {3, 6, 7};
    for (int k = 0; k < 3; k++) {
        const int a = in3[k];
        if ((a == 6 && y == 0) || (a == 7 && y == ny - 1)) continue;  // from the wall
        const R chi = ((F(fs, a, o) - wgt<B>(a) * po) + u_avg * (F(fd, a, b) - wgt<B>(a) * pb)) /
                      (B(1) + u_avg);
        st_pop(fd, a, 9, ps, o, chi + wgt<B>(a) * pout + f_off<MODE, B>(a));
        for (int q = 0; q < 2; q++)
            st_pop(gd, q * 9 + a, 18, ps, o,
                   (G(gs, q, a, o) + u_avg * G(gd, q, a, b)) / (B(1) + u_avg) + g_off<MODE, B>(a));
    }
}

// ---------------------------------------------------------------- init
template <typename T, int MODE>
__global__ void init_kernel(Phys<T> P, double u_max, double r1, double r2, double xcen,
                            double ycen, double xi, void *fv, void *gv, T *macro) {
    using S = typename StoreT<MODE>::type;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    long long n = (long long)y * P.pitch + x;
    const double nyd = P.ny;
    const double u0 = u_max * 4.0 * (y + 0.5) * (nyd - 0.5 - y) / (nyd * nyd);
    double dx = x - xcen;
    dx -= P.nx * floor(dx / P.nx + 0.5);  // nearest periodic image
    const double dy = y - ycen;
    const double r = sqrt(dx * dx + dy * dy);
    const double pout = 0.5 * (1.0 - tanh(2.0 * (r - r2) / xi));
    const double p1 = 0.5 * (1.0 - tanh(2.0 * (r - r1) / xi));
    const double p2 = pout - p1;
    S *f = static_cast<S *>(fv);
    S *g = static_cast<S *>(gv);
    for (int a = 0; a < 9; a++) {
        const double w = wgt<double>(a), eu = cx(a) * u0;
        const double gam = w * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * u0 * u0);
        f[a * P.ps + n] = S((gam - w) + double(f_off<MODE, T>(a)));
        g[a * P.ps + n] = S(p1 * gam + double(g_off<MODE, T>(a)));
        g[(9 + a) * P.ps + n] = S(p2 * gam + double(g_off<MODE, T>(a)));
    }
    if (macro) {
        macro[n] = T(u0);
        macro[P.ps + n] = T(0);
        macro[2 * P.ps + n] = T(0);
    }
}

// ---------------------------------------------------------------- exchange
template <typename T, int MODE>
__global__ void export_kernel(Phys<T> P, const void *fv, const void *gv, double *fo,
                              double *go) {
    using S = typename StoreT<MODE>::type;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    long long n = (long long)y * P.pitch + x, m = (long long)y * P.nx + x;
    long long N = (long long)P.nx * P.ny;
    const S *f = static_cast<const S *>(fv);
    const S *g = static_cast<const S *>(gv);
    for (int a = 0; a < 9; a++) {
        if (fo) fo[a * N + m] = double(T(f[a * P.ps + n]) - f_off<MODE, T>(a));
        if (go) {
            go[a * N + m] = double(T(g[a * P.ps + n]) - g_off<MODE, T>(a));
            go[(9 + a) * N + m] = double(T(g[(9 + a) * P.ps + n]) - g_off<MODE, T>(a));
        }
    }
}

template <typename T, int MODE>
__global__ void import_kernel(Phys<T> P, const double *fi, const double *gi, void *fv,
                              void *gv) {
    using S = typename StoreT<MODE>::type;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    long long n = (long long)y * P.pitch + x, m = (long long)y * P.nx + x;
    long long N = (long long)P.nx * P.ny;
    S *f = static_cast<S *>(fv);
    S *g = static_cast<S *>(gv);
    for (int a = 0; a < 9; a++) {
        if (fi) f[a * P.ps + n] = S(fi[a * N + m] + double(f_off<MODE, T>(a)));
        if (gi) {
            g[a * P.ps + n] = S(gi[a * N + m] + double(g_off<MODE, T>(a)));
            g[(9 + a) * P.ps + n] = S(gi[(9 + a) * N + m] + double(g_off<MODE, T>(a)));
        }
    }
}

template <typename T>
__global__ void plane_to_f64(const T *src, int nx, int ny, int pitch, double *dst) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    dst[(long long)y * nx + x] = double(src[(long long)y * pitch + x]);
}

template <typename T>
__global__ void plane_from_f64(const double *src, int nx, int ny, int pitch, T *dst) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    dst[(long long)y * pitch + x] = T(src[(long long)y * nx + x]);
}

// psi' of a level-0 buffer in the FP64 exchange layout, and back (FP32: the
// hi + lo pair of planes; FP64: one plane).
template <typename T>
__global__ void psi_to_f64(const T *src, int nx, int ny, int pitch, double *dst) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long n = (long long)y * pitch + x;
    double v = double(src[n]);
    if constexpr (psi_planes<T>() == 2) v += double(src[(long long)pitch * ny + n]);
    dst[(long long)y * nx + x] = v;
}

template <typename T>
__global__ void psi_from_f64(const double *src, int nx, int ny, int pitch, T *dst, int comp) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long n = (long long)y * pitch + x;
    const double v = src[(long long)y * nx + x];
    dst[n] = T(v);
    if constexpr (psi_planes<T>() == 2) dst[(long long)pitch * ny + n] = comp ? T(v - double(T(v))) : T(0);
}

template <typename T>
__global__ void phi3_to_f64(const T *p1, const T *p2, int nx, int ny, int pitch, double *dst) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    long long n = (long long)y * pitch + x;
    dst[(long long)y * nx + x] = double(T(1) - p1[n] - p2[n]);
}

// ---------------------------------------------------------------- launchers
static dim3 grid2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

#define FCD_MODE_SWITCH(mode, T, CALL)                                         \
    do {                                                                       \
        if constexpr (sizeof(T) == 8) {                                        \
            constexpr int M = MODE_FP64;                                       \
            CALL;                                                              \
        } else {                                                               \
            if ((mode) == MODE_FP32) {                                         \
                constexpr int M = MODE_FP32;                                   \
                CALL;                                                          \
            } else {                                                           \
                constexpr int M = MODE_FP32_OFFSET;                            \
                CALL;                                                          \
            }                                                                  \
        }                                                                      \
    } while (0)

template <typename T>
void launch_phase(int mode, const Phys<T> &P, const void *g, T *phi1, T *phi2, T *k,
                  PhaseCtl pc, cudaStream_t s) {
    dim3 b(32, 8), gr = grid2(P.nx, P.ny, dim3(32, 16));
    FCD_MODE_SWITCH(mode, T, (phase_kernel<T, M><<<gr, b, 0, s>>>(P, g, phi1, phi2, k, pc)));
}

template <typename T>
void launch_collide(int mode, int tile_h, const LbmArgs<T> &a, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (tile_h == 4) {
            dim3 b(TX, 4), gr = grid2(a.P.nx, a.P.ny, b);
            if (a.open_x) FCD_MODE_SWITCH(mode, T, (collide_kernel<T, M, true, 4, 8><<<gr, b, 0, s>>>(a)));
            else FCD_MODE_SWITCH(mode, T, (collide_kernel<T, M, false, 4, 8><<<gr, b, 0, s>>>(a)));
            return;
        }
    }
    (void)tile_h;
    dim3 b(TX, TY), gr = grid2(a.P.nx, a.P.ny, b);
    if (a.open_x) FCD_MODE_SWITCH(mode, T, (collide_kernel<T, M, true><<<gr, b, 0, s>>>(a)));
    else FCD_MODE_SWITCH(mode, T, (collide_kernel<T, M, false><<<gr, b, 0, s>>>(a)));
}

template <typename T>
void launch_phase_batch(int mode, const BatchLbm<T> *tab, const BatchTile *tiles, int ntiles,
                        cudaStream_t s) {
    if (ntiles <= 0) return;
    dim3 b(32, 8);
    FCD_MODE_SWITCH(mode, T, (phase_batch_kernel<T, M><<<ntiles, b, 0, s>>>(tab, tiles)));
}

template <typename T>
void launch_collide_batch(int mode, int tile_h, const BatchLbm<T> *tab, const BatchTile *tiles,
                          int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return;
    if (tile_h == 4)
        FCD_MODE_SWITCH(mode, T, (collide_batch_kernel<T, M, 4, (sizeof(T) == 8 ? 2 : 8)>
                                  <<<ntiles, dim3(TX, 4), 0, s>>>(tab, tiles)));
    else if (tile_h == 16)
        FCD_MODE_SWITCH(mode, T, (collide_batch_kernel<T, M, 16, (sizeof(T) == 8 ? 1 : 2)>
                                  <<<ntiles, dim3(TX, 16), 0, s>>>(tab, tiles)));
    else
        FCD_MODE_SWITCH(mode, T, (collide_batch_kernel<T, M, 8, (sizeof(T) == 8 ? 1 : 4)>
                                  <<<ntiles, dim3(TX, 8), 0, s>>>(tab, tiles)));
}

void launch_collide_tangent(const LbmArgs<double, DualT> &a, cudaStream_t s) {
    dim3 b(TX, tile_y<MODE_TANGENT>()), gr = grid2(a.P.nx, a.P.ny, b);
    if (a.open_x) collide_kernel<double, MODE_TANGENT, true><<<gr, b, 0, s>>>(a);
    else collide_kernel<double, MODE_TANGENT, false><<<gr, b, 0, s>>>(a);
}

void launch_open_bc_tangent(const Phys<double> &P, const void *f_src, const void *g_src,
                            void *f_dst, void *g_dst, double u_max, double u_avg, cudaStream_t s) {
    const int b = 64, gr = (P.ny + b - 1) / b;
    open_bc_kernel<double, MODE_TANGENT><<<gr, b, 0, s>>>(P, f_src, g_src, f_dst, g_dst, u_max, u_avg);
}

template <typename T>
void launch_open_bc(int mode, const Phys<T> &P, const void *f_src, const void *g_src,
                    void *f_dst, void *g_dst, double u_max, double u_avg, cudaStream_t s) {
    const int b = 64, gr = (P.ny + b - 1) / b;
    FCD_MODE_SWITCH(mode, T, (open_bc_kernel<T, M><<<gr, b, 0, s>>>(P, f_src, g_src, f_dst, g_dst,
                                                                   T(u_max), T(u_avg))));
}

template <typename T>
void launch_init(int mode, const Phys<T> &P, double u_max, double r1, double r2, double xc,
                 double yc, double xi, void *f, void *g, T *macro, cudaStream_t s) {
    dim3 b(32, 8), gr = grid2(P.nx, P.ny, b);
    FCD_MODE_SWITCH(mode, T,
                    (init_kernel<T, M><<<gr, b, 0, s>>>(P, u_max, r1, r2, xc, yc, xi, f, g, macro)));
}

template <typename T>
void launch_export(int mode, const Phys<T> &P, const void *f, const void *g, double *fo,
                   double *go, cudaStream_t s) {
    dim3 b(32, 8), gr = grid2(P.nx, P.ny, b);
    FCD_MODE_SWITCH(mode, T, (export_kernel<T, M><<<gr, b, 0, s>>>(P, f, g, fo, go)));
}

template <typename T>
void launch_import(int mode, const Phys<T> &P, const double *fi, const double *gi, void *f,
                   void *g, cudaStream_t s) {
    dim3 b(32, 8), gr = grid2(P.nx, P.ny, b);
    FCD_MODE_SWITCH(mode, T, (import_kernel<T, M><<<gr, b, 0, s>>>(P, fi, gi, f, g)));
}

template <typename T>
void launch_plane_to_f64(const T *src, int nx, int ny, int pitch, double *dst, cudaStream_t s) {
    dim3 b(32, 8);
    plane_to_f64<T><<<grid2(nx, ny, b), b, 0, s>>>(src, nx, ny, pitch, dst);
}

template <typename T>
void launch_plane_from_f64(const double *src, int nx, int ny, int pitch, T *dst, cudaStream_t s) {
    dim3 b(32, 8);
    plane_from_f64<T><<<grid2(nx, ny, b), b, 0, s>>>(src, nx, ny, pitch, dst);
}

template <typename T>
void launch_psi_to_f64(const T *src, int nx, int ny, int pitch, double *dst, cudaStream_t s) {
    dim3 b(32, 8);
    psi_to_f64<T><<<grid2(nx, ny, b), b, 0, s>>>(src, nx, ny, pitch, dst);
}

template <typename T>
void launch_psi_from_f64(const double *src, int nx, int ny, int pitch, T *dst, int comp,
                         cudaStream_t s) {
    dim3 b(32, 8);
    psi_from_f64<T><<<grid2(nx, ny, b), b, 0, s>>>(src, nx, ny, pitch, dst, comp);
}

template <typename T>
void launch_phi3_to_f64(const T *p1, const T *p2, int nx, int ny, int pitch, double *dst,
                        cudaStream_t s) {
    dim3 b(32, 8);
    phi3_to_f64<T><<<grid2(nx, ny, b), b, 0, s>>>(p1, p2, nx, ny, pitch, dst);
}

#define FCD_INST(T)                                                                           \
    template void launch_phase<T>(int, const Phys<T> &, const void *, T *, T *, T *,          \
                                  PhaseCtl, cudaStream_t);                                    \
    template void launch_phase_batch<T>(int, const BatchLbm<T> *, const BatchTile *, int,      \
                                        cudaStream_t);                                         \
    template void launch_collide_batch<T>(int, int, const BatchLbm<T> *, const BatchTile *,    \
                                          int, cudaStream_t);                                  \
    template void launch_collide<T>(int, int, const LbmArgs<T> &, cudaStream_t);               \
    template void launch_open_bc<T>(int, const Phys<T> &, const void *, const void *, void *,    \
                                    void *, double, double, cudaStream_t);                      \
    template void launch_init<T>(int, const Phys<T> &, double, double, double, double, double, \
                                 double, void *, void *, T *, cudaStream_t);                   \
    template void launch_export<T>(int, const Phys<T> &, const void *, const void *, double *, \
                                   double *, cudaStream_t);                                    \
    template void launch_import<T>(int, const Phys<T> &, const double *, const double *,       \
                                   void *, void *, cudaStream_t);                              \
    template void launch_plane_to_f64<T>(const T *, int, int, int, double *, cudaStream_t);    \
    template void launch_plane_from_f64<T>(const double *, int, int, int, T *, cudaStream_t);  \
    template void launch_phi3_to_f64<T>(const T *, const T *, int, int, int, double *,         \
                                        cudaStream_t);                                         \
    template void launch_psi_to_f64<T>(const T *, int, int, int, double *, cudaStream_t);      \
    template void launch_psi_from_f64<T>(const double *, int, int, int, T *, int, cudaStream_t);
FCD_INST(float)
FCD_INST(double)

}  // namespace fcd
