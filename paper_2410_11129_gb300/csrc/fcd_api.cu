// fcd_api.cu -- C ABI of the coupled ferrofluid compound-droplet step
// (arXiv 2410.11129): parameter mapping, state, CUDA-graph step loop.
//
// One step is captured once per (buffer parity, store-macro flag) into a CUDA
// graph: phase recovery -> coarse permeabilities -> a while node running
// multigrid V-cycles until the device-side control block reports convergence
// or the cycle cap -> fused collide-stream -> step counter. fcd_step(n)
// launches n such graphs; nothing synchronises with the host in between.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <typeinfo>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fcd_adjoint.cuh"

// NVTX range for the duration of a scope (visible to profilers that record
// NVTX; a no-op otherwise). Host-side: a graph-driven step is one range, the
// host-driven step (FCD_NO_GRAPH=1) one range per stage.
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

namespace fcd {
size_t observe_scratch_doubles(int nx, int ny);
}
using namespace fcd;

// ---------------------------------------------------------------- allocator
static fcd_alloc_fn g_alloc = nullptr;
static fcd_free_fn g_free = nullptr;
static void *g_user = nullptr;

static void *default_alloc(size_t bytes, void *) {
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}
static void default_free(void *p, void *) { cudaFree(p); }

extern "C" void fcd_set_allocator(fcd_alloc_fn alloc, fcd_free_fn release, void *user) {
    if (alloc && release) {
        g_alloc = alloc;
        g_free = release;
        g_user = user;
    } else {
        g_alloc = nullptr;
        g_free = nullptr;
        g_user = nullptr;
    }
}

// ---------------------------------------------------------------- parameters
struct Derived {
    double u_avg, s12, s13, s23, gam[3], gamT, tau[3], tau_phi, mu0H0sq, H0, G;
};

// Lattice values of the dimensionless groups. Returns an error text or null.
static const char *derive(const fcd_params *p, Derived *d) {
    if (p->nx < 4 || (p->nx & 1)) return "nx must be even and >= 4";
    if (p->ny < 2) return "ny must be >= 2";
    if (27ll * ((p->nx + 31) / 32 * 32) * p->ny > (1ll << 31) - 1)
        return "lattice too large: 27 population planes must index within 2^31 elements";
    for (int i = 0; i < 3; i++) {
        if (!(p->rho[i] > 0)) return "densities must be positive";
        if (!(p->nu[i] > 0)) return "viscosities must be positive";
        if (!(p->chi[i] >= 0)) return "susceptibilities must be >= 0";
    }
    if (!(p->mobility > 0) || !(p->xi > 0)) return "mobility and xi must be positive";
    if (p->r1 > p->r2) return "core radius exceeds shell radius";
    if (p->precision < FCD_FP64 || p->precision > FCD_FP32_OFFSET) return "unknown precision";
    if (!(p->mag_tol > 0) || p->mag_max_iter < 0) return "mag_tol must be > 0, mag_max_iter >= 0";
    if (!(p->eps_n >= 0)) return "eps_n must be >= 0";
    if (p->open_x != 0 && p->open_x != 1) return "open_x must be 0 or 1";
    if (!(p->s13_over_s12 > 0) || !(p->s23_over_s12 > 0)) return "surface tension ratios must be > 0";
    d->u_avg = 2.0 * p->u_max / 3.0;  // mean of the channel's parabolic profile
    double s23;
    if (p->sigma23 > 0) s23 = p->sigma23;
    else if (p->Ca > 0 && p->u_max > 0) s23 = p->rho[2] * p->nu[2] * d->u_avg / p->Ca;  // Eq. 40
    else return "need Ca > 0 with u_max > 0, or sigma23 > 0";
    const double s12 = s23 / p->s23_over_s12, s13 = p->s13_over_s12 * s12;
    d->s12 = s12;
    d->s13 = s13;
    d->s23 = s23;
    d->gam[0] = s12 + s13 - s23;  // Eq. 27
    d->gam[1] = s12 + s23 - s13;
    d->gam[2] = s13 + s23 - s12;
    // Total spreading (some gamma_i < 0, Eq. 27) needs the eta term of Eq. 28,
    // and a gradient energy sum_i gamma_i |grad phi_i|^2 that stays positive
    // on sum_i grad phi_i = 0 (gamma1 gamma2 + gamma1 gamma3 + gamma2 gamma3 > 0).
    if (!(p->eta >= 0)) return "eta must be >= 0";
    bool total = false;
    for (int i = 0; i < 3; i++) {
        if (d->gam[i] == 0.0) return "a spreading coefficient gamma_i is 0 (Eq. 26 undefined)";
        if (d->gam[i] < 0.0) total = true;
    }
    if (total && !(p->eta > 0)) return "total spreading (a gamma_i < 0) needs eta > 0 (Eq. 28)";
    if (!(d->gam[0] * d->gam[1] + d->gam[0] * d->gam[2] + d->gam[1] * d->gam[2] > 0))
        return "spreading coefficients give a gradient energy that is not positive";
    d->gamT = 3.0 / (1.0 / d->gam[0] + 1.0 / d->gam[1] + 1.0 / d->gam[2]);  // Eq. 26
    for (int i = 0; i < 3; i++) d->tau[i] = 3.0 * p->nu[i];                // Eq. 14
    d->tau_phi = 3.0 * p->mobility;                                        // Eq. 30
    d->mu0H0sq = 0.0;
    if (p->ferro_phase == 1) {
        if (!(p->chi[0] > 0) || !(p->r1 > 0)) return "core ferrofluid needs chi1 > 0 and r1 > 0";
        d->mu0H0sq = 2.0 * s12 * p->Bo_m / (p->chi[0] * p->r1);  // Eq. 41, core
    } else if (p->ferro_phase == 2) {
        const double den = p->chi[1] * (p->r2 * p->r2 - p->r1 * p->r1);
        if (!(den > 0)) return "shell ferrofluid needs chi2 > 0 and r2 > r1";
        d->mu0H0sq = 2.0 * (s12 * p->r1 + s23 * p->r2) * p->Bo_m / den;  // Eq. 41, shell
    } else if (p->ferro_phase != 0) {
        return "ferro_phase must be 0, 1 or 2";
    }
    if (!(d->mu0H0sq >= 0)) return "Bo_m must be >= 0";
    d->H0 = std::sqrt(d->mu0H0sq);
    d->G = 8.0 * p->rho[2] * p->nu[2] * p->u_max / ((double)p->ny * p->ny);
    if (p->open_x) d->G = 0.0;  // the open channel is driven by its inlet
    return nullptr;
}

template <typename T>
static Phys<T> make_phys(const fcd_params *p, const Derived &d, int pitch) {
    Phys<T> P;
    std::memset(&P, 0, sizeof(P));
    P.nx = p->nx;
    P.ny = p->ny;
    P.pitch = pitch;
    P.ps = (long long)pitch * p->ny;
    for (int i = 0; i < 3; i++) {
        P.rho[i] = T(p->rho[i]);
        P.tau[i] = T(d.tau[i]);
        P.ik[i] = T(1.0 / (1.0 + p->chi[i]));
        P.gam[i] = T(d.gam[i]);
        P.lap_coef[i] = T(0.75 * p->xi * d.gam[i]);
    }
    P.dk1 = T(1.0 / (1.0 + p->chi[0]) - 1.0 / (1.0 + p->chi[2]));
    P.dk2 = T(1.0 / (1.0 + p->chi[1]) - 1.0 / (1.0 + p->chi[2]));
    P.s12 = T(d.s12);
    P.s13 = T(d.s13);
    P.s23 = T(d.s23);
    P.eta = T(p->eta);
    P.twelve_over_xi = T(12.0 / p->xi);
    P.four_over_xi = T(4.0 / p->xi);
    P.eps_n = T(p->eps_n);
    const double om = 1.0 / (0.5 + d.tau_phi);
    P.om_phi = T(om);
    P.keep_phi = T(1.0 - om);
    P.src_phi = T(1.0 - 0.5 * om);
    P.H0c = T(d.H0 * std::cos(p->alpha));
    P.H0s = T(d.H0 * std::sin(p->alpha));
    P.G = T(d.G);
    return P;
}

// ---------------------------------------------------------------- context
struct fcd_ctx {
    fcd_params prm;
    Derived D;
    char err[512] = {0};
    cudaStream_t stream = nullptr;
    long step = 0;
    virtual ~fcd_ctx() {}
    virtual fcd_status init() = 0;
    virtual fcd_status do_step(long n) = 0;
    virtual fcd_status solve(double tol, int max_iter, int *iters, double *resid) = 0;
    virtual fcd_status observe(fcd_obs *o) = 0;
    virtual fcd_status field(int which, double *dst, size_t n) = 0;
    virtual fcd_status get_pops(double *f, double *g, double *psi) = 0;
    virtual fcd_status set_pops(const double *f, const double *g, const double *psi, long st) = 0;
    virtual size_t state_bytes() const = 0;
    virtual fcd_status get_state(void *dst, size_t bytes) = 0;
    virtual fcd_status set_state(const void *src, size_t bytes) = 0;
    virtual long launches() const = 0;
    virtual fcd_status solver_stats(long long *out5) = 0;
    virtual fcd_status set_profiling(int on) = 0;
    virtual fcd_status profile(double *ms) = 0;
    virtual int collide_tile_h() const = 0;
    fcd_status fail(fcd_status s, const char *fmt, ...) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, sizeof err, fmt, ap);
        va_end(ap);
        return s;
    }
};

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return fail(FCD_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

struct SnapHeader {
    unsigned magic, version;
    int nx, ny, precision, pitch;
    long long step;
    unsigned long long brk;
    int cur, pad;  // which level-0 potential buffer is current
};
static const unsigned SNAP_VERSION = 4;
static const unsigned SNAP_MAGIC = 0x46434453u;  // "FCDS"

template <typename T>
struct Engine : fcd_ctx {
    using S = T;  // stored type equals the compute type (FP64 or FP32)
    int mode = MODE_FP64;
    int pitch = 0;
    long long ps = 0;
    Phys<T> P;
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *user = nullptr;
    std::vector<void *> mem;
    void *f[2] = {nullptr, nullptr}, *g[2] = {nullptr, nullptr};
    int cur = 0;
    T *phi1 = nullptr, *phi2 = nullptr, *k = nullptr, *psiA = nullptr, *psiB = nullptr,
      *psiP = nullptr, *macro = nullptr;
    MgCtl *ctl = nullptr;
    MgHost<T> *mg = nullptr;
    unsigned long long *brk = nullptr;
    unsigned long long *unst = nullptr;  // first step with a non-finite collision (~0: none)
    long long *d_step = nullptr;
    double *obs_scratch = nullptr;
    ObsOut *obs_out = nullptr;
    MgCtl *h_ctl = nullptr;
    ObsOut *h_obs = nullptr;
    SnapHeader *h_snap = nullptr;  // pinned staging of snapshot headers
    unsigned long long *h_brk = nullptr;
    unsigned long long *h_unst = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    bool use_graph = true;
    bool profiling = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    long host_kernels = 0;
    int reported_nonconv = 0;
    int copies = 1;  // plane sets per field: 1, or 1 + NT for the tangent context
    int tile_h = TY;  // rows per collide tile (FP32: chosen at create, tune_collide)
    int collide_tile_h() const override { return tile_h; }

    // one level-0 potential buffer: psi_planes<T>() planes (FP32: hi and lo)
    size_t psi_bytes() const { return (size_t)psi_planes<T>() * ps * sizeof(T); }
    // FP32 contexts solving below 1e-4 hold psi' as the hi + lo pair: one FP32
    // plane floors the residual at ~2e-5 on the paper's channels (more on
    // larger droplets), and 1e-4 is the tightest tolerance it serves
    static constexpr double COMP_TOL = 1e-4;
    int comp = 0;

    T *dalloc(size_t bytes) {
        void *p = alloc(bytes, user);
        if (p) mem.push_back(p);
        return static_cast<T *>(p);
    }

    ~Engine() override {
        if (stream) cudaStreamSynchronize(stream);
        cudaDeviceSynchronize();
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                if (gexec[a][b]) cudaGraphExecDestroy(gexec[a][b]);
                if (graph[a][b]) cudaGraphDestroy(graph[a][b]);
            }
        if (mg) mg_destroy(mg);
        for (void *p : mem) release(p, user);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (h_obs) cudaFreeHost(h_obs);
        if (h_snap) cudaFreeHost(h_snap);
        if (h_brk) cudaFreeHost(h_brk);
        if (h_unst) cudaFreeHost(h_unst);
        if (cap) cudaStreamDestroy(cap);
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }

    bool magnetic() const { return D.H0 > 0.0; }

    fcd_status init() override {
        mode = prm.precision == FCD_FP64 ? MODE_FP64 : (prm.precision == FCD_FP32 ? MODE_FP32 : MODE_FP32_OFFSET);
        pitch = (prm.nx + 31) / 32 * 32;
        ps = (long long)pitch * prm.ny;
        P = make_phys<T>(&prm, D, pitch);
        comp = sizeof(T) == 4 && prm.mag_tol < COMP_TOL ? 1 : 0;
        const char *nog = getenv("FCD_NO_GRAPH");
        use_graph = !(nog && nog[0] == '1');
        for (int b = 0; b < 2; b++) {
            f[b] = dalloc(9 * copies * ps * sizeof(S));
            g[b] = dalloc(18 * copies * ps * sizeof(S));
        }
        phi1 = dalloc(copies * ps * sizeof(T));
        phi2 = dalloc(copies * ps * sizeof(T));
        k = dalloc(copies * ps * sizeof(T));
        psiA = dalloc(psi_bytes());
        psiB = dalloc(psi_bytes());
        psiP = dalloc(psi_bytes());
        macro = dalloc(3 * ps * sizeof(T));
        ctl = reinterpret_cast<MgCtl *>(dalloc(sizeof(MgCtl)));
        brk = reinterpret_cast<unsigned long long *>(dalloc(sizeof(unsigned long long)));
        unst = reinterpret_cast<unsigned long long *>(dalloc(sizeof(unsigned long long)));
        d_step = reinterpret_cast<long long *>(dalloc(sizeof(long long)));
        obs_scratch = reinterpret_cast<double *>(dalloc(observe_scratch_doubles(prm.nx, prm.ny) * sizeof(double)));
        obs_out = reinterpret_cast<ObsOut *>(dalloc(sizeof(ObsOut)));
        for (void *p : {f[0], f[1], g[0], g[1], (void *)phi1, (void *)phi2, (void *)k, (void *)psiA,
                        (void *)psiB, (void *)psiP, (void *)macro, (void *)ctl, (void *)brk, (void *)unst, (void *)d_step,
                        (void *)obs_scratch, (void *)obs_out})
            if (!p) return fail(FCD_ENOMEM, "device allocation failed");
        CK(cudaMallocHost(&h_ctl, sizeof(MgCtl)));
        CK(cudaMallocHost(&h_obs, sizeof(ObsOut)));
        CK(cudaMallocHost(&h_snap, sizeof(SnapHeader)));
        CK(cudaMallocHost(&h_brk, sizeof(unsigned long long)));
        CK(cudaMallocHost(&h_unst, sizeof(unsigned long long)));
        CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        for (auto &e : ev) CK(cudaEventCreate(&e));
        mg = mg_create<T>(prm.nx, prm.ny, pitch, k, psiA, psiB, ctl, alloc, release, user, err,
                          sizeof err, comp);
        if (!mg) return FCD_ENOMEM;
        cudaStream_t s = stream;
        CK(cudaMemsetAsync(ctl, 0, sizeof(MgCtl), s));
        CK(cudaMemsetAsync(psiA, 0, psi_bytes(), s));
        CK(cudaMemsetAsync(psiB, 0, psi_bytes(), s));
        CK(cudaMemsetAsync(psiP, 0, psi_bytes(), s));
        CK(cudaMemsetAsync(brk, 0xff, sizeof(unsigned long long), s));
        CK(cudaMemsetAsync(unst, 0xff, sizeof(unsigned long long), s));
        CK(cudaMemsetAsync(d_step, 0, sizeof(long long), s));
        // padding columns of every plane stay zero
        for (int b = 0; b < 2; b++) {
            CK(cudaMemsetAsync(f[b], 0, 9 * copies * ps * sizeof(S), s));
            CK(cudaMemsetAsync(g[b], 0, 18 * copies * ps * sizeof(S), s));
        }
        CK(cudaMemsetAsync(phi1, 0, copies * ps * sizeof(T), s));
        CK(cudaMemsetAsync(phi2, 0, copies * ps * sizeof(T), s));
        CK(cudaMemsetAsync(k, 0, copies * ps * sizeof(T), s));
        {
            MgCtl c;
            std::memset(&c, 0, sizeof c);
            c.H0 = D.H0;
            c.tolH0 = prm.mag_tol * D.H0;
            c.max_iter = prm.mag_max_iter;
            *h_ctl = c;
            CK(cudaMemcpyAsync(ctl, h_ctl, sizeof(MgCtl), cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));
        }
        launch_init<T>(mode, P, prm.u_max, prm.r1, prm.r2, prm.xc, prm.yc, prm.xi, f[0], g[0], macro, s);
        host_kernels++;
        CK(cudaGetLastError());
        int it;
        double res;
        fcd_status st = solve(prm.mag_tol, prm.mag_max_iter > 100 ? prm.mag_max_iter : 100, &it, &res);
        if (st != FCD_OK && st != FCD_ENOCONV) return st;
        st = tune_collide();
        if (st != FCD_OK) return st;
        return keep_history();
    }

    // FP32 forms: the collide tile height (4 or 8 rows) that runs this grid
    // faster, timed with events on the context's stream (the best of eight
    // launches each, alternating, after one untimed launch of each; on the
    // 1600 x 200 channel the two differ by about 6%, 1.4 us a launch). The two heights do the
    // same arithmetic per node. The timed launches write the idle population
    // buffers, which the first step overwrites, and record neither breakup nor
    // instability. FCD_COLLIDE_TILE_H=4 or 8 fixes the height instead.
    fcd_status tune_collide() {
        if (sizeof(T) != 4) return FCD_OK;
        const char *env = getenv("FCD_COLLIDE_TILE_H");
        if (env && (atoi(env) == 4 || atoi(env) == 8)) {
            tile_h = atoi(env);
            return FCD_OK;
        }
        LbmArgs<T> a = collide_args(cur, false);
        a.brk = nullptr;
        a.unst = nullptr;
        const int hs[2] = {4, 8};
        float best[2] = {1e30f, 1e30f};
        cudaStream_t s = stream;
        for (int r = 0; r < 9; r++)
            for (int v = 0; v < 2; v++) {
                CK(cudaEventRecord(ev[0], s));
                launch_collide<T>(mode, hs[v], a, s);
                CK(cudaEventRecord(ev[1], s));
                CK(cudaEventSynchronize(ev[1]));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
                if (r > 0) best[v] = std::min(best[v], ms);
            }
        host_kernels += 18;
        tile_h = best[0] < best[1] ? 4 : 8;
        return FCD_OK;
    }

    // The previous potential (for the extrapolated initial guess) := current.
    fcd_status keep_history() {
        if (sync_ctl() != FCD_OK) return FCD_ECUDA;
        CK(cudaMemcpyAsync(psiP, h_ctl->cur ? psiB : psiA, psi_bytes(), cudaMemcpyDeviceToDevice, stream));
        CK(cudaStreamSynchronize(stream));
        return FCD_OK;
    }

    // ---- one step as kernel launches on stream s (the MG loop by while node
    // when capturing, by host polling otherwise)
    fcd_status enqueue_pre(int c, cudaStream_t s) {
        PhaseCtl pc{ctl, magnetic() ? 1 : 0, prm.mag_tol * D.H0, prm.mag_max_iter, d_step,
                    magnetic() ? 1 : 0, psiA, psiB, psiP, comp};
        launch_phase<T>(mode, P, g[c], phi1, phi2, k, pc, s);
        return FCD_OK;
    }
    LbmArgs<T> collide_args(int c, bool store_macro) const {
        LbmArgs<T> a;
        a.P = P;
        a.f_src = f[c];
        a.g_src = g[c];
        a.f_dst = f[c ^ 1];
        a.g_dst = g[c ^ 1];
        a.phi1 = phi1;
        a.phi2 = phi2;
        a.psi0 = psiA;
        a.psi1 = psiB;
        a.ctl = ctl;
        a.macro = store_macro ? macro : nullptr;
        a.brk = brk;
        a.step = &ctl->step_cur;
        a.unst = unst;
        a.open_x = prm.open_x;
        return a;
    }
    void enqueue_post(int c, bool store_macro, cudaStream_t s) {
        launch_collide<T>(mode, tile_h, collide_args(c, store_macro), s);
        if (prm.open_x)
            launch_open_bc<T>(mode, P, f[c], g[c], f[c ^ 1], g[c ^ 1], prm.u_max, D.u_avg, s);
    }
    int post_kernels() const { return prm.open_x ? 2 : 1; }
    // the phase kernel, and in FP64 contexts with a field the solve's
    // coefficient kernel (the multigrid counts its own cycles)
    int pre_kernels() const { return 1 + (magnetic() && sizeof(T) == 8 ? 1 : 0); }

    // One solve with host checks between cycles (hierarchy m with control
    // block c; default: the context's own).
    fcd_status host_mg_loop(cudaStream_t s, MgHost<T> *m = nullptr, MgCtl *c = nullptr) {
        if (!m) {
            m = mg;
            c = ctl;
        }
        mg_presmooth<T>(m, P.H0c, P.H0s, s);
        for (int guard = 0; guard < 1000000; guard++) {
            mg_cycle_head<T>(m, P.H0c, P.H0s, 0, 0, 0, s);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(h_ctl, c, sizeof(MgCtl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (!h_ctl->keep_going) break;
            if (h_ctl->mode == 1) mg_cycle_smooth<T>(m, P.H0c, P.H0s, s);
            else if (h_ctl->mode == 2) mg_cycle_twogrid<T>(m, P.H0c, P.H0s, s);
            else mg_cycle_rest<T>(m, P.H0c, P.H0s, s);
            CK(cudaGetLastError());
        }
        return FCD_OK;
    }

    fcd_status build_graph(int c, int sm) {
        cudaStream_t s = cap;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const fcd_status st = capture_step(c, sm, s);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);  // always leave capture mode
        if (st != FCD_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        CK(e);
        graph[c][sm] = g;
        CK(cudaGraphInstantiate(&gexec[c][sm], graph[c][sm], 0));
        return FCD_OK;
    }

    // The cycle loop of one potential solve in the graph (stream s is capturing;
    // the opening sweeps are already captured), in one of two shapes. Contexts
    // solving to 1e-5 or looser, whose solves mostly stop at their first head
    // (1.0-1.1 heads per step on the FP32 production channels), take the IF
    // form; tighter tolerances (FP64 at 1e-10: about 11 heads per step) the
    // while form. Measured: 1600 x 200 FP32 solve stage 33.9 -> 28.0 us with the
    // IF form; 200 x 40 FP64 0.72 -> 0.78 ms per step with it (one dispatch
    // kernel node more per cycle), hence the split.
    static constexpr double IF_FORM_TOL = 1e-5;
    fcd_status capture_mg_loop(cudaStream_t s, MgHost<T> *m = nullptr) {
        if (!m) m = mg;
        return prm.mag_tol >= IF_FORM_TOL ? capture_mg_if_loop(s, m) : capture_mg_while_loop(s, m);
    }

    // The while form: a while node whose body is the cycle head (the residual
    // kernel, which sets both conditions) and a switch node holding the rest of
    // the chosen cycle. One kernel node fewer per cycle than the IF form, for
    // solves that run many cycles.
    fcd_status capture_mg_while_loop(cudaStream_t s, MgHost<T> *m) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t gcap;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &gcap, &deps, nullptr, &nd));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, gcap, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wnode;
        CK(cudaGraphAddNode(&wnode, gcap, deps, nullptr, nd, &cp));
        // while body: lattice residual, then a switch node holding the rest
        // of the V-cycle (case 0), lattice sweeps only (case 1) or a
        // two-grid cycle (case 2); both conditions are set by the residual
        // kernel
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphConditionalHandle hi;
        CK(cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault));
        cudaStream_t bs;
        CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
        cudaError_t e1 = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal);
        cudaGraph_t out1 = nullptr, out2 = nullptr;
        if (e1 == cudaSuccess) {
            mg_cycle_head<T>(m, P.H0c, P.H0s, h, hi, 1, bs);
            const cudaGraphNode_t *bd = nullptr;
            size_t bn = 0;
            cudaStreamCaptureStatus bcs;
            cudaGraph_t bg;
            e1 = cudaStreamGetCaptureInfo(bs, &bcs, nullptr, &bg, &bd, nullptr, &bn);
            cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
            ip.conditional.handle = hi;
            ip.conditional.type = cudaGraphCondTypeSwitch;
            ip.conditional.size = 3;
            cudaGraphNode_t inode;
            if (e1 == cudaSuccess) e1 = cudaGraphAddNode(&inode, body, bd, nullptr, bn, &ip);
            if (e1 == cudaSuccess)
                e1 = cudaStreamUpdateCaptureDependencies(bs, &inode, nullptr, 1,
                                                         cudaStreamSetCaptureDependencies);
            cudaError_t e2 = cudaStreamEndCapture(bs, &out1);
            if (e1 == cudaSuccess) e1 = e2;
            if (e1 == cudaSuccess)
                e1 = cudaStreamBeginCaptureToGraph(bs, ip.conditional.phGraph_out[0], nullptr,
                                                   nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e1 == cudaSuccess) {
                mg_cycle_rest<T>(m, P.H0c, P.H0s, bs);
                e1 = cudaStreamEndCapture(bs, &out2);
            }
            if (e1 == cudaSuccess)
                e1 = cudaStreamBeginCaptureToGraph(bs, ip.conditional.phGraph_out[1], nullptr,
                                                   nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e1 == cudaSuccess) {
                mg_cycle_smooth<T>(m, P.H0c, P.H0s, bs);
                e1 = cudaStreamEndCapture(bs, &out2);
            }
            if (e1 == cudaSuccess)
                e1 = cudaStreamBeginCaptureToGraph(bs, ip.conditional.phGraph_out[2], nullptr,
                                                   nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e1 == cudaSuccess) {
                mg_cycle_twogrid<T>(m, P.H0c, P.H0s, bs);
                e1 = cudaStreamEndCapture(bs, &out2);
            }
        }
        cudaStreamDestroy(bs);
        CK(e1);
        CK(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
        return FCD_OK;
    }

    // The IF form: the first cycle head as a plain
    // kernel node, then an IF node, entered only when that head chose another
    // cycle, around a while node (condition 1 on entry) whose body dispatches
    // the chosen cycle through a switch node (0 the rest of a V-cycle, 1 lattice
    // sweeps, 2 a two-grid cycle) and ends with the next head, which sets the
    // loop condition. A conditional node costs about 8.7 us whether it runs its
    // body or not (measured on this GPU); a solve that stops at its first head,
    // the common case, pays for the IF node only, not for a while node entered
    // once with a switch node inside (about 14 us).
    fcd_status capture_mg_if_loop(cudaStream_t s, MgHost<T> *m) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t gcap;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &gcap, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle hif;
        CK(cudaGraphConditionalHandleCreate(&hif, gcap, 0, cudaGraphCondAssignDefault));
        mg_cycle_head<T>(m, P.H0c, P.H0s, hif, 0, 3, s);
        CK(cudaGetLastError());
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &gcap, &deps, nullptr, &nd));
        cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
        ip.conditional.handle = hif;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t ifnode;
        CK(cudaGraphAddNode(&ifnode, gcap, deps, nullptr, nd, &ip));
        cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
        // while node inside the IF body, entered with its condition at 1
        cudaGraphConditionalHandle hw;
        CK(cudaGraphConditionalHandleCreate(&hw, ifbody, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
        wp.conditional.handle = hw;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode;
        CK(cudaGraphAddNode(&wnode, ifbody, nullptr, nullptr, 0, &wp));
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        cudaGraphConditionalHandle hs;
        CK(cudaGraphConditionalHandleCreate(&hs, body, 0, cudaGraphCondAssignDefault));
        cudaStream_t bs;
        CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
        cudaGraphNodeParams sp = {cudaGraphNodeTypeConditional};
        sp.conditional.handle = hs;
        sp.conditional.type = cudaGraphCondTypeSwitch;
        sp.conditional.size = 3;
        cudaGraph_t out = nullptr;
        // loop body: dispatch -> switch node -> next head
        cudaError_t e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            mg_cycle_dispatch<T>(m, hs, bs);
            const cudaGraphNode_t *bd = nullptr;
            size_t bn = 0;
            cudaStreamCaptureStatus bcs;
            cudaGraph_t bg;
            e = cudaStreamGetCaptureInfo(bs, &bcs, nullptr, &bg, &bd, nullptr, &bn);
            cudaGraphNode_t snode;
            if (e == cudaSuccess) e = cudaGraphAddNode(&snode, body, bd, nullptr, bn, &sp);
            if (e == cudaSuccess)
                e = cudaStreamUpdateCaptureDependencies(bs, &snode, nullptr, 1,
                                                        cudaStreamSetCaptureDependencies);
            if (e == cudaSuccess) mg_cycle_head<T>(m, P.H0c, P.H0s, hw, 0, 3, bs);
            const cudaError_t e2 = cudaStreamEndCapture(bs, &out);
            if (e == cudaSuccess) e = e2;
        }
        // the three cases of the switch node
        for (int c = 0; c < 3 && e == cudaSuccess; c++) {
            e = cudaStreamBeginCaptureToGraph(bs, sp.conditional.phGraph_out[c], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) break;
            if (c == 0) mg_cycle_rest<T>(m, P.H0c, P.H0s, bs);
            else if (c == 1) mg_cycle_smooth<T>(m, P.H0c, P.H0s, bs);
            else mg_cycle_twogrid<T>(m, P.H0c, P.H0s, bs);
            e = cudaStreamEndCapture(bs, &out);
        }
        cudaStreamDestroy(bs);
        CK(e);
        CK(cudaStreamUpdateCaptureDependencies(s, &ifnode, nullptr, 1, cudaStreamSetCaptureDependencies));
        return FCD_OK;
    }

    // The captured sequence of one step (stream s is in capture mode).
    virtual fcd_status capture_step(int c, int sm, cudaStream_t s) {
        if (profiling) CK(cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal));
        enqueue_pre(c, s);
        if (profiling) CK(cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal));
        if (magnetic()) {
            mg_presmooth<T>(mg, P.H0c, P.H0s, s);
            const fcd_status st = capture_mg_loop(s);
            if (st != FCD_OK) return st;
        }
        if (profiling) CK(cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal));
        enqueue_post(c, sm != 0, s);
        if (profiling) CK(cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal));
        return FCD_OK;
    }

    // One step; sm != 0 also stores the macroscopic fields.
    fcd_status one_step(int sm) {
        cudaStream_t s = stream;
        if (use_graph) {
            if (!gexec[cur][sm]) {
                fcd_status st = build_graph(cur, sm);
                if (st != FCD_OK) return st;
            }
            CK(cudaGraphLaunch(gexec[cur][sm], s));
            host_kernels += pre_kernels() + post_kernels();
        } else {
            if (profiling) CK(cudaEventRecord(ev[0], s));
            {
                NvtxScope r("fcd phase recovery");
                enqueue_pre(cur, s);
            }
            if (profiling) CK(cudaEventRecord(ev[1], s));
            if (magnetic()) {
                NvtxScope r("fcd potential solve");
                fcd_status st = host_mg_loop(s);
                if (st != FCD_OK) return st;
            }
            if (profiling) CK(cudaEventRecord(ev[2], s));
            {
                NvtxScope r("fcd collide-stream");
                enqueue_post(cur, sm != 0, s);
            }
            if (profiling) CK(cudaEventRecord(ev[3], s));
            host_kernels += pre_kernels() + post_kernels();
            CK(cudaGetLastError());
        }
        cur ^= 1;
        step++;
        return FCD_OK;
    }

    fcd_status do_step(long n) override {
        if (n < 0) return fail(FCD_EINVAL, "negative step count");
        for (long i = 0; i < n; i++) {
            const fcd_status st = one_step(i == n - 1 ? 1 : 0);
            if (st != FCD_OK) return st;
        }
        CK(cudaGetLastError());
        return FCD_OK;
    }

    fcd_status sync_ctl() {
        CK(cudaMemcpyAsync(h_ctl, ctl, sizeof(MgCtl), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        return FCD_OK;
    }

    fcd_status solve(double tol, int max_iter, int *iters, double *resid) override {
        if (!(tol > 0)) tol = prm.mag_tol;
        if (max_iter <= 0) max_iter = prm.mag_max_iter;
        cudaStream_t s = stream;
        if (!magnetic()) {
            CK(cudaMemsetAsync(psiA, 0, psi_bytes(), s));
            CK(cudaMemsetAsync(psiB, 0, psi_bytes(), s));
            CK(cudaMemsetAsync(psiP, 0, psi_bytes(), s));
            CK(cudaStreamSynchronize(s));
            if (iters) *iters = 0;
            if (resid) *resid = 0.0;
            return FCD_OK;
        }
        launch_phase<T>(mode, P, g[cur], phi1, phi2, k,
                        PhaseCtl{ctl, 1, tol * D.H0, max_iter, nullptr, 0, nullptr, nullptr, nullptr}, s);
        host_kernels += pre_kernels();  // the opening sweeps are counted with the sweep cycles
        CK(cudaGetLastError());
        fcd_status st = host_mg_loop(s);
        if (st != FCD_OK) return st;
        if (iters) *iters = h_ctl->last_iters;
        if (resid) *resid = h_ctl->last_resid;
        if (!h_ctl->converged) {
            reported_nonconv = h_ctl->nonconv_count;
            return fail(FCD_ENOCONV, "potential solve stopped at %d V-cycles with residual %.3e",
                        h_ctl->last_iters, h_ctl->last_resid);
        }
        return FCD_OK;
    }

    fcd_status observe(fcd_obs *o) override {
        cudaStream_t s = stream;
        launch_observe<T>(mode, P, g[cur], obs_scratch, obs_out, s, prm.open_x);
        host_kernels += 4;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h_obs, obs_out, sizeof(ObsOut), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_brk, brk, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_unst, unst, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_ctl, ctl, sizeof(MgCtl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const ObsOut &r = *h_obs;
        std::memset(o, 0, sizeof *o);
        o->step = step;
        o->t_star = step * D.u_avg / (2.0 * prm.r2);  // Eq. 38
        for (int i = 0; i < 3; i++) o->mass[i] = r.mass[i];
        o->lx_o = r.lx_o; o->ly_o = r.ly_o; o->lx_i = r.lx_i; o->ly_i = r.ly_i;
        o->T_o = (r.lx_o + r.ly_o) > 0 ? (r.ly_o - r.lx_o) / (r.ly_o + r.lx_o) : 0.0;  // Eq. 42
        o->T_i = (r.lx_i + r.ly_i) > 0 ? (r.ly_i - r.lx_i) / (r.ly_i + r.lx_i) : 0.0;
        o->xc_core = r.xc_core; o->yc_core = r.yc_core;
        o->xc_shell = r.xc_shell; o->yc_shell = r.yc_shell;
        long long bstep = -1, bnode = 0;
        if (*h_brk != ~0ull) {
            bstep = (long long)(*h_brk >> 32);
            bnode = (long long)(*h_brk & 0xffffffffull);
        } else if (r.brk_now != ~0ull) {
            bstep = step;
            bnode = (long long)r.brk_now;
        }
        o->b_step = bstep;
        if (bstep >= 0) {
            o->breakup = 1;
            o->xb = double(bnode % prm.nx);
            o->yb = double(bnode / prm.nx);
            o->tb_star = bstep * D.u_avg / (2.0 * prm.r2);
            o->Lb_star = o->xb / prm.ny;
            o->yb_star = std::fabs(o->yb - 0.5 * (prm.ny - 1)) / prm.ny;
        }
        o->mag_iters = magnetic() ? h_ctl->last_iters : 0;
        o->mag_resid = magnetic() ? h_ctl->last_resid : 0.0;
        if (unstable_status() != FCD_OK) return FCD_EUNSTABLE;
        if (r.nonfinite) return fail(FCD_EUNSTABLE, "non-finite phase field at step %ld", step);
        if (h_ctl->nonconv_count > reported_nonconv) {
            reported_nonconv = h_ctl->nonconv_count;
            return fail(FCD_ENOCONV, "a potential solve stopped at the cycle cap (residual %.3e)",
                        h_ctl->last_resid);
        }
        return FCD_OK;
    }

    // FCD_EUNSTABLE once a collision produced a non-finite velocity or
    // pressure; h_unst must have been copied in the caller's synchronised batch.
    fcd_status unstable_status() {
        if (*h_unst == ~0ull) return FCD_OK;
        return fail(FCD_EUNSTABLE, "non-finite velocity or pressure, first in step %llu (now at step %ld)",
                    *h_unst, step);
    }

    double *staging(size_t doubles) {
        void *p = nullptr;
        if (cudaMalloc(&p, doubles * sizeof(double)) != cudaSuccess) return nullptr;
        return static_cast<double *>(p);
    }

    fcd_status field(int which, double *dst, size_t n) override {
        const size_t N = (size_t)prm.nx * prm.ny;
        if (!dst || n < N) return fail(FCD_EINVAL, "destination holds %zu of %zu values", n, N);
        if (which < FCD_FIELD_PHI1 || which > FCD_FIELD_PSI) return fail(FCD_EINVAL, "unknown field %d", which);
        cudaStream_t s = stream;
        double *st = staging(N);
        if (!st) return fail(FCD_ENOMEM, "staging allocation failed");
        fcd_status rc = FCD_OK;
        if (which <= FCD_FIELD_PHI3) {
            launch_phase<T>(mode, P, g[cur], phi1, phi2, nullptr,
                            PhaseCtl{nullptr, 0, 0.0, 0, nullptr, 0, nullptr, nullptr, nullptr}, s);
            if (which == FCD_FIELD_PHI1) launch_plane_to_f64<T>(phi1, prm.nx, prm.ny, pitch, st, s);
            else if (which == FCD_FIELD_PHI2) launch_plane_to_f64<T>(phi2, prm.nx, prm.ny, pitch, st, s);
            else launch_phi3_to_f64<T>(phi1, phi2, prm.nx, prm.ny, pitch, st, s);
            host_kernels += 2;
        } else if (which <= FCD_FIELD_PSTAR) {
            launch_plane_to_f64<T>(macro + (which - FCD_FIELD_UX) * ps, prm.nx, prm.ny, pitch, st, s);
            host_kernels += 1;
        } else {
            if (sync_ctl() != FCD_OK) { cudaFree(st); return FCD_ECUDA; }
            launch_psi_to_f64<T>(h_ctl->cur ? psiB : psiA, prm.nx, prm.ny, pitch, st, s);
            host_kernels += 1;
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, st, N * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_unst, unst, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(FCD_ECUDA, "get_field: %s", cudaGetErrorString(e));
        cudaFree(st);
        if (rc == FCD_OK) rc = unstable_status();  // the field is delivered all the same
        return rc;
    }

    fcd_status get_pops(double *fo, double *go, double *po) override {
        const size_t N = (size_t)prm.nx * prm.ny;
        cudaStream_t s = stream;
        double *st = staging(28 * N);
        if (!st) return fail(FCD_ENOMEM, "staging allocation failed");
        if (sync_ctl() != FCD_OK) { cudaFree(st); return FCD_ECUDA; }
        launch_export<T>(mode, P, f[cur], g[cur], st, st + 9 * N, s);
        launch_psi_to_f64<T>(h_ctl->cur ? psiB : psiA, prm.nx, prm.ny, pitch, st + 27 * N, s);
        host_kernels += 2;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && fo) e = cudaMemcpyAsync(fo, st, 9 * N * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess && go) e = cudaMemcpyAsync(go, st + 9 * N, 18 * N * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess && po) e = cudaMemcpyAsync(po, st + 27 * N, N * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_unst, unst, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(st);
        if (e != cudaSuccess) return fail(FCD_ECUDA, "get_populations: %s", cudaGetErrorString(e));
        return unstable_status();  // the populations are delivered all the same
    }

    fcd_status set_pops(const double *fi, const double *gi, const double *pi, long st_) override {
        const size_t N = (size_t)prm.nx * prm.ny;
        if (st_ < 0) return fail(FCD_EINVAL, "negative step");
        cudaStream_t s = stream;
        double *st = staging(28 * N);
        if (!st) return fail(FCD_ENOMEM, "staging allocation failed");
        cudaError_t e = cudaSuccess;
        if (fi) e = cudaMemcpyAsync(st, fi, 9 * N * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess && gi) e = cudaMemcpyAsync(st + 9 * N, gi, 18 * N * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess && pi) e = cudaMemcpyAsync(st + 27 * N, pi, N * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess) {
            launch_import<T>(mode, P, fi ? st : nullptr, gi ? st + 9 * N : nullptr, f[cur], g[cur], s);
            host_kernels++;
            if (pi) {
                if (sync_ctl() != FCD_OK) { cudaFree(st); return FCD_ECUDA; }
                launch_psi_from_f64<T>(st + 27 * N, prm.nx, prm.ny, pitch, h_ctl->cur ? psiB : psiA, comp, s);
                host_kernels++;
            }
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(brk, 0xff, sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(unst, 0xff, sizeof(unsigned long long), s);
        long long s64 = st_;
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_step, &s64, sizeof(long long), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(st);
        if (e != cudaSuccess) return fail(FCD_ECUDA, "set_populations: %s", cudaGetErrorString(e));
        step = st_;
        return pi ? keep_history() : FCD_OK;
    }

    // Snapshot: header, the 27 stored population planes of the current buffer,
    // both level-0 potential buffers and the previous potential. Both potential
    // buffers travel, with the device's current-buffer index, so neither call
    // needs to read the control block on the host: each is one stream of
    // asynchronous copies and a single synchronisation.
    size_t state_bytes() const override {
        return sizeof(SnapHeader) + 27 * (size_t)ps * sizeof(S) + 3 * psi_bytes();
    }

    fcd_status get_state(void *dst, size_t bytes) override {
        if (!dst || bytes < state_bytes()) return fail(FCD_EINVAL, "snapshot buffer too small");
        cudaStream_t s = stream;
        CK(cudaStreamSynchronize(s));  // the staging header may still be in flight
        SnapHeader &h = *h_snap;
        std::memset(&h, 0, sizeof h);
        h.magic = SNAP_MAGIC;
        h.version = SNAP_VERSION;
        h.nx = prm.nx;
        h.ny = prm.ny;
        h.precision = prm.precision;
        h.pitch = pitch;
        h.step = step;
        char *d = static_cast<char *>(dst);
        CK(cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(d + offsetof(SnapHeader, brk), brk, sizeof(unsigned long long),
                           cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(d + offsetof(SnapHeader, cur), &ctl->cur, sizeof(int), cudaMemcpyDefault, s));
        size_t off = sizeof h;
        CK(cudaMemcpyAsync(d + off, f[cur], 9 * ps * sizeof(S), cudaMemcpyDefault, s));
        off += 9 * ps * sizeof(S);
        CK(cudaMemcpyAsync(d + off, g[cur], 18 * ps * sizeof(S), cudaMemcpyDefault, s));
        off += 18 * ps * sizeof(S);
        for (T *q : {psiA, psiB, psiP}) {
            CK(cudaMemcpyAsync(d + off, q, psi_bytes(), cudaMemcpyDefault, s));
            off += psi_bytes();
        }
        CK(cudaStreamSynchronize(s));
        return FCD_OK;
    }

    fcd_status set_state(const void *src, size_t bytes) override {
        if (!src || bytes < state_bytes()) return fail(FCD_ESTATE, "snapshot too small");
        cudaStream_t s = stream;
        CK(cudaStreamSynchronize(s));
        SnapHeader &h = *h_snap;
        cudaPointerAttributes at;
        const bool host = cudaPointerGetAttributes(&at, src) == cudaSuccess &&
                          at.type != cudaMemoryTypeDevice;
        cudaGetLastError();  // clear the error of an unregistered pointer query
        if (host) {
            std::memcpy(&h, src, sizeof h);
        } else {
            CK(cudaMemcpyAsync(&h, src, sizeof h, cudaMemcpyDefault, s));
            CK(cudaStreamSynchronize(s));
        }
        if (h.magic != SNAP_MAGIC || h.version != SNAP_VERSION || h.nx != prm.nx || h.ny != prm.ny ||
            h.precision != prm.precision || h.pitch != pitch || (h.cur != 0 && h.cur != 1))
            return fail(FCD_ESTATE, "snapshot does not match this context");
        const char *p = static_cast<const char *>(src);
        size_t off = sizeof h;
        CK(cudaMemcpyAsync(f[cur], p + off, 9 * ps * sizeof(S), cudaMemcpyDefault, s));
        off += 9 * ps * sizeof(S);
        CK(cudaMemcpyAsync(g[cur], p + off, 18 * ps * sizeof(S), cudaMemcpyDefault, s));
        off += 18 * ps * sizeof(S);
        for (T *q : {psiA, psiB, psiP}) {
            CK(cudaMemcpyAsync(q, p + off, psi_bytes(), cudaMemcpyDefault, s));
            off += psi_bytes();
        }
        CK(cudaMemcpyAsync(&ctl->cur, &h.cur, sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(brk, &h.brk, sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_step, &h.step, sizeof(long long), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(unst, 0xff, sizeof(unsigned long long), s));
        CK(cudaStreamSynchronize(s));
        step = (long)h.step;
        return FCD_OK;
    }

    fcd_status set_profiling(int on) override {
        if ((on != 0) == profiling) return FCD_OK;
        CK(cudaStreamSynchronize(stream));
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                if (gexec[a][b]) cudaGraphExecDestroy(gexec[a][b]);
                if (graph[a][b]) cudaGraphDestroy(graph[a][b]);
                gexec[a][b] = nullptr;
                graph[a][b] = nullptr;
            }
        profiling = on != 0;
        return FCD_OK;
    }

    fcd_status profile(double *ms) override {
        if (!profiling) return fail(FCD_EINVAL, "profiling is off");
        CK(cudaEventSynchronize(ev[3]));
        float t[3];
        for (int i = 0; i < 3; i++) CK(cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]));
        ms[0] = t[0];
        ms[1] = t[1];
        ms[2] = t[2];
        float tt;
        CK(cudaEventElapsedTime(&tt, ev[0], ev[3]));
        ms[3] = tt;
        return FCD_OK;
    }

    fcd_status solver_stats(long long *o) override {
        if (sync_ctl() != FCD_OK) return FCD_ECUDA;
        o[0] = h_ctl->cycles_launched;
        o[1] = h_ctl->total_cycles;
        o[2] = h_ctl->twogrid_cycles;
        o[3] = h_ctl->smooth_cycles;
        o[4] = h_ctl->nonconv_count;
        return FCD_OK;
    }

    long launches() const override {
        MgCtl c;
        if (cudaMemcpy(&c, ctl, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
        return host_kernels + (long)c.cycles_launched + (long)c.total_cycles * mg_kernels_per_cycle(mg) +
               (long)c.smooth_cycles + 2 * (long)c.twogrid_cycles + (long)c.dispatches;
    }
};


// ---------------------------------------------------------------- tangent
// Constants of the step in dual arithmetic: the value of every constant and its
// derivative along Bo_m, Ca, alpha and nu_r (nu_r = nu_3 / nu_2), from the
// lattice mapping of derive(): sigma_ij ~ 1/Ca (Eq. 40), so gamma_i and the
// Laplacian coefficients too; mu0 H0^2 ~ Bo_m sigma (Eq. 41), H0 its root;
// H0 (cos alpha, sin alpha); tau_2 = 3 nu_3 / nu_r (Eqs. 14, 39).
static Phys<DualT> tangent_phys(const fcd_params *p, const Phys<double> &P) {
    Phys<DualT> Q;
    Q.nx = P.nx;
    Q.ny = P.ny;
    Q.pitch = P.pitch;
    Q.ps = P.ps;
    for (int i = 0; i < 3; i++) {
        Q.rho[i] = DualT(P.rho[i]);
        Q.tau[i] = DualT(P.tau[i]);
        Q.ik[i] = DualT(P.ik[i]);
        Q.gam[i] = DualT(P.gam[i]);
        Q.lap_coef[i] = DualT(P.lap_coef[i]);
    }
    Q.dk1 = DualT(P.dk1);
    Q.dk2 = DualT(P.dk2);
    Q.s12 = DualT(P.s12);
    Q.s13 = DualT(P.s13);
    Q.s23 = DualT(P.s23);
    Q.eta = DualT(P.eta);
    Q.twelve_over_xi = DualT(P.twelve_over_xi);
    Q.four_over_xi = DualT(P.four_over_xi);
    Q.eps_n = DualT(P.eps_n);
    Q.om_phi = DualT(P.om_phi);
    Q.keep_phi = DualT(P.keep_phi);
    Q.src_phi = DualT(P.src_phi);
    Q.H0c = DualT(P.H0c);
    Q.H0s = DualT(P.H0s);
    Q.G = DualT(P.G);
    if (p->ferro_phase != 0 && p->Bo_m > 0) {
        Q.H0c.d[FCD_DIR_BO_M] = P.H0c / (2.0 * p->Bo_m);
        Q.H0s.d[FCD_DIR_BO_M] = P.H0s / (2.0 * p->Bo_m);
    }
    if (!(p->sigma23 > 0)) {
        const double ic = -1.0 / p->Ca;
        Q.s12.d[FCD_DIR_CA] = P.s12 * ic;
        Q.s13.d[FCD_DIR_CA] = P.s13 * ic;
        Q.s23.d[FCD_DIR_CA] = P.s23 * ic;
        for (int i = 0; i < 3; i++) {
            Q.gam[i].d[FCD_DIR_CA] = P.gam[i] * ic;
            Q.lap_coef[i].d[FCD_DIR_CA] = P.lap_coef[i] * ic;
        }
        Q.H0c.d[FCD_DIR_CA] = 0.5 * P.H0c * ic;
        Q.H0s.d[FCD_DIR_CA] = 0.5 * P.H0s * ic;
    }
    Q.H0c.d[FCD_DIR_ALPHA] = -P.H0s;
    Q.H0s.d[FCD_DIR_ALPHA] = P.H0c;
    Q.tau[1].d[FCD_DIR_NU_R] = -P.tau[1] * p->nu[1] / p->nu[2];
    return Q;
}

// FP64 context whose plane sets carry NT tangent copies (see fcd.h). The
// potential solves run with the host loop of the plain context.
struct TangentEngine : Engine<double> {
    int collide_tile_h() const override { return 4; }  // the dual tiles are larger
    Phys<DualT> PT;
    double *psiT = nullptr;   // 1 + NT planes: the step's potential, then its derivatives
    double *dpsiP = nullptr;  // NT planes: derivatives at the previous step (extrapolation)
    // one multigrid hierarchy per direction (own potential buffers, right-hand
    // side and control block; the permeability k is the primal one), so that
    // the NT solves of a step run side by side
    MgHost<double> *mgt[NT] = {};
    MgCtl *ctlt[NT] = {};
    double *tA[NT] = {}, *tB[NT] = {}, *rhst[NT] = {};
    unsigned long long *rmax = nullptr;  // NT values
    cudaStream_t side[NT] = {};
    cudaEvent_t fork = nullptr, join[NT] = {};
    void *tobs = nullptr;
    TanOut *tan_out = nullptr, *h_tan = nullptr;
    int reported_tangent_nonconv = 0;

    ~TangentEngine() override {
        if (stream) cudaStreamSynchronize(stream);
        cudaDeviceSynchronize();
        for (int c = 0; c < NT; c++) {
            if (mgt[c]) mg_destroy(mgt[c]);
            if (side[c]) cudaStreamDestroy(side[c]);
            if (join[c]) cudaEventDestroy(join[c]);
        }
        if (fork) cudaEventDestroy(fork);
        if (h_tan) cudaFreeHost(h_tan);
    }

    fcd_status init() override {
        copies = 1 + NT;
        pitch = (prm.nx + 31) / 32 * 32;
        ps = (long long)pitch * prm.ny;
        psiT = dalloc((1 + NT) * ps * sizeof(double));
        dpsiP = dalloc(NT * ps * sizeof(double));
        rmax = reinterpret_cast<unsigned long long *>(dalloc(NT * sizeof(unsigned long long)));
        tobs = dalloc(tangent_obs_scratch_bytes(prm.nx));
        tan_out = reinterpret_cast<TanOut *>(dalloc(sizeof(TanOut)));
        for (void *q : {(void *)psiT, (void *)dpsiP, (void *)rmax, tobs, (void *)tan_out})
            if (!q) return fail(FCD_ENOMEM, "device allocation failed");
        for (int c = 0; c < NT; c++) {
            tA[c] = dalloc(ps * sizeof(double));
            tB[c] = dalloc(ps * sizeof(double));
            rhst[c] = dalloc(ps * sizeof(double));
            ctlt[c] = reinterpret_cast<MgCtl *>(dalloc(sizeof(MgCtl)));
            if (!tA[c] || !tB[c] || !rhst[c] || !ctlt[c]) return fail(FCD_ENOMEM, "device allocation failed");
            CK(cudaMemsetAsync(tA[c], 0, ps * sizeof(double), stream));
            CK(cudaMemsetAsync(tB[c], 0, ps * sizeof(double), stream));
            CK(cudaMemsetAsync(rhst[c], 0, ps * sizeof(double), stream));
            CK(cudaMemsetAsync(ctlt[c], 0, sizeof(MgCtl), stream));
            CK(cudaStreamCreateWithFlags(&side[c], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&join[c], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        CK(cudaMallocHost(&h_tan, sizeof(TanOut)));
        CK(cudaMemsetAsync(psiT, 0, (1 + NT) * ps * sizeof(double), stream));
        CK(cudaMemsetAsync(dpsiP, 0, NT * ps * sizeof(double), stream));
        CK(cudaStreamSynchronize(stream));
        PT = tangent_phys(&prm, make_phys<double>(&prm, D, pitch));
        fcd_status st = Engine<double>::init();  // the initial solve runs the tangent solves too
        if (st != FCD_OK) return st;
        CK(cudaMemcpyAsync(dpsiP, psiT + ps, NT * ps * sizeof(double), cudaMemcpyDeviceToDevice, stream));
        CK(cudaStreamSynchronize(stream));
        return FCD_OK;
    }

    // Hierarchies of the tangent solves, made once the primal one exists.
    fcd_status make_tangent_mg() {
        for (int c = 0; c < NT && !mgt[c]; c++) {
            // every tangent solve of a step has the primal solve's k, and the
            // primal solve forms the lattice coefficients first: share them
            mgt[c] = mg_create<double>(prm.nx, prm.ny, pitch, k, tA[c], tB[c], ctlt[c], alloc,
                                       release, user, err, sizeof err, 0, mg);
            if (!mgt[c]) return FCD_ENOMEM;
            mg_set_rhs<double>(mgt[c], rhst[c]);
        }
        return FCD_OK;
    }

    // The NT tangent potentials for the current phase fields (derivative
    // planes of k already formed): L(k) dpsi_c = rhs_c on hierarchy c. Graph
    // capture: NT parallel branches forked from s; host loop: one after the
    // other on s. extrap: start from 2 dpsi(t) - dpsi(t-1).
    fcd_status tangent_solves(bool extrap, double tol, int max_iter, cudaStream_t s, bool capture) {
        if (!magnetic()) return FCD_OK;  // no field: every derivative of psi' stays 0
        if (make_tangent_mg() != FCD_OK) return FCD_ENOMEM;
        if (capture) CK(cudaEventRecord(fork, s));
        for (int c = 0; c < NT; c++) {
            cudaStream_t sc = s;
            if (capture) {
                sc = side[c];
                CK(cudaStreamWaitEvent(sc, fork, 0));
            }
            double *dk = k + (c + 1) * ps, *dpsi = psiT + (c + 1) * ps, *prev = dpsiP + c * ps;
            mg_tangent_rhs(mg, dk, P.H0c, P.H0s, PT.H0c.d[c], PT.H0s.d[c], rhst[c], rmax + c, sc);
            if (extrap) mg_psi_io(mgt[c], 2, dpsi, prev, sc);
            else mg_psi_io(mgt[c], 1, dpsi, nullptr, sc);
            mg_reset_scaled(ctlt[c], rmax + c, tol, max_iter, sc);
            fcd_status st;
            if (capture) {
                mg_presmooth<double>(mgt[c], P.H0c, P.H0s, sc);
                st = capture_mg_loop(sc, mgt[c]);
            } else {
                st = host_mg_loop(sc, mgt[c], ctlt[c]);
            }
            if (st != FCD_OK) return st;
            mg_psi_io(mgt[c], 0, dpsi, nullptr, sc);
            CK(cudaGetLastError());
            if (capture) {
                CK(cudaEventRecord(join[c], sc));
                CK(cudaStreamWaitEvent(s, join[c], 0));
            }
        }
        return FCD_OK;
    }

    // kernels of one step outside the multigrid cycles (those are counted on
    // the device): two phase kernels, the primal solve's coefficient kernel and
    // per direction the right-hand side, two copies and the reset, the
    // potential copy and the collision
    long step_kernels() const {
        return 2 + (magnetic() ? 4 * NT + 1 : 0) + 2 + (prm.open_x ? 1 : 0);
    }

    long launches() const override {
        long n = Engine<double>::launches();
        for (int c = 0; c < NT; c++) {
            if (!mgt[c]) continue;
            MgCtl q;
            if (cudaMemcpy(&q, ctlt[c], sizeof q, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            n += (long)q.cycles_launched + (long)q.total_cycles * mg_kernels_per_cycle(mgt[c]) +
                 (long)q.smooth_cycles + 2 * (long)q.twogrid_cycles + (long)q.dispatches;
        }
        return n;
    }

    fcd_status solve(double tol, int max_iter, int *iters, double *resid) override {
        if (!(tol > 0)) tol = prm.mag_tol;
        if (max_iter <= 0) max_iter = prm.mag_max_iter;
        const fcd_status st = Engine<double>::solve(tol, max_iter, iters, resid);
        if (st != FCD_OK && st != FCD_ENOCONV) return st;
        launch_tangent_phase(P, static_cast<const double *>(g[cur]), phi1, phi2, k, stream);
        host_kernels += 1 + (magnetic() ? 4 * NT : 0);  // the tangent phase; per direction 4
        const fcd_status st2 = tangent_solves(false, tol, max_iter, stream, false);
        return st2 != FCD_OK ? st2 : st;
    }

    // One tangent step on s (host loop, or captured when capture is set).
    fcd_status enqueue_tangent_step(int c, bool store_macro, cudaStream_t s, bool capture) {
        enqueue_pre(c, s);
        launch_tangent_phase(P, static_cast<const double *>(g[c]), phi1, phi2, k, s);
        if (magnetic()) {
            fcd_status st;
            if (capture) {
                mg_presmooth<double>(mg, P.H0c, P.H0s, s);
                st = capture_mg_loop(s);
            } else {
                st = host_mg_loop(s);
            }
            if (st != FCD_OK) return st;
            st = tangent_solves(true, prm.mag_tol, prm.mag_max_iter, s, capture);
            if (st != FCD_OK) return st;
        }
        mg_psi_io(mg, 0, psiT, nullptr, s);
        LbmArgs<double, DualT> a;
        a.P = PT;
        a.f_src = f[c];
        a.g_src = g[c];
        a.f_dst = f[c ^ 1];
        a.g_dst = g[c ^ 1];
        a.phi1 = phi1;
        a.phi2 = phi2;
        a.psi0 = psiT;
        a.psi1 = psiT;
        a.ctl = ctl;
        a.macro = store_macro ? macro : nullptr;
        a.brk = brk;
        a.step = d_step;
        a.open_x = prm.open_x;
        launch_collide_tangent(a, s);
        if (prm.open_x)
            launch_open_bc_tangent(P, f[c], g[c], f[c ^ 1], g[c ^ 1], prm.u_max, D.u_avg, s);
        CK(cudaGetLastError());
        return FCD_OK;
    }

    fcd_status capture_step(int c, int sm, cudaStream_t s) override {
        return enqueue_tangent_step(c, sm != 0, s, true);
    }

    fcd_status do_step(long n) override {
        if (n < 0) return fail(FCD_EINVAL, "negative step count");
        cudaStream_t s = stream;
        for (long i = 0; i < n; i++) {
            const int sm = i == n - 1 ? 1 : 0;
            if (use_graph) {
                if (!gexec[cur][sm]) {
                    const fcd_status st = build_graph(cur, sm);
                    if (st != FCD_OK) return st;
                }
                CK(cudaGraphLaunch(gexec[cur][sm], s));
            } else {
                const fcd_status st = enqueue_tangent_step(cur, sm != 0, s, false);
                if (st != FCD_OK) return st;
            }
            host_kernels += step_kernels();
            cur ^= 1;
            step++;
        }
        CK(cudaGetLastError());
        return FCD_OK;
    }

    fcd_status tangent_observe(fcd_tangent_obs *o) {
        fcd_obs po;
        const fcd_status st = observe(&po);  // primal observables (and the seam column)
        if (st != FCD_OK && st != FCD_ENOCONV) return st;
        cudaStream_t s = stream;
        launch_tangent_obs(P, static_cast<const double *>(g[cur]), obs_out, tobs, tan_out, s);
        host_kernels += 1;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h_tan, tan_out, sizeof(TanOut), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        int nonconv = 0;
        for (int c = 0; c < NT; c++) {
            if (!mgt[c]) continue;
            CK(cudaMemcpy(h_ctl, ctlt[c], sizeof(MgCtl), cudaMemcpyDeviceToHost));
            nonconv += h_ctl->nonconv_count;
        }
        std::memset(o, 0, sizeof *o);
        o->step = step;
        o->T_o = h_tan->T_o;
        o->overlap = h_tan->overlap;
        o->lx_o = h_tan->lx;
        o->ly_o = h_tan->ly;
        for (int c = 0; c < NT; c++) {
            o->dT_o[c] = h_tan->dT_o[c];
            o->doverlap[c] = h_tan->doverlap[c];
            o->dlx_o[c] = h_tan->dlx[c];
            o->dly_o[c] = h_tan->dly[c];
        }
        if (nonconv > reported_tangent_nonconv) {
            reported_tangent_nonconv = nonconv;
            return fail(FCD_ENOCONV, "a tangent potential solve stopped at the cycle cap");
        }
        return st;
    }

    size_t state_bytes() const override { return 0; }
    fcd_status get_state(void *, size_t) override {
        return fail(FCD_ESTATE, "state snapshots are not available for tangent contexts");
    }
    fcd_status set_state(const void *, size_t) override {
        return fail(FCD_ESTATE, "state snapshots are not available for tangent contexts");
    }
    fcd_status set_pops(const double *, const double *, const double *, long) override {
        return fail(FCD_ESTATE, "population import is not available for tangent contexts");
    }
    fcd_status set_profiling(int) override {
        return fail(FCD_ESTATE, "step profiling is not available for tangent contexts");
    }
};

// ---------------------------------------------------------------- adjoint
// FP64 periodic context that keeps a checkpoint of its state every K steps
// from step 0 and runs the discrete adjoint of J = wT T_o + wO overlap at its
// current step back to step 0. Two-level checkpointing: the forward pass stores
// one state per K steps; the reverse sweep takes the segments last first,
// recomputes each segment's K states from its checkpoint into slots (every
// step once more, so the sweep costs one extra forward pass) and runs the
// adjoint steps backwards through them. The recomputed states are bitwise the
// ones of the forward pass (same kernels on the same data).
struct AdjointEngine : Engine<double> {
    int K = 1;
    Phys<DualT> PT;                 // constants with their derivatives along theta
    std::vector<double *> ckpt;     // checkpoint c: the state at step c K
    size_t ck_doubles = 0;          // f 9, g 18, psiA, psiB, psiP planes; cur, brk, step
    double *fin = nullptr;          // the final state during a sweep
    double *seg = nullptr;          // K slots: f 9, g 18, psi' 1 plane
    long long slot_stride = 0;
    std::vector<long> slot_step;    // the step whose state slot j holds (-1: none)
    double *ab[2] = {nullptr, nullptr};  // adjoint states (27 planes each)
    double *sb = nullptr, *pb = nullptr, *rhs = nullptr, *lamA = nullptr, *lamB = nullptr;
    double *lamS = nullptr, *lamP = nullptr;  // the last two adjoint potentials (extrapolation)
    double *pacc = nullptr, *hacc = nullptr;
    double *keep = nullptr;  // open channel: the outlet's share of the adjoint before a step
    int nblk_c = 0, nblk_k = 0;
    MgCtl *ctla = nullptr;
    MgHost<double> *mga = nullptr;
    unsigned long long *rmax = nullptr;
    int *d_slot = nullptr;
    void *seed_scr = nullptr;
    AdjOut *adj_out = nullptr, *h_adj = nullptr;
    cudaGraph_t agraph[2] = {nullptr, nullptr};
    cudaGraphExec_t aexec[2] = {nullptr, nullptr};
    int reported_adj_nonconv = 0;

    ~AdjointEngine() override {
        if (stream) cudaStreamSynchronize(stream);
        cudaDeviceSynchronize();
        for (int c = 0; c < 2; c++) {
            if (aexec[c]) cudaGraphExecDestroy(aexec[c]);
            if (agraph[c]) cudaGraphDestroy(agraph[c]);
        }
        if (mga) mg_destroy(mga);
        if (h_adj) cudaFreeHost(h_adj);
    }

    fcd_status init() override {
        const fcd_status st = Engine<double>::init();
        if (st != FCD_OK) return st;
        PT = tangent_phys(&prm, P);
        ck_doubles = 30 * (size_t)ps + 4;
        slot_stride = 28 * ps;
        nblk_c = adj_collide_blocks(prm.nx, prm.ny);
        nblk_k = adj_kbar_blocks(prm.nx, prm.ny);
        for (int c = 0; c < 2; c++) ab[c] = dalloc(27 * ps * sizeof(double));
        sb = dalloc(13 * ps * sizeof(double));
        pb = dalloc(2 * ps * sizeof(double));
        rhs = dalloc(ps * sizeof(double));
        lamA = dalloc(ps * sizeof(double));
        lamB = dalloc(ps * sizeof(double));
        lamS = dalloc(ps * sizeof(double));
        lamP = dalloc(ps * sizeof(double));
        pacc = dalloc((size_t)nblk_c * NPB * sizeof(double));
        hacc = dalloc((size_t)nblk_k * 2 * sizeof(double));
        ctla = reinterpret_cast<MgCtl *>(dalloc(sizeof(MgCtl)));
        rmax = reinterpret_cast<unsigned long long *>(dalloc(sizeof(unsigned long long)));
        d_slot = reinterpret_cast<int *>(dalloc(sizeof(int)));
        seed_scr = dalloc(adj_seed_scratch_bytes(prm.nx));
        adj_out = reinterpret_cast<AdjOut *>(dalloc(sizeof(AdjOut)));
        if (prm.open_x) {
            keep = dalloc((size_t)prm.ny * 27 * sizeof(double));
            if (!keep) return fail(FCD_ENOMEM, "device allocation failed");
        }
        for (void *q : {(void *)ab[0], (void *)ab[1], (void *)sb, (void *)pb, (void *)rhs, (void *)lamA,
                        (void *)lamB, (void *)lamS, (void *)lamP, (void *)pacc, (void *)hacc,
                        (void *)ctla, (void *)rmax,
                        (void *)d_slot, seed_scr, (void *)adj_out})
            if (!q) return fail(FCD_ENOMEM, "device allocation failed");
        // padding columns stay zero in every adjoint plane
        for (int c = 0; c < 2; c++) CK(cudaMemsetAsync(ab[c], 0, 27 * ps * sizeof(double), stream));
        CK(cudaMemsetAsync(sb, 0, 13 * ps * sizeof(double), stream));
        CK(cudaMemsetAsync(pb, 0, 2 * ps * sizeof(double), stream));
        CK(cudaMemsetAsync(rhs, 0, ps * sizeof(double), stream));
        CK(cudaMallocHost(&h_adj, sizeof(AdjOut)));
        return push_checkpoint();
    }

    fcd_status save(double *dst) {
        cudaStream_t s = stream;
        CK(cudaMemcpyAsync(dst, f[cur], 9 * ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst + 9 * ps, g[cur], 18 * ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst + 27 * ps, psiA, ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst + 28 * ps, psiB, ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst + 29 * ps, psiP, ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        double *tail = dst + 30 * ps;
        CK(cudaMemcpyAsync(tail, &ctl->cur, sizeof(int), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(tail + 1, brk, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(tail + 2, d_step, sizeof(long long), cudaMemcpyDeviceToDevice, s));
        return FCD_OK;
    }

    fcd_status restore(const double *src, long at_step) {
        cudaStream_t s = stream;
        CK(cudaMemcpyAsync(f[cur], src, 9 * ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(g[cur], src + 9 * ps, 18 * ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(psiA, src + 27 * ps, ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(psiB, src + 28 * ps, ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(psiP, src + 29 * ps, ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        const double *tail = src + 30 * ps;
        CK(cudaMemcpyAsync(&ctl->cur, tail, sizeof(int), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(brk, tail + 1, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(d_step, tail + 2, sizeof(long long), cudaMemcpyDeviceToDevice, s));
        step = at_step;
        return FCD_OK;
    }

    fcd_status push_checkpoint() {
        double *c = dalloc(ck_doubles * sizeof(double));
        if (!c) return fail(FCD_ENOMEM, "checkpoint allocation failed at step %ld", step);
        ckpt.push_back(c);
        return save(c);
    }

    fcd_status alloc_slots() {
        if (seg) return FCD_OK;
        seg = dalloc((size_t)K * slot_stride * sizeof(double));
        if (!seg)
            return fail(FCD_ENOMEM, "no room for %d recomputed states (%.2f GB); use a smaller "
                        "checkpoint interval", K, K * slot_stride * 8.0 / 1e9);
        slot_step.assign(K, -1);
        return FCD_OK;
    }

    // One forward step that also keeps its state in slot (step mod K): the
    // populations before the step and the potential the step solved for.
    fcd_status record_step(int sm) {
        cudaStream_t s = stream;
        const int j = (int)(step % K);
        double *sl = seg + j * slot_stride;
        const long at = step;
        CK(cudaMemcpyAsync(sl, f[cur], 9 * ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(sl + 9 * ps, g[cur], 18 * ps * sizeof(double), cudaMemcpyDeviceToDevice, s));
        const fcd_status st = one_step(sm);
        if (st != FCD_OK) return st;
        mg_psi_io(mg, 0, sl + 27 * ps, nullptr, s);
        host_kernels += 1;
        slot_step[j] = at;
        return FCD_OK;
    }

    // Forward steps with a checkpoint every K steps; the states of the
    // current segment stay in the slots, so a sweep that starts in this
    // segment need not recompute it.
    fcd_status do_step(long n) override {
        if (n < 0) return fail(FCD_EINVAL, "negative step count");
        fcd_status st = alloc_slots();
        if (st != FCD_OK) return st;
        for (long i = 0; i < n; i++) {
            if (step % K == 0 && (size_t)(step / K) == ckpt.size()) {
                st = push_checkpoint();
                if (st != FCD_OK) return st;
            }
            st = record_step(i == n - 1 ? 1 : 0);
            if (st != FCD_OK) return st;
        }
        CK(cudaGetLastError());
        return FCD_OK;
    }

    // One adjoint step on s: reads the slot *d_slot and ab[c], writes ab[c ^ 1].
    fcd_status enqueue_adj_step(int c, cudaStream_t s, bool capture) {
        // open channel: the boundary kernel ran last in the step, so its transpose runs first
        if (prm.open_x) launch_adj_open_bc(P, ab[c], keep, D.u_avg, s);
        launch_adj_phase(P, seg, d_slot, slot_stride, phi1, phi2, k, s);
        AdjArgs A;
        A.P = P;
        A.seg = seg;
        A.slot = d_slot;
        A.stride = slot_stride;
        A.phi1 = phi1;
        A.phi2 = phi2;
        A.ab_src = ab[c];
        A.ab_dst = ab[c ^ 1];
        A.sb = sb;
        A.pacc = pacc;
        launch_adj_collide(A, prm.open_x, s);
        if (prm.open_x) launch_adj_open_add(P, keep, ab[c ^ 1], s);
        launch_adj_gather(P, sb, phi1, phi2, pb, rhs, rmax, prm.open_x, s);
        if (magnetic()) {
            // initial guess 2 lam(n+1) - lam(n+2), as the plain solve extrapolates psi'
            mg_psi_io(mga, 2, lamS, lamP, s);
            mg_reset_scaled(ctla, rmax, prm.mag_tol, prm.mag_max_iter, s);
            mg_presmooth<double>(mga, P.H0c, P.H0s, s);
            const fcd_status st = capture ? capture_mg_loop(s, mga) : host_mg_loop(s, mga, ctla);
            if (st != FCD_OK) return st;
            mg_psi_io(mga, 0, lamS, nullptr, s);
        }
        AdjKArgs B;
        B.P = P;
        B.seg = seg;
        B.slot = d_slot;
        B.stride = slot_stride;
        B.k = k;
        B.phi1 = phi1;
        B.phi2 = phi2;
        B.pb = pb;
        B.lamA = lamA;
        B.lamB = lamB;
        B.ctl = magnetic() ? ctla : nullptr;
        B.ab = ab[c ^ 1];
        B.hacc = hacc;
        launch_adj_kbar(B, s);
        launch_dec_slot(d_slot, s);
        CK(cudaGetLastError());
        return FCD_OK;
    }
    // kernels of one adjoint step outside the multigrid cycles
    long adj_step_kernels() const { return 6 + (magnetic() ? 5 : 0) + (prm.open_x ? 2 : 0); }

    fcd_status adj_step(int c) {
        cudaStream_t s = stream;
        if (use_graph) {
            if (!aexec[c]) {
                CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
                const fcd_status st = enqueue_adj_step(c, cap, true);
                cudaGraph_t gr = nullptr;
                const cudaError_t e = cudaStreamEndCapture(cap, &gr);
                if (st != FCD_OK) {
                    if (gr) cudaGraphDestroy(gr);
                    return st;
                }
                CK(e);
                agraph[c] = gr;
                CK(cudaGraphInstantiate(&aexec[c], agraph[c], 0));
            }
            CK(cudaGraphLaunch(aexec[c], s));
        } else {
            const fcd_status st = enqueue_adj_step(c, s, false);
            if (st != FCD_OK) return st;
        }
        host_kernels += adj_step_kernels();
        return FCD_OK;
    }

    // seed_f, seed_g (state seed, exchange layout, host or device; either may be
    // null): dJ/d(f, g at the final step) given by the caller instead of the
    // built-in J = wT T_o + wO overlap (then wT = wO = 0).
    // The segments last first: recompute a segment's states into the slots
    // unless the slots already hold them, then its adjoint steps backwards.
    // ca: the adjoint buffer that holds the current adjoint (updated).
    fcd_status sweep(long N, int &ca, long &recomputed) {
        cudaStream_t s = stream;
        const long nseg = (N + K - 1) / K;
        for (long q = nseg - 1; q >= 0; q--) {
            const long n0 = q * K, n1 = std::min(N, n0 + K);
            const int len = (int)(n1 - n0);
            bool have = true;  // the segment's states already in the slots?
            for (int j = 0; j < len && have; j++) have = slot_step[j] == n0 + j;
            if (!have) {
                fcd_status st = restore(ckpt[q], n0);
                if (st != FCD_OK) return st;
                for (int j = 0; j < len; j++) {
                    st = record_step(0);
                    if (st != FCD_OK) return st;
                }
                recomputed += len;
            }
            launch_set_slot(d_slot, len - 1, s);
            host_kernels += 1;
            for (int j = len - 1; j >= 0; j--) {
                const fcd_status st = adj_step(ca);
                if (st != FCD_OK) return st;
                ca ^= 1;
            }
        }
        return FCD_OK;
    }

    fcd_status gradient(double wT, double wO, fcd_adjoint_out *o, double *df0, double *dg0,
                        const double *seed_f = nullptr, const double *seed_g = nullptr) {
        const long N = step;
        const bool state_seed = seed_f || seed_g;
        cudaStream_t s = stream;
        if (!mga && magnetic()) {
            mga = mg_create<double>(prm.nx, prm.ny, pitch, k, lamA, lamB, ctla, alloc, release, user, err,
                                    sizeof err);
            if (!mga) return FCD_ENOMEM;
            mg_set_rhs<double>(mga, rhs);
        }
        if (N > 0) {
            const fcd_status sa = alloc_slots();
            if (sa != FCD_OK) return sa;
        }
        if (!fin) {
            fin = dalloc(ck_doubles * sizeof(double));
            if (!fin) return fail(FCD_ENOMEM, "device allocation failed");
        }
        // J at the final state and its adjoint there
        fcd_obs po;
        fcd_status st = observe(&po);  // plain observables (seam column for l_x)
        if (st != FCD_OK && st != FCD_ENOCONV) return st;
        launch_phase<double>(MODE_FP64, P, g[cur], phi1, phi2, nullptr,
                             PhaseCtl{nullptr, 0, 0.0, 0, nullptr, 0, nullptr, nullptr, nullptr}, s);
        launch_adj_seed(P, phi1, phi2, obs_out, wT, wO, seed_scr, pb, ab[0], adj_out, s);
        host_kernels += 3;
        CK(cudaMemcpyAsync(h_adj, adj_out, sizeof(AdjOut), cudaMemcpyDeviceToHost, s));
        if (state_seed) {  // the caller's dJ/d(f_N, g_N) replaces the seed's planes
            const size_t Nn = (size_t)prm.nx * prm.ny;
            double *stg = staging(27 * Nn);
            if (!stg) return fail(FCD_ENOMEM, "staging allocation failed");
            cudaError_t e = cudaSuccess;
            if (seed_f) e = cudaMemcpyAsync(stg, seed_f, 9 * Nn * sizeof(double), cudaMemcpyDefault, s);
            if (e == cudaSuccess && seed_g)
                e = cudaMemcpyAsync(stg + 9 * Nn, seed_g, 18 * Nn * sizeof(double), cudaMemcpyDefault, s);
            if (e == cudaSuccess) {
                launch_import<double>(MODE_FP64, P, seed_f ? stg : nullptr, seed_g ? stg + 9 * Nn : nullptr,
                                      ab[0], ab[0] + 9 * ps, s);
                host_kernels += 1;
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            cudaFree(stg);
            if (e != cudaSuccess) return fail(FCD_ECUDA, "adjoint seed import: %s", cudaGetErrorString(e));
        }
        if (wT == 0.0 && wO == 0.0 && !df0 && !dg0 && !state_seed) {  // J = 0: values only, zero gradient
            CK(cudaStreamSynchronize(s));
            std::memset(o, 0, sizeof *o);
            o->step = N;
            o->T_o = h_adj->T_o;
            o->overlap = h_adj->overlap;
            return FCD_OK;
        }
        CK(cudaMemsetAsync(pacc, 0, (size_t)nblk_c * NPB * sizeof(double), s));
        CK(cudaMemsetAsync(hacc, 0, (size_t)nblk_k * 2 * sizeof(double), s));
        CK(cudaMemsetAsync(lamA, 0, ps * sizeof(double), s));
        CK(cudaMemsetAsync(lamB, 0, ps * sizeof(double), s));
        CK(cudaMemsetAsync(lamS, 0, ps * sizeof(double), s));
        CK(cudaMemsetAsync(lamP, 0, ps * sizeof(double), s));
        CK(cudaMemsetAsync(ctla, 0, sizeof(MgCtl), s));
        st = save(fin);
        if (st != FCD_OK) return st;
        int ca = 0;
        long recomputed = 0;
        st = sweep(N, ca, recomputed);
        // back to the final state whether or not the sweep completed
        const fcd_status rs = restore(fin, N);
        if (st != FCD_OK) {
            if (rs == FCD_OK) cudaStreamSynchronize(s);
            return st;
        }
        if (rs != FCD_OK) return rs;
        // constants' adjoints, summed block by block in a fixed order
        std::vector<double> hp((size_t)nblk_c * NPB), hh((size_t)nblk_k * 2);
        CK(cudaMemcpyAsync(hp.data(), pacc, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hh.data(), hacc, hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double pbar[NPB] = {0.0};
        for (int b = 0; b < nblk_c; b++)
            for (int q = 0; q < NPB; q++) pbar[q] += hp[(size_t)b * NPB + q];
        for (int b = 0; b < nblk_k; b++) {
            pbar[PB_H0C] += hh[2 * (size_t)b];
            pbar[PB_H0S] += hh[2 * (size_t)b + 1];
        }
        const DualT *dp[NPB] = {&PT.s12, &PT.s13, &PT.s23, &PT.gam[0], &PT.gam[1], &PT.gam[2],
                                &PT.eta, &PT.lap_coef[0], &PT.lap_coef[1], &PT.lap_coef[2],
                                &PT.H0c, &PT.H0s, &PT.tau[0], &PT.tau[1], &PT.tau[2]};
        std::memset(o, 0, sizeof *o);
        o->step = N;
        o->T_o = h_adj->T_o;
        o->overlap = h_adj->overlap;
        o->J = state_seed ? 0.0 : wT * h_adj->T_o + wO * h_adj->overlap;
        o->recomputed_steps = recomputed;
        for (int c = 0; c < NT; c++) {
            double gsum = 0.0;
            for (int q = 0; q < NPB; q++) gsum += pbar[q] * dp[q]->d[c];
            o->grad[c] = gsum;
        }
        if (df0 || dg0) {
            const size_t Nn = (size_t)prm.nx * prm.ny;
            double *stg = staging(27 * Nn);
            if (!stg) return fail(FCD_ENOMEM, "staging allocation failed");
            launch_export<double>(MODE_FP64, P, ab[ca], ab[ca] + 9 * ps, stg, stg + 9 * Nn, s);
            host_kernels += 1;
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess && df0) e = cudaMemcpyAsync(df0, stg, 9 * Nn * sizeof(double), cudaMemcpyDefault, s);
            if (e == cudaSuccess && dg0) e = cudaMemcpyAsync(dg0, stg + 9 * Nn, 18 * Nn * sizeof(double), cudaMemcpyDefault, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            cudaFree(stg);
            if (e != cudaSuccess) return fail(FCD_ECUDA, "adjoint export: %s", cudaGetErrorString(e));
        }
        if (magnetic()) {
            CK(cudaMemcpy(h_ctl, ctla, sizeof(MgCtl), cudaMemcpyDeviceToHost));
            o->solve_cycles = h_ctl->total_cycles + h_ctl->twogrid_cycles + h_ctl->smooth_cycles;
            o->capped_solves = h_ctl->nonconv_count;  // the control block is cleared per sweep
            if (o->capped_solves > 0)
                return fail(FCD_ENOCONV, "%ld adjoint potential solves stopped at the cycle cap",
                            o->capped_solves);
        }
        return FCD_OK;
    }

    long launches() const override {
        long n = Engine<double>::launches();
        if (mga) {
            MgCtl q;
            if (cudaMemcpy(&q, ctla, sizeof q, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            n += (long)q.cycles_launched + (long)q.total_cycles * mg_kernels_per_cycle(mga) +
                 (long)q.smooth_cycles + 2 * (long)q.twogrid_cycles + (long)q.dispatches;
        }
        return n;
    }

    size_t state_bytes() const override { return 0; }
    fcd_status get_state(void *, size_t) override {
        return fail(FCD_ESTATE, "state snapshots are not available for adjoint contexts");
    }
    fcd_status set_state(const void *, size_t) override {
        return fail(FCD_ESTATE, "state snapshots are not available for adjoint contexts");
    }
    fcd_status set_pops(const double *, const double *, const double *, long) override {
        return fail(FCD_ESTATE, "population import is not available for adjoint contexts");
    }
};

// ---------------------------------------------------------------- batch view
namespace fcd {
bool engine_view(fcd_ctx *c, EngineView *v) {
    auto *e = dynamic_cast<Engine<float> *>(c);
    if (!e || e->prm.open_x) return false;
    v->mode = e->mode;
    v->magnetic = e->magnetic() ? 1 : 0;
    v->cur = e->cur;
    v->P = e->P;
    for (int b = 0; b < 2; b++) {
        v->f[b] = e->f[b];
        v->g[b] = e->g[b];
    }
    v->phi1 = e->phi1;
    v->phi2 = e->phi2;
    v->k = e->k;
    v->psiA = e->psiA;
    v->psiB = e->psiB;
    v->psiP = e->psiP;
    v->macro = e->macro;
    v->ctl = e->ctl;
    v->mg = e->mg;
    v->brk = e->brk;
    v->unst = e->unst;
    v->d_step = e->d_step;
    v->tolH0 = e->prm.mag_tol * e->D.H0;
    v->max_iter = e->prm.mag_max_iter;
    v->comp = e->comp;
    return true;
}

fcd_status engine_step1(fcd_ctx *c, int store_macro) {
    // plain contexts only: the tangent and adjoint contexts keep their own step
    if (typeid(*c) == typeid(Engine<float>)) return static_cast<Engine<float> *>(c)->one_step(store_macro);
    if (typeid(*c) == typeid(Engine<double>)) return static_cast<Engine<double> *>(c)->one_step(store_macro);
    return fcd_step(c, 1);
}

void engine_advance(fcd_ctx *c, long steps) {
    auto *e = dynamic_cast<Engine<float> *>(c);
    if (!e) return;
    if (steps & 1) e->cur ^= 1;
    e->step += steps;
}
}  // namespace fcd

// ---------------------------------------------------------------- C ABI
static thread_local char g_last[512];  // reason of the last failed fcd_create on this thread

extern "C" {

fcd_status fcd_create(const fcd_params *params, fcd_ctx **out) {
    if (!out) return FCD_EINVAL;
    *out = nullptr;
    if (!params) return FCD_EINVAL;
    Derived d;
    std::memset(&d, 0, sizeof d);
    const char *why = derive(params, &d);
    if (why) {
        snprintf(g_last, sizeof g_last, "fcd_create: %s", why);
        return FCD_EINVAL;
    }
    fcd_ctx *c = nullptr;
    if (params->precision == FCD_FP64) {
        auto *e = new (std::nothrow) Engine<double>();
        if (e) { e->alloc = g_alloc ? g_alloc : default_alloc; e->release = g_free ? g_free : default_free; e->user = g_alloc ? g_user : nullptr; }
        c = e;
    } else {
        auto *e = new (std::nothrow) Engine<float>();
        if (e) { e->alloc = g_alloc ? g_alloc : default_alloc; e->release = g_free ? g_free : default_free; e->user = g_alloc ? g_user : nullptr; }
        c = e;
    }
    if (!c) return FCD_ENOMEM;
    c->prm = *params;
    c->D = d;
    fcd_status st = c->init();
    if (st != FCD_OK) {
        snprintf(g_last, sizeof g_last, "%s", c->err);
        delete c;
        return st;
    }
    *out = c;
    return FCD_OK;
}

fcd_status fcd_create_tangent(const fcd_params *params, fcd_ctx **out) {
    if (!out) return FCD_EINVAL;
    *out = nullptr;
    if (!params) return FCD_EINVAL;
    fcd_params p = *params;
    p.precision = FCD_FP64;
    Derived d;
    std::memset(&d, 0, sizeof d);
    const char *why = derive(&p, &d);
    if (!why && 18ll * (1 + NT) * ((p.nx + 31) / 32 * 32) * p.ny > (1ll << 31) - 1)
        why = "lattice too large for the tangent copies (90 planes within 2^31 elements)";
    if (!why && p.ferro_phase != 0 && !(p.Bo_m > 0))
        why = "the Bo_m direction needs Bo_m > 0 (H0 ~ sqrt(Bo_m))";
    if (why) {
        snprintf(g_last, sizeof g_last, "fcd_create_tangent: %s", why);
        return FCD_EINVAL;
    }
    auto *e = new (std::nothrow) TangentEngine();
    if (!e) return FCD_ENOMEM;
    e->alloc = g_alloc ? g_alloc : default_alloc;
    e->release = g_free ? g_free : default_free;
    e->user = g_alloc ? g_user : nullptr;
    e->prm = p;
    e->D = d;
    const fcd_status st = e->init();
    if (st != FCD_OK) {
        snprintf(g_last, sizeof g_last, "%s", e->err);
        delete e;
        return st;
    }
    *out = e;
    return FCD_OK;
}

fcd_status fcd_tangent_observables(fcd_ctx *c, fcd_tangent_obs *o) {
    if (!c || !o) return FCD_EINVAL;
    auto *e = dynamic_cast<TangentEngine *>(c);
    if (!e) return c->fail(FCD_EINVAL, "not a tangent context");
    return e->tangent_observe(o);
}

fcd_status fcd_create_adjoint(const fcd_params *params, int checkpoint_interval, fcd_ctx **out) {
    if (!out) return FCD_EINVAL;
    *out = nullptr;
    if (!params) return FCD_EINVAL;
    fcd_params p = *params;
    p.precision = FCD_FP64;
    Derived d;
    std::memset(&d, 0, sizeof d);
    const char *why = derive(&p, &d);
    if (!why && checkpoint_interval < 1) why = "checkpoint_interval must be >= 1";
    if (!why && p.ferro_phase != 0 && !(p.Bo_m > 0))
        why = "the Bo_m direction needs Bo_m > 0 (H0 ~ sqrt(Bo_m))";
    if (why) {
        snprintf(g_last, sizeof g_last, "fcd_create_adjoint: %s", why);
        return FCD_EINVAL;
    }
    auto *e = new (std::nothrow) AdjointEngine();
    if (!e) return FCD_ENOMEM;
    e->alloc = g_alloc ? g_alloc : default_alloc;
    e->release = g_free ? g_free : default_free;
    e->user = g_alloc ? g_user : nullptr;
    e->prm = p;
    e->D = d;
    e->K = checkpoint_interval;
    const fcd_status st = e->init();
    if (st != FCD_OK) {
        snprintf(g_last, sizeof g_last, "%s", e->err);
        delete e;
        return st;
    }
    *out = e;
    return FCD_OK;
}

fcd_status fcd_adjoint_gradient(fcd_ctx *c, double w_T, double w_overlap, fcd_adjoint_out *o,
                                double *df0, double *dg0) {
    if (!c || !o) return FCD_EINVAL;
    auto *e = dynamic_cast<AdjointEngine *>(c);
    if (!e) return c->fail(FCD_EINVAL, "not an adjoint context");
    NvtxScope r("fcd_adjoint_gradient");
    return e->gradient(w_T, w_overlap, o, df0, dg0);
}

fcd_status fcd_adjoint_gradient_state(fcd_ctx *c, const double *seed_f, const double *seed_g,
                                      fcd_adjoint_out *o, double *df0, double *dg0) {
    if (!c || !o) return FCD_EINVAL;
    auto *e = dynamic_cast<AdjointEngine *>(c);
    if (!e) return c->fail(FCD_EINVAL, "not an adjoint context");
    if (!seed_f && !seed_g) return c->fail(FCD_EINVAL, "no seed given");
    return e->gradient(0.0, 0.0, o, df0, dg0, seed_f, seed_g);
}

fcd_status fcd_set_stream(fcd_ctx *c, void *stream) {
    if (!c) return FCD_EINVAL;
    c->stream = static_cast<cudaStream_t>(stream);
    return FCD_OK;
}

fcd_status fcd_step(fcd_ctx *c, long n) {
    NvtxScope r("fcd_step");
    return c ? c->do_step(n) : FCD_EINVAL;
}

fcd_status fcd_solve_magnetic(fcd_ctx *c, double tol, int max_iter, int *iters, double *resid) {
    NvtxScope r("fcd_solve_magnetic");
    return c ? c->solve(tol, max_iter, iters, resid) : FCD_EINVAL;
}

fcd_status fcd_observables(fcd_ctx *c, fcd_obs *o) {
    if (!c || !o) return FCD_EINVAL;
    NvtxScope r("fcd_observables");
    return c->observe(o);
}

fcd_status fcd_get_field(fcd_ctx *c, int which, double *dst, size_t n) {
    return c ? c->field(which, dst, n) : FCD_EINVAL;
}

fcd_status fcd_get_populations(fcd_ctx *c, double *f, double *g, double *psi) {
    return c ? c->get_pops(f, g, psi) : FCD_EINVAL;
}

fcd_status fcd_set_populations(fcd_ctx *c, const double *f, const double *g, const double *psi,
                               long step) {
    return c ? c->set_pops(f, g, psi, step) : FCD_EINVAL;
}

size_t fcd_state_bytes(const fcd_ctx *c) { return c ? c->state_bytes() : 0; }

fcd_status fcd_get_state(fcd_ctx *c, void *dst, size_t bytes) {
    NvtxScope r("fcd_get_state");
    return c ? c->get_state(dst, bytes) : FCD_EINVAL;
}

fcd_status fcd_set_state(fcd_ctx *c, const void *src, size_t bytes) {
    NvtxScope r("fcd_set_state");
    return c ? c->set_state(src, bytes) : FCD_EINVAL;
}

static void derived_out(const Derived &d, double *o) {
    const double v[15] = {d.u_avg, d.s12, d.s13, d.s23, d.gam[0], d.gam[1], d.gam[2], d.gamT,
                          d.tau[0], d.tau[1], d.tau[2], d.tau_phi, d.mu0H0sq, d.H0, d.G};
    std::memcpy(o, v, sizeof v);
}

fcd_status fcd_get_derived(const fcd_ctx *c, double *o) {
    if (!c || !o) return FCD_EINVAL;
    derived_out(c->D, o);
    return FCD_OK;
}

fcd_status fcd_derive_params(const fcd_params *params, double *o) {
    if (!params || !o) {
        std::snprintf(g_last, sizeof g_last, "fcd_derive_params: null argument");
        return FCD_EINVAL;
    }
    Derived d;
    if (const char *why = derive(params, &d)) {
        std::snprintf(g_last, sizeof g_last, "fcd_derive_params: %s", why);
        return FCD_EINVAL;
    }
    derived_out(d, o);
    return FCD_OK;
}

long fcd_kernel_launches(const fcd_ctx *c) { return c ? c->launches() : -1; }

fcd_status fcd_solver_stats(fcd_ctx *c, long long *out5) {
    if (!c || !out5) return FCD_EINVAL;
    return c->solver_stats(out5);
}

fcd_status fcd_collide_tile_height(const fcd_ctx *c, int *rows) {
    if (!c || !rows) return FCD_EINVAL;
    *rows = c->collide_tile_h();
    return FCD_OK;
}

fcd_status fcd_set_profiling(fcd_ctx *c, int enable) { return c ? c->set_profiling(enable) : FCD_EINVAL; }

fcd_status fcd_last_step_profile(fcd_ctx *c, double *ms4) {
    if (!c || !ms4) return FCD_EINVAL;
    return c->profile(ms4);
}

const char *fcd_last_error(const fcd_ctx *c) { return c ? c->err : g_last; }

void fcd_destroy(fcd_ctx *c) { delete c; }

}  // extern "C"
