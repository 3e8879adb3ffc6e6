// fcd_internal.cuh -- shared declarations of the CUDA library (not installed).
//
// Memory layout in HBM (all planes share one row pitch, a multiple of 32 nodes):
//   f      : 9 planes  x ny rows x pitch, double buffered      (storage type S)
//   g      : 18 planes x ny rows x pitch, double buffered      (g[i*9 + a])
//   phi    : 2 planes (phi_1, phi_2) of the current step       (compute type T)
//   macro  : 3 planes (ux, uy, p*) of the most recent collision
//   multigrid level 0: psi' (two buffers), k = 1 + chi (Eq. 8)
// Storage modes: FP64 stores f, g; FP32 plain stores f + w_a (the absolute,
// density-like population) and g; FP32 offset stores f and g - w_a / 2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fcd.h"
#include "fcd_dual.cuh"

namespace fcd {

// MODE_TANGENT: FP64 storage of the primal state and of NT tangent copies
// (forward-mode derivative along NT parameter directions), dual arithmetic.
enum StoreMode { MODE_FP64 = 0, MODE_FP32 = 1, MODE_FP32_OFFSET = 2, MODE_TANGENT = 3 };

constexpr int NT = 4;  // tangent directions: Bo_m, Ca, alpha, nu_r
using DualT = Dual<NT>;

// Arithmetic type of a kernel: the storage type, or dual numbers for tangents.
template <typename T, int MODE>
struct Compute { using type = T; };
template <>
struct Compute<double, MODE_TANGENT> { using type = DualT; };

constexpr int TX = 32;  // collide tile (x)
constexpr int TY = 8;   // collide tile (y)

// D2Q9 (Eq. 20 order: rest, E, N, W, S, NE, NW, SW, SE).
__host__ __device__ constexpr int cx(int a) {
    return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int a) {
    return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int a) {
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5);
}
template <typename T>
__host__ __device__ constexpr T wgt(int a) {
    return a == 0 ? T(4) / T(9) : (a <= 4 ? T(1) / T(9) : T(1) / T(36));
}

// Offsets added to the populations before they are stored.
template <int MODE, typename T>
__host__ __device__ constexpr T f_off(int a) {
    return MODE == MODE_FP32 ? wgt<T>(a) : T(0);
}
template <int MODE, typename T>
__host__ __device__ constexpr T g_off(int a) {
    return MODE == MODE_FP32_OFFSET ? -wgt<T>(a) / T(2) : T(0);
}

// Level-0 potential buffers. FP64 contexts hold psi' in one plane. FP32
// contexts reserve two FP32 planes per buffer (the low plane one plane stride
// after the high one): psi' itself is ~30 H0 on the channels of the paper's
// shape, so one FP32 plane quantises it at ~2e-6 H0, and the 9-point residual
// of that quantisation (~1e-5 H0) hides any smaller residual from the solve's
// stopping test. A context whose tolerance is below that keeps psi' as the
// unevaluated sum hi + lo (Level::comp); the others use the high plane alone
// and leave the low one at 0.
template <typename T>
__host__ __device__ constexpr int psi_planes() { return sizeof(T) == 4 ? 2 : 1; }

// Error-free FP32 sum (Knuth's TwoSum): s + e equals a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <typename T>
__device__ __forceinline__ T clamp01(T v) {
    return v < T(0) ? T(0) : (v > T(1) ? T(1) : v);
}

// Physical constants of one context in the compute type.
template <typename T>
struct Phys {
    int nx, ny, pitch;
    long long ps;                       // plane stride = pitch * ny
    T rho[3], tau[3];                   // Eq. 33 and Eq. 14
    T ik[3];                            // 1 / (1 + chi_i)      (Eq. 8)
    T dk1, dk2;                         // ik[0] - ik[2], ik[1] - ik[2] (Eq. 9)
    T s12, s13, s23, gam[3], eta;       // Eqs. 27, 28
    T twelve_over_xi, lap_coef[3];      // 12 / xi, (3/4) xi gamma_i   (Eq. 25)
    T four_over_xi, eps_n;              // source term of the phase field
    T om_phi, keep_phi, src_phi;        // 1/(1/2 + tau_phi), 1 - om, 1 - om/2
    T H0c, H0s, G;                      // H0 (cos a, sin a), driving force
};

// Multigrid level descriptor (device pointers). Level 0 is the lattice with
// the 9-point link operator; levels >= 1 are merged tensor grids carrying a
// 5-point finite-volume operator. Coordinates are in lattice units with the
// walls at y = 0 and y = ny0 (cell faces) and period nx0 along x.
// Completion counters of the level-0 kernels: tile t of a launch reports to
// group t % MG_GROUPS, the last tile of each group to the control block.
constexpr unsigned MG_GROUPS = 64;
struct alignas(128) MgGroup {
    unsigned count;               // tiles of this group done in the current launch
    unsigned pad_;
    unsigned long long max_bits;  // their max |r| (bits of a double >= 0)
};

template <typename T>
struct Level {
    using value_type = T;
    int nx, ny, pitch;
    T *e, *b, *k;             // correction (level 0: psi'), right-hand side, 1 + chi
    T *r;                     // scratch (level 0: second psi' buffer)
    const int *cx0, *cy0;     // children of cell I: parent columns cx0[I] .. cx0[I+1]-1
    const T *xc, *yc, *wx, *wy;
    const T *ixe;             // 1 / (distance to the east centre), periodic
    const T *iyn, *iys;       // 1 / (distance to the north / south centre or wall)
    T Lx, ylo, yhi;
    // prolongation of the next coarser level onto this one
    const int *px0, *px1, *py0, *py1;  // -1 in py* stands for the wall (value 0)
    const T *pwx, *pwy;
    const T *rhs;  // level 0: explicit right-hand side (nullptr: -L psi0 formed from k)
    // level 0 of FP64 hierarchies: the 9-point coefficients of every node, formed
    // once per solve (planes c_1..c_8, diagonal, its reciprocal, -L psi0)
    T *coef;
    // level 0 of FP32 hierarchies: 1 when psi' is the hi + lo pair (the lo
    // plane one plane stride after each buffer) and the residual is formed in
    // link differences (contexts whose tolerance one FP32 plane cannot reach)
    int comp;
    MgGroup *grp;  // level 0: MG_GROUPS completion groups (zero between launches)
};

// Device-side control block of one potential solve.
struct MgCtl {
    unsigned long long norm_bits;  // max |r| of the current cycle (bits of a double >= 0)
    int cur;                       // which level-0 buffer holds psi'
    int iter;                      // V-cycles done in this solve
    int done;                      // 1 once converged or capped
    int converged;                 // 1 if the tolerance was met
    double tolH0;                  // tol * H0
    int max_iter;
    int keep_going;                // host-visible loop flag
    double last_resid;             // final ||r||_inf / H0
    int last_iters;
    long long total_cycles;        // cumulative V-cycles that ran in full
    long long cycles_launched;     // cumulative cycle heads launched (launch accounting)
    int nonconv_count;             // solves that stopped at the cap
    double H0;
    unsigned int blocks_done;      // blocks of the last kernel of a cycle that finished
    long long step_cur;            // step index of the step in flight (breakup key)
    int mode;                      // decision of the cycle head: 0 V-cycle, 1 lattice sweeps,
                                   // 2 two-grid cycle, 3 stop
    int smooth_left;               // lattice-sweep cycles still allowed in this solve
    int twogrid_left;              // two-grid cycles still allowed in this solve
    long long smooth_cycles;       // cumulative lattice-sweep cycles (launch accounting)
    long long twogrid_cycles;      // cumulative two-grid cycles (launch accounting)
    unsigned batch_visits;         // batched solves: blocks of the current residual launch seen
    long long dispatches;          // cumulative cycle dispatch launches of graph loops (accounting)
};

// What the phase kernel does besides Eq. 32: reset the solve's control block
// (reset != 0) and, when step != nullptr, record the step index in flight in
// ctl->step_cur and advance the device step counter.
struct PhaseCtl {
    MgCtl *ctl;
    int reset;
    double tolH0;
    int max_iter;
    long long *step;
    // extrap != 0: initial guess of the solve psi' <- 2 psi'(t) - psi'(t-1);
    // psi_prev keeps the previous solution (buffers of the compute type)
    int extrap;
    void *psiA, *psiB, *psi_prev;
    int comp;  // FP32: psi' is the hi + lo pair (Level::comp)
};

struct ObsOut {
    double mass[3];
    double xc_core, yc_core, xc_shell, yc_shell;
    double lx_o, ly_o, lx_i, ly_i;
    unsigned long long brk_now;  // touch key of the current state (~0ull if none)
    int xcut;
    int nonfinite;
};

// Tangent observables: values and derivatives along the NT directions.
struct TanOut {
    double T_o, overlap, lx, ly;
    double dT_o[NT], doverlap[NT], dlx[NT], dly[NT];
};

}  // namespace fcd

// ---- host-side launchers (defined in the .cu files) ----
namespace fcd {

// T: element type of the field planes; R: arithmetic type of the constants
// (DualT for the tangent step, whose planes hold the primal value followed by
// NT tangent copies at a stride of one plane set).
template <typename T, typename R = T>
struct LbmArgs {
    Phys<R> P;
    const void *f_src, *g_src;
    void *f_dst, *g_dst;
    const T *phi1, *phi2;
    const T *psi0, *psi1;        // the two level-0 buffers; ctl->cur picks one
    const MgCtl *ctl;
    T *macro;                    // nullptr: do not store the macroscopic fields
    unsigned long long *brk;     // sticky breakup key (nullptr: no check)
    const long long *step;       // device step counter (breakup key)
    // first step whose collision produced a non-finite u or p* (atomicMin of
    // the step index; ~0ull while none; nullptr: no check)
    unsigned long long *unst = nullptr;
    int open_x = 0;              // open channel: no wrap in x (see launch_open_bc)
};

template <typename T>
void launch_phase(int mode, const Phys<T> &P, const void *g, T *phi1, T *phi2, T *k,
                  PhaseCtl pc, cudaStream_t s);

// Batched step over many periodic channels: per instance and buffer parity,
// the collide-stream arguments (lbm; its g_src is also what the phase kernel
// reads) and the phase kernel's outputs and control; a work list of tiles.
template <typename T>
struct BatchLbm {
    LbmArgs<T> lbm;
    PhaseCtl pc;
    T *phi1, *phi2, *k;
};
struct BatchTile {
    int inst;    // instance
    int x0, y0;  // tile origin in that instance's lattice
    int lead;    // 1 for one tile per instance (the phase kernel's control-block reset)
};
template <typename T>
void launch_phase_batch(int mode, const BatchLbm<T> *tab, const BatchTile *tiles, int ntiles,
                        cudaStream_t s);  // 32 x 8 tiles
// tile_h: 4, 8 or 16 rows per tile (the list's tiles are TX x tile_h)
template <typename T>
void launch_collide_batch(int mode, int tile_h, const BatchLbm<T> *tab, const BatchTile *tiles,
                          int ntiles, cudaStream_t s);
// tile_h: rows per collide tile, 4 or 8 for the FP32 forms (the same
// arithmetic per node; the faster one depends on the grid); FP64 uses 8.
template <typename T>
void launch_collide(int mode, int tile_h, const LbmArgs<T> &a, cudaStream_t s);
void launch_collide_tangent(const LbmArgs<double, DualT> &a, cudaStream_t s);
void launch_open_bc_tangent(const Phys<double> &P, const void *f_src, const void *g_src,
                            void *f_dst, void *g_dst, double u_max, double u_avg, cudaStream_t s);
// Open channel: the populations entering through the inlet (x = 0) and the
// outlet (x = nx - 1) after a collide-stream from (f_src, g_src) into
// (f_dst, g_dst); one thread per row.
template <typename T>
void launch_open_bc(int mode, const Phys<T> &P, const void *f_src, const void *g_src,
                    void *f_dst, void *g_dst, double u_max, double u_avg, cudaStream_t s);
template <typename T>
void launch_init(int mode, const Phys<T> &P, double u_max, double r1, double r2, double xc,
                 double yc, double xi, void *f, void *g, T *macro, cudaStream_t s);
template <typename T>
void launch_export(int mode, const Phys<T> &P, const void *f, const void *g, double *fo,
                   double *go, cudaStream_t s);
template <typename T>
void launch_import(int mode, const Phys<T> &P, const double *fi, const double *gi, void *f,
                   void *g, cudaStream_t s);
template <typename T>
void launch_plane_to_f64(const T *src, int nx, int ny, int pitch, double *dst, cudaStream_t s);
template <typename T>
void launch_plane_from_f64(const double *src, int nx, int ny, int pitch, T *dst, cudaStream_t s);
template <typename T>
void launch_phi3_to_f64(const T *p1, const T *p2, int nx, int ny, int pitch, double *dst,
                        cudaStream_t s);
// psi' of a level-0 buffer (psi_planes<T>() planes) to and from FP64
template <typename T>
void launch_psi_to_f64(const T *src, int nx, int ny, int pitch, double *dst, cudaStream_t s);
template <typename T>
void launch_psi_from_f64(const double *src, int nx, int ny, int pitch, T *dst, int comp,
                         cudaStream_t s);  // comp: keep the low part (else the low plane is 0)

// multigrid
template <typename T>
struct MgHost;  // defined in fcd_mg.cu
template <typename T>
MgHost<T> *mg_create(int nx, int ny, int pitch, T *k0, T *psiA, T *psiB, MgCtl *ctl,
                     void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *user,
                     char *err, size_t errlen, int comp = 0,
                     const MgHost<T> *share_coef = nullptr);  // FP64: use its coefficient planes
template <typename T>
void mg_destroy(MgHost<T> *m);
// One V-cycle = head (lattice residual; decides whether the cycle runs) +
// rest (launched only when the head said so: graph if node or host check).
template <typename T>
void mg_cycle_head(MgHost<T> *m, T H0c, T H0s, cudaGraphConditionalHandle hwhile,
                   cudaGraphConditionalHandle hif, int in_graph, cudaStream_t s);
template <typename T>
void mg_cycle_rest(MgHost<T> *m, T H0c, T H0s, cudaStream_t s);
template <typename T>
void mg_cycle_smooth(MgHost<T> *m, T H0c, T H0s, cudaStream_t s);
template <typename T>
void mg_cycle_twogrid(MgHost<T> *m, T H0c, T H0s, cudaStream_t s);
template <typename T>
void mg_presmooth(MgHost<T> *m, T H0c, T H0s, cudaStream_t s);  // opens every solve
template <typename T>
int mg_kernels_per_cycle(const MgHost<T> *m);
// Graph form of the cycle loop: a one-thread kernel at the top of the loop body
// that sets the body's switch node from the mode the last head chose.
template <typename T>
void mg_cycle_dispatch(MgHost<T> *m, cudaGraphConditionalHandle hswitch, cudaStream_t s);
// Tangent solves (FP64): explicit right-hand side on level 0; reset of the
// control block with tolerance tol * max|rhs|; right-hand side along one
// direction, L(k) dpsi' = b(k, dH0) + b(dk, H0) - L(dk) psi'; copies between
// the current level-0 buffer (picked on the device) and a plane:
// op 0 plane <- cur, op 1 cur <- plane, op 2 cur <- 2 plane - prev, prev <- plane.
template <typename T>
void mg_set_rhs(MgHost<T> *m, const T *rhs);
void mg_reset_scaled(MgCtl *ctl, const unsigned long long *scale_bits, double tol, int max_iter,
                     cudaStream_t s);
void mg_tangent_rhs(MgHost<double> *m, const double *dk, double H0c, double H0s, double dH0c,
                    double dH0s, double *rhs, unsigned long long *rmax_bits, cudaStream_t s);
void mg_psi_io(MgHost<double> *m, int op, double *plane, double *prev, cudaStream_t s);
template <typename T>
int mg_levels(const MgHost<T> *m);
// Batched solves of many FP32 hierarchies (one per instance; fields and
// control blocks stay the instances' own): opening sweeps of every solve, and
// the body of the loop that runs until every solve is done.
struct MgBatch;
MgBatch *mg_batch_create(const std::vector<MgHost<float> *> &ms, const std::vector<float> &H0c,
                         const std::vector<float> &H0s, void *(*alloc)(size_t, void *),
                         void (*release)(void *, void *), void *user, char *err, size_t errlen);
void mg_batch_destroy(MgBatch *b);
void mg_batch_presmooth(MgBatch *b, cudaStream_t s);
// one pass of the loop body launched from the host (no graph conditions set)
void mg_batch_body(MgBatch *b, cudaStream_t s);
// the body in parts, for a graph whose while node (hw) holds them: the head
// sets hw when in_graph != 0, and with in_graph == 1 also the conditions of IF
// nodes around the V-cycle (hv) and the two-grid cycle (ht)
void mg_batch_head(MgBatch *b, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hv,
                   cudaGraphConditionalHandle ht, int in_graph, cudaStream_t s);
void mg_batch_vcycle(MgBatch *b, cudaStream_t s);
void mg_batch_twogrid(MgBatch *b, cudaStream_t s);
void mg_batch_close(MgBatch *b, cudaStream_t s);
int mg_batch_body_kernels(const MgBatch *b);
// after a body launched with in_graph = 0: 1 while some solve goes on, 0 when
// all are done, -1 on a CUDA error (synchronises s)
int mg_batch_any(MgBatch *b, cudaStream_t s);

// tangent step (FP64 primal + NT tangent copies)
void launch_tangent_phase(const Phys<double> &P, const double *g, double *phi1, double *phi2,
                          double *k, cudaStream_t s);
size_t tangent_obs_scratch_bytes(int nx);
void launch_tangent_obs(const Phys<double> &P, const double *g, const ObsOut *prim, void *scratch,
                        TanOut *out, cudaStream_t s);

// adjoint step (FP64, periodic channel). A segment of forward states sits in
// slots of `stride` doubles (f 9 planes, g 18 planes, psi' 1 plane); *slot is
// the slot of the step being reversed. Adjoint states hold 27 planes (fb, gb).
struct AdjArgs {
    Phys<double> P;
    const double *seg;
    const int *slot;
    long long stride;
    const double *phi1, *phi2;  // phase fields of the slot's state
    const double *ab_src;       // adjoint after the step
    double *ab_dst;             // adjoint before the step (direct terms)
    double *sb;                 // 13 planes: adjoints of the reduced stencil values
    double *pacc;               // per block: adjoints of the constants (NPB each)
};
struct AdjKArgs {
    Phys<double> P;
    const double *seg;
    const int *slot;
    long long stride;
    const double *k, *phi1, *phi2;
    const double *pb;              // 2 planes: phase-field adjoints from the stencils
    const double *lamA, *lamB;     // adjoint potential buffers
    const MgCtl *ctl;              // its control block (nullptr: no field)
    double *ab;                    // adjoint before the step (gb += phib)
    double *hacc;                  // per block: adjoints of H0 cos(alpha), H0 sin(alpha)
};
struct AdjOut {
    double T_o, overlap, lx, ly;
};
int adj_collide_blocks(int nx, int ny);
int adj_kbar_blocks(int nx, int ny);
size_t adj_seed_scratch_bytes(int nx);
void launch_adj_phase(const Phys<double> &P, const double *seg, const int *slot, long long stride,
                      double *phi1, double *phi2, double *k, cudaStream_t s);
void launch_adj_collide(const AdjArgs &a, int open_x, cudaStream_t s);
void launch_adj_gather(const Phys<double> &P, const double *sb, const double *phi1, const double *phi2,
                       double *pb, double *rhs, unsigned long long *rmax, int open_x, cudaStream_t s);
// open channel: transpose of the boundary kernel on the adjoint after the step
// (keep: ny x 27 doubles, the outlet's dependence on the state before it), and
// the addition of keep into the adjoint before the step
void launch_adj_open_bc(const Phys<double> &P, double *ab, double *keep, double u_avg, cudaStream_t s);
void launch_adj_open_add(const Phys<double> &P, const double *keep, double *ab, cudaStream_t s);
void launch_adj_kbar(const AdjKArgs &a, cudaStream_t s);
void launch_set_slot(int *slot, int v, cudaStream_t s);
void launch_dec_slot(int *slot, cudaStream_t s);
// seed of J = wT T_o + wO overlap at the state whose phase fields are phi1,
// phi2 (prim: the plain observables of that state, for the seam column)
void launch_adj_seed(const Phys<double> &P, const double *phi1, const double *phi2, const ObsOut *prim,
                     double wT, double wO, void *scratch, double *pb, double *ab, AdjOut *out,
                     cudaStream_t s);

// The device state of a plain FP32 periodic context (fcd_create), for the
// batched step: the batch's kernels read and write these buffers directly.
struct EngineView {
    int mode;      // MODE_FP32 or MODE_FP32_OFFSET
    int magnetic;  // a potential solve runs every step
    int cur;       // population buffer of the current state
    Phys<float> P;
    void *f[2], *g[2];
    float *phi1, *phi2, *k, *psiA, *psiB, *psiP, *macro;
    MgCtl *ctl;
    MgHost<float> *mg;
    unsigned long long *brk, *unst;
    long long *d_step;
    double tolH0;
    int max_iter;
    int comp;  // psi' as the hi + lo pair
};
// false (and v untouched) for any other context
bool engine_view(fcd_ctx *c, EngineView *v);
// the host-side record of a context after `steps` steps run by the batch
void engine_advance(fcd_ctx *c, long steps);
// one step of a context on its own stream; store_macro: also store u and p*
fcd_status engine_step1(fcd_ctx *c, int store_macro);

// observables. Scratch layout of one reduction (doubles): phi_1 and phi_2
// planes (nx * ny each, unpadded), then OBS_COLS doubles per column.
constexpr int OBS_COLS = 12;
constexpr size_t observe_scratch_doubles_of(long long nx, long long ny) {
    return 2ull * (size_t)(nx * ny) + (size_t)OBS_COLS * (size_t)nx;
}
size_t observe_scratch_doubles(int nx, int ny);
template <typename T>
void launch_observe(int mode, const Phys<T> &P, const void *g, double *scratch, ObsOut *out,
                    cudaStream_t s, int open_x = 0);

}  // namespace fcd
