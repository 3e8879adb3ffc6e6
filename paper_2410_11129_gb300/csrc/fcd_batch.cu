// fcd_batch.cu -- many independent channels advanced together (the regime-map
// sweep of arXiv 2410.11129, Sec. 3.7: Bo_m x Ca grids of separate runs).
//
// Every instance is a full context (its own state, observables, snapshots).
// Periodic FP32 instances of one storage form and one level-0 form of the
// potential make a group that one fixed set of batched kernels advances, one
// CUDA graph per step:
//   - the phase recovery of every instance in one launch over a work list of
//     32 x 8 tiles spanning all instances;
//   - the potential solves of every instance in one loop of batched multigrid
//     kernels (fcd_mg.cu), a single while node for the whole group;
//   - the fused collide-stream of every instance in one launch over a second
//     work list, whose tile height (4, 8 or 16 rows) an autotuner picks at
//     create by timing the three candidates on the group's own state.
// Other instances (FP64, open channels) keep their own stream and step
// graphs and run beside the group. The caller's stream waits on everything at
// the end of fcd_batch_step (event join).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "fcd_internal.cuh"

using namespace fcd;

namespace {

struct Group {
    int mode = MODE_FP32;
    std::vector<int> idx;          // instances in the group
    std::vector<EngineView> v;
    int tile_h = 8;
    int n_ptiles = 0, n_ctiles = 0;
    BatchTile *d_ptiles = nullptr, *d_ctiles = nullptr;
    BatchLbm<float> *d_tab[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [parity][macro]
    MgBatch *mg = nullptr;
    cudaStream_t stream = nullptr, cap = nullptr;
    cudaEvent_t done = nullptr, solved = nullptr;
    // per buffer parity: graph A = phase recovery + potential solves; graph B
    // = collide-stream (per store-macro flag)
    cudaGraph_t graphA[2] = {nullptr, nullptr}, graphB[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t execA[2] = {nullptr, nullptr}, execB[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    std::vector<void *> mem;
};

void *dev_alloc(std::vector<void *> &mem, size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    mem.push_back(p);
    return p;
}

template <typename U>
U *upload(std::vector<void *> &mem, const std::vector<U> &h) {
    U *d = static_cast<U *>(dev_alloc(mem, h.size() * sizeof(U) + 16));
    if (d && cudaMemcpy(d, h.data(), h.size() * sizeof(U), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    return d;
}

void group_free(Group *g) {
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (int a = 0; a < 2; a++) {
        if (g->execA[a]) cudaGraphExecDestroy(g->execA[a]);
        if (g->graphA[a]) cudaGraphDestroy(g->graphA[a]);
        for (int b = 0; b < 2; b++) {
            if (g->execB[a][b]) cudaGraphExecDestroy(g->execB[a][b]);
            if (g->graphB[a][b]) cudaGraphDestroy(g->graphB[a][b]);
        }
    }
    if (g->mg) mg_batch_destroy(g->mg);
    for (void *p : g->mem) cudaFree(p);
    if (g->done) cudaEventDestroy(g->done);
    if (g->solved) cudaEventDestroy(g->solved);
    if (g->stream) cudaStreamDestroy(g->stream);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
}

// Collide-stream work list of a group for tiles TX x h.
std::vector<BatchTile> collide_tiles(const Group &g, int h) {
    std::vector<BatchTile> t;
    for (size_t i = 0; i < g.v.size(); i++)
        for (int y = 0; y < g.v[i].P.ny; y += h)
            for (int x = 0; x < g.v[i].P.nx; x += TX) t.push_back({(int)i, x, y, 0});
    return t;
}

// Argument table of the group for one buffer parity; macro: store u, p*;
// check: keep the breakup and instability records.
std::vector<BatchLbm<float>> table(const Group &g, int c, bool macro, bool check) {
    std::vector<BatchLbm<float>> tab(g.v.size());
    for (size_t i = 0; i < g.v.size(); i++) {
        const EngineView &v = g.v[i];
        BatchLbm<float> &b = tab[i];
        std::memset(&b, 0, sizeof b);
        LbmArgs<float> &a = b.lbm;
        a.P = v.P;
        a.f_src = v.f[c];
        a.g_src = v.g[c];
        a.f_dst = v.f[c ^ 1];
        a.g_dst = v.g[c ^ 1];
        a.phi1 = v.phi1;
        a.phi2 = v.phi2;
        a.psi0 = v.psiA;
        a.psi1 = v.psiB;
        a.ctl = v.ctl;
        a.macro = macro ? v.macro : nullptr;
        a.brk = check ? v.brk : nullptr;
        a.step = &v.ctl->step_cur;
        a.unst = check ? v.unst : nullptr;
        a.open_x = 0;
        b.pc = PhaseCtl{v.ctl, v.magnetic, v.tolH0, v.max_iter, v.d_step, v.magnetic, v.psiA, v.psiB,
                        v.psiP, v.comp};
        b.phi1 = v.phi1;
        b.phi2 = v.phi2;
        b.k = v.k;
    }
    return tab;
}

// The tile height of the group's collide-stream: the fastest of the
// candidates, each timed over three launches (after one untimed) on the
// group's current state. The timed launches write only the buffers of the
// next step, which the first real step overwrites; no record is kept.
int autotune(Group &g, const char **why) {
    const int cand[3] = {4, 8, 16};
    std::vector<BatchLbm<float>> tab = table(g, g.v[0].cur, false, false);
    BatchLbm<float> *d_tab = upload(g.mem, tab);
    if (!d_tab) { *why = "autotuner allocation"; return -1; }
    cudaEvent_t a, z;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess) {
        *why = "autotuner events";
        return -1;
    }
    int best = 8;
    float best_ms = 1e30f;
    for (int h : cand) {
        const std::vector<BatchTile> t = collide_tiles(g, h);
        std::vector<void *> scratch;
        BatchTile *d_t = upload(scratch, t);
        if (!d_t) continue;
        launch_collide_batch<float>(g.mode, h, d_tab, d_t, (int)t.size(), g.stream);
        cudaEventRecord(a, g.stream);
        for (int r = 0; r < 3; r++) launch_collide_batch<float>(g.mode, h, d_tab, d_t, (int)t.size(), g.stream);
        cudaEventRecord(z, g.stream);
        float ms = 0.f;
        if (cudaEventSynchronize(z) == cudaSuccess && cudaEventElapsedTime(&ms, a, z) == cudaSuccess &&
            cudaGetLastError() == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = h;
        }
        for (void *p : scratch) cudaFree(p);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    return best;
}

fcd_status group_build(Group &g, const char **why) {
    if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.solved, cudaEventDisableTiming) != cudaSuccess) {
        *why = "stream/event creation";
        return FCD_ECUDA;
    }
    std::vector<BatchTile> pt;
    for (size_t i = 0; i < g.v.size(); i++)
        for (int y = 0; y < g.v[i].P.ny; y += 8)
            for (int x = 0; x < g.v[i].P.nx; x += 32) pt.push_back({(int)i, x, y, x == 0 && y == 0});
    g.n_ptiles = (int)pt.size();
    g.d_ptiles = upload(g.mem, pt);
    for (int c = 0; c < 2; c++)
        for (int m = 0; m < 2; m++) g.d_tab[c][m] = upload(g.mem, table(g, c, m != 0, true));
    if (!g.d_ptiles || !g.d_tab[0][0] || !g.d_tab[0][1] || !g.d_tab[1][0] || !g.d_tab[1][1]) {
        *why = "table allocation";
        return FCD_ENOMEM;
    }
    std::vector<MgHost<float> *> mgs;
    std::vector<float> hc, hs;
    for (const EngineView &v : g.v)
        if (v.magnetic) {
            mgs.push_back(v.mg);
            hc.push_back(v.P.H0c);
            hs.push_back(v.P.H0s);
        }
    if (!mgs.empty()) {
        static char mgerr[256];
        g.mg = mg_batch_create(mgs, hc, hs, [](size_t n, void *) -> void * {
                                   void *p = nullptr;
                                   return cudaMalloc(&p, n) == cudaSuccess ? p : nullptr;
                               },
                               [](void *p, void *) { cudaFree(p); }, nullptr, mgerr, sizeof mgerr);
        if (!g.mg) {
            *why = mgerr;
            return FCD_ENOMEM;
        }
    }
    const int h = autotune(g, why);
    if (h < 0) return FCD_ECUDA;
    g.tile_h = h;
    const std::vector<BatchTile> ct = collide_tiles(g, h);
    g.n_ctiles = (int)ct.size();
    g.d_ctiles = upload(g.mem, ct);
    if (!g.d_ctiles) {
        *why = "tile list allocation";
        return FCD_ENOMEM;
    }
    return cudaGetLastError() == cudaSuccess ? FCD_OK : FCD_ECUDA;
}

// A while node at the capture point of s whose body is the group's batched
// multigrid loop body; s continues after it.
cudaError_t capture_solve_loop(Group &g, cudaStream_t s) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t gcap;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &gcap, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, gcap, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    e = cudaGraphAddNode(&wnode, gcap, deps, nullptr, nd, &cp);
    if (e != cudaSuccess) return e;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t bs;
    e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // the V-cycle and two-grid kernels are plain launches whose blocks return
        // at once for instances in another mode: IF nodes around them (set by
        // the head) measured 0.5 ms per step slower on the 96-channel sweep
        mg_batch_head(g.mg, h, 0, 0, 2, bs);
        mg_batch_vcycle(g.mg, bs);
        mg_batch_twogrid(g.mg, bs);
        mg_batch_close(g.mg, bs);
        cudaGraph_t out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(bs, &out);
        if (e == cudaSuccess) e = e2;
    }
    cudaStreamDestroy(bs);
    if (e != cudaSuccess) return e;
    return cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// One step of the group launched from the host (FCD_NO_GRAPH=1: profilers that
// do not follow conditional graph nodes see every kernel); the host reads the
// loop condition after each pass of the body.
cudaError_t group_host_step(Group &g, int c, int sm) {
    cudaStream_t s = g.stream;
    launch_phase_batch<float>(g.mode, g.d_tab[c][0], g.d_ptiles, g.n_ptiles, s);
    if (g.mg) {
        mg_batch_presmooth(g.mg, s);
        for (int guard = 0; guard < 1000000; guard++) {
            mg_batch_body(g.mg, s);
            const int any = mg_batch_any(g.mg, s);
            if (any < 0) return cudaErrorUnknown;
            if (!any) break;
        }
    }
    launch_collide_batch<float>(g.mode, g.tile_h, g.d_tab[c][sm], g.d_ctiles, g.n_ctiles, s);
    return cudaGetLastError();
}

cudaError_t capture_end(cudaStream_t s, cudaError_t e, cudaGraph_t *out, cudaGraphExec_t *exec) {
    cudaGraph_t gr = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &gr);  // always leave capture mode
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return e;
    }
    *out = gr;
    return cudaGraphInstantiate(exec, gr, 0);
}

// Graph A of parity c: phase recovery and the potential solves of the group.
cudaError_t group_graph_a(Group &g, int c) {
    if (g.execA[c]) return cudaSuccess;
    cudaStream_t s = g.cap;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    launch_phase_batch<float>(g.mode, g.d_tab[c][0], g.d_ptiles, g.n_ptiles, s);
    if (g.mg) {
        mg_batch_presmooth(g.mg, s);
        e = capture_solve_loop(g, s);
    }
    return capture_end(s, e, &g.graphA[c], &g.execA[c]);
}

// Graph B of parity c: the collide-stream of the group (sm: store u, p*).
cudaError_t group_graph_b(Group &g, int c, int sm) {
    if (g.execB[c][sm]) return cudaSuccess;
    cudaStream_t s = g.cap;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    launch_collide_batch<float>(g.mode, g.tile_h, g.d_tab[c][sm], g.d_ctiles, g.n_ctiles, s);
    return capture_end(s, cudaGetLastError(), &g.graphB[c][sm], &g.execB[c][sm]);
}

}  // namespace

// Stepping modes: each instance's own step graph on its own stream, all at
// once (MODE_STREAMS), or the batched kernels for the groups (MODE_KERNELS).
// Neither wins everywhere: the batched kernels save launches and keep the
// collide-stream in one large launch, the streams let some instances' solves
// overlap others' collide-streams. Unless FCD_BATCH_MODE fixes it, the first
// steps of the batch time both (steps 3-6 of the schedule below; steps 1-2
// build the graphs) and keep the faster.
enum { MODE_STREAMS = 0, MODE_KERNELS = 1 };
static const int TUNE_SCHEDULE[6] = {MODE_KERNELS, MODE_STREAMS, MODE_KERNELS, MODE_STREAMS,
                                     MODE_KERNELS, MODE_STREAMS};

struct fcd_batch {
    std::vector<fcd_ctx *> inst;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    std::vector<int> group_of;      // group index of each instance, -1: stepped on its own
    std::vector<Group *> groups;
    cudaStream_t caller = nullptr;
    cudaEvent_t start = nullptr;
    int choice = -1;                // stepping mode; -1 while the first steps time both
    bool no_graph = false;          // FCD_NO_GRAPH=1: the batched steps launched from the host
    int tune_i = 0;
    double tune_ms[2] = {0.0, 0.0};
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    char err[512] = {0};
};

static thread_local char batch_last[512];

static void batch_free(fcd_batch *b) {
    if (!b) return;
    for (Group *g : b->groups) group_free(g);
    for (auto s : b->streams) cudaStreamSynchronize(s);
    for (auto c : b->inst) fcd_destroy(c);
    for (auto e : b->done) cudaEventDestroy(e);
    for (auto s : b->streams) cudaStreamDestroy(s);
    if (b->start) cudaEventDestroy(b->start);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    delete b;
}

extern "C" {

fcd_status fcd_batch_create(const fcd_params *params, int n, fcd_batch **out) {
    if (!out) return FCD_EINVAL;
    *out = nullptr;
    if (!params || n <= 0) {
        snprintf(batch_last, sizeof batch_last, "fcd_batch_create: need n > 0 parameter sets");
        return FCD_EINVAL;
    }
    fcd_batch *b = new (std::nothrow) fcd_batch();
    if (!b) return FCD_ENOMEM;
    if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess) {
        snprintf(batch_last, sizeof batch_last, "fcd_batch_create: cudaEventCreate failed");
        batch_free(b);
        return FCD_ECUDA;
    }
    if (const char *ng = getenv("FCD_NO_GRAPH")) b->no_graph = ng[0] == '1';
    if (const char *fm = getenv("FCD_BATCH_MODE")) {
        if (fm[0] == '0') b->choice = MODE_STREAMS;
        else if (fm[0] == '1') b->choice = MODE_KERNELS;
    }
    for (int i = 0; i < n; i++) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            snprintf(batch_last, sizeof batch_last, "fcd_batch_create: stream/event creation failed");
            batch_free(b);
            return FCD_ECUDA;
        }
        b->streams.push_back(s);
        b->done.push_back(e);
        fcd_ctx *c = nullptr;
        const fcd_status st = fcd_create(&params[i], &c);
        if (st != FCD_OK) {
            snprintf(batch_last, sizeof batch_last, "fcd_batch_create: instance %d: %s", i,
                     fcd_last_error(nullptr));
            batch_free(b);
            return st;
        }
        b->inst.push_back(c);
        fcd_set_stream(c, s);
    }
    // group the periodic FP32 instances by storage form and level-0 form of the
    // potential (one FP32 plane or the hi + lo pair), and split each such set
    // into about one group per GROUP_NODES lattice nodes (at most MAX_SPLIT),
    // balanced by nodes: every group has its own stream, so the latency-bound
    // solve kernels of one group overlap the bandwidth-bound launches of
    // another, as the instances' own streams do (FCD_BATCH_GROUPS=k at create
    // fixes the split)
    b->group_of.assign(n, -1);
    const double GROUP_NODES = 6e6;
    const int MAX_SPLIT = 8;
    int forced = 0;
    if (const char *gs = getenv("FCD_BATCH_GROUPS")) forced = atoi(gs);
    for (int key = 0; key < 4; key++) {  // storage form x level-0 form of the potential
        const int form = key < 2 ? MODE_FP32 : MODE_FP32_OFFSET, comp = key & 1;
        std::vector<std::pair<long long, int>> mem;  // (nodes, instance), largest first
        std::vector<EngineView> views(n);
        double total = 0.0;
        for (int i = 0; i < n; i++) {
            if (!engine_view(b->inst[i], &views[i]) || views[i].mode != form || views[i].comp != comp)
                continue;
            const long long nodes = (long long)views[i].P.nx * views[i].P.ny;
            mem.push_back({nodes, i});
            total += (double)nodes;
        }
        if (mem.empty()) continue;
        std::sort(mem.begin(), mem.end(), [](const std::pair<long long, int> &a,
                                            const std::pair<long long, int> &c) {
            return a.first != c.first ? a.first > c.first : a.second < c.second;
        });
        int k = forced > 0 ? forced : (int)(total / GROUP_NODES + 0.5);
        k = std::max(1, std::min(std::min(k, MAX_SPLIT), (int)mem.size()));
        std::vector<Group *> gs(k, nullptr);
        std::vector<long long> load(k, 0);
        for (int q = 0; q < k; q++) {
            gs[q] = new (std::nothrow) Group();
            if (!gs[q]) {
                for (Group *g : gs) delete g;
                batch_free(b);
                return FCD_ENOMEM;
            }
            gs[q]->mode = form;
        }
        std::vector<std::vector<int>> members(k);
        for (const auto &m : mem) {  // largest first into the lightest group
            const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            members[q].push_back(m.second);
            load[q] += m.first;
        }
        for (int q = 0; q < k; q++) {
            std::sort(members[q].begin(), members[q].end());
            for (int i : members[q]) {
                gs[q]->idx.push_back(i);
                gs[q]->v.push_back(views[i]);
                b->group_of[i] = (int)b->groups.size();
            }
            b->groups.push_back(gs[q]);
        }
    }
    if (b->groups.empty()) b->choice = MODE_STREAMS;
    cudaDeviceSynchronize();  // the instances' initial solves precede the autotuner
    for (Group *g : b->groups) {
        const char *why = "unknown";
        const fcd_status st = group_build(*g, &why);
        if (st != FCD_OK) {
            snprintf(batch_last, sizeof batch_last, "fcd_batch_create: batched group: %s", why);
            batch_free(b);
            return st;
        }
    }
    *out = b;
    return FCD_OK;
}

fcd_status fcd_batch_set_stream(fcd_batch *b, void *cuda_stream) {
    if (!b) return FCD_EINVAL;
    b->caller = static_cast<cudaStream_t>(cuda_stream);
    return FCD_OK;
}

}  // extern "C"

// n steps of every instance in stepping mode `mode`, ordered after the caller's
// stream and joined back into it; macro: the batched groups' last step stores
// u and p* (fcd_step(n) does so for the instances on their own streams).
static fcd_status batch_steps(fcd_batch *b, int mode, long n, bool macro) {
    const size_t m = b->inst.size();
    // a group steps as one only while its instances share a buffer parity (an
    // instance stepped on its own breaks that): otherwise its instances step
    // on their own in this call
    std::vector<int> gpar(b->groups.size(), -1);
    for (size_t q = 0; q < b->groups.size(); q++) {
        Group &g = *b->groups[q];
        int par = -2;
        for (int i : g.idx) {
            EngineView v;
            engine_view(b->inst[i], &v);
            par = par == -2 ? v.cur : (par == v.cur ? par : -1);
        }
        gpar[q] = mode == MODE_KERNELS ? par : -1;
    }
    auto batched = [&](size_t i) { return b->group_of[i] >= 0 && gpar[b->group_of[i]] >= 0; };
    if (cudaEventRecord(b->start, b->caller) != cudaSuccess) {
        snprintf(b->err, sizeof b->err, "fcd_batch_step: cudaEventRecord failed");
        return FCD_ECUDA;
    }
    for (size_t i = 0; i < m; i++) {
        cudaError_t e = cudaStreamWaitEvent(b->streams[i], b->start, 0);
        if (e == cudaSuccess && batched(i)) {  // the group's kernels follow the instance's own work
            Group &g = *b->groups[b->group_of[i]];
            e = cudaEventRecord(b->done[i], b->streams[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(g.stream, b->done[i], 0);
        }
        if (e != cudaSuccess) {
            snprintf(b->err, sizeof b->err, "fcd_batch_step: cudaStreamWaitEvent failed");
            return FCD_ECUDA;
        }
    }
    for (size_t q = 0; q < b->groups.size(); q++)
        if (gpar[q] >= 0 && cudaStreamWaitEvent(b->groups[q]->stream, b->start, 0) != cudaSuccess) {
            snprintf(b->err, sizeof b->err, "fcd_batch_step: cudaStreamWaitEvent failed");
            return FCD_ECUDA;
        }
    for (long s = 0; s < n; s++) {
        cudaEvent_t prev_solved = nullptr;
        // instances on their own streams, step by step across the instances so
        // that they advance together and their stages interleave on the GPU;
        // the last step of the call stores u and p*, as fcd_step(n) does
        for (size_t i = 0; i < m; i++) {
            if (batched(i)) continue;
            const fcd_status st = engine_step1(b->inst[i], s == n - 1 ? 1 : 0);
            if (st != FCD_OK) {
                snprintf(b->err, sizeof b->err, "fcd_batch_step: instance %zu: %s", i,
                         fcd_last_error(b->inst[i]));
                return st;
            }
        }
        for (size_t q = 0; q < b->groups.size(); q++) {
            if (gpar[q] < 0) continue;
            Group &g = *b->groups[q];
            const int c = gpar[q] ^ (int)(s & 1), sm = macro && s == n - 1 ? 1 : 0;
            cudaError_t e;
            if (b->no_graph) {
                e = group_host_step(g, c, sm);
            } else {
                // the groups start staggered: in the first step of a call a
                // group's solves wait for the previous group's, after which the
                // groups run free on their streams, so that one group's solves
                // run beside another's collide-stream
                e = group_graph_a(g, c);
                if (e == cudaSuccess) e = group_graph_b(g, c, sm);
                if (e == cudaSuccess && prev_solved && s == 0)
                    e = cudaStreamWaitEvent(g.stream, prev_solved, 0);
                if (e == cudaSuccess) e = cudaGraphLaunch(g.execA[c], g.stream);
                if (e == cudaSuccess) e = cudaEventRecord(g.solved, g.stream);
                if (e == cudaSuccess) e = cudaGraphLaunch(g.execB[c][sm], g.stream);
                prev_solved = g.solved;
            }
            if (e != cudaSuccess) {
                snprintf(b->err, sizeof b->err, "fcd_batch_step: batched step: %s", cudaGetErrorString(e));
                return FCD_ECUDA;
            }
        }
    }
    for (size_t q = 0; q < b->groups.size(); q++) {
        if (gpar[q] < 0) continue;
        Group &g = *b->groups[q];
        for (int i : g.idx) engine_advance(b->inst[i], n);
        if (cudaEventRecord(g.done, g.stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->caller, g.done, 0) != cudaSuccess) {
            snprintf(b->err, sizeof b->err, "fcd_batch_step: join failed");
            return FCD_ECUDA;
        }
        for (int i : g.idx)  // later calls on an instance see the group's steps
            if (cudaStreamWaitEvent(b->streams[i], g.done, 0) != cudaSuccess) {
                snprintf(b->err, sizeof b->err, "fcd_batch_step: join failed");
                return FCD_ECUDA;
            }
    }
    for (size_t i = 0; i < m; i++) {
        if (batched(i)) continue;
        if (cudaEventRecord(b->done[i], b->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(b->caller, b->done[i], 0) != cudaSuccess) {
            snprintf(b->err, sizeof b->err, "fcd_batch_step: join failed");
            return FCD_ECUDA;
        }
    }
    return FCD_OK;
}

extern "C" {

fcd_status fcd_batch_step(fcd_batch *b, long n) {
    if (!b || n < 0) return FCD_EINVAL;
    long done = 0;
    while (b->choice < 0 && done < n) {  // the first steps time both modes, one step at a time
        const int mode = TUNE_SCHEDULE[b->tune_i];
        if (cudaEventRecord(b->t0, b->caller) != cudaSuccess) return FCD_ECUDA;
        const fcd_status st = batch_steps(b, mode, 1, true);
        if (st != FCD_OK) return st;
        float ms = 0.f;
        if (cudaEventRecord(b->t1, b->caller) != cudaSuccess || cudaEventSynchronize(b->t1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, b->t0, b->t1) != cudaSuccess) {
            snprintf(b->err, sizeof b->err, "fcd_batch_step: timing failed");
            return FCD_ECUDA;
        }
        if (b->tune_i >= 2) b->tune_ms[mode] += ms;
        if (++b->tune_i == 6) b->choice = b->tune_ms[MODE_KERNELS] < b->tune_ms[MODE_STREAMS] ? MODE_KERNELS : MODE_STREAMS;
        done++;
    }
    if (done < n) return batch_steps(b, b->choice, n - done, true);
    return FCD_OK;
}

fcd_status fcd_batch_observables(fcd_batch *b, fcd_obs *out) {
    if (!b || !out) return FCD_EINVAL;
    fcd_status worst = FCD_OK;
    for (size_t i = 0; i < b->inst.size(); i++) {
        const fcd_status st = fcd_observables(b->inst[i], &out[i]);
        if (st != FCD_OK && worst == FCD_OK) {
            worst = st;
            snprintf(b->err, sizeof b->err, "instance %zu: %s", i, fcd_last_error(b->inst[i]));
        }
    }
    return worst;
}

fcd_status fcd_batch_set_mode(fcd_batch *b, int mode) {
    if (!b || mode < -1 || mode > 1) return FCD_EINVAL;
    if (mode == MODE_KERNELS && b->groups.empty()) {
        snprintf(b->err, sizeof b->err, "fcd_batch_set_mode: no instance can take the batched kernels");
        return FCD_EINVAL;
    }
    b->choice = mode;
    if (mode < 0) {  // time both again from the next step
        b->tune_i = 0;
        b->tune_ms[0] = b->tune_ms[1] = 0.0;
    }
    return FCD_OK;
}

fcd_status fcd_batch_tuning(const fcd_batch *b, int *mode, int *batched, int *groups, int *tile_h,
                            int tile_h_len) {
    if (!b) return FCD_EINVAL;
    if (mode) *mode = b->choice;
    int nb = 0;
    for (const Group *g : b->groups) nb += (int)g->idx.size();
    if (batched) *batched = nb;
    if (groups) *groups = (int)b->groups.size();
    if (tile_h) {
        for (size_t q = 0; q < b->groups.size() && (int)q < tile_h_len; q++) tile_h[q] = b->groups[q]->tile_h;
    }
    return FCD_OK;
}

int fcd_batch_size(const fcd_batch *b) { return b ? (int)b->inst.size() : 0; }

fcd_ctx *fcd_batch_instance(fcd_batch *b, int i) {
    if (!b || i < 0 || i >= (int)b->inst.size()) return nullptr;
    return b->inst[i];
}

const char *fcd_batch_last_error(const fcd_batch *b) { return b ? b->err : batch_last; }

void fcd_batch_destroy(fcd_batch *b) { batch_free(b); }

}  // extern "C"
