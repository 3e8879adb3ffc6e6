// fcd_batch.cu -- many independent channels advanced together (the regime-map
// sweep of arXiv 2410.11129, Sec. 3.7: Bo_m x Ca grids of separate runs).
//
// Each instance is a full context with its own CUDA stream and its own
// captured step graphs. fcd_batch_step launches, step by step, every
// instance's graph on that instance's stream, so the small latency-bound
// kernels of one instance (phase recovery, multigrid cycle heads and sweeps)
// run concurrently with the bandwidth-bound collide-stream of others. The
// caller's stream waits on all instance streams at the end (event join).
#include <cstdio>
#include <new>
#include <vector>

#include "fcd_internal.cuh"

struct fcd_batch {
    std::vector<fcd_ctx *> inst;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaStream_t caller = nullptr;
    cudaEvent_t start = nullptr;
    char err[512] = {0};
};

static thread_local char batch_last[512];

static void batch_free(fcd_batch *b) {
    if (!b) return;
    for (auto s : b->streams) cudaStreamSynchronize(s);
    for (auto c : b->inst) fcd_destroy(c);
    for (auto e : b->done) cudaEventDestroy(e);
    for (auto s : b->streams) cudaStreamDestroy(s);
    if (b->start) cudaEventDestroy(b->start);
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
    if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
        snprintf(batch_last, sizeof batch_last, "fcd_batch_create: cudaEventCreate failed");
        batch_free(b);
        return FCD_ECUDA;
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
    *out = b;
    return FCD_OK;
}

fcd_status fcd_batch_set_stream(fcd_batch *b, void *cuda_stream) {
    if (!b) return FCD_EINVAL;
    b->caller = static_cast<cudaStream_t>(cuda_stream);
    return FCD_OK;
}

fcd_status fcd_batch_step(fcd_batch *b, long n) {
    if (!b || n < 0) return FCD_EINVAL;
    const size_t m = b->inst.size();
    // instance streams start after the caller's prior work
    if (cudaEventRecord(b->start, b->caller) != cudaSuccess) {
        snprintf(b->err, sizeof b->err, "fcd_batch_step: cudaEventRecord failed");
        return FCD_ECUDA;
    }
    for (size_t i = 0; i < m; i++)
        if (cudaStreamWaitEvent(b->streams[i], b->start, 0) != cudaSuccess) {
            snprintf(b->err, sizeof b->err, "fcd_batch_step: cudaStreamWaitEvent failed");
            return FCD_ECUDA;
        }
    for (long s = 0; s < n; s++)
        for (size_t i = 0; i < m; i++) {
            const fcd_status st = fcd_step(b->inst[i], 1);
            if (st != FCD_OK) {
                snprintf(b->err, sizeof b->err, "fcd_batch_step: instance %zu: %s", i,
                         fcd_last_error(b->inst[i]));
                return st;
            }
        }
    for (size_t i = 0; i < m; i++)
        if (cudaEventRecord(b->done[i], b->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(b->caller, b->done[i], 0) != cudaSuccess) {
            snprintf(b->err, sizeof b->err, "fcd_batch_step: join failed");
            return FCD_ECUDA;
        }
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

int fcd_batch_size(const fcd_batch *b) { return b ? (int)b->inst.size() : 0; }

fcd_ctx *fcd_batch_instance(fcd_batch *b, int i) {
    if (!b || i < 0 || i >= (int)b->inst.size()) return nullptr;
    return b->inst[i];
}

const char *fcd_batch_last_error(const fcd_batch *b) { return b ? b->err : batch_last; }

void fcd_batch_destroy(fcd_batch *b) { batch_free(b); }

}  // extern "C"
