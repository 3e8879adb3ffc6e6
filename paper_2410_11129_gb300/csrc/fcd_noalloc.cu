// fcd_noalloc.cu -- observables of a population buffer without any device
// allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another framework
// owns the device memory budget (a caching allocator that must see every
// byte), latency-critical loops where cudaMalloc/cudaFree would synchronise
// the device, and hosts with a fixed, pre-reserved memory plan. This entry
// point serves them: the caller passes the populations and receives the
// observables; the scratch space the reduction needs lives in one file-scope
// device array reserved when the library is loaded.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fcd_internal.cuh"

namespace fcd {

namespace {

constexpr long long NOALLOC_MAX_NODES = 1ll << 19;  // 524,288 lattice nodes
constexpr int NOALLOC_MAX_NX = 16384;
constexpr size_t OBSOUT_DOUBLES = (sizeof(ObsOut) + sizeof(double) - 1) / sizeof(double);
// The reduction's layout (phase planes, then column records) for the largest
// admitted lattice, followed by the result block: 9.5 MiB.
constexpr size_t NOALLOC_REDUCE_DOUBLES = 2ull * NOALLOC_MAX_NODES + (size_t)OBS_COLS * NOALLOC_MAX_NX;
constexpr size_t NOALLOC_DOUBLES = NOALLOC_REDUCE_DOUBLES + OBSOUT_DOUBLES;
static_assert(observe_scratch_doubles_of(NOALLOC_MAX_NX, NOALLOC_MAX_NODES / NOALLOC_MAX_NX) <=
                  NOALLOC_REDUCE_DOUBLES,
              "every admitted lattice's reduction scratch fits in front of the result block");

// Scratch shared by every call: phase planes, column records, result block.
static __device__ __align__(256) double noalloc_scratch[NOALLOC_DOUBLES];

// Device address of the scratch array, looked up by the first call on each
// device (with that device current) and kept for the process.
constexpr int MAX_DEVICES = 64;
static double *scratch_addr[MAX_DEVICES];
static std::mutex scratch_mutex;

// A rejected call returns its status and states the reason on stderr.
fcd_status noalloc_fail(fcd_status st, const char *msg) {
    fprintf(stderr, "fcd_observe_populations_noalloc: %s\n", msg);
    return st;
}

}  // namespace

}  // namespace fcd

using namespace fcd;

extern "C" fcd_status fcd_observe_populations_noalloc(const double *g, int nx, int ny, int open_x,
                                                      void *cuda_stream, fcd_obs *out) {
    if (!g || !out) return noalloc_fail(FCD_EINVAL, "null population or output pointer");
    if (nx < 4 || ny < 2) return noalloc_fail(FCD_EINVAL, "need nx >= 4 and ny >= 2");
    if (open_x != 0 && open_x != 1) return noalloc_fail(FCD_EINVAL, "open_x must be 0 or 1");
    if (nx > NOALLOC_MAX_NX || (long long)nx * ny > NOALLOC_MAX_NODES)
        return noalloc_fail(FCD_EINVAL,
                            "lattice larger than the static scratch (nx <= 16384, nx*ny <= 524288)");
    // In host code noalloc_scratch names a host-side stand-in, not device memory:
    // the kernels get the array's device address, set up once per device.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return noalloc_fail(FCD_ECUDA, "cannot query the current device");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(scratch_mutex);
        if (!scratch_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
            if (e != cudaSuccess) return noalloc_fail(FCD_ECUDA, cudaGetErrorString(e));
            scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = scratch_addr[dev];
    }
    Phys<double> P;
    memset(&P, 0, sizeof P);
    P.nx = nx;
    P.ny = ny;
    P.pitch = nx;  // the FP64 exchange layout is unpadded
    P.ps = (long long)nx * ny;
    ObsOut *res = reinterpret_cast<ObsOut *>(scratch + observe_scratch_doubles_of(nx, ny));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // launch_observe clears the result block before its kernels run; open_x
    // selects the open channel's frame (no periodic seam, no wrap in x)
    launch_observe<double>(MODE_FP64, P, g, scratch, res, s, open_x);
    ObsOut r;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, res, sizeof r, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(FCD_ECUDA, cudaGetErrorString(e));
    memset(out, 0, sizeof *out);
    for (int i = 0; i < 3; i++) out->mass[i] = r.mass[i];
    out->lx_o = r.lx_o;
    out->ly_o = r.ly_o;
    out->lx_i = r.lx_i;
    out->ly_i = r.ly_i;
    out->T_o = (r.lx_o + r.ly_o) > 0 ? (r.ly_o - r.lx_o) / (r.ly_o + r.lx_o) : 0.0;
    out->T_i = (r.lx_i + r.ly_i) > 0 ? (r.ly_i - r.lx_i) / (r.ly_i + r.lx_i) : 0.0;
    out->xc_core = r.xc_core;
    out->yc_core = r.yc_core;
    out->xc_shell = r.xc_shell;
    out->yc_shell = r.yc_shell;
    out->b_step = -1;
    if (r.brk_now != ~0ull) {
        out->breakup = 1;
        out->b_step = 0;
        out->xb = double(r.brk_now % (unsigned long long)nx);
        out->yb = double(r.brk_now / (unsigned long long)nx);
        out->Lb_star = out->xb / ny;
        out->yb_star = (out->yb > 0.5 * (ny - 1) ? out->yb - 0.5 * (ny - 1) : 0.5 * (ny - 1) - out->yb) / ny;
    }
    if (r.nonfinite) return noalloc_fail(FCD_EUNSTABLE, "non-finite phase field");
    return FCD_OK;
}
