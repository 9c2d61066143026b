// mem_adjoint_noalloc: the tensor-core adjoint for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// that owns all device memory through its own pool or arena (and forbids
// side allocations), plug-ins loaded into such a process, or code that must
// not allocate after start-up (allocation can synchronise the device and is
// not allowed in some latency-critical paths).  They already hold their
// inputs and outputs in device memory; this entry point needs nothing else.
//
// Its scratch space (split-K partial sums and the work list) is a file-scope
// static __device__ array of fixed size.  The array is part of the library's
// device image: every GPU on which the library is loaded holds it (about
// 16 MB) until the process exits.  Every call shares it, so calls that
// overlap on the GPU (different streams, threads or processes sharing a
// context) race; serialise them.  The array keeps the previous call's
// contents; nothing in it needs to start at zero (each partial block is fully
// written before it is read, and the reduction reads only the partials of the
// units this call listed).  The status word is cleared on every call.
//
// The arrays' device addresses are resolved once per device and kept for the
// life of the process; after cudaDeviceReset the library's device image is
// loaded again at new addresses, so the entry point must not be used after a
// device reset in the same process.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/libmemsynth.h"
#include "internal.h"

using namespace msk;

namespace {

constexpr int NOALLOC_MAX_CTAS = 64;
constexpr int NOALLOC_BLK = 256;

static __device__ __align__(256) float g_partial[(size_t)NOALLOC_MAX_CTAS * NOALLOC_BLK * NOALLOC_BLK];
static __device__ __align__(256) AdjUnit g_units[NOALLOC_MAX_CTAS];
// [0, NOALLOC_MAX_CTAS]: per-CTA unit offsets; then 2 entries of per-block offsets
static __device__ __align__(256) int g_offs[NOALLOC_MAX_CTAS + 1 + 2];
static __device__ __align__(256) int g_status;

struct DevPtrs {
    bool ready = false;
    float* partial = nullptr;
    AdjUnit* units = nullptr;
    int* offs = nullptr;
    int* status = nullptr;
    int num_sms = 0;
};

std::mutex g_mu;
DevPtrs g_dev[64];

// Host code cannot use the arrays' names as device addresses; resolve them
// once per device, with that device current.
mem_status setup(int dev, DevPtrs** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return MEM_ECUDA;
    DevPtrs& p = g_dev[dev];
    if (!p.ready) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return MEM_ECUDA;
        if (prop.major != 10 || prop.minor != 3) return MEM_ECUDA;
        if (cudaGetSymbolAddress((void**)&p.partial, g_partial) != cudaSuccess) return MEM_ECUDA;
        if (cudaGetSymbolAddress((void**)&p.units, g_units) != cudaSuccess) return MEM_ECUDA;
        if (cudaGetSymbolAddress((void**)&p.offs, g_offs) != cudaSuccess) return MEM_ECUDA;
        if (cudaGetSymbolAddress((void**)&p.status, g_status) != cudaSuccess) return MEM_ECUDA;
        p.num_sms = prop.multiProcessorCount;
        p.ready = true;
    }
    *out = &p;
    return MEM_OK;
}

}  // namespace

extern "C" mem_status mem_adjoint_noalloc(int32_t n, double dx, double dy, int64_t n_vis,
                                          const double* u_dev, const double* v_dev,
                                          const float* y_dev, const float* pb_dev, float* img_dev,
                                          void* stream) {
    if (n != 64 && n != 128 && n != 256) {
        // the scratch array holds at most one 256 x 256 output block per CTA
        set_global_error("mem_adjoint_noalloc: image side n must be 64, 128 or 256 (the fixed scratch "
                         "array holds one 256 x 256 block per CTA)");
        return MEM_EINVAL;
    }
    if (!(dx > 0) || !(dy > 0) || n_vis < 0 || !pb_dev || !img_dev ||
        (n_vis > 0 && (!u_dev || !v_dev || !y_dev))) {
        set_global_error("mem_adjoint_noalloc: null pointer, negative n_vis or pixel size <= 0");
        return MEM_EINVAL;
    }
    if (((uintptr_t)y_dev & 7) != 0) {
        set_global_error("mem_adjoint_noalloc: y_dev must be 8-byte aligned");
        return MEM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // clear an error the caller may have left pending, so that a failure
    // reported below is this call's own
    cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MEM_ECUDA;
    }
    DevPtrs* P = nullptr;
    mem_status s = setup(dev, &P);
    if (s != MEM_OK) {
        cudaGetLastError();
        set_global_error("mem_adjoint_noalloc: no sm_103 device, or its scratch array could not be resolved");
        return s;
    }

    // Work list: the visibilities' 16-sample stages cut into one contiguous run
    // per CTA (single channel, single output block).
    const int64_t T = (n_vis + TCA_BK - 1) / TCA_BK;
    const int G = (int)std::min<int64_t>(std::min(P->num_sms, NOALLOC_MAX_CTAS), T);
    std::vector<AdjUnit> units;
    int offs[NOALLOC_MAX_CTAS + 1 + 2] = {0};
    for (int g = 0; g < G; ++g) {
        const int64_t s0 = T * g / G, s1 = T * (g + 1) / G;
        AdjUnit un;
        un.chan = 0;
        un.block = 0;
        un.start = s0 * TCA_BK;
        un.count = std::min<int64_t>(n_vis, s1 * TCA_BK) - un.start;
        offs[g] = g;
        units.push_back(un);
    }
    offs[G] = G;
    offs[NOALLOC_MAX_CTAS + 1] = 0;  // block 0 covers units [0, G)
    offs[NOALLOC_MAX_CTAS + 2] = G;

    cudaError_t e = cudaMemsetAsync(P->status, 0, sizeof(int), st);
    if (e == cudaSuccess && G > 0)
        e = cudaMemcpyAsync(P->units, units.data(), units.size() * sizeof(AdjUnit), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->offs, offs, sizeof(offs), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_global_error("mem_adjoint_noalloc: work-list upload failed");
        return MEM_ECUDA;
    }
    DevData d;
    std::memset(&d, 0, sizeof d);
    d.N = n;
    d.C = 1;
    d.n_images = 1;
    d.u = u_dev;
    d.v = v_dev;
    d.beam = pb_dev;
    d.dx = dx;
    d.dy = dy;
    launch_adj_tc_uv(d, P->units, P->offs, G, (const float2*)y_dev, P->partial, (uint64_t)1 << 26,
                     P->status, st);
    launch_adj_tc_reduce_out(n, P->offs + NOALLOC_MAX_CTAS + 1, P->partial, pb_dev, img_dev, st);
    int hs = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, P->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return MEM_ECUDA;
    }
    if (hs & DEV_TIMEOUT) {
        set_global_error("mem_adjoint_noalloc: a bounded device-side wait ran out");
        return MEM_ETIMEOUT;
    }
    return MEM_OK;
}
