// libmemsynth C ABI: context, buffers, work lists, launch sequences and the
// projected conjugate-gradient driver.  Declarations and semantics:
// include/libmemsynth.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "../../include/libmemsynth.h"
#include "internal.h"
#include "solver.h"

using namespace msk;

namespace {

thread_local std::string g_last_error = "";

size_t alloc_cap() {
    const char* s = std::getenv("MEMSYNTH_MAX_BYTES");
    if (!s || !*s) return (size_t)-1;
    return (size_t)std::strtoull(s, nullptr, 10);
}

}  // namespace

struct mem_ctx {
    // problem
    int N = 0, C = 0, n_images = 0, shared = 0, prec = 0;
    double dx = 0, dy = 0, lambda = 0, G = 0;
    uint64_t spin = 0;
    int64_t Z = 0;
    std::vector<int64_t> off;
    cudaStream_t st = nullptr;
    int device = 0, num_sms = 0;
    std::string err;
    int64_t launches = 0;
    size_t bytes = 0, cap = (size_t)-1;
    std::vector<void*> allocs;

    // resident data
    double *u = nullptr, *v = nullptr, *w = nullptr;
    uint64_t *pa = nullptr, *pb = nullptr;
    double2* vo = nullptr;
    float4* vo32 = nullptr;  // V° as FP32 (hi, lo) pairs, for the tensor-core epilogues
    float* w32 = nullptr;
    float* beam = nullptr;
    int64_t* doff = nullptr;

    // work lists: visibility tiles for the direct forms (128) and the
    // tensor-core form (TC_TILE)
    std::vector<VisTile> tiles_h, tiles_tc_h;
    std::vector<int> tile_off_h, tile_off_tc_h;
    VisTile *tiles = nullptr, *tiles_tc = nullptr;
    int *tile_off = nullptr, *tile_off_tc = nullptr;
    int n_tiles = 0, n_tiles_tc = 0;
    std::vector<AdjUnit> units_h;
    std::vector<int> cta_off_h, cb_off_h;
    AdjUnit* units = nullptr;
    int *cta_off = nullptr, *cb_off = nullptr;
    int adj_ctas = 0;

    // scratch
    float2* y32 = nullptr;
    double2* y64 = nullptr;
    double *chi_part = nullptr, *ent_part = nullptr, *gsum = nullptr, *scal = nullptr, *img_tmp = nullptr;
    int gsum_ks = 0;
    float* bf32 = nullptr;
    double* bf64 = nullptr;
    uint16_t* planes = nullptr;
    float* cmean = nullptr;  // column means of the centred tensor-core operand
    float* cscale = nullptr;                    // FP16X3 operand scales per channel
    double* col_psum = nullptr;                 // column-mean partial sums
    float* col_pmax = nullptr;
    unsigned* col_count = nullptr;              // column-mean completion counters (zero between calls)
    float *ymax = nullptr, *ymax_part = nullptr;  // FP16X3: max |y| (adjoint operand scale), partials
    float* partial = nullptr;  // adjoint unit partials (FP32, one BLK x BLK block each)
    int* dstatus = nullptr;
    float* stage = nullptr;  // host-call staging (image, gradient)
    // pinned host words for the scalar and status readback (one copy pair and
    // one stream synchronisation per call; nullptr: pageable fallback)
    double* hscal = nullptr;
    size_t hscal_n = 0;

    // CUDA graphs: each repeated launch sequence is captured once (on a private
    // stream: the legacy default stream cannot be captured) and replayed on st
    struct GraphSlot {
        const void* k1 = nullptr;
        const void* k2 = nullptr;
        int k3 = -1, prec = -1;
        int64_t nlaunch = 0;
        cudaGraphExec_t exec = nullptr;
    };
    bool graphs = true;
    cudaStream_t cap_st = nullptr;
    GraphSlot g_objgrad;
    // the whole solve (evaluations, CG and line-search control) as one graph
    // with conditional WHILE nodes for the iterations and the probes
    struct SolveGraph {
        cudaGraphExec_t exec = nullptr;
        int prec = -1;
        const void* hist = nullptr;
        int64_t n_pro = 0, n_iter = 0, n_probe = 0;  // kernel launches per part
    } g_solve;

    // tensor-core tiling (autotuned): forward kernel (MEM_FWD_STREAM: image
    // operand streamed per tile, column block fwd_bn; MEM_FWD_RESIDENT: image
    // slice resident in shared memory, N <= 256), pipeline depths
    int fwd_kernel = MEM_FWD_STREAM, fwd_bn = 0, fwd_stages = 4, adj_stages = 3;
    double2* vpart = nullptr;  // resident kernel: slice partials [slice][Z]

    // gridded forward (the paper's FFT + bilinear approximation): row
    // spectra and 2-D half spectra for `grid_pad`
    std::vector<double> wsum_h;   // per-channel sum of weights (natural-weights dirty image)
    double* wsum = nullptr;
    int grid_pad = 0;
    float2* grid_R = nullptr;
    float2* grid_F = nullptr;
    std::string gpu_name;

    // optional per-kernel timing (CUDA events on the context stream)
    bool profiling = false;
    struct KEv {
        const char* name;
        cudaEvent_t a, b;
    };
    std::vector<KEv> kev;
    std::vector<cudaEvent_t> ev_pool;
    std::map<std::string, std::pair<double, int64_t>> kacc;

    // solver state
    double *I64 = nullptr, *d64 = nullptr, *g64 = nullptr, *gf64 = nullptr, *gp64 = nullptr;
    double *alpha = nullptr, *beta = nullptr, *dots = nullptr, *dpart = nullptr;
    int* mode = nullptr;
    CgImage* cg_st = nullptr;
    CgControl* cg_ctl = nullptr;
    double* cg_hist = nullptr;
    size_t cg_hist_cap = 0;

    DevData dd() const {
        DevData d;
        d.N = N;
        d.C = C;
        d.n_images = n_images;
        d.shared = shared;
        d.G = G;
        d.lambda = lambda;
        d.pa = pa;
        d.pb = pb;
        d.u = u;
        d.v = v;
        d.vo = vo;
        d.w = w;
        d.vo32 = vo32;
        d.w32 = w32;
        d.beam = beam;
        d.off = doff;
        d.dx = dx;
        d.dy = dy;
        d.fwd_bn = fwd_kernel == MEM_FWD_RESIDENT ? N : fwd_bn;
        d.fwd_stages = fwd_stages;
        d.adj_stages = adj_stages;
        return d;
    }
};

namespace {

cudaEvent_t pool_event(mem_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one kernel launch with CUDA events when profiling is on.
struct KTimer {
    mem_ctx* c;
    const char* name;
    cudaEvent_t a = nullptr;
    KTimer(mem_ctx* ctx, const char* n) : c(ctx), name(n) {
        if (c->profiling) {
            a = pool_event(c);
            cudaEventRecord(a, c->st);
        }
    }
    ~KTimer() {
        if (a) {
            cudaEvent_t b = pool_event(c);
            cudaEventRecord(b, c->st);
            c->kev.push_back({name, a, b});
        }
    }
};

mem_status fail(mem_ctx* c, mem_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    g_last_error = buf;
    return s;
}

mem_status cuda_fail(mem_ctx* c, cudaError_t e, const char* what) {
    return fail(c, MEM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <typename T>
mem_status dalloc(mem_ctx* c, T** p, size_t count);

// Release one tracked allocation.
template <typename T>
void dfree(mem_ctx* c, T** p, size_t count) {
    if (!*p) return;
    for (size_t i = 0; i < c->allocs.size(); ++i)
        if (c->allocs[i] == (void*)*p) {
            c->allocs.erase(c->allocs.begin() + i);
            break;
        }
    cudaFree(*p);
    c->bytes -= std::max<size_t>(count * sizeof(T), 16);
    *p = nullptr;
}

template <typename T>
mem_status dalloc(mem_ctx* c, T** p, size_t count) {
    if (*p) return MEM_OK;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (c->bytes + bytes > c->cap)
        return fail(c, MEM_ENOMEM, "device allocation of %zu bytes exceeds MEMSYNTH_MAX_BYTES", bytes);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MEM_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->bytes += bytes;
    c->allocs.push_back(q);
    *p = (T*)q;
    return MEM_OK;
}

#define TRY(x)                           \
    do {                                 \
        mem_status s_ = (x);             \
        if (s_ != MEM_OK) return s_;     \
    } while (0)

bool tc_shape_ok(int N) { return N == 64 || N == 128 || (N >= 256 && N % 256 == 0); }
bool is_tc(int prec) { return prec == MEM_PREC_BF16X3 || prec == MEM_PREC_FP16X3; }

// Visibility tiles of `size` per channel, in channel order.
void build_tiles(const mem_ctx* c, int size, std::vector<VisTile>& tiles, std::vector<int>& off) {
    tiles.clear();
    off.assign(c->C + 1, 0);
    for (int ch = 0; ch < c->C; ++ch) {
        off[ch] = (int)tiles.size();
        for (int64_t s = c->off[ch]; s < c->off[ch + 1]; s += size) {
            VisTile t;
            t.chan = ch;
            t.start = s;
            t.count = (int)std::min<int64_t>(size, c->off[ch + 1] - s);
            tiles.push_back(t);
        }
    }
    off[c->C] = (int)tiles.size();
}

// Split-K work of the tensor-core adjoint: the (channel, output block)
// segments' 16-visibility stages concatenated and cut into one contiguous run
// per CTA; every (CTA, segment) overlap is a unit with its own partial.
void build_units(mem_ctx* c) {
    const int BLK = tca_blk(c->N), nbx = c->N / BLK, nb = nbx * nbx;
    std::vector<int64_t> seg_st;  // stage count per segment (c, blk)
    int64_t T = 0;
    for (int ch = 0; ch < c->C; ++ch) {
        int64_t z = c->off[ch + 1] - c->off[ch];
        for (int b = 0; b < nb; ++b) {
            int64_t s = (z + TCA_BK - 1) / TCA_BK;
            seg_st.push_back(s);
            T += s;
        }
    }
    c->units_h.clear();
    c->cta_off_h.clear();
    c->cb_off_h.assign((size_t)c->C * nb + 1, 0);
    int G = (int)std::min<int64_t>(c->num_sms, T);
    c->adj_ctas = G;
    if (G <= 0) {
        c->cta_off_h.push_back(0);
        return;
    }
    // CTA g takes global stages [T g / G, T (g+1) / G)
    size_t seg = 0;
    int64_t seg_base = 0;  // first global stage of segment `seg`
    std::vector<int> cb_count((size_t)c->C * nb, 0);
    for (int g = 0; g < G; ++g) {
        c->cta_off_h.push_back((int)c->units_h.size());
        int64_t s0 = T * g / G, s1 = T * (g + 1) / G;
        while (s0 < s1) {
            while (seg < seg_st.size() && seg_base + seg_st[seg] <= s0) {
                seg_base += seg_st[seg];
                ++seg;
            }
            int64_t e = std::min<int64_t>(s1, seg_base + seg_st[seg]);
            int ch = (int)(seg / nb), b = (int)(seg % nb);
            int64_t z0 = c->off[ch], z1 = c->off[ch + 1];
            AdjUnit un;
            un.chan = ch;
            un.block = b;
            un.start = z0 + (s0 - seg_base) * TCA_BK;
            un.count = std::min<int64_t>(z1, z0 + (e - seg_base) * TCA_BK) - un.start;
            c->units_h.push_back(un);
            cb_count[seg] += 1;
            s0 = e;
        }
    }
    c->cta_off_h.push_back((int)c->units_h.size());
    for (size_t i = 0; i < cb_count.size(); ++i) c->cb_off_h[i + 1] = c->cb_off_h[i] + cb_count[i];
}

mem_status check_status(mem_ctx* c) {
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->st), "status readback");
    CK(cudaStreamSynchronize(c->st), "stream synchronize");
    if (hs & DEV_TIMEOUT) {
        cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->st);
        cudaStreamSynchronize(c->st);
        return fail(c, MEM_ETIMEOUT, "a bounded device-side wait ran out (spin_limit %llu)",
                    (unsigned long long)c->spin);
    }
    return MEM_OK;
}

mem_status after_launch(mem_ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return MEM_OK;
}

// Buffers needed by the current precision.
mem_status ensure_buffers(mem_ctx* c) {
    const size_t NN = (size_t)c->N * c->N;
    TRY(dalloc(c, &c->chi_part, (size_t)4 * std::max(std::max(c->n_tiles, c->n_tiles_tc), 1)));
    TRY(dalloc(c, &c->ent_part, (size_t)c->n_images * prep_blocks(c->N)));
    TRY(dalloc(c, &c->scal, (size_t)3 + 3 * c->n_images));
    if (!c->img_tmp) {  // holds the scalar reduction's completion counter, which starts at zero
        TRY(dalloc(c, &c->img_tmp, (size_t)scalars_tmp_doubles(c->n_images)));
        CK(cudaMemsetAsync(c->img_tmp, 0, scalars_tmp_doubles(c->n_images) * sizeof(double), c->st),
           "scalar reduction buffer");
    }
    TRY(dalloc(c, &c->y32, (size_t)std::max<int64_t>(c->Z, 1)));
    if (c->prec == MEM_PREC_FP64_DIRECT) {
        TRY(dalloc(c, &c->y64, (size_t)std::max<int64_t>(c->Z, 1)));
        TRY(dalloc(c, &c->bf64, (size_t)c->C * NN));
    } else if (c->prec == MEM_PREC_FP32_DIRECT) {
        TRY(dalloc(c, &c->bf32, (size_t)c->C * NN));
    } else {
        TRY(dalloc(c, &c->planes, (size_t)2 * c->C * NN));
        TRY(dalloc(c, &c->cmean, (size_t)c->C * c->N));
        if (!c->col_count) {
            TRY(dalloc(c, &c->col_count, (size_t)c->C));
            CK(cudaMemsetAsync(c->col_count, 0, (size_t)c->C * sizeof(unsigned), c->st), "column-mean counters");
        }
        TRY(dalloc(c, &c->col_psum, (size_t)colmean_tmp_count(c->N, c->C)));
        TRY(dalloc(c, &c->col_pmax, (size_t)colmean_tmp_count(c->N, c->C)));
        TRY(dalloc(c, &c->cscale, (size_t)c->C));
        TRY(dalloc(c, &c->ymax, (size_t)1));
        TRY(dalloc(c, &c->ymax_part, (size_t)256));
        const int BLK = tca_blk(c->N);
        TRY(dalloc(c, &c->partial, std::max<size_t>(c->units_h.size(), 1) * BLK * BLK));
        if (c->N <= 256)
            TRY(dalloc(c, &c->vpart, (size_t)(c->N / fwd_rs_ks(c->N)) * std::max<int64_t>(c->Z, 1)));
    }
    int ks = 1;
    if (!is_tc(c->prec)) ks = adj_direct_splits(c->dd(), c->num_sms);
    if (ks > c->gsum_ks) {
        // grow: the old block stays allocated until destroy (rare)
        c->gsum = nullptr;
        TRY(dalloc(c, &c->gsum, (size_t)ks * c->C * NN));
        c->gsum_ks = ks;
    }
    return MEM_OK;
}

int bformat(int prec) {
    return prec == MEM_PREC_FP64_DIRECT   ? BF_F64
           : prec == MEM_PREC_FP32_DIRECT ? BF_F32
           : prec == MEM_PREC_FP16X3      ? BF_F16X3
                                          : BF_BF16X3;
}
void* bbuf(mem_ctx* c) {
    return c->prec == MEM_PREC_FP64_DIRECT ? (void*)c->bf64
           : c->prec == MEM_PREC_FP32_DIRECT ? (void*)c->bf32 : (void*)c->planes;
}

// prep + forward for one image source.  mode: FwdMode.  defer_scalars: the
// objective's scalar reduction is left to a later launch (the gradient's).
mem_status run_forward(mem_ctx* c, const ImgSrc& src, int mode, bool entropy, void* yout,
                       bool defer_scalars = false) {
    DevData d = c->dd();
    const bool tc = is_tc(c->prec);
    const int f16 = c->prec == MEM_PREC_FP16X3;
    // FP16X3: the weighted residual's maximum for the adjoint's operand scale
    // (zeroed by the column-mean kernel)
    float* ymax = (tc && f16 && mode == FWD_RESID) ? c->ymax : nullptr;
    if (tc) {
        KTimer t(c, "colmean");
        launch_colmean(d, src, c->cmean, c->cscale, c->col_psum, c->col_pmax, c->col_count, ymax, c->st);
        c->launches++;
    }
    {
        KTimer t(c, "prep");
        launch_prep(d, src, bformat(c->prec), bbuf(c), entropy ? c->ent_part : nullptr, tc ? c->cmean : nullptr,
                    c->cscale, c->st);
    }
    c->launches++;
    TRY(after_launch(c, "prep kernel"));
    if (tc && c->fwd_kernel == MEM_FWD_RESIDENT) {
        KTimer t(c, "fwd_rs");
        launch_fwd_rs(d, f16, c->tiles_tc, c->n_tiles_tc, c->planes, c->cmean, c->cscale, mode, (float2*)yout,
                      c->chi_part, ymax, c->vpart, c->Z, c->num_sms, c->spin, c->dstatus, c->st);
        if (c->n_tiles_tc > 0) c->launches++;  // + the slice combination
    } else if (tc) {
        KTimer t(c, "fwd_tc");
        launch_fwd_tc(d, f16, c->tiles_tc, c->n_tiles_tc, c->planes, c->cmean, c->cscale, mode, (float2*)yout,
                      c->chi_part, ymax, c->num_sms, c->spin, c->dstatus, c->st);
    } else {
        KTimer t(c, c->prec == MEM_PREC_FP64_DIRECT ? "fwd_direct_f64" : "fwd_direct_f32");
        launch_fwd_direct(d, c->prec == MEM_PREC_FP64_DIRECT, c->tiles, c->n_tiles, bbuf(c), mode, yout,
                          c->chi_part, c->st);
    }
    if ((tc ? c->n_tiles_tc : c->n_tiles) > 0) c->launches++;
    TRY(after_launch(c, "forward kernel"));
    if (mode != FWD_VIS && !defer_scalars) {
        KTimer t(c, "scalars");
        launch_scalars(d, tc ? c->tile_off_tc : c->tile_off, c->chi_part, c->ent_part, entropy ? 1 : 0,
                       c->scal, c->img_tmp, c->st);
        c->launches++;
        TRY(after_launch(c, "scalar reduction"));
    }
    return MEM_OK;
}

// adjoint of y (already in y32 / y64) into gsum; returns ks used.
// ymax_ready: the FP16X3 operand scale's maximum was written by the RESID
// forward that produced y32.
mem_status run_adjoint(mem_ctx* c, int* ks_out, bool ymax_ready = false, bool reduce = true) {
    DevData d = c->dd();
    if (is_tc(c->prec)) {
        const int f16 = c->prec == MEM_PREC_FP16X3;
        if (f16 && !ymax_ready) {
            KTimer t(c, "ymax");
            launch_absmax(2 * c->Z, (const float*)c->y32, c->ymax_part, c->ymax, c->st);
            c->launches += 2;
        }
        if (c->adj_ctas > 0) {
            KTimer t(c, "adj_tc");
            launch_adj_tc(d, f16, c->units, c->cta_off, c->adj_ctas, c->y32, c->ymax, c->partial, c->spin,
                          c->dstatus, c->st);
            c->launches++;
            TRY(after_launch(c, "adjoint kernel"));
        }
        *ks_out = 1;
        if (!reduce) return MEM_OK;
        KTimer t(c, "adj_tc_reduce");
        launch_adj_tc_reduce(d, c->units, c->cb_off, c->partial, f16 ? c->ymax : nullptr, c->gsum, c->st);
        c->launches++;
        TRY(after_launch(c, "adjoint reduction"));
        *ks_out = 1;
    } else {
        int ks = adj_direct_splits(d, c->num_sms);
        const void* y = c->prec == MEM_PREC_FP64_DIRECT ? (const void*)c->y64 : (const void*)c->y32;
        KTimer t(c, c->prec == MEM_PREC_FP64_DIRECT ? "adj_direct_f64" : "adj_direct_f32");
        launch_adj_direct(d, c->prec == MEM_PREC_FP64_DIRECT, y, c->gsum, ks, c->st);
        c->launches++;
        TRY(after_launch(c, "adjoint kernel"));
        *ks_out = ks;
    }
    return MEM_OK;
}

// Objective + gradient at `src`; gradient outputs optional.
mem_status run_objgrad(mem_ctx* c, const ImgSrc& src, int projected, float* out32, double* full64,
                       double* proj64) {
    TRY(ensure_buffers(c));
    void* yout = c->prec == MEM_PREC_FP64_DIRECT ? (void*)c->y64 : (void*)c->y32;
    // images of one channel each: the adjoint's unit-partial sum, the
    // gradient assembly and the objective's scalar reduction are one launch
    const bool fused = is_tc(c->prec) && !c->shared;
    TRY(run_forward(c, src, FWD_RESID, true, yout, fused));
    int ks = 1;
    TRY(run_adjoint(c, &ks, true, !fused));
    if (fused) {
        KTimer t(c, "adj_reduce_grad");
        ScalarArgs sc;
        sc.tile_off = c->tile_off_tc;
        sc.chi_part = c->chi_part;
        sc.ent_part = c->ent_part;
        sc.with_entropy = 1;
        sc.scal = c->scal;
        sc.img_tmp = c->img_tmp;
        launch_adj_tc_reduce_grad(c->dd(), src, c->cb_off, c->partial, c->prec == MEM_PREC_FP16X3 ? c->ymax : nullptr,
                                  projected, out32, full64, proj64, sc, c->st);
    } else {
        KTimer t(c, "finalize");
        launch_finalize(c->dd(), src, c->gsum, ks, projected, out32, full64, proj64, c->st);
    }
    c->launches++;
    return after_launch(c, "gradient assembly");
}

void drop_graph(mem_ctx::GraphSlot& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = mem_ctx::GraphSlot();
}

void drop_graphs(mem_ctx* c) {
    drop_graph(c->g_objgrad);
    if (c->g_solve.exec) cudaGraphExecDestroy(c->g_solve.exec);
    c->g_solve = mem_ctx::SolveGraph();
}

// Run `body` (kernel launches on c->st only) through the graph slot: replay
// when the slot was captured for the same keys, else capture and replay.
// Buffers must already exist (no allocation inside a capture).
mem_status graphed(mem_ctx* c, mem_ctx::GraphSlot& g, const void* k1, const void* k2, int k3,
                   const std::function<mem_status()>& body) {
    if (!c->graphs || c->profiling) return body();
    if (!(g.exec && g.k1 == k1 && g.k2 == k2 && g.k3 == k3 && g.prec == c->prec)) {
        drop_graph(g);
        if (!c->cap_st) CK(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking), "capture stream");
        cudaStream_t user = c->st;
        c->st = c->cap_st;
        const int64_t l0 = c->launches;
        cudaError_t e = cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            c->st = user;
            return cuda_fail(c, e, "begin capture");
        }
        mem_status s = body();
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(c->cap_st, &graph);
        c->st = user;
        const int64_t n = c->launches - l0;
        c->launches = l0;
        if (s != MEM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return cuda_fail(c, e, "graph instantiate");
        }
        g.k1 = k1;
        g.k2 = k2;
        g.k3 = k3;
        g.prec = c->prec;
        g.nlaunch = n;
    }
    CK(cudaGraphLaunch(g.exec, c->st), "graph launch");
    c->launches += g.nlaunch;
    return MEM_OK;
}

mem_status read_scalars(mem_ctx* c, std::vector<double>& out) {
    out.resize(3 + 3 * (size_t)c->n_images);
    const size_t n = out.size();
    if (c->hscal_n < n + 1) {  // the scalars, then the status word
        if (c->hscal) cudaFreeHost(c->hscal);
        c->hscal = nullptr;
        c->hscal_n = 0;
        if (cudaMallocHost((void**)&c->hscal, (n + 1) * sizeof(double)) == cudaSuccess) c->hscal_n = n + 1;
        else cudaGetLastError();  // pageable fallback below
    }
    if (c->hscal) {
        // both words in pinned memory: two asynchronous copies, one synchronisation
        int* hs = (int*)(c->hscal + n);
        CK(cudaMemcpyAsync(c->hscal, c->scal, n * sizeof(double), cudaMemcpyDeviceToHost, c->st), "scalar readback");
        CK(cudaMemcpyAsync(hs, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->st), "status readback");
        CK(cudaStreamSynchronize(c->st), "stream synchronize");
        if (*hs & DEV_TIMEOUT) TRY(check_status(c));
        std::copy(c->hscal, c->hscal + n, out.begin());
    } else {
        CK(cudaMemcpyAsync(out.data(), c->scal, n * sizeof(double), cudaMemcpyDeviceToHost, c->st),
           "scalar readback");
        TRY(check_status(c));
    }
    for (double x : out)
        if (!std::isfinite(x)) return fail(c, MEM_ENUMERIC, "objective is not finite (pixels <= 0?)");
    return MEM_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

void msk::set_global_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {

// ---------------------------------------------------------------------------
// Autotuner.  Candidates: forward image column block BN in {128, 256} (N >=
// 256; the operand planes are laid out per BN) and pipeline depth {3, 4};
// adjoint pipeline depth {2, 3}.  Each candidate is timed with per-kernel
// CUDA events over a few full objective + gradient evaluations of the
// context's own data; the fastest is kept and recorded in a cache file
// (MEMSYNTH_TUNE_CACHE, default $HOME/.cache/libmemsynth_tune.txt) keyed by
// device name, N, log2 of the visibility count, channel count and form.
// ---------------------------------------------------------------------------
std::string tune_key(const mem_ctx* c) {
    int zb = 0;
    while (((int64_t)1 << (zb + 1)) <= std::max<int64_t>(c->Z, 1)) ++zb;
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|N=%d|z=%d|C=%d|prec=%d", c->gpu_name.c_str(), c->N, zb, c->C, c->prec);
    std::string k = buf;
    for (char& ch : k)
        if (ch == ' ') ch = '_';
    return k;
}

std::string tune_path() {
    const char* p = std::getenv("MEMSYNTH_TUNE_CACHE");
    if (p && *p) return p;
    const char* h = std::getenv("HOME");
    return std::string(h ? h : ".") + "/.cache/libmemsynth_tune.txt";
}

bool tune_valid(const mem_ctx* c, const mem_tiling_t& t) {
    if (!(t.adj_stages == 2 || t.adj_stages == 3) || adj_tc_smem_bytes(c->N, t.adj_stages) > 227 * 1024)
        return false;
    if (t.fwd_kernel == MEM_FWD_RESIDENT)
        return c->N <= 256 && t.fwd_stages >= 4 && t.fwd_stages <= fwd_rs_max_stages(c->N);
    if (t.fwd_kernel != MEM_FWD_STREAM) return false;
    // the epilogue reduces 32-column pairs of 16-column chunks
    const int bn = t.fwd_cols;
    if (bn < 32 || bn > 256 || c->N % bn != 0 || bn % 32 != 0) return false;
    if (!(t.fwd_stages == 3 || t.fwd_stages == 4)) return false;
    return fwd_tc_smem_bytes(c->N, bn, t.fwd_stages) <= 227 * 1024;
}

mem_tiling_t tiling_of(const mem_ctx* c) {
    mem_tiling_t t;
    t.fwd_kernel = c->fwd_kernel;
    t.fwd_cols = c->fwd_kernel == MEM_FWD_RESIDENT ? c->N : c->fwd_bn;
    t.fwd_stages = c->fwd_stages;
    t.adj_stages = c->adj_stages;
    return t;
}

void apply_tiling(mem_ctx* c, const mem_tiling_t& t) {
    c->fwd_kernel = t.fwd_kernel;
    c->fwd_bn = t.fwd_kernel == MEM_FWD_RESIDENT ? c->N : t.fwd_cols;
    c->fwd_stages = t.fwd_stages;
    c->adj_stages = t.adj_stages;
}

// N <= 128: the resident kernel (one row slice, no duplicated work; its
// corrections-first order halves the chi^2 error at a solve's final image);
// N >= 256: the streaming kernel (about 1.7x faster than two resident slices).
void default_tiling(mem_ctx* c) {
    mem_tiling_t t;
    if (c->N <= 128) {
        t.fwd_kernel = MEM_FWD_RESIDENT;
        t.fwd_cols = c->N;
        t.fwd_stages = fwd_rs_max_stages(c->N);
    } else {
        t.fwd_kernel = MEM_FWD_STREAM;
        t.fwd_cols = tc_bn(c->N);
        t.fwd_stages = 4;
    }
    t.adj_stages = 3;
    // very large N: the epilogue's column-mean copies leave room for 3 stages
    if (t.fwd_kernel == MEM_FWD_STREAM && fwd_tc_smem_bytes(c->N, t.fwd_cols, 4) > 227 * 1024) t.fwd_stages = 3;
    apply_tiling(c, t);
}

void tune_load(mem_ctx* c) {
    FILE* f = std::fopen(tune_path().c_str(), "r");
    if (!f) return;
    const std::string key = tune_key(c);
    char k[256];
    mem_tiling_t t;
    while (std::fscanf(f, "%255s %d %d %d %d", k, &t.fwd_kernel, &t.fwd_cols, &t.fwd_stages, &t.adj_stages) == 5)
        if (key == k && tune_valid(c, t)) apply_tiling(c, t);
    std::fclose(f);
}

void tune_store(const mem_ctx* c) {
    const std::string path = tune_path();
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        const std::string dir = path.substr(0, slash);
        for (size_t i = 1; i <= dir.size(); ++i)  // create the directory without a shell
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    }
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) return;
    const mem_tiling_t t = tiling_of(c);
    std::fprintf(f, "%s %d %d %d %d\n", tune_key(c).c_str(), t.fwd_kernel, t.fwd_cols, t.fwd_stages, t.adj_stages);
    std::fclose(f);
}

}  // namespace


namespace {

// ---------------------------------------------------------------------------
// The solve's launch sequences (projected PR-CG, Eq. minproblem), shared by
// the graph and by the host-driven path (graphs off, or per-kernel timing).
// Non-zero handles are the conditional nodes the controller kernels steer.
// ---------------------------------------------------------------------------
mem_status solve_prologue(mem_ctx* c, unsigned long long h_outer) {
    ImgSrc src{nullptr, c->I64, nullptr, nullptr, c->G, 0};
    TRY(run_objgrad(c, src, 1, nullptr, c->gf64, c->g64));
    launch_cg_init(c->n_images, c->cg_st, c->cg_ctl, c->scal, c->cg_hist, c->dstatus, h_outer, c->st);
    c->launches++;
    return after_launch(c, "solver start");
}

// beta, direction (and its restart), slope, curvature, first trial step
mem_status solve_iter_head(mem_ctx* c, unsigned long long h_inner) {
    const DevData d = c->dd();
    const int NI = c->n_images;
    cudaStream_t st = c->st;
    launch_dots(d, DOT_BETA, c->g64, c->gp64, nullptr, c->dpart, c->dots, st);
    launch_cg_beta(NI, c->cg_st, c->cg_ctl, c->dots, c->beta, c->mode, st);
    launch_cg_direction(d, c->I64, c->g64, c->beta, c->mode, c->d64, st);
    launch_dots(d, DOT_SLOPE, c->gf64, c->d64, c->g64, c->dpart, c->dots, st);
    launch_cg_slope(NI, c->cg_st, c->dots, c->beta, c->mode, st);
    launch_cg_direction(d, c->I64, c->g64, c->beta, c->mode, c->d64, st);
    launch_dots(d, DOT_SLOPE, c->gf64, c->d64, c->g64, c->dpart, c->dots, st);
    launch_cg_slope2(NI, c->cg_st, c->cg_ctl, c->dots, c->mode, st);
    c->launches += 11;
    TRY(after_launch(c, "search direction"));
    // quadratic model of chi^2 along d: curvature sum w |F(A d)|^2
    ImgSrc src{nullptr, c->d64, nullptr, nullptr, c->G, 0};
    TRY(run_forward(c, src, FWD_CURV, false, nullptr));
    launch_dots(d, DOT_MAX, c->I64, c->d64, nullptr, c->dpart, c->dots, st);
    launch_ls_start(NI, c->cg_st, c->cg_ctl, c->scal, c->dots, c->alpha, c->dstatus, h_inner, st);
    c->launches += 3;
    return after_launch(c, "line search start");
}

// one line-search probe: phi(alpha) = Phi(I) + [Phi(max(I + alpha d, G)) -
// Phi(I)], the change evaluated from the image difference so that its
// rounding error scales with the step, not with Phi
mem_status solve_probe(mem_ctx* c, unsigned long long h_inner) {
    ImgSrc src{nullptr, c->I64, c->d64, c->alpha, c->G, 1};
    void* ybuf = c->prec == MEM_PREC_FP64_DIRECT ? (void*)c->y64 : (void*)c->y32;
    TRY(run_forward(c, src, FWD_DCHI, true, ybuf));
    launch_ls_feed(c->n_images, c->cg_st, c->cg_ctl, c->scal, c->alpha, c->dstatus, h_inner, c->st);
    c->launches++;
    return after_launch(c, "line search");
}

// accepted step, new gradient, history row, loop condition
mem_status solve_iter_tail(mem_ctx* c, unsigned long long h_outer) {
    const DevData d = c->dd();
    const int NI = c->n_images;
    const size_t n = (size_t)NI * c->N * c->N;
    cudaStream_t st = c->st;
    launch_cg_finish(NI, c->cg_st, c->cg_ctl, c->alpha, st);
    launch_cg_step(d, c->I64, c->d64, c->alpha, st);
    c->launches += 2;
    CK(cudaMemcpyAsync(c->gp64, c->g64, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy g");
    ImgSrc src{nullptr, c->I64, nullptr, nullptr, c->G, 0};
    TRY(run_objgrad(c, src, 1, nullptr, c->gf64, c->g64));
    launch_cg_record(NI, c->cg_st, c->cg_ctl, c->scal, c->cg_hist, c->dstatus, h_outer, st);
    c->launches++;
    return after_launch(c, "iteration end");
}

// Capture `body` (launches on c->st) into the existing graph g; the number
// of kernel launches it made goes to *nlaunch.
mem_status capture_into(mem_ctx* c, cudaGraph_t g, const std::function<mem_status()>& body, int64_t* nlaunch) {
    if (!c->cap_st) CK(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking), "capture stream");
    cudaStream_t user = c->st;
    c->st = c->cap_st;
    const int64_t l0 = c->launches;
    cudaError_t e = cudaStreamBeginCaptureToGraph(c->cap_st, g, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c->st = user;
        return cuda_fail(c, e, "begin capture");
    }
    mem_status s = body();
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(c->cap_st, &out);
    c->st = user;
    *nlaunch = c->launches - l0;
    c->launches = l0;
    if (s != MEM_OK) return s;
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    return MEM_OK;
}

// Append a conditional WHILE node after the capture's current last nodes; the
// capture continues after it.  *body receives the loop body graph.
mem_status add_while_here(mem_ctx* c, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(c->st, &cs, nullptr, &g, &deps, &edges, &nd), "capture info");
    if (cs != cudaStreamCaptureStatusActive || !g) return fail(c, MEM_ECUDA, "solve graph: no active capture");
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, edges, nd, &p), "conditional node");
    *body = p.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(c->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
       "capture dependencies");
    return MEM_OK;
}

// prologue -> WHILE(iterations) { head -> WHILE(probes) { probe } -> tail }
mem_status build_solve_graph(mem_ctx* c) {
    if (c->g_solve.exec) cudaGraphExecDestroy(c->g_solve.exec);
    c->g_solve = mem_ctx::SolveGraph();
    cudaGraph_t top = nullptr;
    CK(cudaGraphCreate(&top, 0), "graph create");
    auto done = [&](mem_status s) {
        cudaGraphDestroy(top);
        return s;
    };
    cudaGraphConditionalHandle h_outer = 0, h_inner = 0;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h_outer, top, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "conditional handle"));
    cudaGraph_t body_outer = nullptr, body_inner = nullptr;
    mem_ctx::SolveGraph sg;
    mem_status s = capture_into(c, top, [&]() -> mem_status {
        TRY(solve_prologue(c, h_outer));
        return add_while_here(c, h_outer, &body_outer);
    }, &sg.n_pro);
    if (s != MEM_OK) return done(s);
    e = cudaGraphConditionalHandleCreate(&h_inner, body_outer, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "conditional handle"));
    s = capture_into(c, body_outer, [&]() -> mem_status {
        TRY(solve_iter_head(c, h_inner));
        TRY(add_while_here(c, h_inner, &body_inner));
        return solve_iter_tail(c, h_outer);
    }, &sg.n_iter);
    if (s != MEM_OK) return done(s);
    s = capture_into(c, body_inner, [&]() { return solve_probe(c, h_inner); }, &sg.n_probe);
    if (s != MEM_OK) return done(s);
    e = cudaGraphInstantiate(&sg.exec, top, 0);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "solve graph instantiate"));
    sg.prec = c->prec;
    sg.hist = c->cg_hist;
    c->g_solve = sg;
    return done(MEM_OK);
}

}  // namespace

extern "C" {

const char* mem_status_string(mem_status s) {
    switch (s) {
        case MEM_OK: return "ok";
        case MEM_EINVAL: return "invalid argument";
        case MEM_ENOMEM: return "out of device memory";
        case MEM_ECUDA: return "CUDA error";
        case MEM_ETIMEOUT: return "device wait timed out";
        case MEM_ENUMERIC: return "non-finite objective";
        case MEM_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

const char* mem_last_error(const mem_ctx* c) { return c ? c->err.c_str() : g_last_error.c_str(); }

int64_t mem_num_vis(const mem_ctx* c) { return c ? c->Z : 0; }
int32_t mem_num_images(const mem_ctx* c) { return c ? c->n_images : 0; }
int64_t mem_launch_count(const mem_ctx* c) { return c ? c->launches : 0; }
const double* mem_scalars_dev(const mem_ctx* c) { return c ? c->scal : nullptr; }

mem_status mem_profile(mem_ctx* c, int32_t enable) {
    if (!c) return fail(nullptr, MEM_EINVAL, "null context");
    c->profiling = enable != 0;
    return MEM_OK;
}

int32_t mem_profile_read(mem_ctx* c, int32_t max_kernels, char* names, double* ms_total,
                         int64_t* launches) {
    if (!c) return -1;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return -1;
    for (auto& k : c->kev) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, k.a, k.b);
        auto& acc = c->kacc[k.name];
        acc.first += ms;
        acc.second += 1;
        c->ev_pool.push_back(k.a);
        c->ev_pool.push_back(k.b);
    }
    c->kev.clear();
    int32_t i = 0;
    for (auto& kv : c->kacc) {
        if (i >= max_kernels) break;
        if (names) {
            std::strncpy(names + 32 * i, kv.first.c_str(), 31);
            names[32 * i + 31] = 0;
        }
        if (ms_total) ms_total[i] = kv.second.first;
        if (launches) launches[i] = kv.second.second;
        ++i;
    }
    c->kacc.clear();
    return i;
}

mem_status mem_autotune(mem_ctx* c, const float* image_dev, int32_t reps, mem_tiling_t* choice_out) {
    if (!c || !image_dev) return fail(c, MEM_EINVAL, "null argument");
    if (!is_tc(c->prec)) {
        if (choice_out) *choice_out = tiling_of(c);
        return MEM_OK;  // nothing to tune for the direct forms
    }
    if (reps <= 0) reps = 3;
    TRY(ensure_buffers(c));
    const bool prof0 = c->profiling;
    c->profiling = true;
    // mean per-launch time of the named kernels over `reps` evaluations
    auto time_kernels = [&](std::initializer_list<const char*> names, double* best) -> mem_status {
        ImgSrc src{image_dev, nullptr, nullptr, nullptr, c->G, 0};
        TRY(run_objgrad(c, src, 0, nullptr, nullptr, nullptr));  // warm-up
        mem_profile_read(c, 0, nullptr, nullptr, nullptr);
        for (int r = 0; r < reps; ++r) TRY(run_objgrad(c, src, 0, nullptr, nullptr, nullptr));
        char nm[32 * 32];
        double ms[32];
        int64_t cnt[32];
        const int n = mem_profile_read(c, 32, nm, ms, cnt);
        double tot = 0.0;
        bool seen = false;
        for (int i = 0; i < n; ++i)
            for (const char* want : names)
                if (std::strcmp(nm + 32 * i, want) == 0) {
                    tot += ms[i] / (double)reps;
                    seen = true;
                }
        *best = seen ? tot : 1e300;
        return check_status(c);
    };
    std::vector<mem_tiling_t> fwd;
    for (int k : {MEM_FWD_RESIDENT, MEM_FWD_STREAM})
        for (int bn : {256, 128, 64})
            for (int fs : {6, 5, 4, 3}) {
                mem_tiling_t t{k, k == MEM_FWD_RESIDENT ? c->N : bn, fs, c->adj_stages};
                if (k == MEM_FWD_RESIDENT && bn != 256) continue;  // one column choice
                if (k == MEM_FWD_STREAM && !(bn == tc_bn(c->N) || (c->N >= 256 && bn == 128))) continue;
                if (k == MEM_FWD_STREAM && c->N <= 128) continue;  // accuracy: resident only
                if (tune_valid(c, t)) fwd.push_back(t);
            }
    mem_tiling_t best = tiling_of(c);
    double best_f = 1e300, best_a = 1e300;
    mem_status st = MEM_OK;
    for (const mem_tiling_t& t : fwd) {
        apply_tiling(c, t);
        double ms = 0;
        // the resident kernel's slice combination is part of its cost
        if ((st = time_kernels({"fwd_tc", "fwd_rs"}, &ms)) != MEM_OK) break;
        if (ms < best_f) {
            best_f = ms;
            best = t;
        }
    }
    for (int as : {3, 2}) {
        mem_tiling_t t = best;
        t.adj_stages = as;
        if (st != MEM_OK || !tune_valid(c, t)) continue;
        apply_tiling(c, t);
        double ms = 0;
        if ((st = time_kernels({"adj_tc"}, &ms)) != MEM_OK) break;
        if (ms < best_a) {
            best_a = ms;
            best.adj_stages = as;
        }
    }
    apply_tiling(c, best);
    c->profiling = prof0;
    drop_graphs(c);
    if (st != MEM_OK) return st;
    tune_store(c);
    if (choice_out) *choice_out = best;
    return MEM_OK;
}

mem_status mem_set_tiling(mem_ctx* c, const mem_tiling_t* t) {
    if (!c || !t) return MEM_EINVAL;
    if (!is_tc(c->prec)) return fail(c, MEM_EINVAL, "tiling applies to the tensor-core forms only");
    mem_tiling_t x = *t;
    if (x.fwd_kernel == MEM_FWD_RESIDENT) x.fwd_cols = c->N;
    if (!tune_valid(c, x))
        return fail(c, MEM_EINVAL,
                    "tiling: streaming kernel needs a column block dividing N (32..256, multiple of 32) and 3|4 "
                    "stages; resident kernel N <= 256 and 4..%d stages; adjoint 2|3 stages",
                    c->N <= 256 ? fwd_rs_max_stages(c->N) : 0);
    TRY(mem_sync(c));
    apply_tiling(c, x);
    drop_graphs(c);
    return MEM_OK;
}

mem_status mem_tiling(const mem_ctx* c, mem_tiling_t* out) {
    if (!c || !out) return MEM_EINVAL;
    *out = tiling_of(c);
    return MEM_OK;
}

mem_status mem_forward_gridded(mem_ctx* c, const float* image_dev, int32_t pad, float* vis_dev) {
    if (!c || !image_dev || (!vis_dev && c->Z > 0)) return fail(c, MEM_EINVAL, "null argument");
    if (pad < 1 || pad > 8) return fail(c, MEM_EINVAL, "gridded forward: pad must be 1..8 (got %d)", pad);
    const int M = pad * c->N;
    if (!grid_fft_size_ok(c->N, M))
        return fail(c, MEM_EINVAL, "gridded forward: needs an even N and pad * N <= %d (N = %d, pad = %d)",
                    GRID_FFT_MAX, c->N, pad);
    const size_t H = (size_t)M / 2 + 1;
    if (c->grid_pad != pad) {
        TRY(mem_sync(c));
        if (c->grid_pad) {
            const size_t oM = (size_t)c->grid_pad * c->N, oH = oM / 2 + 1;
            dfree(c, &c->grid_R, (size_t)c->C * oH * c->N);
            dfree(c, &c->grid_F, (size_t)c->C * oM * oH);
        }
        c->grid_pad = 0;
        TRY(dalloc(c, &c->grid_R, (size_t)c->C * H * c->N));
        TRY(dalloc(c, &c->grid_F, (size_t)c->C * M * H));
        c->grid_pad = pad;
    }
    DevData d = c->dd();
    {
        KTimer t(c, "grid_fft");
        launch_grid_fft(d, image_dev, M, c->grid_R, c->grid_F, c->st);
        c->launches += 2;
    }
    TRY(after_launch(c, "gridded forward: 2-D transform"));
    {
        KTimer t(c, "grid_interp");
        launch_grid_interp(d, M, c->grid_F, c->Z, (float2*)vis_dev, c->st);
        if (c->Z > 0) c->launches++;
    }
    return after_launch(c, "gridded forward: interpolation");
}

namespace {
// Shared by the dirty image, the PSF and the residual map: natural weights
// times the chosen visibilities (already in y32 / y64 for residuals), then the
// adjoint without the beam factor.
mem_status dirty_from(mem_ctx* c, int what, float* out_dev) {
    if (!c->wsum) {
        TRY(dalloc(c, &c->wsum, (size_t)c->C));
        CK(cudaMemcpyAsync(c->wsum, c->wsum_h.data(), c->C * sizeof(double), cudaMemcpyHostToDevice, c->st),
           "weight sums");
    }
    DevData d = c->dd();
    launch_dirty_y(d, c->wsum, what, c->Z, c->y32, c->prec == MEM_PREC_FP64_DIRECT ? c->y64 : nullptr, c->st);
    if (c->Z > 0) c->launches++;
    TRY(after_launch(c, "dirty image weights"));
    int ks = 1;
    TRY(run_adjoint(c, &ks));
    launch_dirty_out(d, c->gsum, ks, out_dev, c->st);
    c->launches++;
    return after_launch(c, "dirty image");
}
}  // namespace

mem_status mem_dirty_image(mem_ctx* c, int32_t psf, float* out_dev) {
    if (!c || !out_dev) return fail(c, MEM_EINVAL, "null argument");
    TRY(ensure_buffers(c));
    return dirty_from(c, psf ? 1 : 0, out_dev);
}

mem_status mem_residual_image(mem_ctx* c, const float* image_dev, float* out_dev) {
    if (!c || !out_dev || !image_dev) return fail(c, MEM_EINVAL, "null argument");
    TRY(ensure_buffers(c));
    ImgSrc src{image_dev, nullptr, nullptr, nullptr, c->G, 0};
    void* model = c->prec == MEM_PREC_FP64_DIRECT ? (void*)c->y64 : (void*)c->y32;
    TRY(run_forward(c, src, FWD_VIS, false, model));
    return dirty_from(c, 2, out_dev);
}

mem_status mem_phase_rotate(int64_t n_vis, const double* u, const double* v, double x_p, double y_p,
                            double* vis) {
    if (n_vis < 0 || (n_vis > 0 && (!u || !v || !vis))) return MEM_EINVAL;
    for (int64_t k = 0; k < n_vis; ++k) {
        double t = u[k] * x_p + v[k] * y_p;  // turns
        t -= std::floor(t);
        const double cr = std::cos(2 * M_PI * t), sr = -std::sin(2 * M_PI * t);
        const double re = vis[2 * k], im = vis[2 * k + 1];
        vis[2 * k] = re * cr - im * sr;
        vis[2 * k + 1] = re * sr + im * cr;
    }
    return MEM_OK;
}

mem_status mem_beam_fit(const float* psf, int32_t n, double dx, double dy, double* out4) {
    if (!psf || !out4 || n < 3 || !(dx > 0) || !(dy > 0)) return MEM_EINVAL;
    const int c0 = n / 2;
    const double p0 = psf[(int64_t)c0 * n + c0];
    if (!(p0 > 0)) return MEM_EINVAL;
    // main lobe: 4-connected to the centre, above BEAM_LOBE of the peak
    const double lobe = 0.35;
    std::vector<char> seen((size_t)n * n, 0);
    std::vector<int> stack{c0 * n + c0};
    seen[(size_t)c0 * n + c0] = 1;
    double S[3][3] = {{0}}, R[3] = {0};
    while (!stack.empty()) {
        const int q = stack.back();
        stack.pop_back();
        const int a = q / n, b = q % n;
        const double x = (b - c0) * dx, y = (a - c0) * dy;
        const double f[3] = {x * x, x * y, y * y};
        const double r = -std::log(psf[q] / p0);
        for (int i = 0; i < 3; ++i) {
            R[i] += f[i] * r;
            for (int j = 0; j < 3; ++j) S[i][j] += f[i] * f[j];
        }
        const int nb[4][2] = {{a + 1, b}, {a - 1, b}, {a, b + 1}, {a, b - 1}};
        for (auto& t : nb)
            if (t[0] >= 0 && t[0] < n && t[1] >= 0 && t[1] < n && !seen[(size_t)t[0] * n + t[1]] &&
                psf[(size_t)t[0] * n + t[1]] > lobe * p0) {
                seen[(size_t)t[0] * n + t[1]] = 1;
                stack.push_back(t[0] * n + t[1]);
            }
    }
    // normal equations S (A, B, C) = R by Cramer's rule
    auto det3 = [](double m[3][3]) {
        return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
               m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    };
    const double D = det3(S);
    if (!(std::fabs(D) > 0)) return MEM_ENUMERIC;
    double abc[3];
    for (int k = 0; k < 3; ++k) {
        double T[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) T[i][j] = (j == k) ? R[i] : S[i][j];
        abc[k] = det3(T) / D;
    }
    // quadratic form [[A, B/2], [B/2, C]]: eigenvalues and the major axis
    const double A = abc[0], B2 = abc[1] / 2, C = abc[2];
    const double tr = A + C, disc = std::sqrt(std::max(0.0, (A - C) * (A - C) / 4 + B2 * B2));
    const double l_min = tr / 2 - disc, l_max = tr / 2 + disc;
    if (!(l_min > 0)) return MEM_ENUMERIC;
    const double bmaj = 2 * std::sqrt(std::log(2.0) / l_min), bmin = 2 * std::sqrt(std::log(2.0) / l_max);
    // eigenvector of l_min: (B/2, l_min - A) or (l_min - C, B/2)
    double ex = B2, ey = l_min - A;
    if (std::fabs(ex) + std::fabs(ey) < 1e-300 * (std::fabs(A) + std::fabs(C))) {
        ex = l_min - C;
        ey = B2;
    }
    if (std::fabs(ex) + std::fabs(ey) == 0) {  // circular beam
        ex = 0;
        ey = 1;
    }
    double bpa = std::atan2(ex, ey) * 180.0 / M_PI;
    if (bpa <= -90) bpa += 180;
    if (bpa > 90) bpa -= 180;
    out4[0] = bmaj;
    out4[1] = bmin;
    out4[2] = bpa;
    out4[3] = M_PI / (4 * std::log(2.0)) * bmaj * bmin / (dx * dy);
    return MEM_OK;
}

mem_status mem_use_graphs(mem_ctx* c, int32_t enable) {
    if (!c) return fail(nullptr, MEM_EINVAL, "null context");
    c->graphs = enable != 0;
    if (!c->graphs) drop_graphs(c);
    return MEM_OK;
}

void mem_destroy(mem_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    drop_graphs(c);
    if (c->cap_st) cudaStreamDestroy(c->cap_st);
    for (auto& k : c->kev) {
        cudaEventDestroy(k.a);
        cudaEventDestroy(k.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    if (c->hscal) cudaFreeHost(c->hscal);
    delete c;
}

mem_status mem_set_precision(mem_ctx* c, int32_t prec) {
    if (!c) return fail(nullptr, MEM_EINVAL, "null context");
    if (prec < MEM_PREC_FP64_DIRECT || prec > MEM_PREC_FP16X3)
        return fail(c, MEM_EINVAL, "unknown precision %d", prec);
    if (is_tc(prec) && !tc_shape_ok(c->N))
        return fail(c, MEM_ENOTSUP, "tensor-core forms need N = 64, 128 or a multiple of 256 (N = %d)", c->N);
    c->prec = prec;
    drop_graphs(c);
    default_tiling(c);
    if (is_tc(prec)) tune_load(c);
    return ensure_buffers(c);
}

mem_status mem_create(const mem_config* cfg, const double* u, const double* v, const double* vis_obs,
                      const double* sigma, const float* pb, void* stream, mem_ctx** out) {
    if (!out) return fail(nullptr, MEM_EINVAL, "out is null");
    *out = nullptr;
    if (!cfg || !cfg->vis_offsets || !pb) return fail(nullptr, MEM_EINVAL, "null cfg, vis_offsets or pb");
    const int N = cfg->n, C = cfg->n_channels;
    if (N < 16 || N > 4096 || N % 16 != 0) return fail(nullptr, MEM_EINVAL, "n = %d must be a multiple of 16 in [16, 4096]", N);
    if (C < 1) return fail(nullptr, MEM_EINVAL, "n_channels = %d", C);
    if (!(cfg->dx > 0) || !(cfg->dy > 0)) return fail(nullptr, MEM_EINVAL, "pixel size must be > 0");
    if (!(cfg->G > 0) || !(cfg->lambda >= 0) || !std::isfinite(cfg->G) || !std::isfinite(cfg->lambda))
        return fail(nullptr, MEM_EINVAL, "need G > 0 and lambda >= 0");
    if (cfg->precision < MEM_PREC_FP64_DIRECT || cfg->precision > MEM_PREC_FP16X3)
        return fail(nullptr, MEM_EINVAL, "unknown precision %d", cfg->precision);
    if (cfg->image_mode != MEM_IMAGES_PER_CHANNEL && cfg->image_mode != MEM_IMAGE_SHARED)
        return fail(nullptr, MEM_EINVAL, "unknown image mode %d", cfg->image_mode);
    if (is_tc(cfg->precision) && !tc_shape_ok(N))
        return fail(nullptr, MEM_ENOTSUP, "tensor-core forms need N = 64, 128 or a multiple of 256 (N = %d)", N);
    if (cfg->vis_offsets[0] != 0) return fail(nullptr, MEM_EINVAL, "vis_offsets[0] must be 0");
    for (int i = 0; i < C; ++i)
        if (cfg->vis_offsets[i + 1] < cfg->vis_offsets[i]) return fail(nullptr, MEM_EINVAL, "vis_offsets must not decrease");
    const int64_t Z = cfg->vis_offsets[C];
    if (Z > 0 && (!u || !v || !vis_obs || !sigma)) return fail(nullptr, MEM_EINVAL, "null visibility arrays");
    if (Z >= ((int64_t)1 << 40)) return fail(nullptr, MEM_EINVAL, "too many visibilities");
    for (int64_t k = 0; k < Z; ++k)
        if (!(sigma[k] > 0) || !std::isfinite(sigma[k]) || !std::isfinite(u[k]) || !std::isfinite(v[k]))
            return fail(nullptr, MEM_EINVAL, "sigma must be > 0 and u, v finite (index %lld)", (long long)k);

    mem_ctx* c = new mem_ctx();
    c->N = N;
    c->C = C;
    c->shared = cfg->image_mode == MEM_IMAGE_SHARED;
    c->n_images = c->shared ? 1 : C;
    c->prec = cfg->precision;
    c->dx = cfg->dx;
    c->dy = cfg->dy;
    c->lambda = cfg->lambda;
    c->G = cfg->G;
    c->spin = cfg->spin_limit ? cfg->spin_limit : ((uint64_t)1 << 26);
    c->Z = Z;
    c->off.assign(cfg->vis_offsets, cfg->vis_offsets + C + 1);
    c->st = (cudaStream_t)stream;
    c->cap = alloc_cap();

    auto bail = [&](mem_status s) {
        mem_destroy(c);
        return s;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, c->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(nullptr, MEM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e)));
    }
    if (prop.major != 10 || prop.minor != 3)
        return bail(fail(nullptr, MEM_ECUDA, "libmemsynth is built for sm_103a (GB300); device is sm_%d%d",
                         prop.major, prop.minor));
    c->num_sms = prop.multiProcessorCount;
    c->gpu_name = prop.name;

    const size_t NN = (size_t)N * N;
    mem_status s;
    if ((s = dalloc(c, &c->u, std::max<int64_t>(Z, 1))) || (s = dalloc(c, &c->v, std::max<int64_t>(Z, 1))) ||
        (s = dalloc(c, &c->w, std::max<int64_t>(Z, 1))) || (s = dalloc(c, &c->pa, std::max<int64_t>(Z, 1))) ||
        (s = dalloc(c, &c->pb, std::max<int64_t>(Z, 1))) || (s = dalloc(c, &c->vo, std::max<int64_t>(Z, 1))) ||
        (s = dalloc(c, &c->vo32, std::max<int64_t>(Z, 1))) || (s = dalloc(c, &c->w32, std::max<int64_t>(Z, 1))) ||
        (s = dalloc(c, &c->beam, (size_t)C * NN)) || (s = dalloc(c, &c->doff, (size_t)C + 1)) ||
        (s = dalloc(c, &c->dstatus, 1))) {
        g_last_error = c->err;
        return bail(s);
    }
    std::vector<double> wh((size_t)Z);
    for (int64_t k = 0; k < Z; ++k) wh[k] = 1.0 / (sigma[k] * sigma[k]);
    std::vector<float> w32h((size_t)Z);
    std::vector<float4> vo32h((size_t)Z);
    for (int64_t k = 0; k < Z; ++k) {
        w32h[k] = (float)wh[k];
        const double re = vis_obs[2 * k], im = vis_obs[2 * k + 1];
        const float rh = (float)re, ih = (float)im;
        vo32h[k] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
    }
    c->wsum_h.assign((size_t)C, 0.0);
    for (int ch = 0; ch < C; ++ch)
        for (int64_t k = c->off[ch]; k < c->off[ch + 1]; ++k) c->wsum_h[ch] += wh[k];
    auto cpy = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->st) : cudaSuccess;
    };
    e = cpy(c->u, u, Z * sizeof(double));
    if (e == cudaSuccess) e = cpy(c->v, v, Z * sizeof(double));
    if (e == cudaSuccess) e = cpy(c->w, wh.data(), Z * sizeof(double));
    if (e == cudaSuccess) e = cpy(c->vo, vis_obs, Z * 2 * sizeof(double));
    if (e == cudaSuccess) e = cpy(c->w32, w32h.data(), Z * sizeof(float));
    if (e == cudaSuccess) e = cpy(c->vo32, vo32h.data(), Z * sizeof(float4));
    if (e == cudaSuccess) e = cpy(c->beam, pb, C * NN * sizeof(float));
    if (e == cudaSuccess) e = cpy(c->doff, c->off.data(), (C + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->st);
    if (e != cudaSuccess) {
        cuda_fail(c, e, "upload");
        g_last_error = c->err;
        return bail(MEM_ECUDA);
    }
    launch_phase_prep(Z, c->u, c->v, c->dx, c->dy, c->pa, c->pb, c->st);
    c->launches++;

    build_tiles(c, 128, c->tiles_h, c->tile_off_h);
    build_tiles(c, TC_TILE, c->tiles_tc_h, c->tile_off_tc_h);
    c->n_tiles = (int)c->tiles_h.size();
    c->n_tiles_tc = (int)c->tiles_tc_h.size();
    build_units(c);
    if ((s = dalloc(c, &c->tiles, std::max<size_t>(c->tiles_h.size(), 1))) ||
        (s = dalloc(c, &c->tile_off, c->tile_off_h.size())) ||
        (s = dalloc(c, &c->tiles_tc, std::max<size_t>(c->tiles_tc_h.size(), 1))) ||
        (s = dalloc(c, &c->tile_off_tc, c->tile_off_tc_h.size())) ||
        (s = dalloc(c, &c->units, std::max<size_t>(c->units_h.size(), 1))) ||
        (s = dalloc(c, &c->cta_off, c->cta_off_h.size())) || (s = dalloc(c, &c->cb_off, c->cb_off_h.size()))) {
        g_last_error = c->err;
        return bail(s);
    }
    e = cpy(c->tiles, c->tiles_h.data(), c->tiles_h.size() * sizeof(VisTile));
    if (e == cudaSuccess) e = cpy(c->tile_off, c->tile_off_h.data(), c->tile_off_h.size() * sizeof(int));
    if (e == cudaSuccess) e = cpy(c->tiles_tc, c->tiles_tc_h.data(), c->tiles_tc_h.size() * sizeof(VisTile));
    if (e == cudaSuccess)
        e = cpy(c->tile_off_tc, c->tile_off_tc_h.data(), c->tile_off_tc_h.size() * sizeof(int));
    if (e == cudaSuccess) e = cpy(c->units, c->units_h.data(), c->units_h.size() * sizeof(AdjUnit));
    if (e == cudaSuccess) e = cpy(c->cta_off, c->cta_off_h.data(), c->cta_off_h.size() * sizeof(int));
    if (e == cudaSuccess) e = cpy(c->cb_off, c->cb_off_h.data(), c->cb_off_h.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        cuda_fail(c, e, "context setup");
        g_last_error = c->err;
        return bail(MEM_ECUDA);
    }
    default_tiling(c);
    if (is_tc(c->prec)) tune_load(c);
    if ((s = ensure_buffers(c)) != MEM_OK) {
        g_last_error = c->err;
        return bail(s);
    }
    *out = c;
    return MEM_OK;
}

mem_status mem_sync(mem_ctx* c) {
    if (!c) return fail(nullptr, MEM_EINVAL, "null context");
    CK(cudaGetLastError(), "pending launch error");
    return check_status(c);
}

mem_status mem_forward(mem_ctx* c, const float* image_dev, float* vis_dev) {
    if (!c || !image_dev || (!vis_dev && c->Z > 0)) return fail(c, MEM_EINVAL, "null argument");
    if (!aligned(vis_dev, 8)) return fail(c, MEM_EINVAL, "vis_dev must be 8-byte aligned");
    TRY(ensure_buffers(c));
    ImgSrc src{image_dev, nullptr, nullptr, nullptr, c->G, 0};
    if (c->prec == MEM_PREC_FP64_DIRECT) {
        TRY(run_forward(c, src, FWD_VIS, false, c->y64));
        launch_f64_to_f32(2 * c->Z, (const double*)c->y64, vis_dev, c->st);
        c->launches++;
        return after_launch(c, "conversion");
    }
    return run_forward(c, src, FWD_VIS, false, vis_dev);
}

namespace {
__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
    int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p < n) out[p] = (double)in[p];
}
}  // namespace

mem_status mem_adjoint(mem_ctx* c, const float* y_dev, float* img_dev) {
    if (!c || !img_dev || (!y_dev && c->Z > 0)) return fail(c, MEM_EINVAL, "null argument");
    if (!aligned(y_dev, 8)) return fail(c, MEM_EINVAL, "y_dev must be 8-byte aligned");
    TRY(ensure_buffers(c));
    if (c->Z > 0) {
        if (c->prec == MEM_PREC_FP64_DIRECT) {
            k_f32_to_f64<<<(unsigned)((2 * c->Z + 255) / 256), 256, 0, c->st>>>(2 * c->Z, y_dev, (double*)c->y64);
        } else {
            CK(cudaMemcpyAsync(c->y32, y_dev, (size_t)c->Z * sizeof(float2), cudaMemcpyDeviceToDevice, c->st),
               "copy y");
        }
        c->launches += (c->prec == MEM_PREC_FP64_DIRECT);
    }
    int ks = 1;
    TRY(run_adjoint(c, &ks));
    // beam factor and channel sum only: lambda = 0 view of the assembly
    DevData d = c->dd();
    d.lambda = 0.0;
    ImgSrc src{nullptr, nullptr, nullptr, nullptr, c->G, 0};
    // the assembly reads pixel values only for the entropy term and projection;
    // give it the output buffer as a harmless source (lambda = 0, no projection)
    src.f32 = img_dev;
    launch_finalize(d, src, c->gsum, ks, 0, img_dev, nullptr, nullptr, c->st);
    c->launches++;
    return after_launch(c, "adjoint assembly");
}

mem_status mem_objective_grad(mem_ctx* c, const float* image_dev, float* grad_dev, int32_t projected,
                              double* out3_host) {
    if (!c || !image_dev) return fail(c, MEM_EINVAL, "null argument");
    ImgSrc src{image_dev, nullptr, nullptr, nullptr, c->G, 0};
    TRY(ensure_buffers(c));
    TRY(graphed(c, c->g_objgrad, image_dev, grad_dev, projected ? 1 : 0,
                [&]() { return run_objgrad(c, src, projected, grad_dev, nullptr, nullptr); }));
    if (out3_host) {
        std::vector<double> sc;
        TRY(read_scalars(c, sc));
        out3_host[0] = sc[0];
        out3_host[1] = sc[1];
        out3_host[2] = sc[2];
    }
    return MEM_OK;
}

mem_status mem_objective_grad_host(mem_ctx* c, const float* image_host, float* grad_host, int32_t projected,
                                   double* out3_host) {
    if (!c || !image_host) return fail(c, MEM_EINVAL, "null argument");
    const size_t n = (size_t)c->n_images * c->N * c->N;
    TRY(dalloc(c, &c->stage, 2 * n));
    float* dimg = c->stage;
    float* dgrad = grad_host ? c->stage + n : nullptr;
    CK(cudaMemcpyAsync(dimg, image_host, n * sizeof(float), cudaMemcpyHostToDevice, c->st), "image upload");
    TRY(mem_objective_grad(c, dimg, dgrad, projected, nullptr));
    if (grad_host)
        CK(cudaMemcpyAsync(grad_host, dgrad, n * sizeof(float), cudaMemcpyDeviceToHost, c->st), "gradient download");
    std::vector<double> sc;
    TRY(read_scalars(c, sc));
    if (out3_host) {
        out3_host[0] = sc[0];
        out3_host[1] = sc[1];
        out3_host[2] = sc[2];
    }
    return MEM_OK;
}

mem_status mem_solve(mem_ctx* c, float* image_dev_inout, int32_t n_iter, mem_solve_report* rep,
                     double* hist_host) {
    if (!c || !image_dev_inout || n_iter < 0) return fail(c, MEM_EINVAL, "bad argument");
    const int NI = c->n_images;
    const size_t n = (size_t)NI * c->N * c->N;
    TRY(ensure_buffers(c));
    TRY(dalloc(c, &c->I64, n));
    TRY(dalloc(c, &c->d64, n));
    TRY(dalloc(c, &c->g64, n));
    TRY(dalloc(c, &c->gf64, n));
    TRY(dalloc(c, &c->gp64, n));
    TRY(dalloc(c, &c->alpha, (size_t)NI));
    TRY(dalloc(c, &c->beta, (size_t)NI));
    TRY(dalloc(c, &c->mode, (size_t)NI));
    TRY(dalloc(c, &c->dots, (size_t)2 * NI));
    TRY(dalloc(c, &c->dpart, (size_t)2 * NI * prep_blocks(c->N)));
    TRY(dalloc(c, &c->cg_st, (size_t)NI));
    TRY(dalloc(c, &c->cg_ctl, (size_t)1));
    const size_t hist_n = (size_t)NI * (n_iter + 1) * 6;
    if (hist_n > c->cg_hist_cap) {
        // grow: the old block stays allocated until destroy; the solve graph
        // refers to the history buffer and is rebuilt
        c->cg_hist = nullptr;
        TRY(dalloc(c, &c->cg_hist, std::max(hist_n, (size_t)NI * 51 * 6)));
        c->cg_hist_cap = std::max(hist_n, (size_t)NI * 51 * 6);
    }
    cudaStream_t st = c->st;
    CgControl h0;
    std::memset(&h0, 0, sizeof h0);
    h0.n_iter = n_iter;
    h0.hist_stride = n_iter + 1;
    CK(cudaMemcpyAsync(c->cg_ctl, &h0, sizeof h0, cudaMemcpyHostToDevice, st), "solver control");
    launch_clip_f32_to_f64(c->dd(), image_dev_inout, c->I64, st);
    c->launches++;
    TRY(after_launch(c, "image upload"));

    CgControl hc;
    if (c->graphs && !c->profiling) {
        if (!(c->g_solve.exec && c->g_solve.prec == c->prec && c->g_solve.hist == c->cg_hist))
            TRY(build_solve_graph(c));
        CK(cudaGraphLaunch(c->g_solve.exec, st), "solve graph launch");
        CK(cudaMemcpyAsync(&hc, c->cg_ctl, sizeof hc, cudaMemcpyDeviceToHost, st), "solver control");
        CK(cudaStreamSynchronize(st), "solve");
        c->launches += c->g_solve.n_pro + (int64_t)hc.k * c->g_solve.n_iter + hc.probes * c->g_solve.n_probe;
    } else {
        // the same launch sequence, the loops driven from the host
        auto read_ctl = [&]() -> mem_status {
            CK(cudaMemcpyAsync(&hc, c->cg_ctl, sizeof hc, cudaMemcpyDeviceToHost, st), "solver control");
            CK(cudaStreamSynchronize(st), "solver control");
            return MEM_OK;
        };
        TRY(solve_prologue(c, 0));
        for (;;) {
            TRY(read_ctl());
            if (!hc.outer) break;
            TRY(solve_iter_head(c, 0));
            for (;;) {
                TRY(read_ctl());
                if (!hc.inner) break;
                TRY(solve_probe(c, 0));
            }
            TRY(solve_iter_tail(c, 0));
        }
    }
    launch_f64_to_f32((int64_t)n, c->I64, image_dev_inout, st);
    c->launches++;
    TRY(after_launch(c, "image download"));
    std::vector<CgImage> cg(NI);
    std::vector<double> hist((size_t)NI * (n_iter + 1) * 6, 0.0);
    CK(cudaMemcpyAsync(cg.data(), c->cg_st, NI * sizeof(CgImage), cudaMemcpyDeviceToHost, st), "solver state");
    CK(cudaMemcpyAsync(hist.data(), c->cg_hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
       "solver history");
    TRY(check_status(c));
    if (hc.status & CG_NONFINITE) return fail(c, MEM_ENUMERIC, "objective is not finite (pixels <= 0?)");
    if (hc.status & CG_LOOP) return fail(c, MEM_ENUMERIC, "a line search did not end within its evaluation budget");
    // rows after the last iteration repeat the final objective
    for (int i = 0; i < NI; ++i)
        for (int k = hc.k + 1; k <= n_iter; ++k) {
            double* r = &hist[((size_t)i * (n_iter + 1) + k) * 6];
            r[0] = cg[i].phi;
            r[1] = cg[i].chi;
            r[2] = cg[i].S;
            r[3] = r[4] = r[5] = 0.0;
        }
    if (hist_host) std::memcpy(hist_host, hist.data(), hist.size() * sizeof(double));
    if (rep) {
        rep->iterations = 0;
        rep->evaluations = 0;
        rep->status = MEM_OK;
        rep->stopped_early = hc.stopped_early;
        rep->phi = rep->chi2 = rep->entropy = 0.0;
        for (int i = 0; i < NI; ++i) {
            rep->iterations = std::max(rep->iterations, cg[i].iters);
            rep->evaluations += cg[i].evals;
            rep->phi += cg[i].phi;
            rep->chi2 += cg[i].chi;
            rep->entropy += cg[i].S;
        }
    }
    return MEM_OK;
}

}  // extern "C"
