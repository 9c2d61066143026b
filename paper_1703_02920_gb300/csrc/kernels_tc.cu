// Tensor-core (tcgen05) adjoint of the measurement operator (the forward
// operator is in kernels_fwd.cu).
//
// On the regular pixel grid the phase of Eq. (1) separates,
//   exp(-2 pi i (u x_m + v y_n)) = Ex[k,m] Ey[k,n],
//   Ex[k,m] = exp(-2 pi i u_k x_m),  Ey[k,n] = exp(-2 pi i v_k y_n),
// so the forward sum is   V_k = sum_m Ex[k,m] T[k,m],  T = Ey B^T  (B = A*I),
// and the chi^2 gradient (Eq. chi2gradient, Appendix C) is
//   G[n,m] = sum_k Re(Ey)[k,n] Re(P)[k,m] + Im(Ey)[k,n] Im(P)[k,m],
//   P[k,m] = y_k conj(Ex[k,m]),  y = w r.
// Both contractions run on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, accumulators in TMEM) in a 3-term FP16 or BF16 split: x = hi + lo,
// a b ~= a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32 accumulation.  The phase
// tables are never stored: producer warps generate each tile in shared
// memory from the exact fixed-point phases (one SFU sincos per 8 entries,
// the rest by complex rotation), already split and laid out as UMMA operands.
//
// Every mbarrier wait is bounded; a wait that runs out sets the device status
// word and the whole CTA unwinds, releasing its TMEM.
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace msk {

// ===========================================================================
// Adjoint: split-K over visibilities.  A CTA owns a contiguous run of
// (channel, output block, visibility range) units, accumulates each unit's
// BLK x BLK block of G in TMEM over 16-visibility stages and drains it to an
// FP32 partial buffer; partials are summed in unit order afterwards (compensated
// FP32 two-sum).
// Operands are MN-major (8 consecutive pixels of one visibility per 16-byte
// core-matrix row), the layout the per-visibility phase recurrences produce.
// Roles: warp 4 MMA + TMEM owner; the other 13 warps produce operand stages,
// and warps 0-3 (TMEM lane quadrants 0-3) also drain the accumulator to the
// split-K partials every ADJ_DRAIN stages and at the end of each unit.
// ===========================================================================
constexpr int ADJ_MAX_STAGES = 3;
// Stages (of 16 visibilities) accumulated in TMEM before the accumulator is
// added into the unit's FP32 partial.  The tensor core rounds each MMA's
// addition into its FP32 accumulator toward zero, so an accumulation of K
// MMAs shrinks by up to ~K ulp; bounding K (6 MMAs per stage) bounds that
// bias at ~2.5e-5 relative however many visibilities a unit spans.  The drains
// add with round-to-nearest FP32 reductions, which have no such bias.
constexpr int ADJ_DRAIN = 256;
constexpr int ADJ_THREADS = 448;
constexpr int ADJ_PRODUCER_WARPS = ADJ_THREADS / 32 - 1;  // every warp but the MMA warp

__host__ __device__ inline int adj_rows(int BLK) { return BLK < 128 ? 128 : BLK; }
__host__ __device__ inline int adj_stage_bytes(int BLK) {
    return 4 * adj_rows(BLK) * TCA_BK * 2 + 4 * BLK * TCA_BK * 2;
}
int adj_tc_smem_bytes(int N, int stages) { return stages * adj_stage_bytes(tca_blk(N)) + 1024; }
__host__ __device__ inline uint32_t adj_tmem_cols(int BLK) {
    int c = (adj_rows(BLK) / 128) * BLK;
    uint32_t p = 32;
    while ((int)p < c) p <<= 1;
    return p;
}

// Layout of a unit's partial block (BLK x BLK floats): the element of block
// row n and column m lives at ((mt * BLK/16 + q) * 16 + k) * RB + r, with
// n = mt * 128 + r (r < RB = min(BLK, 128)) and m = 16 q + k.  For a fixed
// column, the rows a warp drains from its TMEM lanes are adjacent, so each
// drain load and store is one coalesced 128-byte access.
__host__ __device__ inline int64_t adj_partial_index(int n, int m, int BLK) {
    const int RB = BLK < 128 ? BLK : 128;
    return ((int64_t)((n / 128) * (BLK / 16) + m / 16) * 16 + (m % 16)) * RB + (n % 128);
}

// Inverse of adj_partial_index: block row and column of partial element i.
__host__ __device__ inline void adj_partial_rc(int64_t i, int BLK, int& n, int& m) {
    const int RB = BLK < 128 ? BLK : 128;
    const int r = (int)(i % RB);
    int64_t t = i / RB;
    const int k = (int)(t % 16);
    t /= 16;
    const int q = (int)(t % (BLK / 16)), mt = (int)(t / (BLK / 16));
    n = mt * 128 + r;
    m = q * 16 + k;
}

// Drain of the TMEM accumulator by warps 0-3 (TMEM lane quadrant = warp):
// partial (one unit's block, layout above) = [partial +] accumulator.  Kept
// out of line so that its registers do not add to the producers' loop.
__device__ __noinline__ void adj_drain(uint32_t tmem, float* out, int BLK, int n_mt, int warp, int lane,
                                       bool first) {
    const int RB = BLK < 128 ? BLK : 128;
    for (int mt = 0; mt < n_mt; ++mt) {
        const int nrow = mt * 128 + warp * 32 + lane;
        const bool row_ok = nrow < BLK;
        const uint32_t lb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * BLK);
        // column m of this lane's row: base[m * RB], coalesced over the warp
        float* base = out + (row_ok ? adj_partial_index(nrow, 0, BLK) : 0);
        // one TMEM wait per 16-column chunk; the unit's first drain stores,
        // later ones add in place with reductions that return nothing, so the
        // drain never waits for a load of the partial (each element is added
        // to by one thread, in program order: the sum keeps its fixed order;
        // the reduction flushes subnormal values, far below any gradient
        // scale, to zero)
        for (int q = 0; q < BLK / 16; ++q) {
            uint32_t r[16];
            tmem_ld16(lb + q * 16, r);
            tmem_ld_wait(r);
            if (row_ok) {
                if (first) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) base[(int64_t)(q * 16 + k) * RB] = __uint_as_float(r[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) atomicAdd(base + (int64_t)(q * 16 + k) * RB, __uint_as_float(r[k]));
                }
            }
        }
    }
}

struct AdjShared {
    uint64_t full[ADJ_MAX_STAGES];
    uint64_t empty[ADJ_MAX_STAGES];
    uint64_t tfull;
    uint64_t tempty;
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

// FROM_UV: phase increments reduced from u, v inside the producers instead of
// read from the prepared arrays.
// F16: FP16X3 operands with y scaled by pow2_scale_for(ymax[0]) (a power of
// two, undone when the partials are summed); otherwise BF16X3.
// ADJ_STAGES: depth of the shared-memory pipeline (autotuned).
template <bool FROM_UV, bool F16, int ADJ_STAGES>
__global__ void __launch_bounds__(ADJ_THREADS, 1)
    k_adj_tc(DevData d, const AdjUnit* __restrict__ units, const int* __restrict__ cta_unit_off,
             const float2* __restrict__ y, const float* __restrict__ ymax, float* __restrict__ partial,
             uint64_t spin, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ AdjShared S;
    const int N = d.N, c0 = N / 2;
    const int BLK = N < 256 ? N : 256;
    const int R = adj_rows(BLK);           // A rows (image rows n, padded to 128)
    const int n_mt = R / 128;
    const int nbx = N / BLK;
    const int a_plane = R * TCA_BK * 2, b_plane = BLK * TCA_BK * 2;
    const int stage_bytes = 4 * a_plane + 4 * b_plane;
    const uint32_t tcols = adj_tmem_cols(BLK);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u0 = cta_unit_off[blockIdx.x], u1 = cta_unit_off[blockIdx.x + 1];
    volatile int* abort = &S.abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ADJ_STAGES; ++s) {
            mbar_init(&S.full[s], ADJ_PRODUCER_WARPS);
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.tfull, 1);
        mbar_init(&S.tempty, 4);
        mbar_init(&S.drain, 1);
        S.abort = 0;
        mbar_fence_init();
    }
    if (warp == 4) {
        tmem_alloc(&S.tmem_base, tcols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;

    if (warp == 4) {
        // The whole warp runs the issue loop, converged (every wait's outcome is
        // made warp-uniform), and one elected lane issues the MMAs and commits.
        {
            const uint32_t idesc = idesc_f16kind(128, BLK, 1, 1, F16 ? 0 : 1);
            const uint32_t sbase = smem_u32(smem);
            const uint32_t lboA = (uint32_t)(R / 8) * 128, lboB = (uint32_t)(BLK / 8) * 128;
            // Operand descriptors of slot 0; another slot or row block only
            // moves the start address, whose field (address >> 4, low 14 bits)
            // takes the offset by plain addition (shared memory < 256 KB).
            // (the four planes of an operand share their strides: plane i is
            // plane 0 moved by i planes)
            const uint64_t d_a = smem_desc(sbase, lboA, 128);
            const uint64_t d_b = smem_desc(sbase + 4 * a_plane, lboB, 128);
            const uint64_t pa16 = (uint64_t)(a_plane >> 4), pb16 = (uint64_t)(b_plane >> 4);
            uint32_t sc = 0;
            bool ok = true;
            uint32_t it = 0;  // accumulation segments so far (tfull / tempty phases)
            for (int u = u0; u < u1 && ok; ++u) {
              const int nst = (int)((units[u].count + TCA_BK - 1) / TCA_BK);
              for (int seg0 = 0; seg0 < nst && ok; seg0 += ADJ_DRAIN, ++it) {
                ok = __all_sync(~0u, mbar_wait(&S.tempty, (it & 1) ^ 1, spin, abort, status));
                if (!ok) break;
                tc_fence_after();
                const int seg1 = min(nst, seg0 + ADJ_DRAIN);
                for (int ks = seg0; ks < seg1; ++ks, ++sc) {
                    const int s = sc % ADJ_STAGES;
                    ok = __all_sync(~0u, mbar_wait(&S.full[s], (sc / ADJ_STAGES) & 1, spin, abort, status));
                    if (!ok) break;
                    tc_fence_after();
                    const uint64_t so = (uint64_t)((uint32_t)(s * stage_bytes) >> 4);
                    const uint64_t bre_h = d_b + so, bre_l = bre_h + pb16;
                    const uint64_t bim_h = bre_h + 2 * pb16, bim_l = bre_h + 3 * pb16;
                    for (int mt = 0; mt < n_mt; ++mt) {
                        const uint64_t are_h = d_a + so + (uint64_t)(mt * 2048 >> 4);  // 16 groups of 8 rows
                        const uint64_t are_l = are_h + pa16, aim_h = are_h + 2 * pa16, aim_l = are_h + 3 * pa16;
                        const uint32_t dt = tmem + (uint32_t)(mt * BLK);
                        const uint32_t acc = ks > seg0 ? 1u : 0u;
                        // products sharing an A tile read it once (collector buffer)
                        umma_f16_elect<MMA_FILL>(dt, are_h, bre_h, idesc, acc);
                        umma_f16_elect<MMA_LASTUSE>(dt, are_h, bre_l, idesc, 1u);
                        umma_f16_elect<MMA_PLAIN>(dt, are_l, bre_h, idesc, 1u);
                        umma_f16_elect<MMA_FILL>(dt, aim_h, bim_h, idesc, 1u);
                        umma_f16_elect<MMA_LASTUSE>(dt, aim_h, bim_l, idesc, 1u);
                        umma_f16_elect<MMA_PLAIN>(dt, aim_l, bim_h, idesc, 1u);
                    }
                    umma_commit_elect(&S.empty[s]);
                }
                if (ok) umma_commit_elect(&S.tfull);
              }
            }
            umma_commit_elect(&S.drain);
            int dummy = 0;
            mbar_wait(&S.drain, 0, drain_limit(spin), (volatile int*)&dummy, status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------ producers (13 warps, 416 thr)
        // A warp-iteration builds two items (8 pixels of 16 visibilities each,
        // one per half-warp).  Whole warps take one side, Ey items (A operand)
        // or P items (B operand), so each thread builds one step table per
        // stage and the halves of a warp never diverge.  A stage has 16
        // warp-iterations per side (N >= 256); the table gives each warp a
        // contiguous run of them such that every SM sub-partition (warp % 4;
        // their FMA pipes are the busy units) carries 8 per stage and no warp
        // more than 3.  Smaller images use the runs' first entries.
        const int pw = warp < 4 ? warp : warp - 1;  // producer warp 0..12
        const int ey_side = (0x3F >> pw) & 1;       // warps 0-3, 5, 6
        const int wi_start = (int)((0xA6EC8039E63C0ull >> (4 * pw)) & 15);
        const int wi_cap = (int)((0x2222233323323ull >> (4 * pw)) & 15);
        const int half = lane >> 4;
        const int jj = lane & 15;           // visibility within the stage
        const int ngA = R / 8, ngB = BLK / 8;
        const int wi_end = min(wi_start + wi_cap, (ey_side ? ngA : ngB) / 2);
        const float ysc = F16 ? pow2_scale_for(ymax[0]) : 1.f;
        uint32_t sc = 0, dr = 0;  // stages produced; accumulator drains (warps 0-3)
        bool ok = true;
        for (int u = u0; u < u1 && ok; ++u) {
            const AdjUnit un = units[u];
            const int blk_n0 = (un.block / nbx) * BLK, blk_m0 = (un.block % nbx) * BLK;
            const int nst = (int)((un.count + TCA_BK - 1) / TCA_BK);
            // per-visibility inputs of the next stage are loaded one stage ahead
            auto fetch = [&](int ks, uint64_t& fa, uint64_t& fb, float2& fy) {
                const int64_t kv = (int64_t)ks * TCA_BK + jj;
                fa = 0;
                fb = 0;
                fy = make_float2(0.f, 0.f);
                if (ks < nst && kv < un.count) {
                    if (FROM_UV) {
                        fa = to_fixed_turns(d.u[un.start + kv] * d.dx);
                        fb = to_fixed_turns(d.v[un.start + kv] * d.dy);
                    } else {
                        fa = d.pa[un.start + kv];
                        fb = d.pb[un.start + kv];
                    }
                    fy = y[un.start + kv];
                }
            };
            uint64_t na, nb;
            float2 ny;
            fetch(0, na, nb, ny);
          for (int seg0 = 0; seg0 < nst && ok; seg0 += ADJ_DRAIN) {
            const int seg1 = min(nst, seg0 + ADJ_DRAIN);
            for (int ks = seg0; ks < seg1; ++ks, ++sc) {
                const int s = sc % ADJ_STAGES;
                const uint64_t pa = na, pb = nb;
                const cf2 yv = {ny.x * ysc, ny.y * ysc};
                const bool valid = (int64_t)ks * TCA_BK + jj < un.count;
                fetch(ks + 1, na, nb, ny);
                // rotation steps exp(-i 2 pi q c), q = 0..7, by powers of one SFU
                // value: c = b for the Ey side, a for the P side (computed before
                // the wait for the ring slot, which they do not need)
                cf2 st[8];
                st[0] = {1.f, 0.f};
                st[1] = cis_neg(ey_side ? pb : pa);
                st[2] = cmul(st[1], st[1]);
                st[4] = cmul(st[2], st[2]);
                st[3] = cmul(st[2], st[1]);
                st[5] = cmul(st[4], st[1]);
                st[6] = cmul(st[4], st[2]);
                st[7] = cmul(st[4], st[3]);
                ok = __all_sync(0xffffffffu, mbar_wait(&S.empty[s], ((sc / ADJ_STAGES) & 1) ^ 1, spin,
                                                       abort, status, 64));
                if (!ok) break;
                unsigned char* A = smem + s * stage_bytes;
                unsigned char* B = A + 4 * a_plane;
                // at most 3 warp-iterations (the table): unrolled so that the
                // items' independent arithmetic interleaves
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int wi = wi_start + r;
                    if (wi >= wi_end) break;
                    const int item = ey_side ? 2 * wi + half : ngA + 2 * wi + half;
                    uint4 rh = {0, 0, 0, 0}, rl = {0, 0, 0, 0}, ih = {0, 0, 0, 0}, il = {0, 0, 0, 0};
                    unsigned char* dst;
                    int plane;
                    if (item < ngA) {
                        const int g = item;
                        const int n0 = blk_n0 + g * 8;
                        if (valid && g * 8 < BLK) {
                            const cf2 base = cis_neg(phase_mul(n0 - c0, pb));
                            cf2 z[8];
#pragma unroll
                            for (int q = 0; q < 8; ++q) z[q] = cmul(base, st[q]);
                            split16x2<F16>(z[0].x, z[1].x, rh.x, rl.x);
                            split16x2<F16>(z[2].x, z[3].x, rh.y, rl.y);
                            split16x2<F16>(z[4].x, z[5].x, rh.z, rl.z);
                            split16x2<F16>(z[6].x, z[7].x, rh.w, rl.w);
                            split16x2<F16>(z[0].y, z[1].y, ih.x, il.x);
                            split16x2<F16>(z[2].y, z[3].y, ih.y, il.y);
                            split16x2<F16>(z[4].y, z[5].y, ih.z, il.z);
                            split16x2<F16>(z[6].y, z[7].y, ih.w, il.w);
                        }
                        dst = A + ((jj >> 3) * ngA + g) * 128 + (jj & 7) * 16;
                        plane = a_plane;
                    } else {
                        const int g = item - ngA;
                        const int m0 = blk_m0 + g * 8;
                        if (valid) {
                            // P = y conj(Ex): conj(base) times conj(steps)
                            const cf2 e = cis_neg(phase_mul(m0 - c0, pa));
                            const cf2 base = cmul(yv, cf2{e.x, -e.y});
                            cf2 z[8];
#pragma unroll
                            for (int q = 0; q < 8; ++q) z[q] = cmul(base, cf2{st[q].x, -st[q].y});
                            split16x2<F16>(z[0].x, z[1].x, rh.x, rl.x);
                            split16x2<F16>(z[2].x, z[3].x, rh.y, rl.y);
                            split16x2<F16>(z[4].x, z[5].x, rh.z, rl.z);
                            split16x2<F16>(z[6].x, z[7].x, rh.w, rl.w);
                            split16x2<F16>(z[0].y, z[1].y, ih.x, il.x);
                            split16x2<F16>(z[2].y, z[3].y, ih.y, il.y);
                            split16x2<F16>(z[4].y, z[5].y, ih.z, il.z);
                            split16x2<F16>(z[6].y, z[7].y, ih.w, il.w);
                        }
                        dst = B + ((jj >> 3) * ngB + g) * 128 + (jj & 7) * 16;
                        plane = b_plane;
                    }
                    *(uint4*)(dst + 0 * plane) = rh;
                    *(uint4*)(dst + 1 * plane) = rl;
                    *(uint4*)(dst + 2 * plane) = ih;
                    *(uint4*)(dst + 3 * plane) = il;
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.full[s]);
            }
            // warps 0-3 drain the accumulator after the last stage of each
            // accumulation segment into the unit's partial
            if (!ok || warp >= 4) continue;
            ok = __all_sync(0xffffffffu, mbar_wait(&S.tfull, dr & 1, spin, abort, status, 1024));
            if (!ok) break;
            tc_fence_after();
            adj_drain(tmem, partial + (int64_t)u * BLK * BLK, BLK, n_mt, warp, lane,
                      seg0 == 0 /* the unit's first segment stores */);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.tempty);
            ++dr;
          }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

template <bool FROM_UV, bool F16, int STAGES>
static void launch_adj_variant(const DevData& d, const AdjUnit* units, const int* cta_unit_off, int n_ctas,
                               const float2* y, const float* ymax, float* partial, uint64_t spin,
                               int* status, cudaStream_t st) {
    const int smem = adj_tc_smem_bytes(d.N, STAGES);
    cudaFuncSetAttribute(k_adj_tc<FROM_UV, F16, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_adj_tc<FROM_UV, F16, STAGES><<<n_ctas, ADJ_THREADS, smem, st>>>(d, units, cta_unit_off, y, ymax,
                                                                      partial, spin, status);
}

void launch_adj_tc(const DevData& d, int f16, const AdjUnit* units, const int* cta_unit_off, int n_ctas,
                   const float2* y, const float* ymax, float* partial, uint64_t spin, int* status,
                   cudaStream_t st) {
    if (n_ctas <= 0) return;
    const bool s2 = d.adj_stages == 2;
    if (f16) {
        if (s2) launch_adj_variant<false, true, 2>(d, units, cta_unit_off, n_ctas, y, ymax, partial, spin, status, st);
        else launch_adj_variant<false, true, 3>(d, units, cta_unit_off, n_ctas, y, ymax, partial, spin, status, st);
    } else {
        if (s2) launch_adj_variant<false, false, 2>(d, units, cta_unit_off, n_ctas, y, ymax, partial, spin, status, st);
        else launch_adj_variant<false, false, 3>(d, units, cta_unit_off, n_ctas, y, ymax, partial, spin, status, st);
    }
}

void launch_adj_tc_uv(const DevData& d, const AdjUnit* units, const int* cta_unit_off, int n_ctas,
                      const float2* y, float* partial, uint64_t spin, int* status, cudaStream_t st) {
    if (n_ctas <= 0) return;
    launch_adj_variant<true, false, ADJ_MAX_STAGES>(d, units, cta_unit_off, n_ctas, y, nullptr, partial, spin,
                                                    status, st);
}

// Single channel: out[p] = A[p] * (unit partials summed in unit order,
// compensated FP32 (two-sum)).
__global__ void __launch_bounds__(256) k_adj_tc_reduce_out(int N, const int* __restrict__ cb_unit_off,
                                                           const float* __restrict__ partial,
                                                           const float* __restrict__ beam,
                                                           float* __restrict__ out) {
    const int64_t NN = (int64_t)N * N;
    const int BLK = N < 256 ? N : 256;
    const int nbx = N / BLK;
    // threads run over the partials' layout (coalesced reads); p is the pixel
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= NN) return;
    const int blk = (int)(i / ((int64_t)BLK * BLK));
    const int64_t loc = i % ((int64_t)BLK * BLK);
    int nl, ml;
    adj_partial_rc(loc, BLK, nl, ml);
    const int64_t p = (int64_t)((blk / nbx) * BLK + nl) * N + (blk % nbx) * BLK + ml;
    float s = 0.f, comp = 0.f;
    for (int u = cb_unit_off[blk]; u < cb_unit_off[blk + 1]; ++u)
        two_sum_acc(s, comp, __ldg(partial + (int64_t)u * BLK * BLK + loc));
    out[p] = beam[p] * (s + comp);
}

void launch_adj_tc_reduce_out(int N, const int* cb_unit_off, const float* partial, const float* beam,
                              float* out, cudaStream_t st) {
    k_adj_tc_reduce_out<<<prep_blocks(N), 256, 0, st>>>(N, cb_unit_off, partial, beam, out);
}

// Sum the unit partials of each (channel, block) in unit order (compensated
// FP32, stored as FP64) into gsum[c][N*N] (without the beam factor).
// Sum of the unit partials [u0, u1) at one element, compensated FP32 (Neumaier).
// A block of 256 threads handles 64 elements with 4 threads each: thread
// group g sums the g-th quarter of the units, and the four quarters are then
// combined in group order, so the sum has a fixed order (independent of the
// launch) and four times the loads in flight of one thread per element.
constexpr int RED_ELEMS = 64;
__device__ __forceinline__ void unit_sum_quarter(const float* __restrict__ src, int64_t stride, int u0, int u1, int g,
                                                 float& s, float& comp) {
    const int ua = u0 + (u1 - u0) * g / 4, ub = u0 + (u1 - u0) * (g + 1) / 4;
    s = 0.f;
    comp = 0.f;
    int u = ua;
    for (; u + 8 <= ub; u += 8) {
        float q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = __ldg(src + (int64_t)(u + k) * stride);
#pragma unroll
        for (int k = 0; k < 8; ++k) two_sum_acc(s, comp, q[k]);
    }
    for (; u < ub; ++u) two_sum_acc(s, comp, __ldg(src + (int64_t)u * stride));
}

// Combine the four groups' (sum, compensation) pairs through shared memory;
// returns the total in group 0's threads.
__device__ __forceinline__ float unit_sum_combine(float s, float comp, int el, int g, float (*sh)[RED_ELEMS][2]) {
    sh[g][el][0] = s;
    sh[g][el][1] = comp;
    __syncthreads();
    float t = sh[0][el][0], c = sh[0][el][1];
    for (int k = 1; k < 4; ++k) {
        two_sum_acc(t, c, sh[k][el][0]);
        c += sh[k][el][1];
    }
    return t + c;
}

__global__ void __launch_bounds__(256) k_adj_tc_reduce(DevData d, const int* __restrict__ cb_unit_off,
                                                       const float* __restrict__ partial,
                                                       const float* __restrict__ ymax,
                                                       double* __restrict__ gsum) {
    __shared__ float sh[4][RED_ELEMS][2];
    const int N = d.N;
    const int64_t NN = (int64_t)N * N;
    const int BLK = N < 256 ? N : 256;
    const int nbx = N / BLK;
    const int c = blockIdx.y;
    const int el = threadIdx.x % RED_ELEMS, g = threadIdx.x / RED_ELEMS;
    // threads run over the partials' layout (coalesced reads); p is the pixel
    const int64_t i = (int64_t)blockIdx.x * RED_ELEMS + el;
    const bool in = i < NN;
    const int blk = in ? (int)(i / ((int64_t)BLK * BLK)) : 0;
    const int64_t loc = in ? i % ((int64_t)BLK * BLK) : 0;
    const int cb = c * nbx * nbx + blk;
    const int u0 = in ? cb_unit_off[cb] : 0, u1 = in ? cb_unit_off[cb + 1] : 0;
    float s, comp;
    unit_sum_quarter(partial + loc, (int64_t)BLK * BLK, u0, u1, g, s, comp);
    const float tot = unit_sum_combine(s, comp, el, g, sh);
    if (g != 0 || !in) return;
    int nl, ml;
    adj_partial_rc(loc, BLK, nl, ml);
    const int64_t p = (int64_t)((blk / nbx) * BLK + nl) * N + (blk % nbx) * BLK + ml;
    const double inv = ymax ? 1.0 / (double)pow2_scale_for(ymax[0]) : 1.0;
    gsum[(int64_t)c * NN + p] = (double)tot * inv;
}

void launch_adj_tc_reduce(const DevData& d, const AdjUnit* units, const int* cb_unit_off,
                          const float* partial, const float* ymax, double* gsum, cudaStream_t st) {
    (void)units;
    const int64_t NN = (int64_t)d.N * d.N;
    dim3 grid((unsigned)((NN + RED_ELEMS - 1) / RED_ELEMS), d.C);
    k_adj_tc_reduce<<<grid, 256, 0, st>>>(d, cb_unit_off, partial, ymax, gsum);
}

// The unit-partial sum of k_adj_tc_reduce followed directly by the gradient
// assembly (Eq. chi2gradient with the beam factor, Eq. Sgradient, the positive
// projection at I = G), for images of one channel each (one image, or a cube):
// the same arithmetic as the separate reduction and assembly, one launch.
// log(I/G) stays FP64: with an FP32 log the 50-iteration solve of the
// 64x64 problem ended 1.4e-3 (relative L2) from the oracle's image in the
// BF16X3 form, against 4.6e-4.
// With sc.scal set, SCAL_SPLIT further blocks per image (the first ones in
// x, so that they start with the first wave) run the objective's scalar
// reduction (scalars_block): it needs only the forward's chi^2 partials and
// the prep's entropy partials, so it shares this launch instead of taking one
// of its own.
__global__ void __launch_bounds__(256) k_adj_tc_reduce_grad(DevData d, ImgSrc src,
                                                            const int* __restrict__ cb_unit_off,
                                                            const float* __restrict__ partial,
                                                            const float* __restrict__ ymax, int projected,
                                                            float* out32, double* full64, double* proj64,
                                                            ScalarArgs sc) {
    __shared__ float sh[4][RED_ELEMS][2];
    const int N = d.N;
    const int64_t NN = (int64_t)N * N;
    const int n_scal = sc.scal ? SCAL_SPLIT : 0;
    if ((int)blockIdx.x < n_scal) {
        scalars_block(d, sc.tile_off, sc.chi_part, sc.ent_part, sc.with_entropy, prep_blocks(N),
                      scalars_part(sc.img_tmp, d.n_images), sc.img_tmp, sc.scal,
                      scalars_counter(sc.img_tmp, d.n_images), blockIdx.y, blockIdx.x);
        return;
    }
    const int BLK = N < 256 ? N : 256;
    const int nbx = N / BLK;
    const int c = blockIdx.y;  // channel = image
    const int el = threadIdx.x % RED_ELEMS, g = threadIdx.x / RED_ELEMS;
    const int64_t i = (int64_t)(blockIdx.x - n_scal) * RED_ELEMS + el;
    const bool in = i < NN;
    const int blk = in ? (int)(i / ((int64_t)BLK * BLK)) : 0;
    const int64_t loc = in ? i % ((int64_t)BLK * BLK) : 0;
    const int cb = c * nbx * nbx + blk;
    const int u0 = in ? cb_unit_off[cb] : 0, u1 = in ? cb_unit_off[cb + 1] : 0;
    float s, comp;
    unit_sum_quarter(partial + loc, (int64_t)BLK * BLK, u0, u1, g, s, comp);
    const float tot = unit_sum_combine(s, comp, el, g, sh);
    if (g != 0 || !in) return;
    int nl, ml;
    adj_partial_rc(loc, BLK, nl, ml);
    const int64_t p = (int64_t)((blk / nbx) * BLK + nl) * N + (blk % nbx) * BLK + ml;
    const double inv = ymax ? 1.0 / (double)pow2_scale_for(ymax[0]) : 1.0;
    const double gchi = (double)tot * inv;
    double gr = (double)d.beam[(int64_t)c * NN + p] * gchi;
    const double x = img_value(src, c, p, NN);
    if (d.lambda != 0.0) gr += d.lambda * (1.0 + log(x / d.G));
    const double gp = (x <= d.G && gr > 0.0) ? 0.0 : gr;
    if (full64) full64[(int64_t)c * NN + p] = gr;
    if (proj64) proj64[(int64_t)c * NN + p] = gp;
    if (out32) out32[(int64_t)c * NN + p] = (float)(projected ? gp : gr);
}

void launch_adj_tc_reduce_grad(const DevData& d, const ImgSrc& src, const int* cb_unit_off, const float* partial,
                               const float* ymax, int projected, float* out32, double* full64, double* proj64,
                               const ScalarArgs& sc, cudaStream_t st) {
    const int64_t NN = (int64_t)d.N * d.N;
    const unsigned gb = (unsigned)((NN + RED_ELEMS - 1) / RED_ELEMS);
    dim3 grid(gb + (sc.scal ? SCAL_SPLIT : 0), d.C);
    k_adj_tc_reduce_grad<<<grid, 256, 0, st>>>(d, src, cb_unit_off, partial, ymax, projected, out32, full64,
                                                proj64, sc);
}

}  // namespace msk
