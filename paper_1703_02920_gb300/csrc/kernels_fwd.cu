// Tensor-core forward operator (Eq. 1 on the pixel grid) with the fused
// per-visibility reduction, residual, weight and chi^2 partials.
//
//   T = Ey B^T  (tcgen05.mma kind::f16, 3-term FP16 or BF16 split, FP32 accumulation)
//   V_k = sum_m Ex[k,m] T[k,m]
//
// The image operand is centred column by column, B'[n][m] = B[n][m] - c_m
// (c_m the column mean), and T = Ey B'^T + c_m S_k with the closed form
//   S_k = sum_n Ey[k,n] = exp(i pi b_k) sin(pi N b_k) / sin(pi b_k),  b_k = frac(v_k dy).
// For low spatial frequencies the uncentred partial sums grow monotonically
// and the tensor core's FP32 accumulation (which rounds towards zero) then
// shrinks T systematically; the centred sums wander around zero instead.
//
// A tile is 64 visibilities.  Its A operand has 128 rows: row
// 32 (j >> 4) + (j & 15) holds Re Ey[j,:] and the row 16 below it Im Ey[j,:]
// (an order that keeps the producers' shared-memory stores free of bank
// conflicts and each visibility's pair of rows in one warp's TMEM lanes), so
// one M=128 MMA produces both the real and the imaginary part of T for 64
// visibilities, and one N <= 256 column block covers an N <= 256 image
// without regenerating Ey.  Two TMEM
// accumulators (2 x BN columns) let the epilogue of one tile overlap the MMAs
// of the next.
//
// Each accumulation covers at most F2_KSEG image rows (a K segment): the
// tensor core adds every MMA's product sum to its FP32 accumulator rounding
// towards zero, a shrink of up to one ulp per MMA that grows with the number
// of MMAs per accumulation.  Larger images run several segments per column
// block, each into a fresh accumulator; the epilogue folds every segment into
// the same compensated per-visibility sums (V is linear in T), so the shrink
// stays at the level of a 256-row image whatever N is.
//
// Roles (448 threads): warps 0-3 epilogue (TMEM lane = A row), warp 4 MMA
// issue (one elected lane) + TMEM owner, warp 5 bulk copies of the image
// operand chunks, warps 6-13 Ey producers.  Every mbarrier wait is bounded.
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace msk {

namespace {

constexpr int F2_MAX_STAGES = 4;
constexpr int F2_THREADS = 448;
constexpr int F2_APLANE = 128 * TC_BK * 2;  // bytes of one A plane (hi or lo), 8 KB
constexpr int F2_ABYTES = 2 * F2_APLANE;
constexpr int F2_KSEG = 256;                 // image rows per accumulation (at most)
// Phase factors advanced by complex recurrence (one product each) between
// SFU evaluations, which are taken every PHASE_REFRESH steps.
constexpr int PHASE_REFRESH = 4;

__host__ __device__ inline int f2_stage_bytes(int BN) { return F2_ABYTES + 2 * BN * TC_BK * 2; }
__host__ __device__ inline uint32_t f2_tmem_cols(int BN) {
    uint32_t c = 32;
    while ((int)c < 2 * BN) c <<= 1;
    return c;
}


struct F2Shared {
    uint64_t full[F2_MAX_STAGES];   // producer warps (8 arrivals) + the copy warp once the stage's image chunk landed
    uint64_t bfull[F2_MAX_STAGES];  // image operand bulk copy (transaction bytes; watched by the copy warp)
    uint64_t empty[F2_MAX_STAGES];  // MMA completion (tcgen05.commit)
    uint64_t tfull[2];
    uint64_t tempty[2];         // 4 epilogue warps
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

// F16: FP16X3 operands (the image planes are scaled by cscale[channel], a
// power of two undone in the epilogue); otherwise BF16X3.
// F2_STAGES: depth of the shared-memory pipeline (autotuned).
template <bool F16, int F2_STAGES>
__global__ void __launch_bounds__(F2_THREADS, 1)
    k_fwd_tc(DevData d, const VisTile* __restrict__ tiles, int n_tiles,
             const uint16_t* __restrict__ planes, const float* __restrict__ cmean,
             const float* __restrict__ cscale, int mode, float2* __restrict__ yout,
             double* __restrict__ chi_part, unsigned* __restrict__ ymax_bits, uint64_t spin, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ F2Shared S;
    const int N = d.N, c0 = N / 2;
    const int BN = d.fwd_bn;
    const int n_mb = N / BN, nk = N / TC_BK;
    // stages per accumulation and accumulations per column block
    const int kseg = nk < F2_KSEG / TC_BK ? nk : F2_KSEG / TC_BK;
    const int n_seg = nk / kseg;
    const int stage_bytes = f2_stage_bytes(BN);
    const uint32_t tcols = f2_tmem_cols(BN);
    const int64_t NN = (int64_t)N * N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abort = &S.abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < F2_STAGES; ++s) {
            mbar_init(&S.full[s], 9);
            mbar_init(&S.bfull[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.tfull[b], 1);
            mbar_init(&S.tempty[b], 4);
        }
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
        // ---------------------------------------------------------------- MMA
        // The whole warp runs the issue loop, converged (every wait's outcome
        // is made warp-uniform), and one elected lane issues the MMAs and
        // commits.
        {
            const uint32_t idesc = idesc_f16kind(128, BN, 0, 0, F16 ? 0 : 1);
            const uint32_t sbase = smem_u32(smem);
            const uint32_t lboB = (uint32_t)(BN / 8) * 128;
            // Operand descriptors of slot 0; another slot or K step only moves
            // the start address, whose field (address >> 4, low 14 bits of the
            // low word) takes the offset by plain 32-bit addition (shared
            // memory < 256 KB, no carry).  A second K step is 2 core-matrix
            // columns on: 2 x 2048 bytes in A, 2 x lboB in B.
            const uint64_t d_ah = smem_desc(sbase, 2048, 128);
            const uint64_t d_al = smem_desc(sbase + F2_APLANE, 2048, 128);
            const uint64_t d_bh = smem_desc(sbase + F2_ABYTES, lboB, 128);
            const uint64_t d_bl = smem_desc(sbase + F2_ABYTES + BN * TC_BK * 2, lboB, 128);
            const uint32_t lo_ah = (uint32_t)d_ah, lo_al = (uint32_t)d_al;
            const uint32_t lo_bh = (uint32_t)d_bh, lo_bl = (uint32_t)d_bl;
            const uint32_t hi_a = (uint32_t)(d_ah >> 32), hi_b = (uint32_t)(d_bh >> 32);
            const uint32_t ka16 = (2u * 2048u) >> 4, kb16 = (2u * lboB) >> 4;
            static_assert(TC_BK == 32, "one stage is two K steps of 16");
            uint32_t sc = 0, it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                for (int u = 0; u < n_mb * n_seg && ok; ++u, ++it) {
                    const int b = it & 1;
                    const int ks0 = (u % n_seg) * kseg;  // first stage of this accumulation
                    ok = __all_sync(~0u, mbar_wait(&S.tempty[b], ((it >> 1) & 1) ^ 1, spin, abort, status));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t dt = tmem + (uint32_t)(b * BN);
                    for (int ks = ks0; ks < ks0 + kseg; ++ks, ++sc) {
                        const int s = sc % F2_STAGES;
                        // one wait: the producers' tables and the image chunk
                        ok = __all_sync(~0u, mbar_wait(&S.full[s], (sc / F2_STAGES) & 1, spin, abort, status));
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t so = (uint32_t)(s * stage_bytes) >> 4;
                        umma6_stage_elect(dt, lo_ah + so, lo_al + so, lo_bh + so, lo_bl + so, hi_a, hi_b, ka16,
                                          kb16, idesc, ks > ks0 ? 1u : 0u);
                        umma_commit_elect(&S.empty[s]);
                    }
                    if (ok) umma_commit_elect(&S.tfull[b]);
                }
            }
            // every issued MMA completes before TMEM is released (its operands
            // were complete when it was issued)
            umma_commit_elect(&S.drain);
            int dummy = 0;
            mbar_wait(&S.drain, 0, drain_limit(spin), (volatile int*)&dummy, status);
        }
        __syncwarp();
    } else if (warp == 5) {
        // --------------------------------------------- image operand copies
        if (lane == 0) {
            uint32_t sc = 0;
            bool ok = true;
            const uint32_t chunk_bytes = 2u * BN * TC_BK * 2;
            // once stage q's chunk has landed (bfull), the copy warp is the
            // ninth arrival on full[q]; it does so one stage behind the copy it
            // issues, so that a copy is always in flight
            auto land = [&](uint32_t q) -> bool {
                if (!mbar_wait(&S.bfull[q % F2_STAGES], (q / F2_STAGES) & 1, spin, abort, status)) return false;
                mbar_arrive(&S.full[q % F2_STAGES]);
                return true;
            };
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int chan = tiles[t].chan;
                const unsigned char* cbase = (const unsigned char*)(planes + (int64_t)chan * 2 * NN);  // 16-bit elements
                for (int mb = 0; mb < n_mb && ok; ++mb) {
                    for (int ks = 0; ks < nk; ++ks, ++sc) {
                        const int s = sc % F2_STAGES;
                        ok = mbar_wait(&S.empty[s], ((sc / F2_STAGES) & 1) ^ 1, spin, abort, status);
                        if (!ok) break;
                        mbar_arrive_expect_tx(&S.bfull[s], chunk_bytes);
                        bulk_g2s(smem + s * stage_bytes + F2_ABYTES,
                                 cbase + (int64_t)(mb * nk + ks) * chunk_bytes, chunk_bytes, &S.bfull[s]);
                        if (sc > 0) {
                            ok = land(sc - 1);
                            if (!ok) {
                                ++sc;  // the copy just issued is in flight too
                                break;
                            }
                        }
                    }
                }
            }
            if (ok && sc > 0) ok = land(sc - 1);
            if (!ok) {
                // copies already issued land on their own; wait for them before
                // the CTA's shared memory is released
                int dummy = 0;
                for (uint32_t q = (sc > F2_STAGES ? sc - F2_STAGES : 0); q < sc; ++q)
                    mbar_wait(&S.bfull[q % F2_STAGES], (q / F2_STAGES) & 1, drain_limit(spin),
                              (volatile int*)&dummy, status);
            }
        }
        __syncwarp();
    } else if (warp >= 6) {
        // ----------------------------------- Ey producers (256 threads)
        // thread -> (visibility j = ptid & 63, k-group g = ptid >> 6): 8 image
        // rows n of one visibility per stage, written as A rows row(j, Re), row(j, Im)
        const int ptid = threadIdx.x - 192;
        const int jv = ptid & 63, g = ptid >> 6;
        // row(j, c) = 32 (j >> 4) + 16 c + (j & 15): the 32 lanes of a store
        // instruction fill four whole 128-byte core matrices (no bank conflicts)
        const int r0 = 32 * (jv >> 4) + (jv & 15);
        const int off = (g * 16 + (r0 >> 3)) * 128 + (r0 & 7) * 16;  // Re row; Im row at +256
        uint32_t sc = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const VisTile tl = tiles[t];
            const bool valid = jv < tl.count;
            const uint64_t pb = valid ? d.pb[tl.start + jv] : 0;
            cf2 step[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) step[q] = cis_neg(phase_mul(q, pb));
            const Rot8 w = rot8_of(step);
            // the group's first row advances by TC_BK rows per stage: its phase
            // factor is the previous one times exp(-2 pi i TC_BK b), refreshed
            // from the SFU every PHASE_REFRESH stages (the products' rounding is
            // unbiased and does not accumulate further)
            const cf2 step_bk = cis_neg(phase_mul(TC_BK, pb));
            for (int mb = 0; mb < n_mb && ok; ++mb) {
                cf2 base = {1.f, 0.f};
                for (int ks = 0; ks < nk; ++ks, ++sc) {
                    const int s = sc % F2_STAGES;
                    // the table values need no ring slot: compute them, then wait
                    uint4 rh = {0, 0, 0, 0}, rl = {0, 0, 0, 0}, ih = {0, 0, 0, 0}, il = {0, 0, 0, 0};
                    if (valid) {
                        const int n0 = ks * TC_BK + g * 8;
                        base = (ks % PHASE_REFRESH) ? cmul(base, step_bk) : cis_neg(phase_mul(n0 - c0, pb));
                        table8_split<F16>(base, w, rh, rl, ih, il);
                    }
                    ok = __all_sync(0xffffffffu, mbar_wait(&S.empty[s], ((sc / F2_STAGES) & 1) ^ 1, spin,
                                                           abort, status, 64));
                    if (!ok) break;
                    unsigned char* A = smem + s * stage_bytes;
                    *(uint4*)(A + off) = rh;
                    *(uint4*)(A + off + 256) = ih;
                    *(uint4*)(A + F2_APLANE + off) = rl;
                    *(uint4*)(A + F2_APLANE + off + 256) = il;
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.full[s]);
                }
            }
        }
    } else {
        // -------------------------------- epilogue (warps 0-3, 128 threads)
        // TMEM lane = A row: warp q holds visibilities 16q .. 16q+15, lane L
        // component L >> 4 (0: Re T, 1: Im T) of visibility 16q + (L & 15).
        // Every lane accumulates (sum ReEx T, sum ImEx T) over its row; lanes L
        // and L ^ 16 combine with one shuffle:
        //   Re V = sum ReEx ReT - ImEx ImT,  Im V = sum ReEx ImT + ImEx ReT.
        const int jv = 16 * warp + (lane & 15), comp = lane >> 4;
        uint32_t it = 0;
        bool ok = true;
        // this warp's copy of the tile channel's column means (read as
        // broadcasts; refreshed when the channel changes)
        float* cmw = (float*)(smem + F2_STAGES * stage_bytes) + warp * N;
        int cm_chan = -1;
        // per-visibility inputs are loaded one tile ahead: the next tile's
        // descriptor and phases arrive while this tile's accumulator drains
        VisTile tl_next{};
        uint64_t pa_next = 0, pb_next = 0;
        auto load_phases = [&](const VisTile& tn) {
            const int64_t jn = tn.start + (jv < tn.count ? jv : 0);
            pa_next = d.pa[jn];
            pb_next = d.pb[jn];
        };
        if ((int)blockIdx.x < n_tiles) {
            tl_next = tiles[blockIdx.x];
            load_phases(tl_next);
        }
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const VisTile tl = tl_next;
            const bool valid = jv < tl.count;
            const int64_t j = tl.start + (valid ? jv : 0);
            const uint64_t pa = pa_next, pb = pb_next;
            if (t + (int)gridDim.x < n_tiles) tl_next = tiles[t + gridDim.x];
            if (tl.chan != cm_chan) {
                __syncwarp();
                const float4* src = (const float4*)(cmean + (int64_t)tl.chan * N);
                for (int i = lane; i < N / 4; i += 32) ((float4*)cmw)[i] = __ldg(src + i);
                __syncwarp();
                cm_chan = tl.chan;
            }
            cf2 step[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) step[q] = cis_neg(phase_mul(q, pa));
            const Rot8 wx8 = rot8_of(step);
            const cf2 step8 = cis_neg(phase_mul(8, pa));
            const cf2 step16 = cis_neg(phase_mul(16, pa));  // chunk to chunk (recurrence below)
            // this lane's component of S_j = sum_n Ey[j,n] (accurate sincospi of
            // the exact half-turn and N/2-multiple phases)
            float scomp;
            {
                const float th = (float)(int64_t)((int64_t)pb >> 1) * 5.421010862427522e-20f;  // b/2, turns
                const float tn = (float)(int64_t)phase_mul(N / 2, pb) * 5.421010862427522e-20f;  // N b/2
                float sh, ch;
                sincospif(2.0f * th, &sh, &ch);          // sin(pi b), cos(pi b)
                const float snb = sinpif(2.0f * tn);      // sin(pi N b)
                const float D = (sh != 0.f) ? snb / sh : (float)N;
                scomp = comp ? sh * D : ch * D;
            }
            const float osc = F16 ? cscale[tl.chan] : 1.f;  // operand scale (power of two)
            scomp *= osc;
            float s0 = 0.f, s1 = 0.f, c0s = 0.f, c1s = 0.f;  // compensated sums
            for (int u = 0; u < n_mb * n_seg; ++u, ++it) {
                const int mb = u / n_seg;
                const int b = it & 1;
                // the column-mean term c_m S_k enters once per column: with the
                // block's first segment only
                const float sterm = (u % n_seg == 0) ? scomp : 0.f;
                ok = __all_sync(0xffffffffu,
                                mbar_wait(&S.tfull[b], (it >> 1) & 1, spin, abort, status, 256));
                if (!ok) break;
                tc_fence_after();
                const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * BN);
                // software pipeline over 16-column chunks: the TMEM load of
                // chunk q+1 is in flight while chunk q is reduced
                const int nq = BN / 16;
                uint32_t tv[2][16];
                auto load_chunk = [&](int q, int slot) { tmem_ld16(lane_base + q * 16, tv[slot]); };
                // sum_k Ex[m0+k] t_k = base * sum_{k<8} step_k t_k + base8 * sum_{k<8} step_k t_{k+8}
                // the chunk's phase factor exp(-2 pi i (m0 - N/2) a): the previous
                // chunk's times step16, refreshed from the SFU every
                // PHASE_REFRESH chunks (chunks run in order)
                cf2 ebase = {1.f, 0.f};
                auto reduce_chunk = [&](int q, int slot) {
                    const int m0 = mb * BN + q * 16;
                    const cf2 base = (q % PHASE_REFRESH) ? cmul(ebase, step16) : cis_neg(phase_mul(m0 - c0, pa));
                    ebase = base;
                    const cf2 base8 = cmul(base, step8);
                    float2 cq[8];
#pragma unroll
                    for (int k = 0; k < 4; ++k) *(float4*)(cq + 2 * k) = ((const float4*)(cmw + m0))[k];
                    // packed pairs (even k, odd k), added at the end
                    const float2 ss = make_float2(sterm, sterm);
                    float2 ux = {0.f, 0.f}, uy = {0.f, 0.f}, wx = {0.f, 0.f}, wy = {0.f, 0.f};
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const float2 tk = __ffma2_rn(cq[p], ss, make_float2(__uint_as_float(tv[slot][2 * p]),
                                                                            __uint_as_float(tv[slot][2 * p + 1])));
                        const float2 tw = __ffma2_rn(cq[p + 4], ss,
                                                     make_float2(__uint_as_float(tv[slot][2 * p + 8]),
                                                                 __uint_as_float(tv[slot][2 * p + 9])));
                        ux = __ffma2_rn(wx8.x[p], tk, ux);
                        uy = __ffma2_rn(wx8.y[p], tk, uy);
                        wx = __ffma2_rn(wx8.x[p], tw, wx);
                        wy = __ffma2_rn(wx8.y[p], tw, wy);
                    }
                    const float sux = ux.x + ux.y, suy = uy.x + uy.y, swx = wx.x + wx.y, swy = wy.x + wy.y;
                    const float a0 = fmaf(base.x, sux, fmaf(-base.y, suy, fmaf(base8.x, swx, -base8.y * swy)));
                    const float a1 = fmaf(base.x, suy, fmaf(base.y, sux, fmaf(base8.x, swy, base8.y * swx)));
                    two_sum_acc(s0, c0s, a0);
                    two_sum_acc(s1, c1s, a1);
                };
                load_chunk(0, 0);
                tmem_ld_wait(tv[0]);
                for (int q = 0; q < nq; q += 2) {
                    load_chunk(q + 1, 1);  // nq is even
                    reduce_chunk(q, 0);
                    tmem_ld_wait(tv[1]);
                    if (q + 2 < nq) load_chunk(q + 2, 0);
                    reduce_chunk(q + 1, 1);
                    if (q + 2 < nq) tmem_ld_wait(tv[0]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.tempty[b]);
            }
            if (!ok) break;
            if (t + (int)gridDim.x < n_tiles) load_phases(tl_next);
            // lane < 16: (sum ReEx ReT, sum ImEx ReT); lane >= 16: (sum ReEx ImT, sum ImEx ImT),
            // each a compensated (hi, lo) pair, unscaled exactly (a power of two).
            // The tail runs in FP32 pair arithmetic: the residual V - V° is an
            // exact pair difference, and chi^2 per visibility needs only FP32
            // relative accuracy (the partials are summed in FP64).
            const float inv = 1.f / osc;
            const float p0h = s0 * inv, p0l = c0s * inv, p1h = s1 * inv, p1l = c1s * inv;
            const float q0h = __shfl_xor_sync(0xffffffffu, p0h, 16), q0l = __shfl_xor_sync(0xffffffffu, p0l, 16);
            const float q1h = __shfl_xor_sync(0xffffffffu, p1h, 16), q1l = __shfl_xor_sync(0xffffffffu, p1l, 16);
            float chi = 0.f;
            float ym = 0.f;  // max |component| of the weighted residual (RESID mode)
            if (valid && comp == 0) {
                const float2 vre = df_add(p0h, p0l, -q1h, -q1l);  // ReEx ReT - ImEx ImT
                const float2 vim = df_add(q0h, q0l, p1h, p1l);    // ReEx ImT + ImEx ReT
                if (mode == FWD_VIS) {
                    yout[j] = make_float2(vre.x + vre.y, vim.x + vim.y);
                } else if (mode == FWD_DCHI) {
                    const float2 yv = yout[j];
                    const float vr = vre.x + vre.y, vi = vim.x + vim.y;
                    chi = yv.x * vr + yv.y * vi + 0.5f * d.w32[j] * (vr * vr + vi * vi);
                } else {
                    float rr = vre.x + vre.y, ri = vim.x + vim.y;
                    if (mode != FWD_CURV) {
                        const float4 o = d.vo32[j];  // (Re hi, Im hi, Re lo, Im lo)
                        const float2 r0 = df_add(vre.x, vre.y, -o.x, -o.z);
                        const float2 r1 = df_add(vim.x, vim.y, -o.y, -o.w);
                        rr = r0.x + r0.y;
                        ri = r1.x + r1.y;
                    }
                    const float w = d.w32[j];
                    chi = 0.5f * w * (rr * rr + ri * ri);
                    if (mode == FWD_RESID) {
                        const float2 yv = make_float2(w * rr, w * ri);
                        yout[j] = yv;
                        ym = fmaxf(fabsf(yv.x), fabsf(yv.y));
                    }
                }
            }
            if (mode == FWD_RESID && ymax_bits) {
                // order-independent maximum (non-negative floats order as their bits)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ym = fmaxf(ym, __shfl_down_sync(0xffffffffu, ym, o));
                if (lane == 0) atomicMax(ymax_bits, __float_as_uint(ym));
            }
            if (mode != FWD_VIS) {
                // one partial per warp (16 visibilities), summed later in a fixed order
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) chi += __shfl_down_sync(0xffffffffu, chi, o);
                if (lane == 0) chi_part[(int64_t)t * 4 + warp] = (double)chi;
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

}  // namespace

// stage ring + the epilogue warps' column-mean copies (4 x N floats) + alignment
int fwd_tc_smem_bytes(int N, int BN, int stages) { return stages * f2_stage_bytes(BN) + 16 * N + 1024; }

template <bool F16, int STAGES>
static void launch_fwd_variant(const DevData& d, const VisTile* tiles, int n_tiles, const void* planes,
                               const float* cmean, const float* cscale, int mode, float2* yout,
                               double* chi_part, unsigned* ymax_bits, int grid, uint64_t spin, int* status,
                               cudaStream_t st) {
    const int smem = fwd_tc_smem_bytes(d.N, d.fwd_bn, STAGES);
    cudaFuncSetAttribute(k_fwd_tc<F16, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_fwd_tc<F16, STAGES><<<grid, F2_THREADS, smem, st>>>(d, tiles, n_tiles, (const uint16_t*)planes, cmean,
                                                          cscale, mode, yout, chi_part, ymax_bits, spin, status);
}

void launch_fwd_tc(const DevData& d, int f16, const VisTile* tiles, int n_tiles, const void* planes,
                   const float* cmean, const float* cscale, int mode, float2* yout, double* chi_part,
                   float* ymax, int grid, uint64_t spin, int* status, cudaStream_t st) {
    unsigned* ymax_bits = (unsigned*)ymax;
    if (n_tiles <= 0) return;
    if (grid > n_tiles) grid = n_tiles;
    const bool s3 = d.fwd_stages == 3;
    if (f16) {
        if (s3) launch_fwd_variant<true, 3>(d, tiles, n_tiles, planes, cmean, cscale, mode, yout, chi_part, ymax_bits, grid, spin, status, st);
        else launch_fwd_variant<true, 4>(d, tiles, n_tiles, planes, cmean, cscale, mode, yout, chi_part, ymax_bits, grid, spin, status, st);
    } else {
        if (s3) launch_fwd_variant<false, 3>(d, tiles, n_tiles, planes, cmean, cscale, mode, yout, chi_part, ymax_bits, grid, spin, status, st);
        else launch_fwd_variant<false, 4>(d, tiles, n_tiles, planes, cmean, cscale, mode, yout, chi_part, ymax_bits, grid, spin, status, st);
    }
}

}  // namespace msk
