// Tensor-core forward operator (Eq. 1 on the pixel grid) for images of side
// N <= 256, with the image operand resident in shared memory.
//
//   T_s = Ey[:, rows of slice s] B'[rows of slice s, :]^T   (tcgen05.mma kind::f16)
//   V_k = sum_s sum_m Ex[k,m] T_s[k,m]  (+ c_m S_k from slice 0)
//
// The image rows (the contraction index n) are cut into slices of at most
// 128 rows.  A persistent CTA owns one slice: it copies that slice of the
// split operand planes (hi and lo, N columns, 128 KB at N = 256) into shared
// memory once per channel and keeps it, so only the phase-table operand Ey
// streams through the pipeline.  Re-streaming the whole image operand for
// every 64-visibility tile is what bounds the streaming kernel (about 5 TB/s
// of L2 traffic at N = 256).  Each slice writes a partial visibility per
// sample (FP64); k_fwd_combine adds the slices in a fixed order and applies
// the residual, weight and chi^2 partials.
//
// Accumulation order.  The tensor core adds each MMA's exact product sum to
// the FP32 accumulator rounding towards zero, so every MMA of an output can
// shrink it by up to one ulp.  The correction products (hi*lo, lo*hi, about
// 2^-11 of the result for the FP16 split, 2^-8 for BF16) are issued first
// over the whole slice, while the accumulator is still small; the hi*hi
// products follow.  Of the 3 KS/16 MMAs per output only the KS/16 hi*hi ones
// then act on an accumulator of full magnitude.  This costs a second pass of
// the phase-table producers (hi plane only) over the slice.
//
// Tile: 64 visibilities, A rows 32 (j >> 4) + (j & 15) (Re Ey) and 16 below
// (Im Ey), as in the streaming kernel.  Roles (416 threads): warps 0-3 epilogue (TMEM lane = A
// row), warp 4 MMA issuer, TMEM owner and resident-operand loader, warps 5-12
// Ey producers.  Every wait is bounded.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace msk {

namespace {

constexpr int RS_THREADS = 416;
constexpr int RS_MAX_STAGES = 6;
constexpr int RS_APLANE = 128 * TC_BK * 2;  // one A plane of a stage (hi or lo), 8 KB
constexpr int RS_ABYTES = 2 * RS_APLANE;


__host__ __device__ inline uint32_t rs_tmem_cols(int N) {
    uint32_t c = 32;
    while ((int)c < 2 * N) c <<= 1;
    return c;
}

struct RsShared {
    uint64_t full[RS_MAX_STAGES];   // 8 producer warps
    uint64_t empty[RS_MAX_STAGES];  // MMA completion (tcgen05.commit)
    uint64_t bres;                  // resident operand copy (transaction bytes)
    uint64_t bfree;                 // MMAs reading the resident operand done
    uint64_t tfull[2];
    uint64_t tempty[2];  // 4 epilogue warps
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

// F16: FP16X3 operands (planes scaled by cscale[channel]); else BF16X3.
template <bool F16, int STAGES>
__global__ void __launch_bounds__(RS_THREADS, 1)
    k_fwd_rs(DevData d, const VisTile* __restrict__ tiles, int n_tiles, const uint16_t* __restrict__ planes,
             const float* __restrict__ cmean, const float* __restrict__ cscale, double2* __restrict__ vpart,
             int64_t z_total, uint64_t spin, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ RsShared S;
    const int N = d.N, c0 = N / 2;
    const int KS = fwd_rs_ks(N), n_slices = N / KS, nks = KS / TC_BK;
    const int slice = blockIdx.x % n_slices;
    const int group = blockIdx.x / n_slices, n_groups = gridDim.x / n_slices;
    // contiguous run of tiles per CTA: few channel changes, so few reloads
    const int t_begin = (int)((int64_t)n_tiles * group / n_groups);
    const int t_end = (int)((int64_t)n_tiles * (group + 1) / n_groups);
    const uint32_t chunk_bytes = 2u * N * TC_BK * 2;  // one 32-row chunk, hi + lo planes
    unsigned char* sB = smem;                         // resident slice: nks chunks
    unsigned char* sA = smem + (size_t)nks * chunk_bytes;
    const uint32_t tcols = rs_tmem_cols(N);
    const int64_t NN = (int64_t)N * N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abort = &S.abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&S.full[s], 8);
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.bres, 1);
        mbar_init(&S.bfree, 1);
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
        // ------------------------------------------ MMA + resident operand
        if (lane == 0) {
            const uint32_t idesc = idesc_f16kind(128, N, 0, 0, F16 ? 0 : 1);
            const uint32_t abase = smem_u32(sA), bbase = smem_u32(sB);
            const uint32_t lboB = (uint32_t)(N / 8) * 128;
            const uint32_t lo_off = (uint32_t)N * TC_BK * 2;  // lo plane within a chunk
            uint32_t sc = 0, it = 0, nres = 0;
            int cur_chan = -1;
            bool ok = true;
            for (int t = t_begin; t < t_end && ok; ++t, ++it) {
                const int chan = tiles[t].chan;
                if (chan != cur_chan) {
                    if (nres > 0) {
                        // every MMA that read the previous channel's slice has completed
                        umma_commit(&S.bfree);
                        ok = mbar_wait(&S.bfree, (nres - 1) & 1, spin, abort, status);
                        if (!ok) break;
                    }
                    const unsigned char* src = (const unsigned char*)(planes + (int64_t)chan * 2 * NN) +
                                               (int64_t)slice * nks * chunk_bytes;
                    mbar_arrive_expect_tx(&S.bres, (uint32_t)nks * chunk_bytes);
                    for (int q = 0; q < nks; ++q)
                        bulk_g2s(sB + (size_t)q * chunk_bytes, src + (size_t)q * chunk_bytes, chunk_bytes, &S.bres);
                    ok = mbar_wait(&S.bres, nres & 1, spin, abort, status);
                    ++nres;
                    if (!ok) break;
                    cur_chan = chan;
                }
                const int b = it & 1;
                ok = mbar_wait(&S.tempty[b], ((it >> 1) & 1) ^ 1, spin, abort, status);
                if (!ok) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(b * N);
                // pass 0: hi*lo and lo*hi over the slice; pass 1: hi*hi
                for (int pass = 0; pass < 2 && ok; ++pass) {
                    for (int ks = 0; ks < nks; ++ks, ++sc) {
                        const int s = sc % STAGES;
                        ok = mbar_wait(&S.full[s], (sc / STAGES) & 1, spin, abort, status);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t A = abase + s * RS_ABYTES;
                        const uint32_t B = bbase + ks * chunk_bytes;
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk) {
                            const uint32_t ao = kk * 2 * 2048, bo = kk * 2 * lboB;
                            const uint64_t a_h = smem_desc(A + ao, 2048, 128);
                            const uint64_t b_h = smem_desc(B + bo, lboB, 128);
                            if (pass == 0) {
                                const uint64_t a_l = smem_desc(A + RS_APLANE + ao, 2048, 128);
                                const uint64_t b_l = smem_desc(B + lo_off + bo, lboB, 128);
                                umma_bf16(dt, a_h, b_l, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
                                umma_bf16(dt, a_l, b_h, idesc, 1u);
                            } else {
                                umma_bf16(dt, a_h, b_h, idesc, 1u);
                            }
                        }
                        umma_commit(&S.empty[s]);
                    }
                }
                if (ok) umma_commit(&S.tfull[b]);
            }
            // every issued MMA completes before TMEM is released, and every
            // resident-operand copy lands before shared memory is released
            umma_commit(&S.drain);
            int dummy = 0;
            mbar_wait(&S.drain, 0, drain_limit(spin), (volatile int*)&dummy, status);
            if (!ok && nres > 0) mbar_wait(&S.bres, (nres - 1) & 1, drain_limit(spin), (volatile int*)&dummy, status);
        }
        __syncwarp();
    } else if (warp >= 5) {
        // --------------------------------------- Ey producers (256 threads)
        // thread -> (visibility j = ptid & 63, row group g = ptid >> 6): 8 image
        // rows of one visibility per stage, written as A rows row(j, Re), row(j, Im)
        const int ptid = threadIdx.x - 160;
        const int jv = ptid & 63, g = ptid >> 6;
        // row(j, c) = 32 (j >> 4) + 16 c + (j & 15): the 32 lanes of a store
        // instruction fill four whole 128-byte core matrices (no bank conflicts)
        const int r0 = 32 * (jv >> 4) + (jv & 15);
        const int off = (g * 16 + (r0 >> 3)) * 128 + (r0 & 7) * 16;  // Re row; Im row at +256
        uint32_t sc = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const VisTile tl = tiles[t];
            const bool valid = jv < tl.count;
            const uint64_t pb = valid ? d.pb[tl.start + jv] : 0;
            cf2 step[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) step[q] = cis_neg(phase_mul(q, pb));
            const Rot8 w = rot8_of(step);
            for (int pass = 0; pass < 2 && ok; ++pass) {
                for (int ks = 0; ks < nks; ++ks, ++sc) {
                    const int s = sc % STAGES;
                    // the table values need no ring slot: compute them, then wait
                    uint4 rh = {0, 0, 0, 0}, rl = {0, 0, 0, 0}, ih = {0, 0, 0, 0}, il = {0, 0, 0, 0};
                    if (valid) {
                        const int n0 = slice * KS + ks * TC_BK + g * 8;
                        table8_split<F16>(cis_neg(phase_mul(n0 - c0, pb)), w, rh, rl, ih, il);
                    }
                    ok = __all_sync(0xffffffffu, mbar_wait(&S.empty[s], ((sc / STAGES) & 1) ^ 1, spin, abort,
                                                           status, 64));
                    if (!ok) break;
                    unsigned char* A = sA + s * RS_ABYTES;
                    *(uint4*)(A + off) = rh;
                    *(uint4*)(A + off + 256) = ih;
                    if (pass == 0) {  // the hi*hi pass reads the hi plane only
                        *(uint4*)(A + RS_APLANE + off) = rl;
                        *(uint4*)(A + RS_APLANE + off + 256) = il;
                    }
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.full[s]);
                }
            }
        }
    } else {
        // -------------------------------- epilogue (warps 0-3, 128 threads)
        // TMEM lane = A row: warp q holds visibilities 16q .. 16q+15, lane L
        // component L >> 4 (0: Re T, 1: Im T) of visibility 16q + (L & 15)
        const int jv = 16 * warp + (lane & 15), comp = lane >> 4;
        uint32_t it = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t, ++it) {
            const VisTile tl = tiles[t];
            const bool valid = jv < tl.count;
            const int64_t j = tl.start + (valid ? jv : 0);
            const uint64_t pa = d.pa[j];
            cf2 step[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) step[q] = cis_neg(phase_mul(q, pa));
            const cf2 step8 = cis_neg(phase_mul(8, pa));
            // slice 0 adds the column-mean part c_m S_k, S_k = sum_n Ey[k,n] in
            // closed form (accurate sincospi of the exact half-turn phases)
            float scomp = 0.f;
            if (slice == 0) {
                const uint64_t pb = d.pb[j];
                const float th = (float)(int64_t)((int64_t)pb >> 1) * 5.421010862427522e-20f;       // b/2, turns
                const float tn = (float)(int64_t)phase_mul(N / 2, pb) * 5.421010862427522e-20f;  // N b/2
                float sh, ch;
                sincospif(2.0f * th, &sh, &ch);      // sin(pi b), cos(pi b)
                const float snb = sinpif(2.0f * tn);  // sin(pi N b)
                const float D = (sh != 0.f) ? snb / sh : (float)N;
                scomp = comp ? sh * D : ch * D;
            }
            const float osc = F16 ? cscale[tl.chan] : 1.f;  // operand scale (power of two)
            scomp *= osc;
            const float* cm = cmean + (int64_t)tl.chan * N;
            float s0 = 0.f, s1 = 0.f, c0s = 0.f, c1s = 0.f;  // compensated sums
            const int b = it & 1;
            ok = __all_sync(0xffffffffu, mbar_wait(&S.tfull[b], (it >> 1) & 1, spin, abort, status, 256));
            if (!ok) break;
            tc_fence_after();
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * N);
            // software pipeline over 16-column chunks (TMEM load and column
            // means of chunk q+1 in flight while chunk q is reduced)
            const int nq = N / 16;
            uint32_t tv[2][16];
            float4 cq4[2][4];
            auto load_chunk = [&](int q, int slot) {
                tmem_ld16(lane_base + q * 16, tv[slot]);
                const float4* src = (const float4*)(cm + q * 16);
#pragma unroll
                for (int k = 0; k < 4; ++k) cq4[slot][k] = __ldg(src + k);
            };
            // sum_k Ex[m0+k] t_k = base * sum_{k<8} step_k t_k + base8 * sum_{k<8} step_k t_{k+8}
            auto reduce_chunk = [&](int q, int slot) {
                const int m0 = q * 16;
                const cf2 base = cis_neg(phase_mul(m0 - c0, pa));
                const cf2 base8 = cmul(base, step8);
                const float* cq = (const float*)cq4[slot];
                float ux = 0.f, uy = 0.f, wx = 0.f, wy = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float tk = fmaf(cq[k], scomp, __uint_as_float(tv[slot][k]));
                    const float tw = fmaf(cq[k + 8], scomp, __uint_as_float(tv[slot][k + 8]));
                    ux = fmaf(step[k].x, tk, ux);
                    uy = fmaf(step[k].y, tk, uy);
                    wx = fmaf(step[k].x, tw, wx);
                    wy = fmaf(step[k].y, tw, wy);
                }
                const float a0 = fmaf(base.x, ux, fmaf(-base.y, uy, fmaf(base8.x, wx, -base8.y * wy)));
                const float a1 = fmaf(base.x, uy, fmaf(base.y, ux, fmaf(base8.x, wy, base8.y * wx)));
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
            // lane < 16: (sum ReEx ReT, sum ImEx ReT); lane >= 16: (sum ReEx ImT, sum ImEx ImT)
            const double inv = 1.0 / (double)osc;
            const double p0 = ((double)s0 + (double)c0s) * inv, p1 = ((double)s1 + (double)c1s) * inv;
            const double q0 = __shfl_xor_sync(0xffffffffu, p0, 16);
            const double q1 = __shfl_xor_sync(0xffffffffu, p1, 16);
            if (valid && comp == 0) vpart[(int64_t)slice * z_total + j] = make_double2(p0 - q1, q0 + p1);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

// One block of 64 threads per tile: V = sum of the slice partials (fixed
// order), then the forward mode (model visibilities, weighted residual,
// chi^2, curvature or line-search difference) and one chi^2 partial per 16
// visibilities, the layout the scalar reduction reads (4 per tile).
__global__ void __launch_bounds__(64) k_fwd_combine(DevData d, const VisTile* __restrict__ tiles,
                                                    const double2* __restrict__ vpart, int n_slices,
                                                    int64_t z_total, int mode, float2* yout, double* chi_part,
                                                    unsigned* ymax_bits) {
    const int t = blockIdx.x;
    const VisTile tl = tiles[t];
    const int jv = threadIdx.x;
    double chi = 0.0;
    float ym = 0.f;  // max |component| of the weighted residual (RESID mode)
    if (jv < tl.count) {
        const int64_t j = tl.start + jv;
        double Vre = 0.0, Vim = 0.0;
        for (int s = 0; s < n_slices; ++s) {
            const double2 p = vpart[(int64_t)s * z_total + j];
            Vre += p.x;
            Vim += p.y;
        }
        if (mode == FWD_VIS) {
            yout[j] = make_float2((float)Vre, (float)Vim);
        } else if (mode == FWD_DCHI) {
            const float2 yv = yout[j];
            chi = (double)yv.x * Vre + (double)yv.y * Vim + 0.5 * d.w[j] * (Vre * Vre + Vim * Vim);
        } else {
            double rr = Vre, ri = Vim;
            if (mode != FWD_CURV) {
                rr -= d.vo[j].x;
                ri -= d.vo[j].y;
            }
            const double w = d.w[j];
            chi = 0.5 * w * (rr * rr + ri * ri);
            if (mode == FWD_RESID) {
                const float2 yv = make_float2((float)(w * rr), (float)(w * ri));
                yout[j] = yv;
                ym = fmaxf(fabsf(yv.x), fabsf(yv.y));
            }
        }
    }
    if (mode == FWD_RESID && ymax_bits) {
        // order-independent maximum (non-negative floats order as their bits)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ym = fmaxf(ym, __shfl_down_sync(0xffffffffu, ym, o));
        if ((jv & 31) == 0) atomicMax(ymax_bits, __float_as_uint(ym));
    }
    if (mode != FWD_VIS) {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) chi += __shfl_down_sync(0xffffffffu, chi, o, 16);
        if ((jv & 15) == 0) chi_part[(int64_t)t * 4 + (jv >> 4)] = chi;
    }
}

template <bool F16, int STAGES>
void launch_rs_variant(const DevData& d, const VisTile* tiles, int n_tiles, const void* planes, const float* cmean,
                       const float* cscale, double2* vpart, int64_t z_total, int grid, uint64_t spin, int* status,
                       cudaStream_t st) {
    const int smem = fwd_rs_smem_bytes(d.N, STAGES);
    cudaFuncSetAttribute(k_fwd_rs<F16, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_fwd_rs<F16, STAGES><<<grid, RS_THREADS, smem, st>>>(d, tiles, n_tiles, (const uint16_t*)planes, cmean,
                                                          cscale, vpart, z_total, spin, status);
}

}  // namespace

int fwd_rs_smem_bytes(int N, int stages) { return fwd_rs_ks(N) * N * 4 + stages * RS_ABYTES + 1024; }

int fwd_rs_max_stages(int N) {
    int s = RS_MAX_STAGES;
    while (s > 2 && fwd_rs_smem_bytes(N, s) > 227 * 1024) --s;
    return s;
}

void launch_fwd_rs(const DevData& d, int f16, const VisTile* tiles, int n_tiles, const void* planes,
                   const float* cmean, const float* cscale, int mode, float2* yout, double* chi_part,
                   float* ymax, double2* vpart, int64_t z_total, int num_sms, uint64_t spin, int* status,
                   cudaStream_t st) {
    if (n_tiles <= 0) return;
    const int n_slices = d.N / fwd_rs_ks(d.N);
    // CTAs per slice: one per SM, at most one per tile
    const int per = std::max(1, std::min(num_sms / n_slices, n_tiles));
    const int grid = per * n_slices;
    const int stages = d.fwd_stages;
#define MSK_RS(F, S) launch_rs_variant<F, S>(d, tiles, n_tiles, planes, cmean, cscale, vpart, z_total, grid, spin, status, st)
    if (f16) {
        if (stages <= 4) MSK_RS(true, 4);
        else if (stages == 5) MSK_RS(true, 5);
        else MSK_RS(true, 6);
    } else {
        if (stages <= 4) MSK_RS(false, 4);
        else if (stages == 5) MSK_RS(false, 5);
        else MSK_RS(false, 6);
    }
#undef MSK_RS
    k_fwd_combine<<<n_tiles, 64, 0, st>>>(d, tiles, vpart, n_slices, z_total, mode, yout, chi_part,
                                          (unsigned*)ymax);
}

}  // namespace msk
