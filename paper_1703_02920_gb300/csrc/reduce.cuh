// Block-level reductions shared by the SIMT kernels and the adjoint's
// reduction kernel: a fixed-order block sum and the ordered FP64 reduction of
// the chi^2 tile partials and entropy partials into the objective scalars.
#pragma once

#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace msk {

// ---------------------------------------------------------------------------
// block reductions (fixed tree: deterministic)
// ---------------------------------------------------------------------------
template <int BLOCK>
__device__ __forceinline__ double block_sum(double x, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < BLOCK / 32; ++i) r += sh[i];
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// Ordered FP64 reductions of tile partials into per-image and total scalars.
// scal layout: [0..2] = Phi, chi^2, S totals; [3 + 3i ...] per image.
// ---------------------------------------------------------------------------
// SCAL_SPLIT blocks per image; block (i, q) sums a contiguous share of image
// i's chi^2 partials and entropy partials in a fixed order; the last of the
// n_images x SCAL_SPLIT blocks to finish adds the shares in order.
constexpr int SCAL_SPLIT = 32;

// img_tmp: 3 * n_images totals, 2 * SCAL_SPLIT * n_images partials, then the
// completion counter (zero between evaluations)
__device__ __host__ inline double* scalars_part(double* img_tmp, int n_images) { return img_tmp + 3 * n_images; }
__device__ __host__ inline unsigned* scalars_counter(double* img_tmp, int n_images) {
    return (unsigned*)(scalars_part(img_tmp, n_images) + 2 * SCAL_SPLIT * n_images);
}

// Every thread of the block calls this (block-wide barriers inside).
__device__ __forceinline__ void scalars_block(const DevData& d, const int* __restrict__ tile_off,
                                              const double* __restrict__ chi_part,
                                              const double* __restrict__ ent_part, int with_entropy,
                                              int n_ent_blocks, double* part, double* img_tmp, double* scal,
                                              unsigned* counter, int i, int q) {
    __shared__ double sh[8];
    __shared__ bool last;
    int c_lo = d.shared ? 0 : i, c_hi = d.shared ? d.C : i + 1;
    const int64_t t0 = 4LL * tile_off[c_lo], t1 = 4LL * tile_off[c_hi];  // channels are contiguous
    const int64_t len = t1 - t0;
    const int64_t a = t0 + len * q / SCAL_SPLIT, b = t0 + len * (q + 1) / SCAL_SPLIT;
    double x = 0.0;
    for (int64_t t = a + threadIdx.x; t < b; t += 256) x += chi_part[t];
    const double chi = block_sum<256>(x, sh);
    double S = 0.0;
    if (with_entropy) {
        const int e0 = (int)((int64_t)n_ent_blocks * q / SCAL_SPLIT), e1 = (int)((int64_t)n_ent_blocks * (q + 1) / SCAL_SPLIT);
        double y = 0.0;
        for (int e = e0 + threadIdx.x; e < e1; e += 256) y += ent_part[(int64_t)i * n_ent_blocks + e];
        S = block_sum<256>(y, sh);
    }
    if (threadIdx.x == 0) {
        part[((int64_t)i * SCAL_SPLIT + q) * 2] = chi;
        part[((int64_t)i * SCAL_SPLIT + q) * 2 + 1] = S;
        // the last block to finish forms the totals
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)(d.n_images * SCAL_SPLIT) - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // Stage 2 (last block): one thread per image sums its SCAL_SPLIT partials
    // in order (read through L2); thread 0 then forms the totals in image order
    for (int im = threadIdx.x; im < d.n_images; im += blockDim.x) {
        double c2 = 0.0, s2 = 0.0;
        for (int k = 0; k < SCAL_SPLIT; ++k) {
            c2 += __ldcg(part + ((int64_t)im * SCAL_SPLIT + k) * 2);
            s2 += __ldcg(part + ((int64_t)im * SCAL_SPLIT + k) * 2 + 1);
        }
        img_tmp[3 * im] = c2 - d.lambda * s2;
        img_tmp[3 * im + 1] = c2;
        img_tmp[3 * im + 2] = s2;
        scal[3 + 3 * im] = c2 - d.lambda * s2;
        scal[4 + 3 * im] = c2;
        scal[5 + 3 * im] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0, tb = 0, tc = 0;
        for (int im = 0; im < d.n_images; ++im) {
            ta += img_tmp[3 * im];
            tb += img_tmp[3 * im + 1];
            tc += img_tmp[3 * im + 2];
        }
        scal[0] = ta;
        scal[1] = tb;
        scal[2] = tc;
        *counter = 0;  // ready for the next evaluation
    }
}

}  // namespace msk
