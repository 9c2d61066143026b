// SIMT kernels of libmemsynth: per-visibility phase preparation, the
// attenuation/operand preparation, the plain direct-sum operator pair in FP64
// and FP32 (one exponential per visibility-pixel pair, the comparators of the
// tensor-core form), gradient assembly with the entropy term and positivity
// projection, ordered FP64 reductions and the CG vector updates.
#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace msk {

// ---------------------------------------------------------------------------
// a1: per-visibility phase increments.  frac(u dx) reduced in FP64 and held as
// a 64-bit fixed-point fraction of a turn; pixel phases are then exact integer
// multiples (Eq. 1 on the grid x_m = (m - N/2) dx).
// ---------------------------------------------------------------------------
__global__ void k_phase_prep(int64_t Z, const double* __restrict__ u, const double* __restrict__ v,
                             double dx, double dy, uint64_t* __restrict__ pa,
                             uint64_t* __restrict__ pb) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Z) return;
    pa[k] = to_fixed_turns(u[k] * dx);
    pb[k] = to_fixed_turns(v[k] * dy);
}

void launch_phase_prep(int64_t Z, const double* u, const double* v, double dx, double dy,
                       uint64_t* pa, uint64_t* pb, cudaStream_t st) {
    if (Z <= 0) return;
    k_phase_prep<<<(unsigned)((Z + 255) / 256), 256, 0, st>>>(Z, u, v, dx, dy, pa, pb);
}


template <int BLOCK>
__device__ __forceinline__ double block_max(double x, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        r = sh[0];
        for (int i = 1; i < BLOCK / 32; ++i) r = fmax(r, sh[i]);
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ int image_of(const DevData& d, int c) { return d.shared ? 0 : c; }


// ---------------------------------------------------------------------------
// a2: attenuation and operand preparation.  B_c = A_c * I.  The BF16x3 form
// stores hi/lo planes pre-arranged in the tensor-core operand layout of the
// forward kernel: per channel, chunks (m-block mb, n-stage ks) of BN x BK
// elements, K-major interleaved 8x8 core matrices, hi plane then lo plane.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t tc_plane_index(int n, int m, int N, int BN) {
    int nk = N / TC_BK;
    int mb = m / BN, r = m % BN, ks = n / TC_BK, k = n % TC_BK;
    int64_t chunk = (int64_t)mb * nk + ks;
    int64_t chunk_elems = (int64_t)2 * BN * TC_BK;  // hi + lo
    int64_t off = ((int64_t)(k / 8) * (BN / 8) + r / 8) * 64 + (r % 8) * 8 + (k % 8);
    return chunk * chunk_elems + off;  // in bf16 elements; lo at + BN*BK
}

// Column means c_m = (1/N) sum_n B[n][m] per channel (the operand of the
// tensor-core forward is centred column by column, see k_fwd_tc), in two
// stages with a fixed summation order.  Stage 1: block (column block of 32,
// row block rb of N/COL_RB rows, channel) -> partial sums and max |B| per
// column.  Stage 2, run by the channel's last stage-1 block to finish (a
// completion counter per channel, which that block resets): c_m, then the
// bound max_n |B[n][m] - c_m| <= max|B| + |c_m| maximised over the channel,
// and from it the channel's power-of-two FP16X3 operand scale.
constexpr int COL_RB = 16;

__global__ void __launch_bounds__(256) k_colsum(DevData d, ImgSrc src, double* __restrict__ psum,
                                                float* __restrict__ pmax, unsigned* __restrict__ count,
                                                float* __restrict__ cmean, float* __restrict__ cscale,
                                                float* __restrict__ ymax_clear) {
    __shared__ double sh[8][33];
    __shared__ float shm[8][33];
    __shared__ bool last;
    const int N = d.N;
    const int64_t NN = (int64_t)N * N;
    const int c = blockIdx.z, rb = blockIdx.y;
    const int i = image_of(d, c);
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * 32 + lane;
    const int rg = threadIdx.x >> 5;
    // the FP16X3 residual maximum of the forward that follows starts at zero
    if (ymax_clear && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) *ymax_clear = 0.f;
    const int n0 = (int)((int64_t)N * rb / COL_RB), n1 = (int)((int64_t)N * (rb + 1) / COL_RB);
    double acc = 0.0;
    float amax = 0.f;
    if (m < N) {
        for (int n = n0 + rg; n < n1; n += 8) {
            const int64_t p = (int64_t)n * N + m;
            double x = img_value(src, i, p, NN);
            if (src.diff) x -= src.f64[(int64_t)i * NN + p];
            const double b = (double)d.beam[(int64_t)c * NN + p] * x;
            acc += b;
            amax = fmaxf(amax, (float)fabs(b));
        }
    }
    sh[rg][lane] = acc;
    shm[rg][lane] = amax;
    __syncthreads();
    if (rg == 0 && m < N) {
        double t = 0.0;
        float mx = 0.f;
        for (int k = 0; k < 8; ++k) {
            t += sh[k][lane];
            mx = fmaxf(mx, shm[k][lane]);
        }
        psum[((int64_t)c * COL_RB + rb) * N + m] = t;
        pmax[((int64_t)c * COL_RB + rb) * N + m] = mx;
        __threadfence();  // each writer's partials visible device-wide before the count below
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&count[c], 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // stage 2: the partials of channel c in row-block order (read through L2)
    float bound = 0.f;
    for (int mm = threadIdx.x; mm < N; mm += blockDim.x) {
        double t = 0.0;
        float mx = 0.f;
#pragma unroll
        for (int r = 0; r < COL_RB; ++r) {
            t += __ldcg(psum + ((int64_t)c * COL_RB + r) * N + mm);
            mx = fmaxf(mx, __ldcg(pmax + ((int64_t)c * COL_RB + r) * N + mm));
        }
        const float cm = (float)(t / N);
        cmean[(int64_t)c * N + mm] = cm;
        bound = fmaxf(bound, mx + fabsf(cm));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bound = fmaxf(bound, __shfl_down_sync(0xffffffffu, bound, o));
    if (lane == 0) shm[0][rg] = bound;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mx = 0.f;
        for (int k = 0; k < 8; ++k) mx = fmaxf(mx, shm[0][k]);
        cscale[c] = pow2_scale_for(mx);
        count[c] = 0;  // ready for the next evaluation
    }
}

void launch_colmean(const DevData& d, const ImgSrc& src, float* cmean, float* cscale, double* psum, float* pmax,
                    unsigned* count, float* ymax_clear, cudaStream_t st) {
    k_colsum<<<dim3(colmean_blocks(d.N), COL_RB, d.C), 256, 0, st>>>(d, src, psum, pmax, count, cmean, cscale,
                                                                    ymax_clear);
}

int colmean_tmp_count(int N, int C) { return COL_RB * N * C; }

// max |y| over n floats: 256 block maxima, then one block forms the scale.
__global__ void __launch_bounds__(256) k_absmax_part(int64_t n, const float* __restrict__ y,
                                                     float* __restrict__ part) {
    float mx = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < n; k += (int64_t)gridDim.x * 256)
        mx = fmaxf(mx, fabsf(y[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    __shared__ float sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = sh[0];
        for (int k = 1; k < 8; ++k) t = fmaxf(t, sh[k]);
        part[blockIdx.x] = t;
    }
}

__global__ void k_absmax_final(const float* __restrict__ part, float* ymax) {
    if (threadIdx.x != 0) return;
    float t = 0.f;
    for (int k = 0; k < 256; ++k) t = fmaxf(t, part[k]);
    ymax[0] = t;
}

void launch_absmax(int64_t n, const float* y, float* part, float* ymax, cudaStream_t st) {
    k_absmax_part<<<256, 256, 0, st>>>(n, y, part);
    k_absmax_final<<<1, 32, 0, st>>>(part, ymax);
}

__global__ void __launch_bounds__(256) k_prep(DevData d, ImgSrc src, int fmt, void* bout,
                                              double* ent_part, const float* __restrict__ cmean,
                                              const float* __restrict__ cscale) {
    __shared__ double sh[8];
    const int N = d.N;
    const int64_t NN = (int64_t)N * N;
    const int c = blockIdx.y;
    const int i = image_of(d, c);
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    // the entropy partial of an image is formed by its first channel only
    // (the others would repeat it in the shared-image mode)
    const bool ent = ent_part && !(d.shared && c != 0);
    double e = 0.0;
    if (p < NN) {
        double x = img_value(src, i, p, NN);
        double xb = x;
        if (src.diff) {
            // line-search probe as a difference from the base image I: the
            // operand is delta = max(I + alpha d, G) - I, the entropy term the
            // change of sum x log(x/G)
            const double x0 = src.f64[(int64_t)i * NN + p];
            xb = x - x0;
            if (ent) e = x * log(x / src.G) - x0 * log(x0 / src.G);
        } else if (ent) {
            e = x * log(x / src.G);
        }
        double b = (double)d.beam[(int64_t)c * NN + p] * xb;
        if (fmt == BF_F32) {
            ((float*)bout)[(int64_t)c * NN + p] = (float)b;
        } else if (fmt == BF_F64) {
            ((double*)bout)[(int64_t)c * NN + p] = b;
        } else {
            int n = (int)(p / N), m = (int)(p % N);
            int BN = d.fwd_bn;
            const double cb = b - (cmean ? (double)cmean[(int64_t)c * N + m] : 0.0);
            const int64_t q = tc_plane_index(n, m, N, BN);
            if (fmt == BF_BF16X3) {
                const float bf = (float)cb;
                __nv_bfloat16 hi = __float2bfloat16_rn(bf);
                __nv_bfloat16 lo = __float2bfloat16_rn(bf - __bfloat162float(hi));
                __nv_bfloat16* base = (__nv_bfloat16*)bout + (int64_t)c * 2 * NN;
                base[q] = hi;
                base[q + (int64_t)BN * TC_BK] = lo;
            } else {
                const float sc = cscale[c];
                const float bf = (float)(cb * (double)sc);
                __half hi = __float2half_rn(bf);
                __half lo = __float2half_rn(bf - __half2float(hi));
                __half* base = (__half*)bout + (int64_t)c * 2 * NN;
                base[q] = hi;
                base[q + (int64_t)BN * TC_BK] = lo;
            }
        }
    }
    if (ent) {  // uniform over the block (one channel per block row)
        double s = block_sum<256>(e, sh);
        if (threadIdx.x == 0) ent_part[(int64_t)i * gridDim.x + blockIdx.x] = -s;
    }
}


void launch_prep(const DevData& d, const ImgSrc& src, int fmt, void* bout, double* ent_part,
                 const float* cmean, const float* cscale, cudaStream_t st) {
    dim3 grid(prep_blocks(d.N), d.C);
    k_prep<<<grid, 256, 0, st>>>(d, src, fmt, bout, ent_part, cmean, cscale);
}

// ---------------------------------------------------------------------------
// a12: direct-sum forward, one thread per visibility, one exponential per
// (visibility, pixel) pair.  Image rows are staged in shared memory; each row's
// sum is formed in the working precision and added to an FP64 accumulator.
// Fused epilogue (Algorithm 2 + the reduction of Algorithm 1): residual,
// weight, chi^2 tile partial.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cis_minus(uint64_t p, T& c, T& s);
template <>
__device__ __forceinline__ void cis_minus<float>(uint64_t p, float& c, float& s) {
    __sincosf(phase_to_angle_f32(p), &s, &c);
}
template <>
__device__ __forceinline__ void cis_minus<double>(uint64_t p, double& c, double& s) {
    sincospi(2.0 * phase_to_turns_f64(p), &s, &c);
}

template <typename T>
__global__ void __launch_bounds__(128) k_fwd_direct(DevData d, const VisTile* __restrict__ tiles,
                                                    const T* __restrict__ B, int mode, void* yout,
                                                    double* __restrict__ chi_part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* row = (T*)smraw;
    const VisTile t = tiles[blockIdx.x];
    const int N = d.N, c0 = N / 2;
    const int64_t NN = (int64_t)N * N;
    const bool valid = (int)threadIdx.x < t.count;
    const int64_t j = t.start + (valid ? threadIdx.x : 0);
    const uint64_t a = d.pa[j], b = d.pb[j];
    const T* Bc = B + (int64_t)t.chan * NN;
    double re = 0.0, im = 0.0;
    const uint64_t pstart = phase_mul(-c0, a);
    for (int n = 0; n < N; ++n) {
        __syncthreads();
        for (int m = threadIdx.x; m < N; m += 128) row[m] = Bc[(int64_t)n * N + m];
        __syncthreads();
        uint64_t p = pstart + phase_mul(n - c0, b);
        T rr = 0, ri = 0;
        for (int m = 0; m < N; ++m) {
            T cs, sn;
            cis_minus<T>(p, cs, sn);
            T bv = row[m];
            rr += bv * cs;
            ri -= bv * sn;
            p += a;
        }
        re += (double)rr;
        im += (double)ri;
    }
    double chi = 0.0;
    if (valid) {
        if (mode == FWD_VIS) {
            if (sizeof(T) == 8) ((double2*)yout)[j] = make_double2(re, im);
            else ((float2*)yout)[j] = make_float2((float)re, (float)im);
        } else if (mode == FWD_DCHI) {
            double yr, yi;
            if (sizeof(T) == 8) { double2 q = ((const double2*)yout)[j]; yr = q.x; yi = q.y; }
            else { float2 q = ((const float2*)yout)[j]; yr = q.x; yi = q.y; }
            chi = yr * re + yi * im + 0.5 * d.w[j] * (re * re + im * im);
        } else {
            double rr = re, ri = im;
            if (mode != FWD_CURV) { rr -= d.vo[j].x; ri -= d.vo[j].y; }
            double w = d.w[j];
            chi = 0.5 * w * (rr * rr + ri * ri);
            if (mode == FWD_RESID) {
                if (sizeof(T) == 8) ((double2*)yout)[j] = make_double2(w * rr, w * ri);
                else ((float2*)yout)[j] = make_float2((float)(w * rr), (float)(w * ri));
            }
        }
    }
    if (mode != FWD_VIS) {
        // one partial per warp (32 visibilities), summed later in a fixed order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) chi += __shfl_down_sync(0xffffffffu, chi, o);
        if ((threadIdx.x & 31) == 0) chi_part[(int64_t)blockIdx.x * 4 + (threadIdx.x >> 5)] = chi;
    }
}

void launch_fwd_direct(const DevData& d, int fp64, const VisTile* tiles, int n_tiles, const void* B,
                       int mode, void* yout, double* chi_part, cudaStream_t st) {
    if (n_tiles <= 0) return;
    if (fp64) {
        k_fwd_direct<double><<<n_tiles, 128, d.N * sizeof(double), st>>>(d, tiles, (const double*)B,
                                                                        mode, yout, chi_part);
    } else {
        k_fwd_direct<float><<<n_tiles, 128, d.N * sizeof(float), st>>>(d, tiles, (const float*)B,
                                                                      mode, yout, chi_part);
    }
}

// ---------------------------------------------------------------------------
// a12: direct-sum adjoint (the gradient kernel of Section 2.5): each thread
// owns ADJ_PPT adjacent pixels of a row and loops over a slice of the
// channel's visibilities staged in shared memory; slices (blockIdx.z) are
// summed later in a fixed order.  Sixteen pixels per thread share each
// visibility's phase set-up (two 64-bit products) among sixteen pairs, which
// leaves the FP32 form bound by its two SFU operations per pair (2 -> 16:
// 43 -> 31 ms per launch at 256^2 with 999,600 visibilities).
// ---------------------------------------------------------------------------
constexpr int ADJ_PPT = 16;
constexpr int ADJ_CHUNK = 256;

template <typename T, typename T2>
__global__ void __launch_bounds__(128) k_adj_direct(DevData d, const T2* __restrict__ y,
                                                    double* __restrict__ gsum, int ks) {
    __shared__ uint64_t sa[ADJ_CHUNK], sb[ADJ_CHUNK];
    __shared__ T syr[ADJ_CHUNK], syi[ADJ_CHUNK];
    const int N = d.N, c0 = N / 2;
    const int64_t NN = (int64_t)N * N;
    const int c = blockIdx.y;
    const int64_t pix = ((int64_t)blockIdx.x * 128 + threadIdx.x) * ADJ_PPT;
    const bool valid = pix < NN;
    const int n = valid ? (int)(pix / N) : 0, m0 = valid ? (int)(pix % N) : 0;
    const int64_t v0 = d.off[c], v1 = d.off[c + 1];
    const int64_t len = v1 - v0;
    const int64_t k0 = v0 + len * blockIdx.z / ks, k1 = v0 + len * (blockIdx.z + 1) / ks;
    double acc[ADJ_PPT];
#pragma unroll
    for (int q = 0; q < ADJ_PPT; ++q) acc[q] = 0.0;
    for (int64_t base = k0; base < k1; base += ADJ_CHUNK) {
        int cnt = (int)((k1 - base) < ADJ_CHUNK ? (k1 - base) : ADJ_CHUNK);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += 128) {
            sa[q] = d.pa[base + q];
            sb[q] = d.pb[base + q];
            T2 yy = y[base + q];
            syr[q] = yy.x;
            syi[q] = yy.y;
        }
        __syncthreads();
        T part[ADJ_PPT];
#pragma unroll
        for (int q = 0; q < ADJ_PPT; ++q) part[q] = 0;
        for (int k = 0; k < cnt; ++k) {
            uint64_t p = phase_mul(m0 - c0, sa[k]) + phase_mul(n - c0, sb[k]);
            T yr = syr[k], yi = syi[k];
#pragma unroll
            for (int q = 0; q < ADJ_PPT; ++q) {
                T cs, sn;
                cis_minus<T>(p, cs, sn);
                // Re(y e^{+i theta}) = yr cos - yi sin
                part[q] += yr * cs - yi * sn;
                p += sa[k];
            }
        }
#pragma unroll
        for (int q = 0; q < ADJ_PPT; ++q) acc[q] += (double)part[q];
    }
    if (valid) {
        double* out = gsum + ((int64_t)blockIdx.z * d.C + c) * NN + pix;
#pragma unroll
        for (int q = 0; q < ADJ_PPT; ++q) out[q] = acc[q];
    }
}

int adj_direct_splits(const DevData& d, int num_sms) {
    int64_t NN = (int64_t)d.N * d.N;
    int64_t blocks = (NN / ADJ_PPT + 127) / 128 * d.C;
    int64_t want = 4LL * num_sms;
    int ks = (int)((want + blocks - 1) / blocks);
    if (ks < 1) ks = 1;
    if (ks > 64) ks = 64;
    return ks;
}

void launch_adj_direct(const DevData& d, int fp64, const void* y, double* gsum, int ks,
                       cudaStream_t st) {
    int64_t NN = (int64_t)d.N * d.N;
    dim3 grid((unsigned)((NN / ADJ_PPT + 127) / 128), d.C, ks);
    if (fp64) k_adj_direct<double, double2><<<grid, 128, 0, st>>>(d, (const double2*)y, gsum, ks);
    else k_adj_direct<float, float2><<<grid, 128, 0, st>>>(d, (const float2*)y, gsum, ks);
}

// ---------------------------------------------------------------------------
// a7: gradient assembly.  grad chi^2 of image i is the sum over its channels
// of A_c times the channel's adjoint sum (Eq. chi2gradient with the beam
// factor; Eq. chi2-multi for a shared image), plus lambda (1 + log(I/G))
// (Eq. Sgradient), then the positive projection at the bound I = G.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finalize(DevData d, ImgSrc src,
                                                  const double* __restrict__ gsum, int ks,
                                                  int projected, float* out32, double* full64,
                                                  double* proj64) {
    const int N = d.N;
    const int64_t NN = (int64_t)N * N;
    const int i = blockIdx.y;
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p >= NN) return;
    int c_lo = d.shared ? 0 : i, c_hi = d.shared ? d.C : i + 1;
    double g = 0.0;
    for (int c = c_lo; c < c_hi; ++c) {
        double s = 0.0;
        for (int k = 0; k < ks; ++k) s += gsum[((int64_t)k * d.C + c) * NN + p];
        g += (double)d.beam[(int64_t)c * NN + p] * s;
    }
    double x = img_value(src, i, p, NN);
    if (d.lambda != 0.0) g += d.lambda * (1.0 + log(x / d.G));
    double gp = (x <= d.G && g > 0.0) ? 0.0 : g;
    if (full64) full64[(int64_t)i * NN + p] = g;
    if (proj64) proj64[(int64_t)i * NN + p] = gp;
    if (out32) out32[(int64_t)i * NN + p] = (float)(projected ? gp : g);
}

void launch_finalize(const DevData& d, const ImgSrc& src, const double* gsum, int ks, int projected,
                     float* out32, double* full64, double* proj64, cudaStream_t st) {
    dim3 grid(prep_blocks(d.N), d.n_images);
    k_finalize<<<grid, 256, 0, st>>>(d, src, gsum, ks, projected, out32, full64, proj64);
}

// ---------------------------------------------------------------------------
// Ordered FP64 reductions of tile partials into per-image and total scalars.
// scal layout: [0..2] = Phi, chi^2, S totals; [3 + 3i ...] per image.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scalars(DevData d, const int* __restrict__ tile_off,
                                                 const double* __restrict__ chi_part,
                                                 const double* __restrict__ ent_part, int with_entropy,
                                                 int n_ent_blocks, double* part, double* img_tmp, double* scal,
                                                 unsigned* counter) {
    scalars_block(d, tile_off, chi_part, ent_part, with_entropy, n_ent_blocks, part, img_tmp, scal, counter,
                  blockIdx.x, blockIdx.y);
}

void launch_scalars(const DevData& d, const int* tile_off, const double* chi_part,
                    const double* ent_part, int with_entropy, double* scal, double* img_tmp,
                    cudaStream_t st) {
    double* part = scalars_part(img_tmp, d.n_images);
    unsigned* counter = scalars_counter(img_tmp, d.n_images);
    k_scalars<<<dim3(d.n_images, SCAL_SPLIT), 256, 0, st>>>(d, tile_off, chi_part, ent_part, with_entropy,
                                                             prep_blocks(d.N), part, img_tmp, scal, counter);
}

int scalars_tmp_doubles(int n_images) { return 3 * n_images + 2 * SCAL_SPLIT * n_images + 1; }

// ---------------------------------------------------------------------------
// a8: CG vector kernels (FP64), per image.
// DOT_BETA : out[2i] = gprev.gprev, out[2i+1] = (g - gprev).g   (Polak-Ribiere)
// DOT_SLOPE: out[2i] = gfull.d,     out[2i+1] = g.g
// DOT_MAX  : out[2i] = max I,       out[2i+1] = max |d|
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dots_part(DevData d, int which, const double* __restrict__ a,
                                                   const double* __restrict__ b,
                                                   const double* __restrict__ c, double* part) {
    __shared__ double sh[8];
    const int64_t NN = (int64_t)d.N * d.N;
    const int i = blockIdx.y;
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double x0 = 0.0, x1 = 0.0;
    if (p < NN) {
        const int64_t q = (int64_t)i * NN + p;
        if (which == DOT_BETA) {          // a = g, b = gprev
            x0 = b[q] * b[q];
            x1 = (a[q] - b[q]) * a[q];
        } else if (which == DOT_SLOPE) {  // a = gfull, b = d, c = g
            x0 = a[q] * b[q];
            x1 = c[q] * c[q];
        } else {                          // a = I, b = d
            x0 = a[q];
            x1 = fabs(b[q]);
        }
    }
    double r0, r1;
    if (which == DOT_MAX) {
        r0 = block_max<256>(x0, sh);
        r1 = block_max<256>(x1, sh);
    } else {
        r0 = block_sum<256>(x0, sh);
        r1 = block_sum<256>(x1, sh);
    }
    if (threadIdx.x == 0) {
        part[((int64_t)i * gridDim.x + blockIdx.x) * 2] = r0;
        part[((int64_t)i * gridDim.x + blockIdx.x) * 2 + 1] = r1;
    }
}

__global__ void __launch_bounds__(256) k_dots_final(int which, int nblk, const double* __restrict__ part,
                                                    double* out) {
    __shared__ double sh[8];
    const int i = blockIdx.x;
    double x0 = (which == DOT_MAX) ? 0.0 : 0.0, x1 = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 256) {
        double p0 = part[((int64_t)i * nblk + b) * 2], p1 = part[((int64_t)i * nblk + b) * 2 + 1];
        if (which == DOT_MAX) { x0 = fmax(x0, p0); x1 = fmax(x1, p1); }
        else { x0 += p0; x1 += p1; }
    }
    double r0, r1;
    if (which == DOT_MAX) { r0 = block_max<256>(x0, sh); r1 = block_max<256>(x1, sh); }
    else { r0 = block_sum<256>(x0, sh); r1 = block_sum<256>(x1, sh); }
    if (threadIdx.x == 0) { out[2 * i] = r0; out[2 * i + 1] = r1; }
}

void launch_dots(const DevData& d, int which, const double* a, const double* b, const double* c,
                 double* part, double* out, cudaStream_t st) {
    int nblk = prep_blocks(d.N);
    k_dots_part<<<dim3(nblk, d.n_images), 256, 0, st>>>(d, which, a, b, c, part);
    k_dots_final<<<d.n_images, 256, 0, st>>>(which, nblk, part, out);
}

// Search direction per image, mode_i: 0 keep, 1 d = -g + beta_i d, 2 d = -g;
// then the bound projection: a pixel at I = G cannot move down.
__global__ void __launch_bounds__(256) k_cg_direction(DevData d, const double* __restrict__ I,
                                                      const double* __restrict__ g,
                                                      const double* __restrict__ beta,
                                                      const int* __restrict__ mode, double* dir) {
    const int64_t NN = (int64_t)d.N * d.N;
    const int i = blockIdx.y;
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p >= NN || mode[i] == 0) return;
    const int64_t q = (int64_t)i * NN + p;
    double nd = mode[i] == 2 ? -g[q] : -g[q] + beta[i] * dir[q];
    if (I[q] <= d.G && nd < 0.0) nd = 0.0;
    dir[q] = nd;
}

void launch_cg_direction(const DevData& d, const double* I, const double* g, const double* beta,
                         const int* mode, double* dir, cudaStream_t st) {
    k_cg_direction<<<dim3(prep_blocks(d.N), d.n_images), 256, 0, st>>>(d, I, g, beta, mode, dir);
}

// I = max(I + alpha_i d, G) for images with alpha_i > 0.
__global__ void __launch_bounds__(256) k_cg_step(DevData d, double* I, const double* __restrict__ dir,
                                                 const double* __restrict__ alpha) {
    const int64_t NN = (int64_t)d.N * d.N;
    const int i = blockIdx.y;
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p >= NN || !(alpha[i] > 0.0)) return;
    const int64_t q = (int64_t)i * NN + p;
    I[q] = fmax(I[q] + alpha[i] * dir[q], d.G);
}

void launch_cg_step(const DevData& d, double* I, const double* dir, const double* alpha,
                    cudaStream_t st) {
    k_cg_step<<<dim3(prep_blocks(d.N), d.n_images), 256, 0, st>>>(d, I, dir, alpha);
}

__global__ void k_clip_f32_to_f64(int64_t n, const float* __restrict__ in, double* __restrict__ out,
                                  double G) {
    int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p < n) out[p] = fmax((double)in[p], G);
}

void launch_clip_f32_to_f64(const DevData& d, const float* in, double* out, cudaStream_t st) {
    int64_t n = (int64_t)d.n_images * d.N * d.N;
    k_clip_f32_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, in, out, d.G);
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p < n) out[p] = (float)in[p];
}

void launch_f64_to_f32(int64_t n, const double* in, float* out, cudaStream_t st) {
    if (n <= 0) return;
    k_f64_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, in, out);
}

}  // namespace msk

namespace msk {

// ---------------------------------------------------------------------------
// Dirty image and PSF (Appendix A, Eq. dirty and Eq. PSF): the adjoint of
// y_k = omega_k V_k (or omega_k), omega_k = w_k / (sum of w over the channel);
// the sum of the adjoint's splits per channel, without the primary beam.
// ---------------------------------------------------------------------------
// what: 0 measured visibilities, 1 PSF (V = 1), 2 residuals V° - V, with the
// model V read from y64 (FP64 form) or y32 at the same index it overwrites.
__global__ void __launch_bounds__(256) k_dirty_y(DevData d, const double* __restrict__ wsum, int what,
                                                 int64_t z_total, float2* __restrict__ y32,
                                                 double2* __restrict__ y64) {
    const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (j >= z_total) return;
    int lo = 0, hi = d.C;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (d.off[mid] <= j) lo = mid;
        else hi = mid;
    }
    const double om = d.w[j] / wsum[lo];
    double2 v = what == 1 ? make_double2(1.0, 0.0) : d.vo[j];
    if (what == 2) {
        const double2 m = y64 ? y64[j] : make_double2((double)y32[j].x, (double)y32[j].y);
        v.x -= m.x;
        v.y -= m.y;
    }
    y32[j] = make_float2((float)(om * v.x), (float)(om * v.y));
    if (y64) y64[j] = make_double2(om * v.x, om * v.y);
}

__global__ void __launch_bounds__(256) k_dirty_out(DevData d, const double* __restrict__ gsum, int ks,
                                                   float* __restrict__ out) {
    const int64_t NN = (int64_t)d.N * d.N;
    const int c = blockIdx.y;
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p >= NN) return;
    double s = 0.0;
    for (int k = 0; k < ks; ++k) s += gsum[((int64_t)k * d.C + c) * NN + p];
    out[(int64_t)c * NN + p] = (float)s;
}

void launch_dirty_y(const DevData& d, const double* wsum, int what, int64_t z_total, float2* y32, double2* y64,
                    cudaStream_t st) {
    if (z_total <= 0) return;
    k_dirty_y<<<(unsigned)((z_total + 255) / 256), 256, 0, st>>>(d, wsum, what, z_total, y32, y64);
}

void launch_dirty_out(const DevData& d, const double* gsum, int ks, float* out, cudaStream_t st) {
    dim3 grid(prep_blocks(d.N), d.C);
    k_dirty_out<<<grid, 256, 0, st>>>(d, gsum, ks, out);
}

}  // namespace msk
