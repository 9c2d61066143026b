// The paper's gridded forward (Section 2.4, the steps of the objective
// evaluation; Algorithm alg:chi2gpu): attenuation, zero padding to
// M = pad N, a 2-D FFT of every channel's image on the grid, the
// phase-centre modulation and bilinear interpolation at each sample's grid
// coordinates.  An approximation of Eq. (1): its error against the exact sum
// falls about as 1/pad^2 (bilinear interpolation of a band-limited grid).
//
// The 2-D real-to-complex transform is this file's own:
//   rows    : the N non-zero rows of the padded image, two real rows per
//             complex transform of length M (z = row_a + i row_b; the two
//             spectra follow from Hermitian symmetry), half spectrum
//             k = 0..M/2 written column-major, R[c][k][n];
//   columns : for each of the M/2 + 1 frequency columns, a complex
//             transform of length M over the padded rows (only the N window
//             rows are non-zero), giving F[c][l][k].
// Each transform runs in one CTA in shared memory: a Stockham (autosorting,
// ping-pong) mixed-radix FFT with radix-4 and radix-2 stages and, for the
// odd factor of pad (3, 5, 7), one stage of direct small DFTs; twiddles from
// sincospif of exact fractions of a turn.  FP32 throughout.
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace msk {

namespace {

constexpr int FFT_THREADS = 256;

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// exp(-2 pi i q / d) for integers 0 <= q < d
__device__ __forceinline__ float2 c_root(int q, int d) {
    float s, c;
    sincospif(2.0f * (float)q / (float)d, &s, &c);
    return make_float2(c, -s);
}

// The radices of M (product = M): 4s, then one 2, then one odd factor.
struct FftPlan {
    int n_st;
    int r[16];
};

__device__ __forceinline__ FftPlan fft_plan(int M) {
    FftPlan p;
    p.n_st = 0;
    int odd = M;
    while (!(odd & 1)) odd >>= 1;
    int two = M / odd;
    while (two % 4 == 0) {
        p.r[p.n_st++] = 4;
        two /= 4;
    }
    if (two == 2) p.r[p.n_st++] = 2;
    if (odd > 1) p.r[p.n_st++] = odd;
    return p;
}

// Forward DFT, X[k] = sum_t x[t] exp(-2 pi i k t / M), of the M values in
// a[] (shared memory; b[] is the ping-pong buffer).  Returns the buffer that
// holds the result.  All threads of the block take part.
__device__ float2* fft_shared(float2* a, float2* b, int M) {
    const FftPlan p = fft_plan(M);
    int Ns = 1;
    for (int st = 0; st < p.n_st; ++st) {
        const int R = p.r[st];
        const int nb = M / R;
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            const int jm = j % Ns;
            float2 v[7];
            // load with twiddles exp(-2 pi i r jm / (Ns R))
            for (int r = 0; r < R; ++r) {
                const float2 x = a[j + r * nb];
                v[r] = r == 0 ? x : c_mul(x, c_root((r * jm) % (Ns * R), Ns * R));
            }
            float2 o[7];
            if (R == 4) {
                const float2 s02 = c_add(v[0], v[2]), d02 = c_sub(v[0], v[2]);
                const float2 s13 = c_add(v[1], v[3]), d13 = c_sub(v[1], v[3]);
                const float2 md13 = make_float2(d13.y, -d13.x);  // -i (v1 - v3)
                o[0] = c_add(s02, s13);
                o[1] = c_add(d02, md13);
                o[2] = c_sub(s02, s13);
                o[3] = c_sub(d02, md13);
            } else if (R == 2) {
                o[0] = c_add(v[0], v[1]);
                o[1] = c_sub(v[0], v[1]);
            } else {
                for (int s = 0; s < R; ++s) {
                    float2 acc = v[0];
                    for (int t = 1; t < R; ++t) acc = c_add(acc, c_mul(v[t], c_root((s * t) % R, R)));
                    o[s] = acc;
                }
            }
            const int base = (j / Ns) * Ns * R + jm;
            for (int r = 0; r < R; ++r) b[base + r * Ns] = o[r];
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// Row pass: CTA (pair q, channel c) transforms rows 2q and 2q + 1 of the N x N
// window of A_c * I (centred in the M x M padded image) and writes their half
// spectra to R[c][k][n], k = 0..M/2.
__global__ void __launch_bounds__(FFT_THREADS) k_fft_rows(DevData d, const float* __restrict__ img, int M,
                                                          float2* __restrict__ R) {
    extern __shared__ float2 sh[];
    float2* a = sh;
    float2* b = sh + M;
    const int N = d.N, o = (M - N) / 2, H = M / 2 + 1;
    const int c = blockIdx.y, n0 = 2 * blockIdx.x;
    const int i = d.shared ? 0 : c;
    const int64_t NN = (int64_t)N * N;
    const float* A = d.beam + (int64_t)c * NN;
    const float* I = img + (int64_t)i * NN;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int x = m - o;
        float2 z = make_float2(0.f, 0.f);
        if (x >= 0 && x < N) {
            const int64_t p0 = (int64_t)n0 * N + x, p1 = p0 + N;
            z = make_float2(A[p0] * I[p0], A[p1] * I[p1]);
        }
        a[m] = z;
    }
    __syncthreads();
    const float2* Zs = fft_shared(a, b, M);
    float2* Rc = R + (int64_t)c * H * N;
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
        const float2 zk = Zs[k];
        const float2 zc = Zs[(M - k) % M];
        // X_a = (Z_k + conj Z_{M-k}) / 2,  X_b = (Z_k - conj Z_{M-k}) / (2i)
        const float2 xa = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
        const float2 xb = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
        Rc[(int64_t)k * N + n0] = xa;
        Rc[(int64_t)k * N + n0 + 1] = xb;
    }
}

// Column pass: CTA (column k, channel c) transforms R[c][k][.] placed at the
// window rows of a length-M column and writes F[c][l][k].
__global__ void __launch_bounds__(FFT_THREADS) k_fft_cols(int N, int M, const float2* __restrict__ R,
                                                          float2* __restrict__ F) {
    extern __shared__ float2 sh[];
    float2* a = sh;
    float2* b = sh + M;
    const int o = (M - N) / 2, H = M / 2 + 1;
    const int k = blockIdx.x, c = blockIdx.y;
    const float2* Rk = R + ((int64_t)c * H + k) * N;
    for (int l = threadIdx.x; l < M; l += blockDim.x) {
        const int n = l - o;
        a[l] = (n >= 0 && n < N) ? Rk[n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* Y = fft_shared(a, b, M);
    float2* Fc = F + (int64_t)c * M * H;
    for (int l = threadIdx.x; l < M; l += blockDim.x) Fc[(int64_t)l * H + k] = Y[l];
}

// Value of the modulated transform at integer grid frequency (k, l) from the
// half spectrum (columns 0..M/2; the rest by Hermitian symmetry of a real
// image's transform), times (-1)^(k+l) for the phase centre at pixel N/2.
__device__ __forceinline__ float2 grid_value(const float2* __restrict__ F, int M, int64_t k, int64_t l) {
    int kk = (int)(((k % M) + M) % M), ll = (int)(((l % M) + M) % M);
    float2 z;
    const int H = M / 2 + 1;
    if (kk < H) {
        z = F[(int64_t)ll * H + kk];
    } else {
        const float2 f = F[(int64_t)((M - ll) % M) * H + (M - kk)];
        z = make_float2(f.x, -f.y);
    }
    if ((k + l) & 1) z = make_float2(-z.x, -z.y);
    return z;
}

__global__ void __launch_bounds__(256) k_grid_interp(DevData d, int M, const float2* __restrict__ F,
                                                     int64_t z_total, float2* __restrict__ vis) {
    const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (j >= z_total) return;
    // channel of sample j (offsets ascending)
    int lo = 0, hi = d.C;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (d.off[mid] <= j) lo = mid;
        else hi = mid;
    }
    const float2* Fc = F + (int64_t)lo * M * (M / 2 + 1);
    const double gu = d.u[j] * (double)M * d.dx, gv = d.v[j] * (double)M * d.dy;
    const double k0 = floor(gu), l0 = floor(gv);
    const float fx = (float)(gu - k0), fy = (float)(gv - l0);
    const int64_t k = (int64_t)k0, l = (int64_t)l0;
    const float2 a = grid_value(Fc, M, k, l), b = grid_value(Fc, M, k + 1, l);
    const float2 e = grid_value(Fc, M, k, l + 1), f = grid_value(Fc, M, k + 1, l + 1);
    const float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy), w01 = (1.f - fx) * fy, w11 = fx * fy;
    vis[j] = make_float2(w00 * a.x + w10 * b.x + w01 * e.x + w11 * f.x,
                         w00 * a.y + w10 * b.y + w01 * e.y + w11 * f.y);
}

}  // namespace

bool grid_fft_size_ok(int N, int M) {
    if (N < 2 || (N & 1) || M < N || M > GRID_FFT_MAX) return false;
    int odd = M;
    while (!(odd & 1)) odd >>= 1;
    return odd == 1 || odd == 3 || odd == 5 || odd == 7;
}

void launch_grid_fft(const DevData& d, const float* img, int M, float2* R, float2* F, cudaStream_t st) {
    const int H = M / 2 + 1;
    const int smem = 2 * M * (int)sizeof(float2);
    cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_fft_rows<<<dim3(d.N / 2, d.C), FFT_THREADS, smem, st>>>(d, img, M, R);
    k_fft_cols<<<dim3(H, d.C), FFT_THREADS, smem, st>>>(d.N, M, R, F);
}

void launch_grid_interp(const DevData& d, int M, const float2* F, int64_t z_total, float2* vis, cudaStream_t st) {
    if (z_total <= 0) return;
    k_grid_interp<<<(unsigned)((z_total + 255) / 256), 256, 0, st>>>(d, M, F, z_total, vis);
}

}  // namespace msk
