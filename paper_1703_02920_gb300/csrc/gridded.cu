// The paper's gridded forward (Section 2.4, the steps of the objective
// evaluation; Algorithm alg:chi2gpu): attenuation, zero padding to
// M = pad N, a 2-D FFT of every channel's image on the grid, the
// phase-centre modulation and bilinear interpolation at each sample's grid
// coordinates.  An approximation of Eq. (1): its error against the exact sum
// falls about as 1/pad^2 (bilinear interpolation of a band-limited grid).
//
// The FFT is a plain cuFFT real-to-complex transform, batched over channels;
// the padding and the modulated interpolation are the kernels below.
#include <cufft.h>

#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace msk {

namespace {

// P[c][n'][m'] = A_c[n][m] I[n][m] inside the centred N x N window, else 0.
__global__ void __launch_bounds__(256) k_grid_pad(DevData d, const float* __restrict__ img, int M,
                                                  float* __restrict__ P) {
    const int N = d.N, o = (M - N) / 2;
    const int c = blockIdx.y;
    const int64_t MM = (int64_t)M * M, NN = (int64_t)N * N;
    const int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (q >= MM) return;
    const int n = (int)(q / M) - o, m = (int)(q % M) - o;
    float x = 0.f;
    if (n >= 0 && n < N && m >= 0 && m < N) {
        const int i = d.shared ? 0 : c;
        const int64_t p = (int64_t)n * N + m;
        x = d.beam[(int64_t)c * NN + p] * img[(int64_t)i * NN + p];
    }
    P[(int64_t)c * MM + q] = x;
}

// Value of the modulated transform at integer grid frequency (k, l) from the
// half spectrum (columns 0..M/2; the rest by Hermitian symmetry of a real
// image's transform), times (-1)^(k+l) for the phase centre at pixel N/2.
__device__ __forceinline__ float2 grid_value(const cufftComplex* __restrict__ F, int M, int64_t k, int64_t l) {
    int kk = (int)(((k % M) + M) % M), ll = (int)(((l % M) + M) % M);
    float2 z;
    const int H = M / 2 + 1;
    if (kk < H) {
        const cufftComplex f = F[(int64_t)ll * H + kk];
        z = make_float2(f.x, f.y);
    } else {
        const cufftComplex f = F[(int64_t)((M - ll) % M) * H + (M - kk)];
        z = make_float2(f.x, -f.y);
    }
    if ((k + l) & 1) z = make_float2(-z.x, -z.y);
    return z;
}

__global__ void __launch_bounds__(256) k_grid_interp(DevData d, int M, const cufftComplex* __restrict__ F,
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
    const cufftComplex* Fc = F + (int64_t)lo * M * (M / 2 + 1);
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

void launch_grid_pad(const DevData& d, const float* img, int M, float* P, cudaStream_t st) {
    const int64_t MM = (int64_t)M * M;
    dim3 grid((unsigned)((MM + 255) / 256), d.C);
    k_grid_pad<<<grid, 256, 0, st>>>(d, img, M, P);
}

void launch_grid_interp(const DevData& d, int M, const void* F, int64_t z_total, float2* vis, cudaStream_t st) {
    if (z_total <= 0) return;
    k_grid_interp<<<(unsigned)((z_total + 255) / 256), 256, 0, st>>>(d, M, (const cufftComplex*)F, z_total, vis);
}

}  // namespace msk
