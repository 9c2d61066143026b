// Internal interfaces of libmemsynth: device data views and kernel launchers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace msk {

// Device status word bits (the host maps them to mem_status).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BADARG = 2 };

// Consecutive visibilities of one channel (the forward kernels' unit: 128 for
// the direct forms, TC_TILE for the tensor-core form).
struct VisTile {
    int32_t chan;
    int32_t count;
    int64_t start;
};

// Split-K unit of the tensor-core adjoint: one output block of one channel
// over a visibility range.
struct AdjUnit {
    int32_t chan;
    int32_t block;   // output block index (row-major over N/BLK x N/BLK)
    int64_t start;   // first visibility (global index)
    int64_t count;
};

// Read-only problem data resident on the device.
struct DevData {
    int N;
    int C;
    int n_images;
    int shared;          // 1: one image for all channels
    double G;
    double lambda;
    const uint64_t* pa;  // frac(u dx) as 64-bit fixed-point turns
    const uint64_t* pb;  // frac(v dy)
    const double* u;
    const double* v;
    const double2* vo;   // observed visibilities
    const double* w;     // 1/sigma^2
    const float4* vo32;  // observed visibilities as FP32 pairs (Re hi, Im hi, Re lo, Im lo)
    const float* w32;    // 1/sigma^2 in FP32
    const float* beam;   // C*N*N
    const int64_t* off;  // C+1
    double dx, dy;       // pixel size (radians)
    // tensor-core tiling chosen by the autotuner (defaults: tc_bn(N), 4, 3)
    int fwd_bn;          // forward image column block (divides N, <= 256; N for the resident kernel)
    int fwd_stages;      // forward pipeline depth (streaming 3|4, resident 4..6)
    int adj_stages;      // adjoint pipeline depth (2 or 3)
};

// Where pixel values come from: the caller's FP32 image, or the solver's FP64
// state, optionally moved along a direction and clipped: max(I + alpha_i d, G).
struct ImgSrc {
    const float* f32;
    const double* f64;
    const double* dir;
    const double* alpha;  // per image (device)
    double G;
    int diff;             // operand is max(I + alpha d, G) - I, entropy as a difference
};

enum BFormat { BF_F32 = 0, BF_F64 = 1, BF_BF16X3 = 2, BF_F16X3 = 3 };
// FWD_VIS: write V.  FWD_RESID: write y = w (V - V^o), chi^2 partials.
// FWD_CHI: chi^2 partials only.  FWD_CURV: 1/2 w |V|^2 partials.
// FWD_DCHI: chi^2 change for an operand that is an image difference delta,
//   Re(conj(y) F(A delta)) + 1/2 w |F(A delta)|^2, with y = w r of the base
//   image read from the y buffer.
enum FwdMode { FWD_VIS = 0, FWD_RESID = 1, FWD_CHI = 2, FWD_CURV = 3, FWD_DCHI = 4 };

// Forward tensor-core tiling: 64 visibilities per tile, image column block
// width BN and image rows per pipeline stage.
constexpr int TC_BK = 32;
constexpr int TC_TILE = 64;
__host__ __device__ inline int tc_bn(int N) { return N < 256 ? N : 256; }
// Adjoint tensor-core tiling: output block side and visibilities per stage.
constexpr int TCA_BK = 16;
inline int tca_blk(int N) { return N < 256 ? N : 256; }

// Message returned by mem_last_error(NULL) (thread-local).
void set_global_error(const char* msg);

// ---- launchers (all asynchronous on `st`) ----
void launch_phase_prep(int64_t Z, const double* u, const double* v, double dx, double dy,
                       uint64_t* pa, uint64_t* pb, cudaStream_t st);

// B_c = A_c * img(c) for every channel in the requested format; entropy
// partials S_i per (image, block) when ent_part != nullptr.  The tensor-core
// formats hold B - c_m (c_m the column mean from launch_colmean); F16X3 also
// scales each channel by cscale[c] (a power of two, from launch_colmean).
void launch_prep(const DevData& d, const ImgSrc& src, int fmt, void* bout, double* ent_part,
                 const float* cmean, const float* cscale, cudaStream_t st);
// Column means of B_c per channel into cmean[C][N] and the channel's FP16X3
// operand scale into cscale[C] (from the bound max_m (max_n |B| + |c_m|)).
// psum (double) and pmax (float) hold colmean_tmp_count(N, C) entries each;
// count holds C completion counters, zero between calls (each call leaves
// them zero).  ymax_clear (nullable) is set to zero.
void launch_colmean(const DevData& d, const ImgSrc& src, float* cmean, float* cscale, double* psum, float* pmax,
                    unsigned* count, float* ymax_clear, cudaStream_t st);
int colmean_tmp_count(int N, int C);
__host__ __device__ inline int colmean_blocks(int N) { return (N + 31) / 32; }
// max |component| of n floats into ymax[0]; the FP16X3 adjoint scales y by
// pow2_scale_for(ymax[0]).  The forward writes the same maximum of the y it
// produces (RESID mode) when given ymax (zeroed before).
void launch_absmax(int64_t n, const float* y, float* part, float* ymax, cudaStream_t st);
__host__ __device__ inline int prep_blocks(int N) { return (int)(((int64_t)N * N + 255) / 256); }

void launch_fwd_direct(const DevData& d, int fp64, const VisTile* tiles, int n_tiles, const void* B,
                       int mode, void* yout, double* chi_part, cudaStream_t st);
// gsum: [ks][C][N*N] doubles, per-channel sums without the beam factor.
void launch_adj_direct(const DevData& d, int fp64, const void* y, double* gsum, int ks,
                       cudaStream_t st);
int adj_direct_splits(const DevData& d, int num_sms);

// Tensor-core forms.
int fwd_tc_smem_bytes(int N, int BN, int stages);
// Resident-operand forward (N <= 256): the image rows are cut into slices of
// fwd_rs_ks(N); each CTA keeps one slice of the operand planes in shared
// memory; slice partials (FP64, [slice][visibility]) are combined by a second
// kernel that also applies the forward mode.
__host__ __device__ inline int fwd_rs_ks(int N) { return N < 128 ? N : 128; }
int fwd_rs_smem_bytes(int N, int stages);
// The paper's gridded forward: the 2-D real-to-complex transform of every
// channel's A_c * I zero-padded to M x M (image centred), as this library's
// own FFT kernels (rows into R[C][M/2+1][N], columns into F[C][M][M/2+1]),
// then the modulated bilinear interpolation of the half spectra.
constexpr int GRID_FFT_MAX = 8192;  // M <= 8192: two M-point buffers per CTA in shared memory
bool grid_fft_size_ok(int N, int M);  // N even, M = 2^a q with q in {1, 3, 5, 7}, M <= GRID_FFT_MAX
void launch_grid_fft(const DevData& d, const float* img, int M, float2* R, float2* F, cudaStream_t st);
// Dirty image / PSF / residual map: weighted adjoint inputs (what: 0 data,
// 1 PSF, 2 residuals against the model in y32 / y64), and the per-channel
// image from the adjoint's FP64 sums (no primary-beam factor).
void launch_dirty_y(const DevData& d, const double* wsum, int what, int64_t z_total, float2* y32, double2* y64,
                    cudaStream_t st);
void launch_dirty_out(const DevData& d, const double* gsum, int ks, float* out, cudaStream_t st);
void launch_grid_interp(const DevData& d, int M, const float2* F, int64_t z_total, float2* vis, cudaStream_t st);
int fwd_rs_max_stages(int N);
void launch_fwd_rs(const DevData& d, int f16, const VisTile* tiles, int n_tiles, const void* planes,
                   const float* cmean, const float* cscale, int mode, float2* yout, double* chi_part,
                   float* ymax, double2* vpart, int64_t z_total, int num_sms, uint64_t spin, int* status,
                   cudaStream_t st);
// f16 = 1: FP16X3 operands (planes scaled by cscale[c]); 0: BF16X3.
// ymax (nullable, RESID mode): max |component| of the weighted residual
// written to yout is combined into ymax[0] (which the caller zeroes).
void launch_fwd_tc(const DevData& d, int f16, const VisTile* tiles, int n_tiles, const void* planes,
                   const float* cmean, const float* cscale, int mode, float2* yout, double* chi_part,
                   float* ymax, int grid, uint64_t spin, int* status, cudaStream_t st);
int adj_tc_smem_bytes(int N, int stages);
// units sorted by CTA: CTA b runs units [cta_unit_off[b], cta_unit_off[b+1]).
// f16 = 1: FP16X3 with y scaled by pow2_scale_for(ymax[0]) (partials carry the scale).
void launch_adj_tc(const DevData& d, int f16, const AdjUnit* units, const int* cta_unit_off, int n_ctas,
                   const float2* y, const float* ymax, float* partial, uint64_t spin, int* status,
                   cudaStream_t st);
// Variant reading u, v (FP64, wavelengths) instead of the prepared phase
// increments: the caller passes d.u, d.v, d.dx, d.dy; d.pa / d.pb are unused.
void launch_adj_tc_uv(const DevData& d, const AdjUnit* units, const int* cta_unit_off, int n_ctas,
                      const float2* y, float* partial, uint64_t spin, int* status, cudaStream_t st);
// out[p] = A[p] * sum of unit partials (single channel, unit order,
// compensated FP32 two-sum).
void launch_adj_tc_reduce_out(int N, const int* cb_unit_off, const float* partial, const float* beam,
                              float* out, cudaStream_t st);
// Sum unit partials per channel (unit order) into gsum[C][N*N].
// ymax (nullable, FP16X3): partials are divided by pow2_scale_for(ymax[0]).
void launch_adj_tc_reduce(const DevData& d, const AdjUnit* units, const int* unit_off_by_chan_blk,
                          const float* partial, const float* ymax, double* gsum, cudaStream_t st);
// Inputs of the objective's scalar reduction (launch_scalars) when it runs
// inside another launch; scal == nullptr: not run.
struct ScalarArgs {
    const int* tile_off = nullptr;
    const double* chi_part = nullptr;
    const double* ent_part = nullptr;
    int with_entropy = 0;
    double* scal = nullptr;
    double* img_tmp = nullptr;
};
// Unit-partial sum plus gradient assembly in one launch, for images of one
// channel each (not the shared-image mode); with sc.scal set, the same launch
// also forms the objective scalars (as launch_scalars).
void launch_adj_tc_reduce_grad(const DevData& d, const ImgSrc& src, const int* cb_unit_off, const float* partial,
                               const float* ymax, int projected, float* out32, double* full64, double* proj64,
                               const ScalarArgs& sc, cudaStream_t st);

// grad_i = sum_{c in image i} A_c * sum_k gsum[k][c] + lambda (1 + log(I/G)); optional projection.
void launch_finalize(const DevData& d, const ImgSrc& src, const double* gsum, int ks, int projected,
                     float* out32, double* full64, double* proj64, cudaStream_t st);

// chi_part holds 4 partials per visibility tile (one per 32 visibilities).
// Per-image chi^2 / S / Phi into scal[3 + 3 i ...] and totals into scal[0..2].
void launch_scalars(const DevData& d, const int* tile_off, const double* chi_part,
                    const double* ent_part, int with_entropy, double* scal, double* img_tmp,
                    cudaStream_t st);
int scalars_tmp_doubles(int n_images);

// Solver vector kernels (FP64, per image).
void launch_dots(const DevData& d, int which, const double* a, const double* b, const double* c,
                 double* part, double* out, cudaStream_t st);
void launch_cg_direction(const DevData& d, const double* I, const double* g, const double* beta,
                         const int* mode, double* dir, cudaStream_t st);
void launch_cg_step(const DevData& d, double* I, const double* dir, const double* alpha,
                    cudaStream_t st);
void launch_clip_f32_to_f64(const DevData& d, const float* in, double* out, cudaStream_t st);
void launch_f64_to_f32(int64_t n, const double* in, float* out, cudaStream_t st);

enum DotKind { DOT_BETA = 0, DOT_SLOPE = 1, DOT_MAX = 2 };

}  // namespace msk
