// Device-side helpers shared by the libmemsynth kernels: exact phase
// arithmetic, bounded mbarrier waits, and the sm_100-family PTX used by the
// tensor-core kernels (tcgen05 MMA / TMEM, bulk async copies).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace msk {

// ---------------------------------------------------------------------------
// Phase arithmetic.
//
// Each visibility carries a = frac(u dx) and b = frac(v dy) as 64-bit
// fixed-point turns (two's complement, 1 turn = 2^64).  The phase of pixel
// (m, n) is (m - N/2) a + (n - N/2) b modulo one turn, which wraps exactly in
// unsigned 64-bit arithmetic: the only rounding is the one FP64 reduction of
// u dx (and v dy) per visibility.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t phase_mul(int64_t k, uint64_t a) {
    return (uint64_t)k * a;
}

// frac(t) as a 64-bit fixed-point fraction of a turn (FP64 reduction).
__device__ __forceinline__ uint64_t to_fixed_turns(double t) {
    double f = t - rint(t);  // [-0.5, 0.5]
    if (f >= 0.5) f -= 1.0;  // same turn, keeps f * 2^64 inside int64
    return (uint64_t)__double2ll_rn(f * 18446744073709551616.0);
}

// Angle in radians in [-pi, pi) from the top 32 bits of a fixed-point phase.
__device__ __forceinline__ float phase_to_angle_f32(uint64_t p) {
    const float k2pi_2m32 = 6.283185307179586f / 4294967296.0f;
    return (float)(int32_t)(uint32_t)(p >> 32) * k2pi_2m32;
}

// Turns in [-0.5, 0.5) as FP64 from all 64 bits.
__device__ __forceinline__ double phase_to_turns_f64(uint64_t p) {
    return (double)(int64_t)p * 5.421010862427522e-20;  // 2^-64
}

// Compensated accumulation (Neumaier): s + c carries the sum of the added
// terms to about twice FP32 precision, in a fixed order.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
    s = t;
}

// (ah + al) + (bh + bl) for double-float pairs (|al| <= ulp(ah)/2, likewise
// b), as a normalized pair (hi, lo): Knuth's two-sum of the high parts, then
// the low parts.  Exact when the high parts cancel (Sterbenz), which is the
// case for a residual V - V° of a good model.
__device__ __forceinline__ float2 df_add(float ah, float al, float bh, float bl) {
    const float s = ah + bh;
    const float bb = s - ah;
    const float e = (ah - (s - bb)) + (bh - bb);
    const float lo = e + (al + bl);
    const float hi = s + lo;
    return make_float2(hi, lo - (hi - s));
}

// exp(-i * angle) components for the forward sign convention are (c, -s).
struct cf2 { float x, y; };

// Pixel p of image i from an image source: the caller's FP32 image, or the
// solver's FP64 state moved along its direction and clipped, max(I + alpha d, G).
__device__ __forceinline__ double img_value(const ImgSrc& s, int i, int64_t p, int64_t NN) {
    if (s.f32) return (double)s.f32[(int64_t)i * NN + p];
    double x = s.f64[(int64_t)i * NN + p];
    if (s.dir) x = fmax(x + s.alpha[i] * s.dir[(int64_t)i * NN + p], s.G);
    return x;
}


__device__ __forceinline__ cf2 cmul(cf2 a, cf2 b) {
    return {fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)};
}

// ---------------------------------------------------------------------------
// Shared-memory addresses, mbarriers
// ---------------------------------------------------------------------------
// e^{-2 pi i p / 2^64} from the SFU sine and cosine, rescaled to unit
// modulus: with x = c^2 + s^2 = 1 + e, the factor 1.5 - x/2 = 1/sqrt(x) + O(e^2)
// removes a systematic modulus error of the approximations, which would
// otherwise scale every product of table entries (four per term of Eq. 1).
__device__ __forceinline__ cf2 cis_neg(uint64_t p) {
    float s, c;
    __sincosf(phase_to_angle_f32(p), &s, &c);
    const float r = fmaf(-0.5f, fmaf(c, c, s * s), 1.5f);
    return {c * r, -s * r};
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait: gives up after `limit` polls or when another role of the CTA
// has already given up (*abort != 0); on give-up sets the device status and
// the CTA's abort flag.  Returns true when the phase completed.  sleep_ns > 0
// backs off between polls (for long waits, so that waiting warps leave the
// issue slots to working ones); the poll bound is then limit / 16.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit,
                                          volatile int* abort, int* status, unsigned sleep_ns = 0) {
    uint64_t it = 0;
    const uint64_t lim = sleep_ns ? (limit >> 4 ? limit >> 4 : 1) : limit;
    while (!mbar_try_wait(bar, parity)) {
        if (++it >= lim || *abort) {
            *abort = 1;
            atomicOr(status, DEV_TIMEOUT);
            return false;
        }
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    return true;
}

// Bound for the end-of-kernel waits on the CTA's own in-flight tensor-core
// operations and bulk copies.  Those were issued with complete operands and
// finish within microseconds, but they must finish before TMEM or shared
// memory is released, so the bound is the context's spin limit and never fewer
// than 2^24 polls (a spin limit small enough to force a timeout elsewhere must
// not cut these waits short).
__device__ __forceinline__ uint64_t drain_limit(uint64_t spin) {
    return spin > (1ull << 24) ? spin : (1ull << 24);
}

// 1-D bulk async copy global -> shared, completion counted on an mbarrier.
// Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Make generic-proxy shared-memory writes visible to the async proxy (tensor core).
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// tcgen05: TMEM allocation, MMA, commit, loads
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols));
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (bf16 inputs, fp32 accumulate).
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Arrive on an mbarrier once all previously issued tcgen05 ops of this thread complete.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Whole-warp forms of the MMA issue and commit.  Every lane of the warp
// executes them, converged, and elect.sync picks the issuing lane.  For a
// full member mask the election is deterministic (the same lane on every
// call), so one thread issues all of the warp's MMAs and its commits track
// them.  A converged issue loop with an elected lane issues MMAs in fewer
// clocks than a loop run by one lane alone.  MMA_FILL keeps the MMA's A tile
// in the tensor core's collector buffer for the issuing thread's next MMA,
// MMA_LASTUSE takes A from that buffer and releases it: two consecutive
// products with the same A tile read it from shared memory once.
enum MmaCollect { MMA_PLAIN, MMA_FILL, MMA_LASTUSE };
template <MmaCollect OP>
__device__ __forceinline__ void umma_f16_elect(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
    if (OP == MMA_FILL)
        asm volatile(
            "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    else if (OP == MMA_LASTUSE)
        asm volatile(
            "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    else
        asm volatile(
            "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit_elect(uint64_t* bar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
            smem_u32(bar))
        : "memory");
}


// The six MMAs of one streaming-forward stage (two K steps, each hi x hi,
// hi x lo, lo x hi; the first two share their A tile through the collector
// buffer) in one block, whole-warp form (elect.sync picks the issuing lane, as
// in umma_f16_elect).  Each descriptor is assembled from its low word (start
// address field already moved to the stage's slot; ka / kb move it to the
// second K step) and the high word it shares with its operand's other planes.
// acc = 0 starts a fresh accumulation with the first MMA.
__device__ __forceinline__ void umma6_stage_elect(uint32_t dt, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl,
                                                  uint32_t hia, uint32_t hib, uint32_t ka, uint32_t kb,
                                                  uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p, one, e;\n .reg .b64 d0, d1, d2, d3, d4, d5, d6, d7;\n .reg .b32 t0, t1, t2, t3;\n"
        " setp.ne.b32 p, %10, 0;\n setp.ne.b32 one, %11, 0;\n"
        " elect.sync _|e, 0xffffffff;\n"
        " mov.b64 d0, {%1, %5};\n mov.b64 d1, {%2, %5};\n mov.b64 d2, {%3, %6};\n mov.b64 d3, {%4, %6};\n"
        " add.u32 t0, %1, %7;\n add.u32 t1, %2, %7;\n add.u32 t2, %3, %8;\n add.u32 t3, %4, %8;\n"
        " mov.b64 d4, {t0, %5};\n mov.b64 d5, {t1, %5};\n mov.b64 d6, {t2, %6};\n mov.b64 d7, {t3, %6};\n"
        " @e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], d0, d2, %9, p;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], d0, d3, %9, one;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], d1, d2, %9, one;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], d4, d6, %9, one;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], d4, d7, %9, one;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], d5, d6, %9, one;\n}\n" ::"r"(dt),
        "r"(ah), "r"(al), "r"(bh), "r"(bl), "r"(hia), "r"(hib), "r"(ka), "r"(kb), "r"(idesc), "r"(acc), "r"(1u));
}

// 32 lanes x 16 consecutive 32-bit columns; thread i of the warp gets lane
// (warp's lane quarter base + i).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%"
        "15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Wait for outstanding TMEM loads and tie the given destination registers to
// the wait, so that no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_ld_wait(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
                   "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

// Shared-memory matrix descriptor, no swizzle (interleaved 8x16-byte core
// matrices).  lbo: byte step between core matrices along K (K-major) / along
// K groups (MN-major); sbo: byte step between 8-row groups along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;
}

// Instruction descriptor, kind::f16: D f32, A and B both bf16 (bf16 = 1) or
// both f16 (bf16 = 0), dense.
__host__ __device__ constexpr uint32_t idesc_f16kind(int M, int N, int a_mn_major, int b_mn_major,
                                                     int bf16) {
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)a_mn_major << 15) |
           ((uint32_t)b_mn_major << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn_major, int b_mn_major) {
    return idesc_f16kind(M, N, a_mn_major, b_mn_major, 1);
}

// Split x into f16 hi + lo with x ~= hi + lo (|x - hi - lo| <~ 2^-22 |x| in the
// normal range; callers scale operands so that they stay in range).
__device__ __forceinline__ void split_f16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    __half2 h = __floats2half2_rn(a, b);
    float2 hf = __half22float2(h);
    __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

// 2^(14 - e) for the exponent e of x > 0 (x * scale in [2^14, 2^15)); 1 for x <= 0.
__host__ __device__ __forceinline__ float pow2_scale_for(float x) {
    if (!(x > 0.f)) return 1.f;
    int e;
    frexpf(x, &e);  // x = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, 15 - e);
}

// Split x into bf16 hi + lo with x ~= hi + lo (|x - hi - lo| <~ 2^-16 |x|).
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    float2 hf = __bfloat1622float2(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

// Split into the 16-bit format of the tensor-core form (F16: f16, else bf16).
template <bool F16>
__device__ __forceinline__ void split16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if (F16) split_f16x2(a, b, hi, lo);
    else split_bf16x2(a, b, hi, lo);
}

// ---------------------------------------------------------------------------
// Packed FP32x2 forms (sm_100 and later) of the table arithmetic above.
// Results are bit-identical to cmul / split16x2: every component sees the
// same roundings in the same order, two lanes per instruction.
// ---------------------------------------------------------------------------

// Eight rotation factors w_0..w_7 in planar pairs: x[p] = (Re w_2p, Re w_2p+1),
// y[p] the imaginary parts.
struct Rot8 {
    float2 x[4], y[4];
};

__device__ __forceinline__ Rot8 rot8_of(const cf2 (&w)[8]) {
    Rot8 r;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        r.x[p] = make_float2(w[2 * p].x, w[2 * p + 1].x);
        r.y[p] = make_float2(w[2 * p].y, w[2 * p + 1].y);
    }
    return r;
}

// z_q = base w_q for q = 0..7 as planar pairs re[p] = (Re z_2p, Re z_2p+1),
// im[p] likewise: Re z = fma(bx, wx, (-by) wy), Im z = fma(bx, wy, by wx),
// exactly as cmul(base, w_q).
__device__ __forceinline__ void rotate8(cf2 base, const Rot8& w, float2 (&re)[4], float2 (&im)[4]) {
    const float2 bx = make_float2(base.x, base.x), by = make_float2(base.y, base.y);
    const float2 nby = make_float2(-base.y, -base.y);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        re[p] = __ffma2_rn(bx, w.x[p], __fmul2_rn(nby, w.y[p]));
        im[p] = __ffma2_rn(bx, w.y[p], __fmul2_rn(by, w.x[p]));
    }
}

// split16x2 of the pair v = (a, b): the residual a - hi, b - hi in one
// packed subtraction.
template <bool F16>
__device__ __forceinline__ void split16x2p(float2 v, uint32_t& hi, uint32_t& lo) {
    if (F16) {
        const __half2 h = __float22half2_rn(v);
        const float2 hf = __half22float2(h);
        const __half2 l = __float22half2_rn(__fadd2_rn(v, make_float2(-hf.x, -hf.y)));
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __float22bfloat162_rn(__fadd2_rn(v, make_float2(-hf.x, -hf.y)));
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// Eight rotated entries split into the four 16-byte operand rows of one
// 8-element group: Re hi/lo and Im hi/lo.
template <bool F16>
__device__ __forceinline__ void table8_split(cf2 base, const Rot8& w, uint4& rh, uint4& rl, uint4& ih,
                                             uint4& il) {
    float2 re[4], im[4];
    rotate8(base, w, re, im);
    split16x2p<F16>(re[0], rh.x, rl.x);
    split16x2p<F16>(re[1], rh.y, rl.y);
    split16x2p<F16>(re[2], rh.z, rl.z);
    split16x2p<F16>(re[3], rh.w, rl.w);
    split16x2p<F16>(im[0], ih.x, il.x);
    split16x2p<F16>(im[1], ih.y, il.y);
    split16x2p<F16>(im[2], ih.z, il.z);
    split16x2p<F16>(im[3], ih.w, il.w);
}

}  // namespace msk
