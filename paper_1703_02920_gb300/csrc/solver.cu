// Device-side control of the projected Polak-Ribiere CG (Eq. minproblem):
// the conjugate-gradient bookkeeping, the line-search state machine and the
// loop conditions run in single-block controller kernels, so that a whole
// solve is one launch of a CUDA graph whose loops are conditional WHILE
// nodes (the host reads the results once, at the end).
//
// Per iteration (every scalar in FP64):
//   beta_i = max(0, (g - g_prev).g / g_prev.g_prev)  (0 on restarts: the first
//            iteration, every RESTART-th, and when d is not a descent direction)
//   d_i    = -g + beta_i d (bound-projected), slope_i = grad Phi . d
//   alpha0 = -slope / sum w |F(A d)|^2  (the minimiser of chi^2's quadratic
//            model along d), or max I / max |d| without curvature
//   line search on phi(alpha) = Phi(max(I + alpha d, G)): bracketing (shrink by
//            SHRINK until phi < phi(0), else expand by GOLD while phi falls),
//            Brent's method (Brent 1973, ch. 5), then one Newton step on
//            central differences over x -/+ h, h = min(POLISH alpha0, x / 2),
//            clamped to that interval
//   I      = max(I + alpha d, G)
// Images of a cube are independent CGs that share every batched evaluation.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "solver.h"

namespace msk {

namespace {

// Constants of this library's reading of the paper's Numerical-Recipes style
// CG (Section 4.2 names the method, not its constants).
constexpr double GOLD = 1.618033988749895;    // bracket expansion ratio
constexpr double CGOLD = 0.3819660112501051;  // golden-section fraction
constexpr double SHRINK = 0.25;               // trial-step reduction
constexpr int LS_MAX_EVALS = 20;              // objective evaluations per line search (+2 for the last step)
constexpr double LS_TOL = 1e-3;               // relative step tolerance (Brent)
constexpr double LS_EPS = 1e-10;              // absolute tolerance / first trial step
constexpr int RESTART = 50;                   // steepest-descent restart period
constexpr double POLISH = 0.2;                // half-width of the final 3-point Newton step / step
constexpr int CTL_THREADS = 256;

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// Line search on phi(alpha), alpha >= 0, as a resumable state machine: start()
// sets the first request, feed() takes phi(req) and sets the next request
// until the phase is DONE (alpha = the accepted step, 0 when no decrease was
// found within the budget).
__device__ void ls_finish(LineSearchState& s, double al, double f) {
    if (al > 0.0) {
        s.px = al;
        s.pfx = f;
        s.ph = fmin(POLISH * s.a0, 0.5 * al);
        s.req = s.px + s.ph;
        s.phase = LS_POL_P;
        return;
    }
    s.alpha = al;
    s.phase = LS_DONE;
}

__device__ void ls_brent_step(LineSearchState& s) {
    if (s.nb >= s.budget) {
        s.evals += s.nb;
        ls_finish(s, s.x, s.fx);
        return;
    }
    const double xm = 0.5 * (s.lo + s.hi);
    const double tol1 = LS_TOL * fabs(s.x) + s.eps;
    const double tol2 = 2.0 * tol1;
    if (fabs(s.x - xm) <= tol2 - 0.5 * (s.hi - s.lo)) {
        s.evals += s.nb;
        ls_finish(s, s.x, s.fx);
        return;
    }
    bool golden = true;
    if (fabs(s.e) > tol1) {
        // parabola through (v, fv), (w, fw), (x, fx)
        const double r = (s.x - s.w) * (s.fx - s.fv);
        double q = (s.x - s.v) * (s.fx - s.fw);
        double p = (s.x - s.v) * q - (s.x - s.w) * r;
        q = 2.0 * (q - r);
        if (q > 0.0) p = -p;
        else q = -q;
        const double e_prev = s.e;
        s.e = s.d;
        if (fabs(p) < fabs(0.5 * q * e_prev) && p > q * (s.lo - s.x) && p < q * (s.hi - s.x)) {
            s.d = p / q;
            const double t = s.x + s.d;
            if ((t - s.lo) < tol2 || (s.hi - t) < tol2) s.d = (xm >= s.x) ? tol1 : -tol1;
            golden = false;
        }
    }
    if (golden) {
        s.e = (s.x >= xm) ? (s.lo - s.x) : (s.hi - s.x);
        s.d = CGOLD * s.e;
    }
    s.req = (fabs(s.d) >= tol1) ? s.x + s.d : s.x + (s.d >= 0.0 ? tol1 : -tol1);
}

__device__ void ls_brent_start(LineSearchState& s) {
    s.lo = s.a;
    s.hi = s.c;
    s.x = s.w = s.v = s.b;
    s.fx = s.fw = s.fv = s.fb;
    s.d = s.e = 0.0;
    s.nb = 0;
    s.budget = LS_MAX_EVALS - s.evals;
    s.phase = LS_BRENT;
    ls_brent_step(s);
}

__device__ void ls_shrink_check(LineSearchState& s) {
    if (s.fb >= s.fa && s.evals < LS_MAX_EVALS) {
        s.c = s.b;
        s.fc = s.fb;
        s.b = s.b * SHRINK;
        s.req = s.b;
        s.phase = LS_SHRINK;
    } else if (s.fb >= s.fa) {
        ls_finish(s, 0.0, s.f0);
    } else {
        ls_brent_start(s);
    }
}

__device__ void ls_expand_check(LineSearchState& s) {
    if (s.fc < s.fb && s.evals < LS_MAX_EVALS) {
        s.a = s.b;
        s.fa = s.fb;
        s.b = s.c;
        s.fb = s.fc;
        s.c = s.b + GOLD * (s.b - s.a);
        s.req = s.c;
        s.phase = LS_EXPAND;
    } else if (s.fc < s.fb) {
        ls_finish(s, s.c, s.fc);
    } else {
        ls_brent_start(s);
    }
}

__device__ void ls_start(LineSearchState& s, double phi0, double alpha0) {
    s.a0 = alpha0;
    s.f0 = phi0;
    s.eps = LS_EPS * alpha0;
    s.a = 0.0;
    s.fa = phi0;
    s.b = alpha0;
    s.req = s.b;
    s.evals = 0;
    s.alpha = 0.0;
    s.phase = LS_INIT;
}

__device__ void ls_feed(LineSearchState& s, double f) {
    switch (s.phase) {
        case LS_INIT:
            s.fb = f;
            s.evals = 1;
            if (s.fb >= s.fa) {
                s.c = s.b;
                s.fc = s.fb;
                ls_shrink_check(s);
            } else {
                s.c = s.b + GOLD * (s.b - s.a);
                s.req = s.c;
                s.phase = LS_EXPAND;
            }
            break;
        case LS_SHRINK:
            s.fb = f;
            s.evals += 1;
            ls_shrink_check(s);
            break;
        case LS_EXPAND:
            s.fc = f;
            s.evals += 1;
            ls_expand_check(s);
            break;
        case LS_BRENT: {
            const double t = s.req, ft = f;
            s.nb += 1;
            if (ft <= s.fx) {
                if (t >= s.x) s.lo = s.x;
                else s.hi = s.x;
                s.v = s.w;
                s.fv = s.fw;
                s.w = s.x;
                s.fw = s.fx;
                s.x = t;
                s.fx = ft;
            } else {
                if (t < s.x) s.lo = t;
                else s.hi = t;
                if (ft <= s.fw || s.w == s.x) {
                    s.v = s.w;
                    s.fv = s.fw;
                    s.w = t;
                    s.fw = ft;
                } else if (ft <= s.fv || s.v == s.x || s.v == s.w) {
                    s.v = t;
                    s.fv = ft;
                }
            }
            ls_brent_step(s);
            break;
        }
        case LS_POL_P:
            s.pfp = f;
            s.evals += 1;
            s.req = s.px - s.ph;
            s.phase = LS_POL_M;
            break;
        case LS_POL_M: {
            const double fm = f;
            s.evals += 1;
            double x = s.px;
            const double curv = s.pfp - 2.0 * s.pfx + fm;
            if (curv > 0.0) {
                const double t = s.px - s.ph * (s.pfp - fm) / (2.0 * curv);
                x = fmin(fmax(t, s.px - s.ph), s.px + s.ph);
            }
            s.alpha = x;
            s.phase = LS_DONE;
            break;
        }
        default:
            break;
    }
}

// Block-wide OR of a flag; every thread gets the result.
__device__ int block_any(int x) { return __syncthreads_or(x); }

// The loop condition: written to ctl (read by the host when graphs are off)
// and, inside a graph, to the conditional node's handle.
__device__ void set_cond(CgControl* ctl, int which, int value, unsigned long long handle) {
    if (threadIdx.x != 0) return;
    if (which == 0) ctl->outer = value;
    else ctl->inner = value;
    if (handle) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, value ? 1u : 0u);
}

__device__ void hist_row(const CgControl* ctl, double* hist, int i, int k, double phi, double chi, double S,
                         double alpha, double beta, double evals) {
    double* h = hist + ((int64_t)i * ctl->hist_stride + k) * 6;
    h[0] = phi;
    h[1] = chi;
    h[2] = S;
    h[3] = alpha;
    h[4] = beta;
    h[5] = evals;
}

// After the first objective + gradient: per-image state and history row 0.
__global__ void __launch_bounds__(CTL_THREADS) k_cg_init(int NI, CgImage* st, CgControl* ctl, const double* scal,
                                                         double* hist, const int* dstatus,
                                                         unsigned long long h_outer) {
    int any = 0, bad = 0;
    for (int i = threadIdx.x; i < NI; i += CTL_THREADS) {
        CgImage& s = st[i];
        s.phi = scal[3 + 3 * i];
        s.chi = scal[4 + 3 * i];
        s.S = scal[5 + 3 * i];
        s.beta = s.slope = s.alpha = 0.0;
        s.iters = s.evals = 0;
        s.ls.phase = LS_DONE;
        s.active = 1;
        if (!(finite(s.phi) && finite(s.chi) && finite(s.S))) {
            bad = 1;
            s.active = 0;
        }
        hist_row(ctl, hist, i, 0, s.phi, s.chi, s.S, 0.0, 0.0, 0.0);
        any |= s.active;
    }
    any = block_any(any);
    bad = block_any(bad);
    if (threadIdx.x == 0) {
        if (bad) ctl->status |= CG_NONFINITE;
        if (*dstatus) ctl->status |= CG_DEVICE;
    }
    __syncthreads();
    set_cond(ctl, 0, any && ctl->k < ctl->n_iter && ctl->status == 0, h_outer);
}

// Polak-Ribiere beta from dots = (g_prev.g_prev, (g - g_prev).g) per image;
// direction mode 1 (d = -g + beta d) or 2 (d = -g) for active images, 0 keep.
__global__ void __launch_bounds__(CTL_THREADS) k_cg_beta(int NI, CgImage* st, const CgControl* ctl,
                                                         const double* dots, double* beta, int* mode) {
    const int k = ctl->k;
    for (int i = threadIdx.x; i < NI; i += CTL_THREADS) {
        double b = 0.0;
        if (k > 0 && k % RESTART != 0) {
            const double gg = dots[2 * i], pr = dots[2 * i + 1];
            if (gg > 0.0) b = fmax(0.0, pr / gg);
        }
        st[i].beta = b;
        beta[i] = b;
        mode[i] = st[i].active ? (b == 0.0 ? 2 : 1) : 0;
    }
}

// slope = grad Phi . d; an active image whose d is not a descent direction
// restarts with d = -g (mode 2, beta 0); the others keep d (mode 0).
__global__ void __launch_bounds__(CTL_THREADS) k_cg_slope(int NI, CgImage* st, const double* dots, double* beta,
                                                          int* mode) {
    for (int i = threadIdx.x; i < NI; i += CTL_THREADS) {
        CgImage& s = st[i];
        s.slope = dots[2 * i];
        mode[i] = 0;
        if (s.active && s.slope >= 0.0) {
            mode[i] = 2;
            s.beta = 0.0;
            beta[i] = 0.0;
        }
    }
}

// Slopes of the restarted directions; an image still without descent stops.
__global__ void __launch_bounds__(CTL_THREADS) k_cg_slope2(int NI, CgImage* st, CgControl* ctl, const double* dots,
                                                           const int* mode) {
    int stopped = 0;
    for (int i = threadIdx.x; i < NI; i += CTL_THREADS) {
        CgImage& s = st[i];
        if (mode[i] == 2) s.slope = dots[2 * i];
        if (s.active && s.slope >= 0.0) {
            s.active = 0;
            stopped = 1;
        }
    }
    stopped = block_any(stopped);
    if (threadIdx.x == 0 && stopped) ctl->stopped_early = 1;
}

// First trial step and line-search start.  scal holds 1/2 sum w |F(A d)|^2 per
// image in its chi^2 slot (curvature pass); dots = (max I, max |d|).
__global__ void __launch_bounds__(CTL_THREADS) k_ls_start(int NI, CgImage* st, CgControl* ctl, const double* scal,
                                                          const double* dots, double* alpha, const int* dstatus,
                                                          unsigned long long h_inner) {
    int run = 0, bad = 0;
    for (int i = threadIdx.x; i < NI; i += CTL_THREADS) {
        CgImage& s = st[i];
        alpha[i] = 0.0;
        s.ls.phase = LS_DONE;
        if (!s.active) continue;
        const double curv = 2.0 * scal[4 + 3 * i];
        if (!finite(curv)) bad = 1;
        double a0 = curv > 0.0 ? -s.slope / curv : 0.0;
        if (!(a0 > 0.0)) a0 = dots[2 * i] / dots[2 * i + 1];
        ls_start(s.ls, s.phi, a0);
        alpha[i] = s.ls.req;
        run = 1;
    }
    run = block_any(run);
    bad = block_any(bad);
    if (threadIdx.x == 0) {
        ctl->rounds = 0;
        if (bad) ctl->status |= CG_NONFINITE;
        if (*dstatus) ctl->status |= CG_DEVICE;
    }
    __syncthreads();
    set_cond(ctl, 1, run && ctl->status == 0, h_inner);
}

// One probe evaluated: scal holds Phi(max(I + alpha d, G)) - Phi(I) per image.
__global__ void __launch_bounds__(CTL_THREADS) k_ls_feed(int NI, CgImage* st, CgControl* ctl, const double* scal,
                                                         double* alpha, const int* dstatus,
                                                         unsigned long long h_inner) {
    int run = 0, bad = 0;
    for (int i = threadIdx.x; i < NI; i += CTL_THREADS) {
        CgImage& s = st[i];
        if (s.active && s.ls.phase != LS_DONE) {
            const double f = s.phi + scal[3 + 3 * i];
            if (!finite(f)) bad = 1;
            ls_feed(s.ls, f);
        }
        const bool r = s.active && s.ls.phase != LS_DONE;
        alpha[i] = r ? s.ls.req : 0.0;
        run |= r;
    }
    run = block_any(run);
    bad = block_any(bad);
    if (threadIdx.x == 0) {
        ctl->rounds += 1;
        ctl->probes += 1;
        if (bad) ctl->status |= CG_NONFINITE;
        if (*dstatus) ctl->status |= CG_DEVICE;
        // every line search ends within LS_MAX_EVALS + 2 probes; the cap only
        // guards the loop against a state that should not occur
        if (ctl->rounds >= LS_MAX_EVALS + 8) ctl->status |= CG_LOOP;
    }
    __syncthreads();
    set_cond(ctl, 1, run && ctl->status == 0, h_inner);
}

// Accepted steps: alpha per image (0 for images that stop: no decrease found).
__global__ void __launch_bounds__(CTL_THREADS) k_cg_finish(int NI, CgImage* st, CgControl* ctl, double* alpha) {
    int stopped = 0;
    const int fail = ctl->status != 0;
    for (int i = threadIdx.x; i < NI; i += CTL_THREADS) {
        CgImage& s = st[i];
        double a = 0.0;
        if (s.active) {
            if (fail || s.ls.phase != LS_DONE || !(s.ls.alpha > 0.0)) {
                s.active = 0;
                stopped = 1;
            } else {
                a = s.ls.alpha;
            }
        }
        s.alpha = a;
        alpha[i] = a;
    }
    stopped = block_any(stopped);
    if (threadIdx.x == 0 && stopped && !fail) ctl->stopped_early = 1;
}

// After the step's objective + gradient: history row k + 1, counters and the
// outer loop condition.
__global__ void __launch_bounds__(CTL_THREADS) k_cg_record(int NI, CgImage* st, CgControl* ctl, const double* scal,
                                                           double* hist, const int* dstatus,
                                                           unsigned long long h_outer) {
    const int k = ctl->k;
    int any = 0, bad = 0;
    for (int i = threadIdx.x; i < NI; i += CTL_THREADS) {
        CgImage& s = st[i];
        if (s.alpha > 0.0) {
            const double ev = (double)(s.ls.evals + 2);
            s.iters = k + 1;
            s.evals += s.ls.evals + 2;
            s.phi = scal[3 + 3 * i];
            s.chi = scal[4 + 3 * i];
            s.S = scal[5 + 3 * i];
            if (!(finite(s.phi) && finite(s.chi) && finite(s.S))) bad = 1;
            hist_row(ctl, hist, i, k + 1, s.phi, s.chi, s.S, s.alpha, s.beta, ev);
        } else {
            hist_row(ctl, hist, i, k + 1, s.phi, s.chi, s.S, 0.0, 0.0, 0.0);
        }
        any |= s.active;
    }
    any = block_any(any);
    bad = block_any(bad);
    if (threadIdx.x == 0) {
        ctl->k = k + 1;
        if (bad) ctl->status |= CG_NONFINITE;
        if (*dstatus) ctl->status |= CG_DEVICE;
    }
    __syncthreads();
    set_cond(ctl, 0, any && k + 1 < ctl->n_iter && ctl->status == 0, h_outer);
}

}  // namespace

void launch_cg_init(int NI, CgImage* st, CgControl* ctl, const double* scal, double* hist, const int* dstatus,
                    unsigned long long h_outer, cudaStream_t s) {
    k_cg_init<<<1, CTL_THREADS, 0, s>>>(NI, st, ctl, scal, hist, dstatus, h_outer);
}
void launch_cg_beta(int NI, CgImage* st, const CgControl* ctl, const double* dots, double* beta, int* mode,
                    cudaStream_t s) {
    k_cg_beta<<<1, CTL_THREADS, 0, s>>>(NI, st, ctl, dots, beta, mode);
}
void launch_cg_slope(int NI, CgImage* st, const double* dots, double* beta, int* mode, cudaStream_t s) {
    k_cg_slope<<<1, CTL_THREADS, 0, s>>>(NI, st, dots, beta, mode);
}
void launch_cg_slope2(int NI, CgImage* st, CgControl* ctl, const double* dots, const int* mode, cudaStream_t s) {
    k_cg_slope2<<<1, CTL_THREADS, 0, s>>>(NI, st, ctl, dots, mode);
}
void launch_ls_start(int NI, CgImage* st, CgControl* ctl, const double* scal, const double* dots, double* alpha,
                     const int* dstatus, unsigned long long h_inner, cudaStream_t s) {
    k_ls_start<<<1, CTL_THREADS, 0, s>>>(NI, st, ctl, scal, dots, alpha, dstatus, h_inner);
}
void launch_ls_feed(int NI, CgImage* st, CgControl* ctl, const double* scal, double* alpha, const int* dstatus,
                    unsigned long long h_inner, cudaStream_t s) {
    k_ls_feed<<<1, CTL_THREADS, 0, s>>>(NI, st, ctl, scal, alpha, dstatus, h_inner);
}
void launch_cg_finish(int NI, CgImage* st, CgControl* ctl, double* alpha, cudaStream_t s) {
    k_cg_finish<<<1, CTL_THREADS, 0, s>>>(NI, st, ctl, alpha);
}
void launch_cg_record(int NI, CgImage* st, CgControl* ctl, const double* scal, double* hist, const int* dstatus,
                      unsigned long long h_outer, cudaStream_t s) {
    k_cg_record<<<1, CTL_THREADS, 0, s>>>(NI, st, ctl, scal, hist, dstatus, h_outer);
}

}  // namespace msk
