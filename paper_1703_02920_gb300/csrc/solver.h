// Device-resident state of the projected CG solve and its controller kernels
// (solver.cu).  The host copies CgImage / CgControl back once, at the end of
// a solve.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace msk {

enum LsPhase : int { LS_INIT = 0, LS_SHRINK, LS_EXPAND, LS_BRENT, LS_POL_P, LS_POL_M, LS_DONE };

// One line search (bracketing, Brent, final Newton step), resumable per probe.
struct LineSearchState {
    double f0, a, fa, b, fb, c, fc, eps, a0;
    double lo, hi, x, w, v, fx, fw, fv, d, e;
    double px, pfx, ph, pfp;
    double req, alpha;
    int phase, evals, nb, budget;
};

// Per image: the iterate's objective terms, CG scalars and counters.
struct CgImage {
    LineSearchState ls;
    double phi, chi, S;
    double beta, slope, alpha;
    int active, iters, evals, pad;
};

// CgControl.status bits: a non-finite objective, a device-side wait that ran
// out (the context's status word), a line search that did not end.
enum : int { CG_NONFINITE = 1, CG_DEVICE = 2, CG_LOOP = 4 };

struct CgControl {
    int k;            // iterations done
    int n_iter;       // iterations requested (set by the host before a solve)
    int hist_stride;  // rows per image in the history buffer (n_iter + 1)
    int stopped_early;
    int status;
    int rounds;       // probes of the current line search
    int outer, inner; // loop conditions (read by the host when graphs are off)
    long long probes; // probes over the whole solve
};

// Controller kernels (one block each).  A non-zero handle is the conditional
// node whose condition the kernel sets (outer: iterations; inner: probes).
void launch_cg_init(int NI, CgImage* st, CgControl* ctl, const double* scal, double* hist, const int* dstatus,
                    unsigned long long h_outer, cudaStream_t s);
void launch_cg_beta(int NI, CgImage* st, const CgControl* ctl, const double* dots, double* beta, int* mode,
                    cudaStream_t s);
void launch_cg_slope(int NI, CgImage* st, const double* dots, double* beta, int* mode, cudaStream_t s);
void launch_cg_slope2(int NI, CgImage* st, CgControl* ctl, const double* dots, const int* mode, cudaStream_t s);
void launch_ls_start(int NI, CgImage* st, CgControl* ctl, const double* scal, const double* dots, double* alpha,
                     const int* dstatus, unsigned long long h_inner, cudaStream_t s);
void launch_ls_feed(int NI, CgImage* st, CgControl* ctl, const double* scal, double* alpha, const int* dstatus,
                    unsigned long long h_inner, cudaStream_t s);
void launch_cg_finish(int NI, CgImage* st, CgControl* ctl, double* alpha, cudaStream_t s);
void launch_cg_record(int NI, CgImage* st, CgControl* ctl, const double* scal, double* hist, const int* dstatus,
                      unsigned long long h_outer, cudaStream_t s);

}  // namespace msk
