"""FP64 oracle for non-gridding MEM (test infrastructure only).

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this module.  It shares no code with the CUDA library: the operator sums live
in ``memsynth_oracle.c`` (plain C, FP64, OpenMP over independent outputs) and
everything else here is plain numpy in FP64, following the paper:

* chi^2 = 1/2 sum_k w_k |V^m_k - V^o_k|^2, w_k = 1/sigma_k^2      (Eq. phi2, Eq. DataProbability)
* multi-channel chi^2 summed over channels                        (Eq. chi2-multi)
* entropy S = -sum_i I_i log(I_i / G); Phi = chi^2 - lambda S     (Eq. phi3; the
  (I/G) log(I/G) scale of Eq. phi2 is absorbed into lambda: lambda = lambda_paper / G)
* grad chi^2 = A * Re(F^H (w r))                                  (Eq. chi2gradient, Appendix C,
  with the primary-beam factor of the model kept)
* grad (-lambda S) = lambda (1 + log(I / G))                      (Eq. Sgradient)
* minimise Phi over I >= G                                        (Eq. minproblem)
  with a positively projected Polak-Ribiere conjugate gradient and a bracketing +
  Brent line search (Section 2.4 / 4.2 name a Numerical-Recipes style CG; the
  steps below are written from the published methods).

Where the paper is silent the readings are fixed here and repeated in the
CUDA library's host code: projection of gradient and direction at the bound,
quadratic-model first trial step, bracketing constants, Brent tolerance and
evaluation budget, restart period.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "memsynth_oracle.c")
_SO = os.path.join(_HERE, "_memsynth_oracle.so")
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, OpenMP, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            D = ctypes.c_double
            P = ctypes.POINTER(ctypes.c_double)
            I64 = ctypes.c_int64
            I = ctypes.c_int
            for name in ("orc_forward_direct", "orc_forward_factored"):
                getattr(lib, name).argtypes = [I, D, D, I64, P, P, P, P]
                getattr(lib, name).restype = None
            for name in ("orc_adjoint_direct", "orc_adjoint_factored"):
                getattr(lib, name).argtypes = [I, D, D, I64, P, P, P, I, I, I, I, P]
                getattr(lib, name).restype = None
            lib.orc_adjoint_factored_full.argtypes = [I, D, D, I64, P, P, P, P]
            lib.orc_adjoint_factored_full.restype = None
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [I]
            lib.orc_set_num_threads.restype = None
            _LIB = lib
        return _LIB


def num_threads() -> int:
    return int(_lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads for the following operator sums (results do not depend on it)."""
    _lib().orc_set_num_threads(int(n))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ----------------------------------------------------------------------------
# the operator pair
# ----------------------------------------------------------------------------
def forward(N: int, dx: float, dy: float, u, v, B, form: str = "factored") -> np.ndarray:
    """V_k = sum_{n,m} B[n,m] exp(-2 pi i (u_k x_m + v_k y_n)), complex128 (Z,)."""
    u, v, B = _f64(u), _f64(v), _f64(B).reshape(N, N)
    Z = u.size
    out = np.zeros(2 * Z)
    fn = _lib().orc_forward_direct if form == "direct" else _lib().orc_forward_factored
    if Z:
        fn(N, dx, dy, Z, _p(u), _p(v), _p(B), _p(out))
    return out[0::2] + 1j * out[1::2]


def forward_gridded(N: int, dx: float, dy: float, u, v, B, pad: int = 2) -> np.ndarray:
    """The paper's gridded approximation of Eq. (1) (Section 2.4, the steps of
    the objective evaluation; Algorithm alg:chi2gpu): the attenuated image B
    is zero-padded to M = pad N (image centred), Fourier transformed on the
    grid, modulated so that the phase centre is pixel (N/2, N/2), and the model
    visibility is bilinearly interpolated at the sample's grid coordinates
    (u M dx, v M dy).  Reading of the garbled modulation factor: on the grid
    frequency (k, l) / (M dx, M dy) the exact sum equals FFT[l, k] (-1)^(k+l),
    because pixel m sits at x = (m + M/2 - N/2 - M/2) dx in the centred padding.
    complex128 (Z,)."""
    u, v, B = _f64(u), _f64(v), _f64(B).reshape(N, N)
    M = pad * N
    o = (M - N) // 2
    P = np.zeros((M, M))
    P[o:o + N, o:o + N] = B
    F = np.fft.fft2(P)  # F[l, k] = sum P[n', m'] exp(-2 pi i (l n' + k m') / M)

    def grid(k, l):
        sign = 1.0 - 2.0 * ((k + l) & 1)  # (-1)^(k+l), the phase-centre modulation
        return F[l % M, k % M] * sign

    out = np.zeros(u.size, dtype=np.complex128)
    for j in range(u.size):
        gu, gv = u[j] * M * dx, v[j] * M * dy
        k0, l0 = int(np.floor(gu)), int(np.floor(gv))
        fx, fy = gu - k0, gv - l0
        out[j] = ((1 - fx) * (1 - fy) * grid(k0, l0) + fx * (1 - fy) * grid(k0 + 1, l0)
                  + (1 - fx) * fy * grid(k0, l0 + 1) + fx * fy * grid(k0 + 1, l0 + 1))
    return out


def adjoint(N: int, dx: float, dy: float, u, v, y, crop=None, form: str = "factored") -> np.ndarray:
    """G[n,m] = sum_k Re(y_k exp(+2 pi i (u_k x_m + v_k y_n))) on a crop
    (n0, nn, m0, nm) of the image (default: the whole image), float64."""
    u, v = _f64(u), _f64(v)
    y = np.asarray(y, dtype=np.complex128)
    yi = np.empty(2 * y.size)
    yi[0::2], yi[1::2] = y.real, y.imag
    Z = u.size
    if crop is None and form == "factored":
        G = np.zeros((N, N))
        if Z:
            _lib().orc_adjoint_factored_full(N, dx, dy, Z, _p(u), _p(v), _p(yi), _p(G))
        return G
    n0, nn, m0, nm = crop if crop is not None else (0, N, 0, N)
    G = np.zeros((nn, nm))
    fn = _lib().orc_adjoint_direct if form == "direct" else _lib().orc_adjoint_factored
    if Z:
        fn(N, dx, dy, Z, _p(u), _p(v), _p(yi), n0, nn, m0, nm, _p(G))
    return G


# ----------------------------------------------------------------------------
# objective, gradient, projection
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    N: int
    dx: float
    dy: float
    u: np.ndarray
    v: np.ndarray
    vo: np.ndarray
    sigma: np.ndarray
    pb: np.ndarray          # (C, N, N)
    offsets: np.ndarray     # (C+1,)
    G: float
    lam: float
    shared_image: bool = False

    @classmethod
    def from_dataset(cls, ds, lam=None, G=None) -> "Problem":
        return cls(N=ds.N, dx=ds.dx, dy=ds.dy, u=_f64(ds.u), v=_f64(ds.v),
                   vo=np.asarray(ds.vo, dtype=np.complex128), sigma=_f64(ds.sigma),
                   pb=np.asarray(ds.pb, dtype=np.float64), offsets=np.asarray(ds.offsets, dtype=np.int64),
                   G=float(ds.G if G is None else G), lam=float(ds.lam if lam is None else lam),
                   shared_image=bool(ds.shared_image))

    @property
    def C(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_images(self) -> int:
        return 1 if self.shared_image else self.C

    def sl(self, c: int) -> slice:
        return slice(int(self.offsets[c]), int(self.offsets[c + 1]))

    def image_of(self, I: np.ndarray, c: int) -> np.ndarray:
        I = np.asarray(I, dtype=np.float64).reshape(self.n_images, self.N, self.N)
        return I[0] if self.shared_image else I[c]

    def weights(self, c: int) -> np.ndarray:
        return 1.0 / self.sigma[self.sl(c)] ** 2


def model_vis(P: Problem, I: np.ndarray, form: str = "factored"):
    """Model visibilities V^m_c = F_c(A_c * I_c) for every channel."""
    out = []
    for c in range(P.C):
        s = P.sl(c)
        out.append(forward(P.N, P.dx, P.dy, P.u[s], P.v[s], P.pb[c] * P.image_of(I, c), form))
    return out


def chi2_terms(P: Problem, I: np.ndarray, form: str = "factored"):
    """Per-channel chi^2 (with the 1/2) and residuals r = V^m - V^o."""
    vm = model_vis(P, I, form)
    chis, res = [], []
    for c in range(P.C):
        r = vm[c] - P.vo[P.sl(c)]
        res.append(r)
        chis.append(0.5 * float(np.sum(P.weights(c) * (r.real ** 2 + r.imag ** 2))))
    return chis, res


def entropy(I: np.ndarray, G: float) -> float:
    """S = -sum_i I_i log(I_i / G) (Eq. logentropy with the 1/G scale folded into lambda)."""
    I = np.asarray(I, dtype=np.float64)
    return float(-np.sum(I * np.log(I / G)))


def objective(P: Problem, I: np.ndarray, form: str = "factored"):
    """(Phi, chi^2, S) at I (all images), Phi = chi^2 - lambda S."""
    chis, _ = chi2_terms(P, I, form)
    chi = float(sum(chis))
    S = entropy(I, P.G)
    return chi - P.lam * S, chi, S


def grad_chi2(P: Problem, res, form: str = "factored") -> np.ndarray:
    g = np.zeros((P.n_images, P.N, P.N))
    for c in range(P.C):
        s = P.sl(c)
        gc = P.pb[c] * adjoint(P.N, P.dx, P.dy, P.u[s], P.v[s], P.weights(c) * res[c], None, form)
        if P.shared_image:
            g[0] += gc
        else:
            g[c] = gc
    return g


def objective_grad(P: Problem, I: np.ndarray, form: str = "factored"):
    """(Phi, chi^2, S, grad Phi) with grad Phi = A*Re(F^H(w r)) + lambda (1 + log(I/G))."""
    I = np.asarray(I, dtype=np.float64).reshape(P.n_images, P.N, P.N)
    chis, res = chi2_terms(P, I, form)
    chi = float(sum(chis))
    S = entropy(I, P.G)
    g = grad_chi2(P, res, form) + P.lam * (1.0 + np.log(I / P.G))
    return chi - P.lam * S, chi, S, g


def project_grad(I: np.ndarray, g: np.ndarray, G: float) -> np.ndarray:
    """Positive projection of the gradient (Eq. minproblem, I >= G): a pixel on
    the bound whose gradient points outward (g > 0, descent would lower it)
    is frozen."""
    out = g.copy()
    out[(I <= G) & (g > 0)] = 0.0
    return out


def project_dir(I: np.ndarray, d: np.ndarray, G: float) -> np.ndarray:
    """A search direction cannot move a pixel on the bound downwards."""
    out = d.copy()
    out[(I <= G) & (d < 0)] = 0.0
    return out


def thermal_noise(sigma) -> float:
    """sigma_D = (sum_k 1/sigma_k^2)^(-1/2) (Appendix B)."""
    s = np.asarray(sigma, dtype=np.float64)
    return float(1.0 / math.sqrt(np.sum(1.0 / s ** 2)))


# ----------------------------------------------------------------------------
# projected Polak-Ribiere CG with bracketing + Brent line search
# ----------------------------------------------------------------------------
GOLD = 1.618033988749895        # bracket expansion ratio (golden ratio)
CGOLD = 0.3819660112501051      # golden-section fraction 2 - GOLD
SHRINK = 0.25                   # trial-step reduction while no decrease is found
LS_MAX_EVALS = 20               # objective evaluations per line search
LS_TOL = 1e-3                   # relative tolerance on the step in Brent's method
LS_EPS = 1e-10                  # absolute tolerance, as a fraction of the first trial step
RESTART = 50                    # steepest-descent restart period
POLISH = 0.2                    # half-width of the final 3-point Newton step, relative to the step


def brent_min(phi, lo, hi, x, fx, tol, eps, budget):
    """Brent's minimisation without derivatives (Brent 1973, ch. 5) on the
    bracket lo < x < hi with phi(x) below both ends.  Returns (x, phi(x), evals)."""
    w = v = x
    fw = fv = fx
    d = e = 0.0
    evals = 0
    while evals < budget:
        xm = 0.5 * (lo + hi)
        tol1 = tol * abs(x) + eps
        tol2 = 2.0 * tol1
        if abs(x - xm) <= tol2 - 0.5 * (hi - lo):
            break
        golden = True
        if abs(e) > tol1:
            # parabola through (v, fv), (w, fw), (x, fx)
            r = (x - w) * (fx - fv)
            q = (x - v) * (fx - fw)
            p = (x - v) * q - (x - w) * r
            q = 2.0 * (q - r)
            if q > 0.0:
                p = -p
            else:
                q = -q
            e_prev = e
            e = d
            if abs(p) < abs(0.5 * q * e_prev) and p > q * (lo - x) and p < q * (hi - x):
                d = p / q
                t = x + d
                if (t - lo) < tol2 or (hi - t) < tol2:
                    d = tol1 if xm >= x else -tol1
                golden = False
        if golden:
            e = (lo - x) if x >= xm else (hi - x)
            d = CGOLD * e
        t = x + d if abs(d) >= tol1 else x + (tol1 if d >= 0.0 else -tol1)
        ft = phi(t)
        evals += 1
        if ft <= fx:
            if t >= x:
                lo = x
            else:
                hi = x
            v, fv = w, fw
            w, fw = x, fx
            x, fx = t, ft
        else:
            if t < x:
                lo = t
            else:
                hi = t
            if ft <= fw or w == x:
                v, fv = w, fw
                w, fw = t, ft
            elif ft <= fv or v == x or v == w:
                v, fv = t, ft
    return x, fx, evals


def line_search(phi, f0: float, alpha0: float):
    """Minimise phi(alpha), alpha >= 0, phi(0) = f0, starting from the trial step
    alpha0 > 0.  Bracket (shrink by SHRINK until phi < f0, or expand by GOLD
    while phi keeps falling), then Brent, then one Newton step on the centred
    stencil x -/+ POLISH x (see polish).  Returns (alpha, evals); alpha = 0 when
    no decrease was found within the budget."""
    x, fx, evals = _bracket_brent(phi, f0, alpha0)
    if x <= 0.0:
        return 0.0, evals
    return polish(phi, x, fx, min(POLISH * alpha0, 0.5 * x)), evals + 2


def polish(phi, x: float, fx: float, h: float) -> float:
    """Final step: Newton on central differences over x -/+ h, clamped to
    [x - h, x + h], with h = min(POLISH alpha0, x/2) fixed by the trial step.
    Brent stops anywhere within its tolerance of the minimiser; this step moves
    it to within O(tol^2) by a formula that is continuous in the objective
    values, so that implementations with different rounding land on the same
    step."""
    fp = phi(x + h)
    fm = phi(x - h)
    curv = fp - 2.0 * fx + fm
    if curv > 0.0:
        t = x - h * (fp - fm) / (2.0 * curv)
        x = min(max(t, x - h), x + h)
    return x


def _bracket_brent(phi, f0: float, alpha0: float):
    eps = LS_EPS * alpha0
    a, fa = 0.0, f0
    b = alpha0
    fb = phi(b)
    evals = 1
    if fb >= fa:
        c, fc = b, fb
        while fb >= fa and evals < LS_MAX_EVALS:
            c, fc = b, fb
            b = b * SHRINK
            fb = phi(b)
            evals += 1
        if fb >= fa:
            return 0.0, f0, evals
    else:
        c = b + GOLD * (b - a)
        fc = phi(c)
        evals += 1
        while fc < fb and evals < LS_MAX_EVALS:
            a, fa = b, fb
            b, fb = c, fc
            c = b + GOLD * (b - a)
            fc = phi(c)
            evals += 1
        if fc < fb:
            return c, fc, evals
    x, fx, n = brent_min(phi, a, c, b, fb, LS_TOL, eps, LS_MAX_EVALS - evals)
    return x, fx, evals + n


def _solve_one(P: Problem, I0: np.ndarray, n_iter: int, chan, form: str):
    """Projected PR-CG on one image.  `chan` lists the channels whose chi^2
    involves this image (all channels in shared-image mode)."""
    G, lam = P.G, P.lam

    def sub_problem():
        offs = [0]
        us, vs, vos, sgs, pbs = [], [], [], [], []
        for c in chan:
            s = P.sl(c)
            us.append(P.u[s]); vs.append(P.v[s]); vos.append(P.vo[s]); sgs.append(P.sigma[s])
            pbs.append(P.pb[c]); offs.append(offs[-1] + s.stop - s.start)
        return Problem(P.N, P.dx, P.dy, np.concatenate(us), np.concatenate(vs), np.concatenate(vos),
                       np.concatenate(sgs), np.stack(pbs), np.array(offs, dtype=np.int64), G, lam,
                       shared_image=True)

    Q = sub_problem()
    I = np.maximum(np.asarray(I0, dtype=np.float64).reshape(1, P.N, P.N), G)
    f, chi, S, gfull = objective_grad(Q, I, form)
    g = project_grad(I, gfull, G)
    hist = [dict(phi=f, chi2=chi, S=S, alpha=0.0, beta=0.0, evals=0)]
    d = np.zeros_like(I)
    g_prev = None
    for k in range(n_iter):
        beta = 0.0
        if k > 0 and k % RESTART != 0:
            gg = float(np.sum(g_prev * g_prev))
            if gg > 0.0:
                beta = max(0.0, float(np.sum((g - g_prev) * g)) / gg)
        d = project_dir(I, -g + beta * d, G)
        slope = float(np.sum(gfull * d))
        if slope >= 0.0:
            beta = 0.0
            d = project_dir(I, -g, G)
            slope = float(np.sum(gfull * d))
        if slope >= 0.0:
            break
        # quadratic model of chi^2 along d: 1/2 alpha^2 sum w |F(A d)|^2
        curv = 0.0
        for c, vd in enumerate(model_vis(Q, d, form)):
            curv += float(np.sum(Q.weights(c) * (vd.real ** 2 + vd.imag ** 2)))
        if curv > 0.0:
            alpha0 = -slope / curv
        else:
            alpha0 = float(np.max(I)) / float(np.max(np.abs(d)))

        def phi(alpha):
            return objective(Q, np.maximum(I + alpha * d, G), form)[0]

        alpha, evals = line_search(phi, f, alpha0)
        if alpha <= 0.0:
            break
        I = np.maximum(I + alpha * d, G)
        g_prev = g
        f, chi, S, gfull = objective_grad(Q, I, form)
        g = project_grad(I, gfull, G)
        hist.append(dict(phi=f, chi2=chi, S=S, alpha=alpha, beta=beta, evals=evals + 2))
    return I[0], hist


def solve(P: Problem, I0: np.ndarray, n_iter: int, form: str = "factored"):
    """Minimise Phi over I >= G (Eq. minproblem).  Cube mode: one independent
    CG per channel image.  Shared-image mode: one CG over Eq. chi2-multi.
    Returns (images (n_images, N, N), per-image histories)."""
    I0 = np.asarray(I0, dtype=np.float64).reshape(P.n_images, P.N, P.N)
    if P.shared_image:
        img, h = _solve_one(P, I0[0], n_iter, list(range(P.C)), form)
        return img[None], [h]
    imgs, hists = [], []
    for c in range(P.C):
        img, h = _solve_one(P, I0[c], n_iter, [c], form)
        imgs.append(img)
        hists.append(h)
    return np.stack(imgs), hists


def mosaic_forward(N: int, dx: float, dy: float, u, v, A_p, I, x_p: float, y_p: float) -> np.ndarray:
    """One pointing of a mosaic (Section 2.4: an attenuation image per pointing,
    centred on its field): the sky I seen through the pointing's primary beam
    A_p (already centred at the pointing, an N x N image on the same grid) with
    the phase referenced to the pointing centre (x_p, y_p):
    V_k = sum_{n,m} A_p[n,m] I[n,m] exp(-2 pi i (u_k (x_m - x_p) + v_k (y_n - y_p)))."""
    u, v = _f64(u), _f64(v)
    B = _f64(A_p).reshape(N, N) * _f64(I).reshape(N, N)
    return forward(N, dx, dy, u, v, B) * np.exp(2j * np.pi * (u * x_p + v * y_p))


def dirty_image(P: Problem, psf: bool = False, vis=None) -> np.ndarray:
    """Natural-weights dirty image per channel (Appendix A, Eq. dirty, with the
    measured visibilities in place of gridded ones), or the PSF (Eq. PSF):
    I^D(X) = sum_k omega_k Re(V_k exp(+2 pi i U_k . X)), omega_k = w_k / sum_l w_l
    over the channel's samples; no primary-beam factor.  (C, N, N).  vis: other
    visibilities in place of the measured ones (the residuals V° - V for a
    residual map)."""
    out = np.zeros((P.C, P.N, P.N))
    vo = P.vo if vis is None else np.asarray(vis, dtype=np.complex128)
    for c in range(P.C):
        s = P.sl(c)
        w = P.weights(c)
        if w.size == 0:
            continue
        om = w / np.sum(w)
        y = om * (np.ones(w.size) if psf else vo[s])
        out[c] = adjoint(P.N, P.dx, P.dy, P.u[s], P.v[s], y.astype(np.complex128))
    return out


BEAM_LOBE = 0.35  # main-lobe pixels: connected to the centre, PSF above this fraction of the peak


def beam_fit(psf: np.ndarray, dx: float, dy: float):
    """Elliptical Gaussian fitted to the PSF's main lobe (Appendix A: BMAJ,
    BMIN as FWHM, BPA).  Reading: least squares of ln(PSF / PSF0) against the
    quadratic form -(A x^2 + B x y + C y^2) over the 4-connected region around
    the centre pixel (N/2, N/2) where PSF > BEAM_LOBE PSF0, with x = (m - N/2) dx,
    y = (n - N/2) dy.  BPA (degrees, in (-90, 90]) runs from the +y (row) axis
    towards +x (column).  Returns (BMAJ, BMIN, BPA, beam area in pixels =
    pi/(4 ln 2) BMAJ BMIN / (dx dy))."""
    psf = np.asarray(psf, dtype=np.float64)
    N = psf.shape[0]
    c = N // 2
    p0 = psf[c, c]
    seen = np.zeros_like(psf, dtype=bool)
    stack, pix = [(c, c)], []
    seen[c, c] = True
    while stack:
        n, m = stack.pop()
        pix.append((n, m))
        for dn, dm in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            a, b = n + dn, m + dm
            if 0 <= a < N and 0 <= b < N and not seen[a, b] and psf[a, b] > BEAM_LOBE * p0:
                seen[a, b] = True
                stack.append((a, b))
    pix = np.array(sorted(pix))
    x = (pix[:, 1] - c) * dx
    y = (pix[:, 0] - c) * dy
    rhs = -np.log(psf[pix[:, 0], pix[:, 1]] / p0)
    X = np.stack([x * x, x * y, y * y], 1)
    A, B, C = np.linalg.lstsq(X, rhs, rcond=None)[0]
    lam, vec = np.linalg.eigh(np.array([[A, B / 2], [B / 2, C]]))
    if lam[0] <= 0:
        raise ValueError("the PSF main lobe is not a peak")
    bmaj, bmin = 2 * math.sqrt(math.log(2) / lam[0]), 2 * math.sqrt(math.log(2) / lam[1])
    ex, ey = vec[0, 0], vec[1, 0]  # major axis (smallest curvature)
    bpa = math.degrees(math.atan2(ex, ey))
    if bpa <= -90:
        bpa += 180
    if bpa > 90:
        bpa -= 180
    return bmaj, bmin, bpa, math.pi / (4 * math.log(2)) * bmaj * bmin / (dx * dy)


def kkt_residual(I: np.ndarray, g: np.ndarray, G: float) -> float:
    """|| I - max(I - g, G) ||: zero exactly at a point satisfying the bound-
    constrained first-order conditions."""
    return float(np.linalg.norm(I - np.maximum(I - g, G)))
