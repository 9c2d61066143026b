"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: expected values come from
numpy's FFT (the direct sum on the FFT grid), continuous Fourier transforms of
Gaussians and points, conjugate symmetry, the adjoint identity, finite
differences, Appendix B's noise formula, scipy's bounded minimisers, and
closed-form minima.  Each test names the passage it follows.
"""
import math

import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

FORMS = ["direct", "factored"]


def _grid_uv(N, dx, dy, kx, ky):
    return np.asarray(kx) / (N * dx), np.asarray(ky) / (N * dy)


@pytest.mark.parametrize("form", FORMS)
def test_forward_on_fft_grid_equals_fft2(oracle_mod, form):
    """Eq. (1) on the pixel grid at u = kx/(N dx), v = ky/(N dy) is a 2-D DFT:
    V = exp(+2 pi i (kx + ky) c / N) * FFT2(B)[ky, kx], c = N/2 (the pixel
    origin of the gradient kernel, Section 2.5).  dx != dy catches a swapped axis."""
    N, dx, dy = 16, 3e-7, 5e-7
    rng = np.random.default_rng(1)
    B = rng.random((N, N))
    kx = np.array([0, 1, 3, -2, 5, 7, -8, 4])
    ky = np.array([0, 2, -1, 4, -7, 1, 3, -8])
    u, v = _grid_uv(N, dx, dy, kx, ky)
    V = oracle_mod.forward(N, dx, dy, u, v, B, form)
    c = N // 2
    expect = np.fft.fft2(B)[ky % N, kx % N] * np.exp(2j * np.pi * (kx + ky) * c / N)
    assert np.max(np.abs(V - expect)) <= 1e-13 * np.max(np.abs(expect))


@pytest.mark.parametrize("form", FORMS)
def test_adjoint_on_fft_grid_equals_ifft2(oracle_mod, form):
    """Eq. (chi2gradient)'s sum Re(sum_k y_k exp(+2 pi i U_k.X)) on grid points is
    N^2 * IFFT2 of the gridded, phase-shifted y."""
    N, dx, dy = 16, 4e-7, 2e-7
    rng = np.random.default_rng(2)
    Z = 40
    kx = rng.integers(-N // 2, N // 2, Z)
    ky = rng.integers(-N // 2, N // 2, Z)
    u, v = _grid_uv(N, dx, dy, kx, ky)
    y = rng.standard_normal(Z) + 1j * rng.standard_normal(Z)
    c = N // 2
    Yg = np.zeros((N, N), dtype=complex)
    np.add.at(Yg, (ky % N, kx % N), y * np.exp(-2j * np.pi * (kx + ky) * c / N))
    expect = np.real(N * N * np.fft.ifft2(Yg))
    if form == "factored":
        G = oracle_mod.adjoint(N, dx, dy, u, v, y)
    else:
        G = oracle_mod.adjoint(N, dx, dy, u, v, y, crop=(0, N, 0, N), form="direct")
    assert np.max(np.abs(G - expect)) <= 1e-12 * np.max(np.abs(expect))


@pytest.mark.parametrize("form", FORMS)
def test_point_source_at_phase_centre(oracle_mod, form):
    """A point source of flux f at the phase centre gives V = f * A(0) for every (u,v)."""
    N, dx = 32, S.ARCSEC * 0.1
    rng = np.random.default_rng(3)
    Z = 64
    u = rng.uniform(-0.45, 0.45, Z) / dx
    v = rng.uniform(-0.45, 0.45, Z) / dx
    A = S.gaussian_beam(N, dx, dx, 20 * dx).astype(np.float64)
    I = np.zeros((N, N))
    I[N // 2, N // 2] = 0.37
    V = oracle_mod.forward(N, dx, dx, u, v, A * I, form)
    assert A[N // 2, N // 2] == 1.0
    assert np.max(np.abs(V - 0.37)) <= 1e-14


@pytest.mark.parametrize("form", FORMS)
def test_offset_point_source_phase_ramp(oracle_mod, form):
    """A point at pixel (n0, m0) gives the phase ramp f A exp(-2 pi i (u x0 + v y0))
    with x0 = (m0 - N/2) dx, y0 = (n0 - N/2) dy (asymmetric in x/y)."""
    N, dx, dy = 32, S.ARCSEC * 0.1, S.ARCSEC * 0.15
    rng = np.random.default_rng(4)
    Z = 64
    u = rng.uniform(-0.45, 0.45, Z) / dx
    v = rng.uniform(-0.45, 0.45, Z) / dy
    A = S.gaussian_beam(N, dx, dy, 20 * dx).astype(np.float64)
    n0, m0, f = 5, 23, 0.8
    I = np.zeros((N, N))
    I[n0, m0] = f
    x0, y0 = (m0 - N // 2) * dx, (n0 - N // 2) * dy
    V = oracle_mod.forward(N, dx, dy, u, v, A * I, form)
    expect = f * A[n0, m0] * np.exp(-2j * np.pi * (u * x0 + v * y0))
    assert np.max(np.abs(V - expect)) <= 1e-13


def test_gaussian_times_beam_closed_form(oracle_mod):
    """A well-sampled elliptical Gaussian times a Gaussian beam: the pixel sum
    equals the continuous transform (Poisson summation; aliases and edge
    truncation below 1e-10 for these widths)."""
    N, dx = 96, S.ARCSEC * 0.1
    comps = [S.Gaussian(flux=0.6, x0=0.3 * S.ARCSEC, y0=-0.2 * S.ARCSEC,
                        fwhm_maj=1.0 * S.ARCSEC, fwhm_min=0.8 * S.ARCSEC, pa=0.6)]
    beam = 6.0 * S.ARCSEC
    rng = np.random.default_rng(5)
    Z = 80
    u = rng.uniform(-0.3, 0.3, Z) / dx
    v = rng.uniform(-0.3, 0.3, Z) / dx
    img = S.sky_image(comps, N, dx, dx)
    x = (np.arange(N) - N // 2) * dx
    A = np.exp(-0.5 * (x[:, None] ** 2 + x[None, :] ** 2) / (beam * S.FWHM_TO_SIGMA) ** 2)
    V = oracle_mod.forward(N, dx, dx, u, v, A * img, "factored")
    expect = S.sky_visibilities(comps, u, v, beam)
    assert np.max(np.abs(V - expect)) <= 1e-10 * np.max(np.abs(expect))


def test_circular_gaussian_textbook_transform(oracle_mod):
    """Circular Gaussian of peak I0 (Jy/pixel) at the centre times a circular
    Gaussian beam: V(u,v) = I0 * 2 pi s_e^2 / (dx dy) * exp(-2 pi^2 s_e^2 (u^2+v^2)),
    s_e^2 = s_s^2 s_b^2 / (s_s^2 + s_b^2)."""
    N, dx = 128, S.ARCSEC * 0.05
    ss, sb = 4.0 * dx, 10.0 * dx
    x = (np.arange(N) - N // 2) * dx
    r2 = x[:, None] ** 2 + x[None, :] ** 2
    I0 = 0.02
    img = I0 * np.exp(-0.5 * r2 / ss ** 2)
    A = np.exp(-0.5 * r2 / sb ** 2)
    rng = np.random.default_rng(6)
    Z = 50
    u = rng.uniform(-0.2, 0.2, Z) / dx
    v = rng.uniform(-0.2, 0.2, Z) / dx
    se2 = ss ** 2 * sb ** 2 / (ss ** 2 + sb ** 2)
    expect = I0 * 2 * np.pi * se2 / (dx * dx) * np.exp(-2 * np.pi ** 2 * se2 * (u ** 2 + v ** 2))
    V = oracle_mod.forward(N, dx, dx, u, v, A * img, "factored")
    assert np.max(np.abs(V - expect)) <= 1e-10 * expect.max()


@pytest.mark.parametrize("form", FORMS)
def test_hermitian_symmetry(oracle_mod, form):
    """Real images have Hermitian visibilities: V(-u,-v) = conj V(u,v)."""
    N, dx = 24, S.ARCSEC * 0.1
    rng = np.random.default_rng(7)
    B = rng.random((N, N))
    u = rng.uniform(-0.45, 0.45, 30) / dx
    v = rng.uniform(-0.45, 0.45, 30) / dx
    V1 = oracle_mod.forward(N, dx, dx, u, v, B, form)
    V2 = oracle_mod.forward(N, dx, dx, -u, -v, B, form)
    assert np.max(np.abs(V2 - np.conj(V1))) <= 1e-13 * np.max(np.abs(V1))


@pytest.mark.parametrize("form", FORMS)
def test_degenerate_frequencies_closed_forms(oracle_mod, form):
    """Eq. 1 on the pixel grid x_m = (m - N/2) dx at frequencies where it has a
    plain value: the origin gives sum B; u dx = 1/2 gives the alternating sum
    sum_m (-1)^(m - N/2) B[n, m] (rows likewise for v); a whole turn per pixel
    (u dx = 1) aliases to u = 0, and any u + 1/dx aliases to u."""
    N, dx, dy = 32, 2.1e-7, 1.7e-7
    rng = np.random.default_rng(13)
    B = rng.random((N, N))
    sgn = (-1.0) ** (np.arange(N) - N // 2)
    u0, v0 = 0.31 / dx, -0.22 / dy
    u = np.array([0.0, 0.5 / dx, 0.0, 0.5 / dx, 1.0 / dx, u0 + 1.0 / dx, u0, -1.5 / dx])
    v = np.array([0.0, 0.0, 0.5 / dy, -0.5 / dy, 0.0, v0 - 2.0 / dy, v0, 0.0])
    V = oracle_mod.forward(N, dx, dy, u, v, B, form)
    scale = B.sum()
    assert abs(V[0] - B.sum()) <= 1e-13 * scale
    assert abs(V[1] - (B * sgn[None, :]).sum()) <= 1e-12 * scale
    assert abs(V[2] - (B * sgn[:, None]).sum()) <= 1e-12 * scale
    assert abs(V[3] - (B * sgn[:, None] * sgn[None, :]).sum()) <= 1e-12 * scale
    assert abs(V[4] - V[0]) <= 1e-12 * scale
    assert abs(V[5] - V[6]) <= 1e-12 * scale
    assert abs(V[7] - V[1]) <= 1e-12 * scale


@pytest.mark.parametrize("form", FORMS)
def test_adjoint_identity(oracle_mod, form):
    """Re<F x, y> = <x, Re(F^H y)> for real x, complex y (Appendix C pairs the
    model's derivative with the chi^2 gradient)."""
    N, dx, dy = 20, S.ARCSEC * 0.1, S.ARCSEC * 0.12
    rng = np.random.default_rng(8)
    Z = 70
    u = rng.uniform(-0.45, 0.45, Z) / dx
    v = rng.uniform(-0.45, 0.45, Z) / dy
    x = rng.standard_normal((N, N))
    y = rng.standard_normal(Z) + 1j * rng.standard_normal(Z)
    lhs = np.real(np.vdot(y, oracle_mod.forward(N, dx, dy, u, v, x, form)))
    G = oracle_mod.adjoint(N, dx, dy, u, v, y, crop=(0, N, 0, N), form=form)
    rhs = float(np.sum(x * G))
    assert abs(lhs - rhs) <= 1e-12 * (np.sum(np.abs(x)) * np.sum(np.abs(y)))


def test_factored_and_direct_agree(oracle_mod):
    """The factored evaluation order reproduces the direct sum to rounding."""
    N, dx, dy = 32, S.ARCSEC * 0.1, S.ARCSEC * 0.07
    rng = np.random.default_rng(9)
    Z = 100
    u = rng.uniform(-0.45, 0.45, Z) / dx * 3  # several turns across the field
    v = rng.uniform(-0.45, 0.45, Z) / dy * 3
    B = rng.random((N, N))
    y = rng.standard_normal(Z) + 1j * rng.standard_normal(Z)
    Vd = oracle_mod.forward(N, dx, dy, u, v, B, "direct")
    Vf = oracle_mod.forward(N, dx, dy, u, v, B, "factored")
    assert np.max(np.abs(Vd - Vf)) <= 1e-12 * np.max(np.abs(Vd))
    Gd = oracle_mod.adjoint(N, dx, dy, u, v, y, crop=(0, N, 0, N), form="direct")
    Gf = oracle_mod.adjoint(N, dx, dy, u, v, y)
    Gc = oracle_mod.adjoint(N, dx, dy, u, v, y, crop=(3, 10, 7, 12), form="factored")
    assert np.max(np.abs(Gd - Gf)) <= 1e-12 * np.max(np.abs(Gd))
    assert np.max(np.abs(Gc - Gd[3:13, 7:19])) <= 1e-12 * np.max(np.abs(Gd))


def _tiny_problem(seed=10, N=8, Z=50, C=1, shared=False, lam=2.0):
    ds = S.random_problem(N, Z, seed, C=C, shared_image=shared, lam=lam, G=1e-3)
    return ds


def test_chi2_gradient_central_differences_exact(oracle_mod):
    """chi^2 is quadratic in I, so central differences are exact for any step
    (Eq. phi2): [chi2(I + h e_p) - chi2(I - h e_p)] / 2h = d chi2 / d I_p."""
    ds = _tiny_problem()
    P = oracle_mod.Problem.from_dataset(ds, lam=0.0)
    I = ds.truth.astype(np.float64)
    _, _, _, g = oracle_mod.objective_grad(P, I)
    rng = np.random.default_rng(11)
    for p in rng.choice(P.N * P.N, 12, replace=False):
        h = 0.05
        e = np.zeros_like(I).ravel()
        e[p] = h
        e = e.reshape(I.shape)
        fp = oracle_mod.objective(P, I + e)[1]
        fm = oracle_mod.objective(P, I - e)[1]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g.ravel()[p]) <= 1e-9 * max(1.0, abs(g.ravel()[p]))


@pytest.mark.parametrize("C,shared", [(1, False), (2, True), (3, False)])
def test_objective_gradient_finite_differences(oracle_mod, C, shared):
    """grad Phi = A Re(F^H w r) + lambda (1 + log(I/G)) against central differences
    of Phi (Eq. phi3, Eq. Sgradient, Eq. chi2-multi for the shared image)."""
    ds = _tiny_problem(seed=12 + C, C=C, shared=shared)
    P = oracle_mod.Problem.from_dataset(ds)
    I = ds.truth.astype(np.float64) + 0.01
    phi, _, _, g = oracle_mod.objective_grad(P, I)
    rng = np.random.default_rng(13)
    for p in rng.choice(I.size, 10, replace=False):
        h = 1e-6
        e = np.zeros(I.size)
        e[p] = h
        e = e.reshape(I.shape)
        fd = (oracle_mod.objective(P, I + e)[0] - oracle_mod.objective(P, I - e)[0]) / (2 * h)
        assert abs(fd - g.ravel()[p]) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_zero_gradient_at_exact_data(oracle_mod):
    """With V^o = F(A I) the chi^2 residuals vanish and so does grad chi^2; at
    I = 0 the gradient is -A Re(F^H(w V^o)) (a weighted dirty image, Appendix A)."""
    ds = _tiny_problem(seed=20)
    P = oracle_mod.Problem.from_dataset(ds, lam=0.0)
    I = ds.truth.astype(np.float64)
    P.vo = oracle_mod.model_vis(P, I)[0]
    phi, chi, _, g = oracle_mod.objective_grad(P, np.maximum(I, 1e-300))
    assert chi <= 1e-25 and np.max(np.abs(g)) <= 1e-10
    P2 = oracle_mod.Problem.from_dataset(ds, lam=0.0)
    chis, res = oracle_mod.chi2_terms(P2, np.zeros_like(I))
    g0 = oracle_mod.grad_chi2(P2, res)
    w = 1.0 / ds.sigma ** 2
    dirty = oracle_mod.adjoint(P2.N, P2.dx, P2.dy, ds.u, ds.v, w * ds.vo)
    assert np.max(np.abs(g0[0] + ds.pb[0] * dirty)) <= 1e-12 * np.max(np.abs(g0))


def test_entropy_maximal_at_prior_on_feasible_set(oracle_mod):
    """S = -sum I log(I/G): stationary at I = G/e (dS/dI = -(1 + log(I/G))),
    decreasing for I > G/e, so on I >= G it is largest at I = G (Eq. minproblem)."""
    G = 1e-3
    rng = np.random.default_rng(14)
    s_prior = oracle_mod.entropy(np.full(64, G), G)
    assert s_prior == 0.0
    for _ in range(20):
        I = G + rng.random(64) * rng.choice([1e-4, 1e-2, 1.0])
        assert oracle_mod.entropy(I, G) < s_prior
    # stationary point of the unconstrained entropy
    h = 1e-9
    s = lambda t: oracle_mod.entropy(np.array([t]), G)
    d = (s(G / math.e + h) - s(G / math.e - h)) / (2 * h)
    assert abs(d) < 1e-6
    assert s(G / math.e) > s(G / math.e * 1.01) and s(G / math.e) > s(G / math.e * 0.99)


def test_thermal_noise_appendix_b(oracle_mod):
    """Appendix B: a noise-only natural-weight dirty pixel has standard deviation
    sigma_D = (sum 1/sigma^2)^(-1/2), whatever the (u,v) coverage."""
    N, dx = 8, S.ARCSEC * 0.1
    rng = np.random.default_rng(15)
    Z = 40
    u = rng.uniform(-0.45, 0.45, Z) / dx
    v = rng.uniform(-0.45, 0.45, Z) / dx
    sigma = rng.uniform(0.5, 2.0, Z)
    w = 1.0 / sigma ** 2
    omega = w / w.sum()
    vals = []
    for s in range(1500):
        r = np.random.default_rng(1000 + s)
        noise = sigma * (r.standard_normal(Z) + 1j * r.standard_normal(Z))
        vals.append(oracle_mod.adjoint(N, dx, dx, u, v, omega * noise, crop=(2, 1, 5, 1))[0, 0])
    sd = np.std(vals)
    assert abs(sd / oracle_mod.thermal_noise(sigma) - 1.0) < 0.08


def test_generator_visibilities_match_pixel_sum(oracle_mod):
    """The generator's closed-form visibilities of well-sampled Gaussians and
    pixel-centred points equal the oracle's pixel sum of its pixelised sky."""
    N, dx = 128, S.ARCSEC * 0.1
    comps = [S.Gaussian(0.5, 0.5 * S.ARCSEC, 0.3 * S.ARCSEC, 1.5 * S.ARCSEC, 1.2 * S.ARCSEC, 1.1),
             S.Gaussian(0.3, -1.0 * S.ARCSEC, 0.2 * S.ARCSEC, 1.2 * S.ARCSEC, 1.0 * S.ARCSEC, 0.2),
             S.Point(0.2, 0.4 * S.ARCSEC, -0.8 * S.ARCSEC)]
    beam = 12 * S.ARCSEC
    rng = np.random.default_rng(16)
    u = rng.uniform(-0.3, 0.3, 60) / dx
    v = rng.uniform(-0.3, 0.3, 60) / dx
    A = S.gaussian_beam(N, dx, dx, beam).astype(np.float64)
    x = (np.arange(N) - N // 2) * dx
    A64 = np.exp(-0.5 * (x[:, None] ** 2 + x[None, :] ** 2) / (beam * S.FWHM_TO_SIGMA) ** 2)
    V = oracle_mod.forward(N, dx, dx, u, v, A64 * S.sky_image(comps, N, dx, dx))
    expect = S.sky_visibilities(comps, u, v, beam)
    assert np.max(np.abs(V - expect)) <= 1e-9 * np.max(np.abs(expect))
    assert np.max(np.abs(A - A64)) < 1e-7


def test_brent_matches_scipy_bounded_minimiser(oracle_mod):
    """The line-search core (Brent 1973) finds the same minimiser as scipy's
    bounded Brent on smooth unimodal functions."""
    from scipy.optimize import minimize_scalar
    fns = [lambda t: (t - 0.7) ** 2 + 0.1 * t ** 4,
           lambda t: math.exp(t) - 3 * t,
           lambda t: t * math.log(t) if t > 0 else 0.0]
    for f in fns:
        x, fx, n = oracle_mod.brent_min(f, 1e-3, 3.0, 1.0, f(1.0), 1e-8, 1e-12, 200)
        ref = minimize_scalar(f, bounds=(1e-3, 3.0), method="bounded", options=dict(xatol=1e-10))
        assert abs(x - ref.x) < 1e-6 and fx <= ref.fun + 1e-12


def test_line_search_brackets_and_converges(oracle_mod):
    """Bracketing by shrinking or golden expansion, then Brent: the accepted
    step is within the tolerance of the true minimiser, from either side."""
    for a_true, a0 in [(3.0, 0.1), (0.01, 5.0), (1.0, 1.0)]:
        f = lambda t, a=a_true: (t - a) ** 2 / a + 1.0
        alpha, n = oracle_mod.line_search(f, f(0.0), a0)
        # on a parabola the final Newton step is exact
        assert abs(alpha - a_true) <= 1e-12 * a_true
        assert n <= oracle_mod.LS_MAX_EVALS + 2
    # non-quadratic: x log x - x has its minimum at 1; the final central-
    # difference Newton step carries its truncation term (h^2 / 6) g3 / g2 with
    # g3 / g2 = -1 there (h <= x / 2), identical for every implementation
    g = lambda t: t * math.log(t) - t if t > 0 else 0.0
    alpha, n = oracle_mod.line_search(g, 0.0, 0.3)
    assert abs(alpha - 1.0) <= 1.2 * 0.5 ** 2 / 6
    alpha, n = oracle_mod.line_search(lambda t: 1.0 + t, 1.0, 1.0)
    assert alpha == 0.0


def test_polish_is_continuous_in_the_start(oracle_mod):
    """Two Brent results at the two ends of a 2e-3 tolerance window polish to
    steps that agree about 100x more closely: what is left depends on the start
    only through a term of order h^2 (x - x*) (third derivative of the test
    function relative to its curvature)."""
    from scipy.optimize import minimize_scalar
    f = lambda t: math.exp(t) - 3 * t + 0.1 * t ** 4
    xs = minimize_scalar(f, bounds=(0.1, 3.0), method="bounded", options=dict(xatol=1e-12)).x
    h = oracle_mod.POLISH * xs
    a = oracle_mod.polish(f, xs * (1 - 1e-3), f(xs * (1 - 1e-3)), h)
    b = oracle_mod.polish(f, xs * (1 + 1e-3), f(xs * (1 + 1e-3)), h)
    assert abs(a - b) <= 2e-5 * xs


def test_polish_is_exact_on_a_parabola_and_stays_in_its_window(oracle_mod):
    """The central-difference Newton step lands on a parabola's vertex from any
    start within h of it, and never leaves [x - h, x + h] (it is a clamped
    step, so a vertex farther away is approached by h only)."""
    f = lambda t: 3.0 * (t - 1.7) ** 2 - 2.0
    for x in (1.55, 1.7, 1.84):
        assert abs(oracle_mod.polish(f, x, f(x), 0.2) - 1.7) <= 1e-12
    assert oracle_mod.polish(f, 1.0, f(1.0), 0.2) == pytest.approx(1.2, abs=1e-15)
    assert oracle_mod.polish(f, 2.5, f(2.5), 0.2) == pytest.approx(2.3, abs=1e-15)
    # no curvature (a line, or a concave stencil): the step stays where it is
    assert oracle_mod.polish(lambda t: -t, 0.8, -0.8, 0.1) == 0.8
    assert oracle_mod.polish(lambda t: -(t - 1) ** 2, 0.8, -0.04, 0.1) == 0.8


def test_projection_rules(oracle_mod):
    """Positive projection at the bound I = G (Eq. minproblem): a pixel on the
    bound keeps a gradient component only if descent (-g) raises it, and a
    search direction only if it does not lower it.  Pixels above the bound
    are never touched."""
    G = 1e-3
    I = np.array([G, G, 2 * G, 3 * G, G, 0.5 * G])
    g = np.array([1.0, -1.0, 1.0, -1.0, 0.0, 2.0])
    assert np.array_equal(oracle_mod.project_grad(I, g, G), [0.0, -1.0, 1.0, -1.0, 0.0, 0.0])
    d = np.array([-1.0, 1.0, -1.0, 1.0, 0.0, -3.0])
    assert np.array_equal(oracle_mod.project_dir(I, d, G), [0.0, 1.0, -1.0, 1.0, 0.0, 0.0])
    # the inputs are not modified in place
    assert np.array_equal(g, [1.0, -1.0, 1.0, -1.0, 0.0, 2.0])
    assert np.array_equal(d, [-1.0, 1.0, -1.0, 1.0, 0.0, -3.0])


def test_cg_terminates_on_a_quadratic(oracle_mod):
    """With lambda = 0 and the bound inactive Phi = chi^2 is a convex quadratic
    in n = N^2 unknowns.  Polak-Ribiere CG with an exact line search is then
    linear CG, which reaches the minimiser in at most n steps in exact
    arithmetic (Hestenes and Stiefel 1952); the line search is exact here
    because the first trial step is the quadratic model's minimiser and the
    final Newton step is exact on a parabola.  Steepest descent (beta = 0), a
    wrong sign of beta or of the direction update stall far above it."""
    N = 4
    ds = S.random_problem(N, 40, 31, C=1, shared_image=False, lam=0.0, G=1e-12)
    P = oracle_mod.Problem.from_dataset(ds)
    rng = np.random.default_rng(5)
    truth = 1.0 + rng.random((1, N, N))
    P.vo = oracle_mod.model_vis(P, truth)[0]
    I0 = truth + 0.3 * rng.standard_normal((1, N, N))
    assert I0.min() > 0.5
    img, hists = oracle_mod.solve(P, I0, N * N + 4)
    phis = [h["phi"] for h in hists[0]]
    assert np.max(np.abs(img - truth)) <= 1e-9
    assert phis[-1] <= 1e-15 * phis[0]
    # after n steps only rounding is left (a factor 1e6 below the start at least)
    assert phis[min(N * N, len(phis) - 1)] <= 1e-5 * phis[0]


@pytest.mark.parametrize("lam", [50.0, 2.0])
def test_solver_reaches_bounded_minimiser(oracle_mod, lam):
    """For lambda > 0 Phi is strictly convex on I >= G (quadratic chi^2 plus
    I log I), so the minimiser of Eq. minproblem is unique: the projected CG
    lands on the point scipy's L-BFGS-B finds with the same bounds, Phi never
    increases, every iterate stays feasible and the bound-constrained KKT
    residual falls by 1e3 at least."""
    from scipy.optimize import minimize
    ds = _tiny_problem(seed=21, N=8, Z=60, lam=lam)
    P = oracle_mod.Problem.from_dataset(ds)
    I0 = np.full((1, 8, 8), P.G)
    img, hists = oracle_mod.solve(P, I0, 150)
    phis = [h["phi"] for h in hists[0]]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(phis, phis[1:]))
    assert img.min() >= P.G
    # the bound is active somewhere, so the projection is exercised
    assert np.count_nonzero(img <= P.G) > 0

    def fg(x):
        phi, _, _, g = oracle_mod.objective_grad(P, x.reshape(1, 8, 8))
        return phi, g.ravel()

    ref = minimize(fg, np.full(64, 2 * P.G), jac=True, method="L-BFGS-B",
                   bounds=[(P.G, None)] * 64, options=dict(maxiter=5000, ftol=1e-15, gtol=1e-12))
    rel = np.linalg.norm(img.ravel() - ref.x) / np.linalg.norm(ref.x)
    assert rel < 1e-3, rel
    assert phis[-1] <= ref.fun * (1 + 1e-12)
    _, _, _, g = oracle_mod.objective_grad(P, img)
    k_end = oracle_mod.kkt_residual(img, g, P.G)
    _, _, _, g0 = oracle_mod.objective_grad(P, np.maximum(I0, P.G))
    assert k_end < 1e-3 * oracle_mod.kkt_residual(np.maximum(I0, P.G), g0, P.G)


def test_shared_image_solve_reaches_the_summed_minimiser(oracle_mod):
    """Shared-image mode (Eq. chi2-multi): one image, chi^2 summed over the
    channels, each with its own beam.  The solve lands on L-BFGS-B's bounded
    minimiser of that summed objective."""
    from scipy.optimize import minimize
    ds = _tiny_problem(seed=23, N=8, Z=30, C=3, shared=True, lam=20.0)
    P = oracle_mod.Problem.from_dataset(ds)
    assert P.shared_image and P.C == 3
    I0 = np.full((1, 8, 8), P.G)
    img, hists = oracle_mod.solve(P, I0, 150)
    assert img.shape == (1, 8, 8) and len(hists) == 1

    def fg(x):
        phi, _, _, g = oracle_mod.objective_grad(P, x.reshape(1, 8, 8))
        return phi, g.ravel()

    ref = minimize(fg, np.full(64, 2 * P.G), jac=True, method="L-BFGS-B",
                   bounds=[(P.G, None)] * 64, options=dict(maxiter=5000, ftol=1e-15, gtol=1e-12))
    rel = np.linalg.norm(img.ravel() - ref.x) / np.linalg.norm(ref.x)
    assert rel < 1e-3, rel


def test_cube_mode_solves_channels_independently(oracle_mod):
    """Cube mode (independent channel images): solving the cube equals solving
    each channel alone, bit for bit."""
    ds = _tiny_problem(seed=22, C=2, N=8, Z=40, lam=20.0)
    P = oracle_mod.Problem.from_dataset(ds)
    assert not P.shared_image
    I0 = np.full((2, 8, 8), P.G)
    imgs, _ = oracle_mod.solve(P, I0, 10)
    for c in range(2):
        s = P.sl(c)
        Pc = oracle_mod.Problem(P.N, P.dx, P.dy, P.u[s], P.v[s], P.vo[s], P.sigma[s], P.pb[c:c + 1],
                                np.array([0, s.stop - s.start]), P.G, P.lam)
        ic, _ = oracle_mod.solve(Pc, I0[c:c + 1], 10)
        assert np.array_equal(ic[0], imgs[c])
    # and the two channels really differ (their data do)
    assert not np.array_equal(imgs[0], imgs[1])


# ---------------------------------------------------------------------------
# the paper's gridded forward (Section 2.4 steps, Algorithm alg:chi2gpu)
# ---------------------------------------------------------------------------
def _gridded_case(N=16, seed=3):
    rng = np.random.default_rng(seed)
    dx, dy = 1.3e-6, 0.9e-6
    B = rng.random((N, N))
    return N, dx, dy, B, rng


def test_gridded_forward_on_grid_points_equals_the_direct_sum(oracle_mod):
    """At grid frequencies (k, l) / (M dx, M dy) there is no interpolation:
    FFT plus modulation must reproduce the direct sum of Eq. (1)."""
    N, dx, dy, B, rng = _gridded_case()
    for pad in (1, 2, 3):
        M = pad * N
        k = rng.integers(-M, M, 40)
        l = rng.integers(-M, M, 40)
        u, v = k / (M * dx), l / (M * dy)
        g = oracle_mod.forward_gridded(N, dx, dy, u, v, B, pad)
        d = oracle_mod.forward(N, dx, dy, u, v, B, "direct")
        assert np.max(np.abs(g - d)) <= 1e-12 * np.max(np.abs(d)), pad


def test_gridded_forward_is_the_bilinear_blend_of_grid_values(oracle_mod):
    """Between grid points the result is the bilinear blend of the exact sums
    at the four surrounding grid frequencies."""
    N, dx, dy, B, rng = _gridded_case(seed=4)
    pad = 2
    M = pad * N
    gu, gv = rng.uniform(-M, M, 30), rng.uniform(-M, M, 30)
    u, v = gu / (M * dx), gv / (M * dy)
    g = oracle_mod.forward_gridded(N, dx, dy, u, v, B, pad)
    k0, l0 = np.floor(gu), np.floor(gv)
    fx, fy = gu - k0, gv - l0
    corner = lambda dk, dl: oracle_mod.forward(N, dx, dy, (k0 + dk) / (M * dx), (l0 + dl) / (M * dy), B, "direct")
    ref = ((1 - fx) * (1 - fy) * corner(0, 0) + fx * (1 - fy) * corner(1, 0)
           + (1 - fx) * fy * corner(0, 1) + fx * fy * corner(1, 1))
    assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_gridded_forward_is_hermitian_and_converges_with_padding(oracle_mod):
    """Real image: V(-u,-v) = conj V(u,v); the interpolation error against the
    exact sum falls as the grid is refined by zero padding (smooth image)."""
    N = 32
    dx = dy = 1e-6
    yy, xx = np.mgrid[0:N, 0:N] - N / 2
    B = np.exp(-(xx ** 2 + yy ** 2) / (2 * 3.0 ** 2))
    rng = np.random.default_rng(5)
    r = rng.uniform(0, 0.45 / dx, 200)
    t = rng.uniform(0, 2 * np.pi, 200)
    u, v = r * np.cos(t), r * np.sin(t)
    d = oracle_mod.forward(N, dx, dy, u, v, B, "direct")
    errs = []
    for pad in (1, 2, 4, 8):
        g = oracle_mod.forward_gridded(N, dx, dy, u, v, B, pad)
        gm = oracle_mod.forward_gridded(N, dx, dy, -u, -v, B, pad)
        assert np.max(np.abs(gm - np.conj(g))) <= 1e-12 * np.max(np.abs(g))
        errs.append(np.max(np.abs(g - d)) / np.max(np.abs(d)))
    assert errs[0] > errs[1] > errs[2] > errs[3], errs
    assert errs[3] < 0.05 * errs[0], errs


# ---------------------------------------------------------------------------
# dirty image, PSF and beam (Appendix A)
# ---------------------------------------------------------------------------
def test_psf_peaks_at_one_and_point_source_dirty_image_is_shifted_psf(oracle_mod):
    """sum omega = 1 puts the PSF's peak (1) at the phase centre.  A noiseless
    point source of flux f at pixel (n0, m0) has V_k = f exp(-2 pi i U_k . X0),
    so by the shift theorem its dirty image is f PSF(X - X0)."""
    ds = S.random_problem(32, 300, 91)
    N, c = ds.N, ds.N // 2
    f, n0, m0 = 0.7, 19, 11
    x0, y0 = (m0 - c) * ds.dx, (n0 - c) * ds.dy
    ds.vo = f * np.exp(-2j * np.pi * (ds.u * x0 + ds.v * y0))
    P = oracle_mod.Problem.from_dataset(ds)
    psf = oracle_mod.dirty_image(P, psf=True)[0]
    assert psf[c, c] == pytest.approx(1.0, abs=1e-12)
    assert np.max(psf) == pytest.approx(1.0, abs=1e-12)
    dirty = oracle_mod.dirty_image(P)[0]
    dn, dm = n0 - c, m0 - c
    # dirty[n, m] = f psf[n - dn, m - dm] wherever both indices are on the grid
    sub = dirty[max(dn, 0):N + min(dn, 0), max(dm, 0):N + min(dm, 0)]
    ref = f * psf[max(-dn, 0):N + min(-dn, 0), max(-dm, 0):N + min(-dm, 0)]
    assert np.max(np.abs(sub - ref)) <= 1e-12
    assert np.unravel_index(np.argmax(dirty), dirty.shape) == (n0, m0)


def test_beam_fit_recovers_an_elliptical_gaussian(oracle_mod):
    N = 64
    dx, dy = 0.05e-6, 0.07e-6
    for bmaj, bmin, bpa in [(9e-7, 5e-7, 30.0), (1.2e-6, 1.2e-6 * 0.999, -75.0), (8e-7, 3e-7, 90.0)]:
        n, m = np.mgrid[0:N, 0:N]
        x, y = (m - N // 2) * dx, (n - N // 2) * dy
        t = np.radians(bpa)
        a = x * np.sin(t) + y * np.cos(t)   # along the major axis (from +y towards +x)
        b = x * np.cos(t) - y * np.sin(t)
        s2 = 1 / (8 * np.log(2))
        psf = np.exp(-(a ** 2 / (s2 * bmaj ** 2) + b ** 2 / (s2 * bmin ** 2)) / 2)
        got = oracle_mod.beam_fit(psf, dx, dy)
        assert got[0] == pytest.approx(bmaj, rel=1e-9)
        assert got[1] == pytest.approx(bmin, rel=1e-9)
        if bmaj / bmin > 1.01:
            assert (got[2] - bpa + 90) % 180 - 90 == pytest.approx(0.0, abs=1e-6)
        assert got[3] == pytest.approx(np.pi / (4 * np.log(2)) * bmaj * bmin / (dx * dy), rel=1e-9)


# ---------------------------------------------------------------------------
# mosaic pointing (Section 2.4: one attenuation image per pointing)
# ---------------------------------------------------------------------------
def test_mosaic_pointing_of_a_point_source_is_its_closed_form(oracle_mod):
    """A point source of flux f at X_s seen by a pointing centred at X_p:
    V = f A_p(X_s) exp(-2 pi i U . (X_s - X_p))."""
    N, dx = 48, 1e-6
    c = N // 2
    rng = np.random.default_rng(6)
    u, v = rng.uniform(-4e5, 4e5, 50), rng.uniform(-4e5, 4e5, 50)
    ns, ms_ = 30, 17
    I = np.zeros((N, N))
    I[ns, ms_] = 0.8
    xp, yp = 7 * dx, -5 * dx
    n, m = np.mgrid[0:N, 0:N]
    A = np.exp(-(((m - c) * dx - xp) ** 2 + ((n - c) * dx - yp) ** 2) / (2 * (12 * dx) ** 2))
    V = oracle_mod.mosaic_forward(N, dx, dx, u, v, A, I, xp, yp)
    xs, ys = (ms_ - c) * dx, (ns - c) * dx
    ref = 0.8 * A[ns, ms_] * np.exp(-2j * np.pi * (u * (xs - xp) + v * (ys - yp)))
    assert np.max(np.abs(V - ref)) <= 1e-12
