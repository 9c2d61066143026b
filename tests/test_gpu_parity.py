"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
identical seeded inputs.

Tolerances (stated for the split-precision tensor-core form; the direct FP64
form agrees to the float32 rounding of the ABI's outputs):
  model visibilities   max|dV| / max|V|          <= 1e-5
  gradient             ||dg||_2 / ||g||_2        <= 1e-4
  objective            |dPhi| / |Phi|            <= 1e-6
Sizes span several tiles (128 visibilities, 128/256-pixel blocks) and a ragged
tail; cube cases include an empty channel.
"""
import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

pytestmark = pytest.mark.gpu

# The FP64 form computes in FP64 but returns visibilities and gradients as
# float32 through the ABI, so it agrees to float32 rounding of its outputs.
TOL_V = {"fp64_direct": 2e-7, "fp32_direct": 1e-5, "bf16x3": 1e-5, "fp16x3": 1e-5}
TOL_G = {"fp64_direct": 2e-7, "fp32_direct": 1e-4, "bf16x3": 1e-4, "fp16x3": 1e-4}
# chi^2 and Phi at a given image.  The objective bound of 1e-6 is held at
# the solve's final image (test_gpu_solver); at arbitrary images, where the
# model can dominate the residual (R = sum w Re(conj(r) V) / sum w |r|^2 near
# 1), chi^2 moves by about 2R times a relative model bias:
#   FP16x3: up to 3N/16 = 48 truncating accumulations per output at N = 256,
#           ~1.4e-6 relative worst case, so 3e-6;
#   BF16x3: the 8+8-bit table split leaves up to 2^-17 per entry, so 1e-5.
TOL_PHI = {"fp64_direct": 1e-11, "fp32_direct": 1e-6, "bf16x3": 1e-5, "fp16x3": 3e-6}
TOL_CHI = TOL_PHI
FORMS = ["fp64_direct", "fp32_direct", "bf16x3", "fp16x3"]


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1703_02920_gb300 import memsynth
    memsynth.load()
    return memsynth


def _oracle_vis(oracle_mod, ds, img):
    P = oracle_mod.Problem.from_dataset(ds)
    return np.concatenate(oracle_mod.model_vis(P, np.asarray(img, dtype=np.float64)))


def _rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    dict(N=64, Z=1000, C=1, shared=False, seed=1),
    dict(N=128, Z=777, C=1, shared=False, seed=2),
    dict(N=256, Z=300, C=1, shared=False, seed=3),
    dict(N=64, Z=0, C=3, shared=False, seed=4, z_list=[257, 0, 130]),
    dict(N=128, Z=0, C=3, shared=True, seed=5, z_list=[200, 129, 64]),
]


def _case(c):
    return S.random_problem(c["N"], c["Z"], c["seed"], C=c["C"], shared_image=c["shared"],
                            z_list=c.get("z_list"), lam=3.0)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_forward_parity(ms, oracle_mod, form, ci):
    import torch
    ds = _case(CASES[ci])
    ctx = ms.Context(ds, precision=form)
    img = ds.truth
    V = ctx.forward(torch.from_numpy(img).cuda()).cpu().numpy().astype(np.float64)
    ref = _oracle_vis(oracle_mod, ds, img)
    got = V[:, 0] + 1j * V[:, 1]
    assert _rel_max(got, ref) <= TOL_V[form]
    ctx.close()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_adjoint_parity(ms, oracle_mod, form, ci):
    import torch
    ds = _case(CASES[ci])
    ctx = ms.Context(ds, precision=form)
    y = S.random_complex(ds.Z, 100 + ci).astype(np.complex64)
    yt = torch.from_numpy(np.stack([y.real, y.imag], 1)).cuda()
    G = ctx.adjoint(yt).cpu().numpy().astype(np.float64)
    P = oracle_mod.Problem.from_dataset(ds)
    y64 = y.astype(np.complex128)
    ref = np.zeros((P.n_images, P.N, P.N))
    for c in range(P.C):
        s = P.sl(c)
        gc = P.pb[c] * oracle_mod.adjoint(P.N, P.dx, P.dy, P.u[s], P.v[s], y64[s])
        ref[0 if P.shared_image else c] += gc
    assert _rel_l2(G, ref) <= TOL_G[form]
    ctx.close()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_objective_gradient_parity(ms, oracle_mod, form, ci):
    import torch
    ds = _case(CASES[ci])
    ctx = ms.Context(ds, precision=form)
    img = ds.truth
    phi, chi, Sv, g = ctx.objective_grad(torch.from_numpy(img).cuda())
    P = oracle_mod.Problem.from_dataset(ds)
    rphi, rchi, rS, rg = oracle_mod.objective_grad(P, img.astype(np.float64))
    assert abs(phi - rphi) <= TOL_PHI[form] * abs(rphi)
    assert abs(chi - rchi) <= TOL_PHI[form] * abs(rchi)
    assert abs(Sv - rS) <= 1e-12 * abs(rS)
    assert _rel_l2(g.cpu().numpy().astype(np.float64), rg) <= TOL_G[form]
    # projected gradient: the bound rule applied on the device
    _, _, _, gp = ctx.objective_grad(torch.from_numpy(img).cuda(), projected=True)
    rgp = oracle_mod.project_grad(img.astype(np.float64), rg, P.G)
    assert _rel_l2(gp.cpu().numpy().astype(np.float64), rgp) <= TOL_G[form]
    ctx.close()


def _degenerate(N, seed):
    """A random problem plus visibilities on the degenerate frequencies of the
    separable forward: the origin (twice), the axes (frac(v dy) = 0, the
    closed-form column sum's sin(pi b) = 0 branch), exact grid frequencies
    k / (N dx), the Nyquist edge |u dx| = 1/2, beyond it (aliased), and a whole
    turn per pixel (u dx = 1).  213 visibilities: ragged tiles."""
    import dataclasses
    base = S.random_problem(N, 201, seed, lam=3.0)
    dx, g = base.dx, 1.0 / (N * base.dx)
    su = np.array([0, 0, 0.5 / dx, -0.5 / dx, 0.7 / dx, 3 * g, -5 * g, 1.0 / dx, 0.25 / dx, 0, 7 * g, 0])
    sv = np.array([0, 0.5 / dx, 0, 3 * g, -0.7 / dx, 0, 2 * g, 1.0 / dx, -0.25 / dx, -9 * g, 0, 0])
    k = su.size
    rng = np.random.default_rng(seed)
    return dataclasses.replace(
        base, name=f"degenerate{N}", u=np.concatenate([su, base.u]), v=np.concatenate([sv, base.v]),
        vo=np.concatenate([(rng.standard_normal(k) + 1j * rng.standard_normal(k)) * 0.3, base.vo]),
        sigma=np.concatenate([np.full(k, 0.05), base.sigma]),
        offsets=np.array([0, k + base.u.size], dtype=np.int64))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("N,tiling", [(64, None), (256, None), (256, ("resident", 256, 4, 3))])
def test_degenerate_frequencies(ms, oracle_mod, form, N, tiling):
    import torch
    ds = _degenerate(N, 70 + N)
    ctx = ms.Context(ds, precision=form)
    if tiling is not None and form in ("bf16x3", "fp16x3"):
        ctx.set_tiling(*tiling)
    img = torch.from_numpy(ds.truth).cuda()
    V = ctx.forward(img).cpu().numpy().astype(np.float64)
    ref = _oracle_vis(oracle_mod, ds, ds.truth)
    assert _rel_max(V[:, 0] + 1j * V[:, 1], ref) <= TOL_V[form]
    phi, chi, Sv, g = ctx.objective_grad(img)
    P = oracle_mod.Problem.from_dataset(ds)
    rphi, rchi, rS, rg = oracle_mod.objective_grad(P, ds.truth.astype(np.float64))
    assert abs(chi - rchi) <= TOL_CHI[form] * abs(rchi)
    assert _rel_l2(g.cpu().numpy().astype(np.float64), rg) <= TOL_G[form]
    ctx.close()


@pytest.mark.parametrize("form", FORMS)
def test_single_visibility(ms, oracle_mod, form):
    """Z = 1: one tile holding one visibility, one adjoint unit."""
    import torch
    ds = S.random_problem(128, 1, 81, lam=3.0)
    ctx = ms.Context(ds, precision=form)
    img = torch.from_numpy(ds.truth).cuda()
    V = ctx.forward(img).cpu().numpy().astype(np.float64)
    assert _rel_max(V[:, 0] + 1j * V[:, 1], _oracle_vis(oracle_mod, ds, ds.truth)) <= TOL_V[form]
    phi, chi, Sv, g = ctx.objective_grad(img)
    P = oracle_mod.Problem.from_dataset(ds)
    rphi, rchi, rS, rg = oracle_mod.objective_grad(P, ds.truth.astype(np.float64))
    assert abs(chi - rchi) <= TOL_CHI[form] * abs(rchi)
    assert _rel_l2(g.cpu().numpy().astype(np.float64), rg) <= TOL_G[form]
    ctx.close()


@pytest.mark.parametrize("form", FORMS)
def test_host_buffer_entry_matches_device_entry(ms, form):
    import torch
    ds = _case(CASES[0])
    ctx = ms.Context(ds, precision=form)
    a = ctx.objective_grad(torch.from_numpy(ds.truth).cuda())
    b = ctx.objective_grad_host(ds.truth)
    assert a[:3] == b[:3]
    assert np.array_equal(a[3].cpu().numpy(), b[3])
    ctx.close()


def test_precision_switch_reuses_context(ms, oracle_mod):
    import torch
    ds = _case(CASES[1])
    ctx = ms.Context(ds, precision="fp64_direct")
    ref = _oracle_vis(oracle_mod, ds, ds.truth)
    for form in ["bf16x3", "fp32_direct", "fp16x3", "fp64_direct", "bf16x3"]:
        ctx.set_precision(form)
        V = ctx.forward(torch.from_numpy(ds.truth).cuda()).cpu().numpy().astype(np.float64)
        assert _rel_max(V[:, 0] + 1j * V[:, 1], ref) <= TOL_V[form]
    ctx.close()


def test_deterministic_repeat(ms):
    """Fixed-order reductions: two evaluations are bitwise identical."""
    import torch
    ds = _case(CASES[2])
    ctx = ms.Context(ds, precision="bf16x3")
    img = torch.from_numpy(ds.truth).cuda()
    a = ctx.objective_grad(img)
    b = ctx.objective_grad(img)
    assert a[:3] == b[:3] and torch.equal(a[3], b[3])
    ctx.close()


# every tiling the autotuner can choose (and a narrower column block) against
# the oracle, on images that take one and two column blocks / row slices
TILINGS = [("resident", 256, 6, 3), ("resident", 256, 5, 2), ("resident", 256, 4, 3),
           ("stream", 256, 4, 3), ("stream", 128, 4, 3), ("stream", 256, 3, 2), ("stream", 128, 3, 2),
           ("stream", 64, 4, 3)]


@pytest.mark.parametrize("form", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("tiling", TILINGS)
def test_tiling_variants_parity(ms, oracle_mod, form, tiling):
    import torch
    ds = S.random_problem(256, 1500, 61, lam=3.0)
    ctx = ms.Context(ds, precision=form)
    ctx.set_tiling(*tiling)
    assert ctx.tiling() == tiling
    img = ds.truth
    V = ctx.forward(torch.from_numpy(img).cuda()).cpu().numpy().astype(np.float64)
    got = V[:, 0] + 1j * V[:, 1]
    assert _rel_max(got, _oracle_vis(oracle_mod, ds, img)) <= TOL_V[form]
    phi, chi, Sv, g = ctx.objective_grad(torch.from_numpy(img).cuda())
    P = oracle_mod.Problem.from_dataset(ds)
    rphi, rchi, rS, rg = oracle_mod.objective_grad(P, img.astype(np.float64))
    assert _rel_l2(g.cpu().numpy().astype(np.float64), rg) <= TOL_G[form]
    assert abs(chi - rchi) <= TOL_CHI[form] * abs(rchi)
    ctx.close()


@pytest.mark.parametrize("N", [64, 128])
def test_resident_kernel_small_images(ms, oracle_mod, N):
    """One row slice (N <= 128): forward and chi^2 against the oracle, cube
    with an empty channel (three channels: a reload of the resident slice at
    each channel change)."""
    import torch
    ds = S.random_problem(N, 0, 64 + N, C=3, z_list=[700, 0, 333], lam=3.0)
    for form in ["bf16x3", "fp16x3"]:
        ctx = ms.Context(ds, precision=form)
        ctx.set_tiling("resident", N, 4, 3)
        V = ctx.forward(torch.from_numpy(ds.truth).cuda()).cpu().numpy().astype(np.float64)
        assert _rel_max(V[:, 0] + 1j * V[:, 1], _oracle_vis(oracle_mod, ds, ds.truth)) <= TOL_V[form]
        ctx.close()


def test_tiling_rejects_bad_shapes(ms):
    ds = S.random_problem(128, 100, 62)
    ctx = ms.Context(ds, precision="fp16x3")
    for bad in [("stream", 256, 4, 3), ("stream", 48, 4, 3), ("stream", 128, 5, 3), ("stream", 128, 4, 4),
                ("stream", 96, 4, 3), ("resident", 128, 3, 3), ("resident", 128, 9, 3)]:
        with pytest.raises(ms.MemError):
            ctx.set_tiling(*bad)
    ctx.set_tiling("stream", 64, 3, 2)
    assert ctx.tiling() == ("stream", 64, 3, 2)
    ctx.close()
    ctx = ms.Context(ds, precision="fp32_direct")
    with pytest.raises(ms.MemError):
        ctx.set_tiling("stream", 128, 4, 3)
    ctx.close()
    big = S.random_problem(512, 50, 65)
    ctx = ms.Context(big, precision="bf16x3")
    assert ctx.tiling()[0] == "stream"
    with pytest.raises(ms.MemError):
        ctx.set_tiling("resident", 512, 4, 3)
    ctx.close()


def test_autotune_choice_and_cache(ms, oracle_mod, tmp_path, monkeypatch):
    import torch
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("MEMSYNTH_TUNE_CACHE", str(cache))
    ds = S.random_problem(256, 4000, 63, lam=3.0)
    ctx = ms.Context(ds, precision="fp16x3")
    img = torch.from_numpy(ds.truth).cuda()
    choice = ctx.autotune(img, reps=2)
    kern, cols, fs, ast = choice
    assert (kern == "resident" and cols == 256 and fs in (4, 5, 6)) or \
        (kern == "stream" and cols in (128, 256) and fs in (3, 4))
    assert ast in (2, 3)
    assert ctx.tiling() == choice
    V = ctx.forward(img).cpu().numpy().astype(np.float64)
    assert _rel_max(V[:, 0] + 1j * V[:, 1], _oracle_vis(oracle_mod, ds, ds.truth)) <= TOL_V["fp16x3"]
    ctx.close()
    text = cache.read_text()
    code = {"stream": 0, "resident": 1}[kern]
    assert "N=256" in text and text.strip().endswith(f"{code} {cols} {fs} {ast}")
    # a new context for the same shape and form starts from the cached choice
    ctx = ms.Context(ds, precision="fp16x3")
    assert ctx.tiling() == choice
    ctx.close()
