"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The oracle cannot evaluate 10^6 - 10^7 visibilities x 10^5 - 10^6 pixels, so:
  * forward: full launch, a sample of visibilities recomputed one by one by
    the oracle's direct sum;
  * adjoint: full launch with a seeded input that is non-zero on a sample of
    visibilities only, compared on a pixel crop;
  * objective / gradient: internal consistency that holds at any size
    (chi^2 equals 1/2 sum w |V - V^o|^2 of the forward output; the gradient
    equals the adjoint of w r plus the entropy term).
"""
import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1703_02920_gb300 import memsynth
    memsynth.load()
    return memsynth


@pytest.fixture(scope="module")
def ds2():
    return S.make(2)


@pytest.fixture(scope="module", params=["fp16x3", "bf16x3"])
def cfg2(ms, ds2, request):
    ctx = ms.Context(ds2, precision=request.param)
    yield ds2, ctx
    ctx.close()


def _sample(Z, n, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(Z, n, replace=False))


def test_config2_forward_sampled(cfg2, oracle_mod):
    import torch
    ds, ctx = cfg2
    img = np.maximum(ds.truth, ds.G)
    V = ctx.forward(torch.from_numpy(img).cuda()).cpu().numpy().astype(np.float64)
    idx = _sample(ds.Z, 256, 1)
    ref = oracle_mod.forward(ds.N, ds.dx, ds.dy, ds.u[idx], ds.v[idx],
                             ds.pb[0].astype(np.float64) * img[0].astype(np.float64), "direct")
    got = V[idx, 0] + 1j * V[idx, 1]
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5


def test_config2_adjoint_sampled(cfg2, oracle_mod):
    import torch
    ds, ctx = cfg2
    idx = _sample(ds.Z, 20000, 2)
    t = S.random_complex(idx.size, 3)
    y = np.zeros((ds.Z, 2), dtype=np.float32)
    y[idx, 0], y[idx, 1] = t.real, t.imag
    G = ctx.adjoint(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)[0]
    n0, m0 = 100, 37
    crop = (n0, 32, m0, 32)
    ref = oracle_mod.adjoint(ds.N, ds.dx, ds.dy, ds.u[idx], ds.v[idx],
                             y[idx, 0].astype(np.float64) + 1j * y[idx, 1].astype(np.float64), crop=crop)
    ref = ref * ds.pb[0, n0:n0 + 32, m0:m0 + 32].astype(np.float64)
    got = G[n0:n0 + 32, m0:m0 + 32]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4


def test_config2_objective_gradient_consistency(cfg2):
    import torch
    ds, ctx = cfg2
    img = torch.from_numpy(np.maximum(ds.truth, ds.G)).cuda()
    phi, chi, Sv, g = ctx.objective_grad(img)
    V = ctx.forward(img).cpu().numpy().astype(np.float64)
    r = V[:, 0] + 1j * V[:, 1] - ds.vo
    w = 1.0 / ds.sigma ** 2
    chi_host = 0.5 * np.sum(w * np.abs(r) ** 2)
    assert abs(chi - chi_host) <= 1e-6 * chi_host
    I64 = img.cpu().numpy().astype(np.float64)
    S_host = -np.sum(I64 * np.log(I64 / ds.G))
    assert abs(Sv - S_host) <= 1e-9 * abs(S_host)
    assert abs(phi - (chi - ds.lam * Sv)) <= 1e-12 * abs(phi)
    wr = (w * r).astype(np.complex64)
    adj = ctx.adjoint(torch.from_numpy(np.stack([wr.real, wr.imag], 1)).cuda()).cpu().numpy().astype(np.float64)
    expect = adj + ds.lam * (1.0 + np.log(I64 / ds.G))
    got = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - expect) / np.linalg.norm(expect) <= 1e-4


def test_config3_autograd_full_size(ms, oracle_mod):
    """512 x 512 image, 10^7 visibilities, split-BF16 form: backward against
    exact central differences of a linear functional on 64 random pixels and
    against the oracle's adjoint on a 32 x 32 crop."""
    import torch
    ds = S.make(3)
    ctx = ms.Context(ds, precision="bf16x3")
    op = ms.MemOperator()
    idx = _sample(ds.Z, 20000, 4)
    t = S.random_complex(idx.size, 5)
    tt = np.zeros((ds.Z, 2), dtype=np.float32)
    tt[idx, 0], tt[idx, 1] = t.real, t.imag
    ttd = torch.from_numpy(tt).cuda()
    base = torch.from_numpy(np.maximum(ds.truth, ds.G)).cuda()
    img = base.clone().requires_grad_(True)
    (op.apply(img, ctx) * ttd).sum().backward()
    g = img.grad.detach().cpu().numpy().astype(np.float64)[0]
    n0, m0 = 240, 250
    ref = oracle_mod.adjoint(ds.N, ds.dx, ds.dy, ds.u[idx], ds.v[idx],
                             tt[idx, 0].astype(np.float64) + 1j * tt[idx, 1].astype(np.float64),
                             crop=(n0, 32, m0, 32))
    ref = ref * ds.pb[0, n0:n0 + 32, m0:m0 + 32].astype(np.float64)
    assert np.linalg.norm(g[n0:n0 + 32, m0:m0 + 32] - ref) / np.linalg.norm(ref) <= 1e-4
    rng = np.random.default_rng(6)
    h = 1.0
    tt64 = ttd.double()
    gmax = np.max(np.abs(g))
    for p in rng.choice(ds.N * ds.N, 64, replace=False):
        e = torch.zeros_like(base).view(-1)
        e[p] = h
        e = e.view_as(base)
        with torch.no_grad():
            lp = (ctx.forward(base + e).double() * tt64).sum().item()
            lm = (ctx.forward(base - e).double() * tt64).sum().item()
        assert abs((lp - lm) / (2 * h) - g.ravel()[p]) <= 1e-4 * gmax
    ctx.close()


@pytest.fixture(scope="module")
def cfg4(ms):
    ds = S.make(4)
    ctx = ms.Context(ds, precision="fp16x3")
    yield ds, ctx
    ctx.close()


def test_config4_cube_forward_sampled(cfg4, oracle_mod):
    """64-channel cube, uneven per-channel counts, one batched launch chain:
    sampled visibilities of several channels against the oracle's direct sum
    with that channel's beam."""
    import torch
    ds, ctx = cfg4
    img = np.maximum(ds.truth, ds.G)
    V = ctx.forward(torch.from_numpy(img).cuda()).cpu().numpy().astype(np.float64)
    for c in [0, 17, 40, ds.C - 1]:
        a, b = int(ds.offsets[c]), int(ds.offsets[c + 1])
        idx = a + _sample(b - a, 96, 10 + c)
        ref = oracle_mod.forward(ds.N, ds.dx, ds.dy, ds.u[idx], ds.v[idx],
                                 ds.pb[c].astype(np.float64) * img[c].astype(np.float64), "direct")
        got = V[idx, 0] + 1j * V[idx, 1]
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5, c


def test_config4_cube_batched_equals_single_channel(cfg4, ms):
    """The batched forward of a channel equals that channel run alone, bit for
    bit (the same tiles, column means and operand scale); chi^2 per image
    matches the host sum over the forward's output."""
    import torch
    ds, ctx = cfg4
    img = np.maximum(ds.truth, ds.G)
    V = ctx.forward(torch.from_numpy(img).cuda()).cpu().numpy()
    for c in [5, 40]:
        one = ds.subset([c])
        cc = ms.Context(one, precision="fp16x3")
        cc.set_tiling(*ctx.tiling())
        V1 = cc.forward(torch.from_numpy(np.ascontiguousarray(img[c:c + 1])).cuda()).cpu().numpy()
        a, b = int(ds.offsets[c]), int(ds.offsets[c + 1])
        assert np.array_equal(V1, V[a:b]), c
        cc.close()
    phi, chi, Sv, g = ctx.objective_grad(torch.from_numpy(img).cuda())
    r = V[:, 0].astype(np.float64) + 1j * V[:, 1].astype(np.float64) - ds.vo
    chi_host = 0.5 * np.sum(np.abs(r) ** 2 / ds.sigma ** 2)
    assert abs(chi - chi_host) <= 1e-6 * chi_host


def test_config5_forward_and_adjoint_sampled(ms, oracle_mod):
    """1024 x 1024 image, 2.0e7 visibilities (four 256-column blocks per tile,
    16 adjoint output blocks), FP16x3 in the default launch configuration:
    sampled visibilities against the oracle's direct sum, and the adjoint of
    an input that is non-zero on 20,000 visibilities on a 32 x 32 crop."""
    import torch
    ds = S.make(5)
    ctx = ms.Context(ds, precision="fp16x3")
    img = np.maximum(ds.truth, ds.G)
    V = ctx.forward(torch.from_numpy(img).cuda()).cpu().numpy().astype(np.float64)
    idx = _sample(ds.Z, 128, 51)
    ref = oracle_mod.forward(ds.N, ds.dx, ds.dy, ds.u[idx], ds.v[idx],
                             ds.pb[0].astype(np.float64) * img[0].astype(np.float64), "direct")
    got = V[idx, 0] + 1j * V[idx, 1]
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5
    del V
    idx = _sample(ds.Z, 20000, 52)
    t = S.random_complex(idx.size, 53)
    y = np.zeros((ds.Z, 2), dtype=np.float32)
    y[idx, 0], y[idx, 1] = t.real, t.imag
    G = ctx.adjoint(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)[0]
    for n0, m0 in [(500, 470), (3, 990)]:
        ref = oracle_mod.adjoint(ds.N, ds.dx, ds.dy, ds.u[idx], ds.v[idx],
                                 y[idx, 0].astype(np.float64) + 1j * y[idx, 1].astype(np.float64),
                                 crop=(n0, 32, m0, 32))
        ref = ref * ds.pb[0, n0:n0 + 32, m0:m0 + 32].astype(np.float64)
        got = G[n0:n0 + 32, m0:m0 + 32]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4, (n0, m0)
    ctx.close()


@pytest.mark.parametrize("config, crop", [(2, 32), (5, 16)])
def test_adjoint_full_data(ms, oracle_mod, config, crop):
    """Every visibility non-zero (the weighted residual at the truth image),
    so each CTA accumulates its whole share of the data set: the gradient
    term against the oracle's adjoint over all Z visibilities on two pixel
    crops.  This is where accumulation bias would show (it grows with the
    visibilities a CTA sums)."""
    import torch
    ds = S.make(config)
    ctx = ms.Context(ds, precision="fp16x3")
    img = np.maximum(ds.truth, ds.G)
    V = ctx.forward(torch.from_numpy(img).cuda()).cpu().numpy().astype(np.float64)
    y = ((V[:, 0] + 1j * V[:, 1] - ds.vo) / ds.sigma ** 2).astype(np.complex64)
    del V
    G = ctx.adjoint(torch.from_numpy(np.stack([y.real, y.imag], 1)).cuda()).cpu().numpy().astype(np.float64)[0]
    ctx.close()
    for n0, m0 in [(ds.N // 2 - crop // 2, ds.N // 2 - crop // 2), (5, ds.N - crop - 9)]:
        ref = oracle_mod.adjoint(ds.N, ds.dx, ds.dy, ds.u, ds.v, y.astype(np.complex128),
                                 crop=(n0, crop, m0, crop))
        ref = ref * ds.pb[0, n0:n0 + crop, m0:m0 + crop].astype(np.float64)
        got = G[n0:n0 + crop, m0:m0 + crop]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4, (n0, m0)
