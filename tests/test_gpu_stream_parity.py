"""The streaming tensor-core forward (the default for N >= 256) against the
FP64 oracle at the image sizes the product runs.

* A 256 x 256 MEM solve (Eq. minproblem) on the config-2 array geometry with
  16 Earth-rotation dumps (19,600 visibilities), 40 CG iterations from
  I = G, in both split forms: final image within 1e-3 (relative L2) of the
  oracle's solve, Phi non-increasing, and the objective at the solve's final
  image within the form's bound of the oracle's value at that same image.
* chi^2, Phi, visibilities and gradient at N = 512 and N = 1024 (about 5e3
  visibilities each, config-3 and config-5 geometry) at the sky image and at
  a random positive image.

Bounds.  FP16x3 (the default form) is held to the task's 1e-6 on the
objective at the final image.  BF16x3 splits each operand into 8 + 8
significant bits, so every product carries up to about 3 * 2^-18 of
representation and dropped-term error (against 2^-22 for FP16x3); at a
solve's final image, where the model visibilities dominate the residuals,
its objective error is of order 1e-6 by arithmetic alone, so it is held to
3e-6 there.  At arbitrary images chi^2 is held to the per-form bounds derived
from the arithmetic (3e-6 FP16x3, 1e-5 BF16x3): every accumulation of the
streaming kernel covers at most 256 image rows (48 truncating MMA additions),
whatever N is, so the N = 256 derivation holds at N = 512 and 1024.
"""
import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

pytestmark = pytest.mark.gpu

FORMS = ["fp16x3", "bf16x3"]
TOL_PHI_FINAL = {"fp16x3": 1e-6, "bf16x3": 3e-6}
# the 40-iteration trajectory is far from converged and amplifies evaluation
# errors (a 1e-7 max|V| perturbation of the oracle's own forward moves the
# config-1 final objective by 6e-5); BF16x3's errors are about 10x FP16x3's.
# One-sided: the form's objective must have fallen at least about as far.
TRAJ_PHI = {"fp16x3": 2e-5, "bf16x3": 1e-4}
TOL_CHI = {"fp16x3": 3e-6, "bf16x3": 1e-5}
TOL_V = 1e-5
TOL_G = 1e-4
N_ITER = 40


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1703_02920_gb300 import memsynth
    memsynth.load()
    return memsynth


def _start(ds):
    # the same start on both sides: float32(G), clipped at G as the library does
    return np.full((1, ds.N, ds.N), max(float(np.float32(ds.G)), ds.G))


@pytest.fixture(scope="module")
def solve256(oracle_mod):
    ds = S.make_continuum(2, dumps=16)
    P = oracle_mod.Problem.from_dataset(ds)
    img, hist = oracle_mod.solve(P, _start(ds), N_ITER)
    return ds, P, img, hist[0]


@pytest.mark.parametrize("form", FORMS)
def test_stream_solve_256_matches_oracle(ms, solve256, oracle_mod, form):
    import torch
    ds, P, ref_img, ref_hist = solve256
    assert ds.N == 256 and ds.Z == 19600
    ctx = ms.Context(ds, precision=form)
    assert ctx.tiling()[0] == "stream"
    I0 = torch.from_numpy(_start(ds).astype(np.float32)).cuda()
    img, rep, hist = ctx.solve(I0, N_ITER)
    img = img.cpu().numpy().astype(np.float64)
    ctx.close()
    assert rep.iterations == N_ITER
    phis = hist[0, : rep.iterations + 1, 0]
    assert np.all(np.diff(phis) <= 1e-12 * np.abs(phis[:-1]))
    assert img.min() >= np.float32(ds.G) * (1 - 1e-7)
    rel = np.linalg.norm(img - ref_img) / np.linalg.norm(ref_img)
    assert rel <= 1e-3, rel
    own_phi, own_chi, _ = oracle_mod.objective(P, img)
    assert abs(rep.phi - own_phi) <= TOL_PHI_FINAL[form] * abs(own_phi), (rep.phi, own_phi)
    # and along the way the objective fell at least as far as the oracle's did
    # (an unconverged trajectory may well end lower: its own objective at its
    # own image is checked above)
    ref_phi = ref_hist[-1]["phi"]
    assert rep.phi - ref_phi <= TRAJ_PHI[form] * abs(ref_phi), (rep.phi, ref_phi)


def _cases():
    out = []
    for cfg, dumps in ((3, 4), (5, 3)):
        ds = S.make_continuum(cfg, dumps=dumps)
        rng = np.random.default_rng(90 + cfg)
        rand = (ds.G + 0.02 * rng.random((1, ds.N, ds.N)) ** 4 * (ds.G / 1e-4)).astype(np.float32)
        out.append((ds, "sky", np.maximum(ds.truth, np.float32(ds.G)).astype(np.float32)))
        out.append((ds, "random", rand))
    return out


@pytest.fixture(scope="module")
def large_cases(oracle_mod):
    res = []
    for ds, label, img in _cases():
        P = oracle_mod.Problem.from_dataset(ds)
        I = img.astype(np.float64)
        phi, chi, _, g = oracle_mod.objective_grad(P, I)
        V = oracle_mod.model_vis(P, I)[0]
        res.append((ds, label, img, phi, chi, g, V))
    return res


@pytest.mark.parametrize("form", FORMS)
def test_stream_objective_at_512_and_1024(ms, large_cases, form):
    import torch
    for ds, label, img, rphi, rchi, rg, rV in large_cases:
        assert ds.N in (512, 1024) and 4000 <= ds.Z <= 7000
        ctx = ms.Context(ds, precision=form)
        assert ctx.tiling()[0] == "stream"
        t = torch.from_numpy(img).cuda()
        phi, chi, _, g = ctx.objective_grad(t)
        V = ctx.forward(t).cpu().numpy().astype(np.float64)
        g = g.cpu().numpy().astype(np.float64)
        ctx.close()
        V = V[:, 0] + 1j * V[:, 1]
        what = (ds.N, label, form)
        assert abs(chi - rchi) <= TOL_CHI[form] * abs(rchi), (what, chi, rchi)
        assert abs(phi - rphi) <= TOL_CHI[form] * abs(rphi), (what, phi, rphi)
        assert np.max(np.abs(V - rV)) <= TOL_V * np.max(np.abs(rV)), what
        assert np.linalg.norm(g - rg) / np.linalg.norm(rg) <= TOL_G, what
