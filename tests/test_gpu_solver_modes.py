"""Split-form solves in the cube and shared-image modes against the FP64 oracle.

Cube: independent per-channel objectives (Eq. minproblem per image), batched
in every launch; one channel has no visibilities.  Shared image: one image for
all channels, chi^2 summed over them (Eq. chi2-multi).  A 64 x 64 problem with
three channels, 10 projected-CG iterations from I = G in the FP16x3 and
BF16x3 forms:
* every image within 1e-3 (relative L2) of the oracle's solve, every pixel
  >= G, each image's Phi non-increasing;
* the objective the form reports at its final image(s) within the form's
  evaluation bound of the oracle's objective at the same image(s): 1e-6 for
  FP16x3, 3e-6 for BF16x3 (its 8 + 8-bit split carries errors of order 1e-6
  where the model visibilities dominate the residuals).
"""
import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

pytestmark = pytest.mark.gpu

N_ITER = 10
TOL_PHI = {"fp16x3": 1e-6, "bf16x3": 3e-6}


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1703_02920_gb300 import memsynth
    memsynth.load()
    return memsynth


def _problem(mode):
    if mode == "cube":
        return S.random_problem(64, 0, seed=41, C=3, z_list=[600, 0, 400], lam=20.0, G=1e-3)
    return S.random_problem(64, 0, seed=42, C=3, z_list=[500, 300, 400], lam=20.0, G=1e-3, shared_image=True)


@pytest.fixture(scope="module")
def refs(oracle_mod):
    out = {}
    for mode in ("cube", "shared"):
        ds = _problem(mode)
        P = oracle_mod.Problem.from_dataset(ds)
        # the same float32 start on both sides (float32(1e-3) lies just above G)
        I0 = np.full((P.n_images, ds.N, ds.N), P.G).astype(np.float32)
        ref, _ = oracle_mod.solve(P, I0.astype(np.float64), N_ITER)
        out[mode] = (ds, P, I0, ref)
    return out


@pytest.mark.parametrize("mode", ["cube", "shared"])
@pytest.mark.parametrize("form", ["fp16x3", "bf16x3"])
def test_split_form_solve_matches_oracle(ms, oracle_mod, refs, mode, form):
    import torch
    ds, P, I0, ref = refs[mode]
    ctx = ms.Context(ds, precision=form)
    img, rep, hist = ctx.solve(torch.from_numpy(I0).cuda(), N_ITER)
    ctx.close()
    img = img.cpu().numpy().astype(np.float64)
    assert rep.status == 0
    assert img.shape == ref.shape == (P.n_images, ds.N, ds.N)
    assert img.min() >= np.float32(P.G) * (1 - 1e-7)
    for i in range(P.n_images):
        # (iterations after an early stop repeat the last values)
        phis = hist[i, : N_ITER + 1, 0]
        assert np.all(np.diff(phis) <= 1e-12 * np.abs(phis[:-1])), (i, phis)
        rel = np.linalg.norm(img[i] - ref[i]) / np.linalg.norm(ref[i])
        assert rel <= 1e-3, (mode, form, i, rel)
    own = oracle_mod.objective(P, img)[0]
    assert abs(rep.phi - own) <= TOL_PHI[form] * abs(own), (mode, form, rep.phi, own)
