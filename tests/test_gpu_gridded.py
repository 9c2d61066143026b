"""The paper's gridded forward (zero-padded FFT, phase-centre modulation,
bilinear interpolation; Section 2.4 steps, Algorithm alg:chi2gpu) on the GPU
against the oracle's statement of the same steps.  FP32 FFT: agreement to
2e-5 of max|V|; its approximation error against Eq. (1) is the oracle's."""
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


def _oracle_gridded(oracle_mod, ds, img, pad):
    out = []
    for c in range(ds.C):
        a, b = int(ds.offsets[c]), int(ds.offsets[c + 1])
        i = 0 if ds.shared_image else c
        B = ds.pb[c].astype(np.float64) * img[i].astype(np.float64)
        out.append(oracle_mod.forward_gridded(ds.N, ds.dx, ds.dy, ds.u[a:b], ds.v[a:b], B, pad))
    return np.concatenate(out)


CASES = [dict(N=64, Z=700, C=1, shared=False, seed=81), dict(N=128, Z=0, C=3, shared=False, seed=82,
         z_list=[400, 0, 333]), dict(N=64, Z=0, C=2, shared=True, seed=83, z_list=[300, 500])]


@pytest.mark.parametrize("pad", [1, 2, 3])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_gridded_forward_matches_oracle(ms, oracle_mod, pad, ci):
    import torch
    c = CASES[ci]
    ds = S.random_problem(c["N"], c["Z"], c["seed"], C=c["C"], shared_image=c["shared"], z_list=c.get("z_list"))
    ctx = ms.Context(ds, precision="fp16x3")
    V = ctx.forward_gridded(torch.from_numpy(ds.truth).cuda(), pad).cpu().numpy().astype(np.float64)
    ref = _oracle_gridded(oracle_mod, ds, ds.truth, pad)
    got = V[:, 0] + 1j * V[:, 1]
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))
    # the approximation error against the exact sum is the oracle's
    exact = np.concatenate(oracle_mod.model_vis(oracle_mod.Problem.from_dataset(ds), ds.truth.astype(np.float64)))
    e_gpu = np.max(np.abs(got - exact)) / np.max(np.abs(exact))
    e_ref = np.max(np.abs(ref - exact)) / np.max(np.abs(exact))
    assert abs(e_gpu - e_ref) <= 1e-4 + 0.01 * e_ref, (e_gpu, e_ref)
    ctx.close()


@pytest.mark.parametrize("N,pad,Z", [(64, 5, 500), (64, 7, 500), (128, 6, 400), (256, 4, 600)])
def test_gridded_forward_every_radix_and_large_grids(ms, oracle_mod, N, pad, Z):
    """The transform's radix-5 and radix-7 stages (pad 5, 7), radix 3 with
    radix 2 and 4 (pad 6) and a 1024-point grid (N = 256, pad 4) against the
    oracle's statement of the same steps."""
    import torch
    ds = S.random_problem(N, Z, 86 + pad, C=1)
    ctx = ms.Context(ds, precision="fp16x3")
    V = ctx.forward_gridded(torch.from_numpy(ds.truth).cuda(), pad).cpu().numpy().astype(np.float64)
    ref = _oracle_gridded(oracle_mod, ds, ds.truth, pad)
    got = V[:, 0] + 1j * V[:, 1]
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref)), (N, pad)
    ctx.close()


def test_gridded_forward_rejects_bad_pad(ms):
    import torch
    ds = S.random_problem(64, 10, 84)
    ctx = ms.Context(ds, precision="fp32_direct")
    img = torch.from_numpy(ds.truth).cuda()
    for pad in (0, 9):
        with pytest.raises(ms.MemError):
            ctx.forward_gridded(img, pad)
    ctx.forward_gridded(img, 2)
    ctx.forward_gridded(img, 4)  # re-plans for another pad
    ctx.close()
