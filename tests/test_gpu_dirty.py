"""Natural-weights dirty image, PSF and residual map (Appendix A) on the GPU,
per channel and form, against the oracle; the PSF peaks at 1 on the phase
centre."""
import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = {"fp64_direct": 1e-6, "fp32_direct": 1e-5, "bf16x3": 1e-4, "fp16x3": 1e-4}


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1703_02920_gb300 import memsynth
    memsynth.load()
    return memsynth


@pytest.mark.parametrize("form", list(TOL))
def test_dirty_image_and_psf_match_oracle(ms, oracle_mod, form):
    ds = S.random_problem(128, 0, 95, C=3, z_list=[900, 0, 512])
    P = oracle_mod.Problem.from_dataset(ds)
    ctx = ms.Context(ds, precision=form)
    for psf in (False, True):
        got = ctx.dirty_image(psf).cpu().numpy().astype(np.float64)
        ref = oracle_mod.dirty_image(P, psf)
        for c in (0, 2):
            assert np.linalg.norm(got[c] - ref[c]) / np.linalg.norm(ref[c]) <= TOL[form], (psf, c)
        assert np.all(got[1] == 0)  # the empty channel
        if psf:
            assert got[0][64, 64] == pytest.approx(1.0, abs=1e-5)
    ctx.close()


@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("form", list(TOL))
def test_residual_map_matches_oracle(ms, oracle_mod, form, shared):
    """Dirty image of V° - V(I): the oracle's dirty image of its own residuals
    (per channel; one model image for all channels in the shared-image mode);
    a model equal to the data leaves an empty map."""
    import dataclasses
    ds = S.random_problem(128, 0, 96, C=3, z_list=[900, 0, 512], shared_image=shared)
    P = oracle_mod.Problem.from_dataset(ds)
    img = ds.truth.astype(np.float64)
    V = np.concatenate(oracle_mod.model_vis(P, img))
    ctx = ms.Context(ds, precision=form)
    got = ctx.residual_image(ds.truth).cpu().numpy().astype(np.float64)
    ctx.close()
    ref = oracle_mod.dirty_image(P, vis=P.vo - V)
    for c in (0, 2):
        assert np.linalg.norm(got[c] - ref[c]) / np.linalg.norm(ref[c]) <= TOL[form], c
    assert np.all(got[1] == 0)  # the empty channel
    # data = model: only the forward's rounding remains
    exact = dataclasses.replace(ds, vo=V)
    ctx = ms.Context(exact, precision=form)
    zero = ctx.residual_image(ds.truth).cpu().numpy().astype(np.float64)
    ctx.close()
    dirty = oracle_mod.dirty_image(oracle_mod.Problem.from_dataset(exact))
    assert np.max(np.abs(zero)) <= 10 * TOL[form] * np.max(np.abs(dirty))


def test_config1_beam_from_gpu_psf(ms, oracle_mod):
    """The beam fitted to the GPU's PSF equals the oracle's fit of the oracle's PSF."""
    ds = S.make(1)
    ctx = ms.Context(ds, precision="fp16x3")
    psf = ctx.dirty_image(True).cpu().numpy()[0]
    ctx.close()
    got = ms.mem_beam_fit(psf, ds.dx, ds.dy)
    ref = oracle_mod.beam_fit(oracle_mod.dirty_image(oracle_mod.Problem.from_dataset(ds), True)[0], ds.dx, ds.dy)
    assert got[0] == pytest.approx(ref[0], rel=1e-3)
    assert got[1] == pytest.approx(ref[1], rel=1e-3)
    assert got[3] == pytest.approx(ref[3], rel=2e-3)
