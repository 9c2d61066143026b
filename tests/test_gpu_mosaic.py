"""Mosaic (Section 2.4: one attenuation image per pointing): three pointings
with their own phase centres and beams, data made by the oracle's statement
of a pointing; after mem_phase_rotate the pointings are the channels of a
shared-image context, whose chi^2 must be the mosaic's by definition."""
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


def _mosaic(oracle_mod, N=64, seed=97):
    rng = np.random.default_rng(seed)
    dx = 0.1 * S.ARCSEC
    c = N // 2
    n, m = np.mgrid[0:N, 0:N]
    sky = (1e-4 + 0.02 * rng.random((N, N)) ** 6).astype(np.float32)
    us, vs, vos, sgs, pbs, offs, raw = [], [], [], [], [], [0], []
    for k, (px, py) in enumerate([(-9, 4), (8, 6), (1, -10)]):
        xp, yp = px * dx, py * dx
        A = np.exp(-(((m - c) * dx - xp) ** 2 + ((n - c) * dx - yp) ** 2) / (2 * (14 * dx) ** 2)).astype(np.float32)
        z = 400 + 100 * k
        r = 0.45 / dx * np.sqrt(rng.random(z))
        t = 2 * np.pi * rng.random(z)
        u, v = r * np.cos(t), r * np.sin(t)
        sig = np.full(z, 0.01)
        V = oracle_mod.mosaic_forward(N, dx, dx, u, v, A, sky, xp, yp)
        V = V + sig * (rng.standard_normal(z) + 1j * rng.standard_normal(z))
        raw.append((u, v, V, xp, yp))
        us.append(u); vs.append(v); sgs.append(sig); pbs.append(A); offs.append(offs[-1] + z)
    return dx, sky, raw, us, vs, sgs, pbs, offs


def test_rotated_pointings_give_the_mosaic_objective(ms, oracle_mod):
    import torch
    N = 64
    dx, sky, raw, us, vs, sgs, pbs, offs = _mosaic(oracle_mod, N)
    vos = [ms.mem_phase_rotate(u, v, V, xp, yp) for (u, v, V, xp, yp) in raw]
    ds = S.Dataset(name="mosaic3", N=N, dx=dx, dy=dx, u=np.concatenate(us), v=np.concatenate(vs),
                   vo=np.concatenate(vos), sigma=np.concatenate(sgs), pb=np.stack(pbs),
                   offsets=np.array(offs, dtype=np.int64), truth=sky[None], G=1e-4, lam=5.0, n_iter=8,
                   shared_image=True)
    img = np.maximum(sky, np.float32(1e-4))[None]
    # the mosaic's chi^2 straight from its definition (phase per pointing)
    chi_def = 0.0
    for (u, v, V, xp, yp), A, sig in zip(raw, pbs, sgs):
        Vm = oracle_mod.mosaic_forward(N, dx, dx, u, v, A, img[0], xp, yp)
        chi_def += 0.5 * np.sum(np.abs(Vm - V) ** 2 / sig ** 2)
    for form, tol in [("fp64_direct", 1e-10), ("fp16x3", 3e-6)]:
        ctx = ms.Context(ds, precision=form)
        phi, chi, Sv, g = ctx.objective_grad(torch.from_numpy(img).cuda())
        assert abs(chi - chi_def) <= tol * chi_def, (form, chi, chi_def)
        ctx.close()
    # and the solve over the mosaic matches the oracle's on the same problem
    P = oracle_mod.Problem.from_dataset(ds)
    I0 = np.full((1, N, N), np.float32(ds.G))
    ref, hist = oracle_mod.solve(P, I0.astype(np.float64), ds.n_iter)
    ctx = ms.Context(ds, precision="fp64_direct")
    out, rep, _ = ctx.solve(torch.from_numpy(I0).cuda(), ds.n_iter)
    ctx.close()
    out = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-6
