"""The allocation-free adjoint entry point (mem_adjoint_noalloc).

It serves callers that cannot allocate device memory themselves (code inside a
framework that owns all device memory through its own pool, or that must not
allocate after start-up): they pass device inputs and outputs only, and the
call's scratch lives in a fixed static array inside the library.  Checked
through the C ABI against the ordinary entry point (mem_adjoint, split-BF16
tensor-core form, which allocates its scratch per context) and against the
FP64 oracle's adjoint times the beam (Eq. chi2gradient), within the gradient
tolerance the other tests use, on calls in a row: the shared scratch keeps
the previous call's contents, so a call with fewer CTAs than the one before
must ignore the stale partials, and a call without visibilities must write
zeros.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-4  # relative L2, as for every adjoint / gradient comparison


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1703_02920_gb300 import memsynth
    memsynth.load()
    return memsynth


def _noalloc(ms, ds, y, n_vis=None):
    import torch
    z = ds.Z if n_vis is None else n_vis
    u = torch.from_numpy(np.ascontiguousarray(ds.u[:z])).cuda()
    v = torch.from_numpy(np.ascontiguousarray(ds.v[:z])).cuda()
    pb = torch.from_numpy(ds.pb[0]).cuda().contiguous()
    yt = torch.from_numpy(np.stack([y.real, y.imag], 1).astype(np.float32)).cuda().reshape(z, 2)
    out = torch.full((ds.N, ds.N), float("nan"), dtype=torch.float32, device="cuda")
    ms.mem_adjoint_noalloc(ds.N, ds.dx, ds.dy, u if z else None, v if z else None, yt if z else None, pb,
                           out, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), yt


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,Z,seed", [(256, 5000, 71), (128, 3000, 73), (64, 1000, 72)])
def test_noalloc_adjoint_matches_mem_adjoint_and_oracle_twice(ms, oracle_mod, N, Z, seed):
    ds = S.random_problem(N, Z, seed, lam=0.0)
    ctx = ms.Context(ds, precision="bf16x3")
    for call in range(2):
        y = S.random_complex(Z, seed * 10 + call)
        out, yt = _noalloc(ms, ds, y)
        ref = ctx.adjoint(yt)[0].double().cpu().numpy()
        assert _rel(out, ref) <= TOL, (call, _rel(out, ref))
        exact = ds.pb[0] * oracle_mod.adjoint(N, ds.dx, ds.dy, ds.u, ds.v, y.astype(np.complex64))
        assert _rel(out, exact) <= TOL, (call, _rel(out, exact))
    ctx.close()


def test_noalloc_fewer_ctas_after_more_then_no_visibilities(ms, oracle_mod):
    """A call over many visibilities fills every CTA's partial block; the next,
    over 100 visibilities (7 stages of 16, so 7 CTAs), must use only its own
    units; then a call with no visibilities returns the zero image."""
    ds = S.random_problem(256, 40000, 74, lam=0.0)
    y = S.random_complex(ds.Z, 741)
    out, yt = _noalloc(ms, ds, y)
    ctx = ms.Context(ds, precision="bf16x3")
    ref = ctx.adjoint(yt)[0].double().cpu().numpy()
    ctx.close()
    assert _rel(out, ref) <= TOL
    small = S.random_problem(256, 100, 75, lam=0.0)
    ys = S.random_complex(small.Z, 751)
    out_s, yts = _noalloc(ms, small, ys)
    ctx = ms.Context(small, precision="bf16x3")
    ref_s = ctx.adjoint(yts)[0].double().cpu().numpy()
    ctx.close()
    assert _rel(out_s, ref_s) <= TOL
    exact = small.pb[0] * oracle_mod.adjoint(256, small.dx, small.dy, small.u, small.v, ys.astype(np.complex64))
    assert _rel(out_s, exact) <= TOL
    out0, _ = _noalloc(ms, small, np.zeros(0, dtype=complex), n_vis=0)
    assert np.array_equal(out0, np.zeros((256, 256)))


def test_noalloc_rejects_sizes_beyond_its_scratch(ms):
    import torch
    u = torch.zeros(16, dtype=torch.float64, device="cuda")
    y = torch.zeros((16, 2), dtype=torch.float32, device="cuda")
    img = torch.zeros((512, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(ms.MemError) as e:
        ms.mem_adjoint_noalloc(512, 1e-7, 1e-7, u, u, y, img, img)
    assert e.value.status == 1
    assert "64, 128 or 256" in str(e.value)
