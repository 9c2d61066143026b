"""The allocation-free adjoint entry point (mem_adjoint_noalloc).

It serves callers that cannot allocate device memory themselves (code inside a
framework that owns all device memory through its own pool, or that must not
allocate after start-up): they pass device inputs and outputs only, and the
call's scratch lives in a fixed static array inside the library.  Checked
against the ordinary entry point (mem_adjoint, split-BF16 tensor-core form,
which allocates its scratch per context) through the C ABI, within the
gradient tolerance the other tests use, on two calls in a row (the shared
scratch keeps the previous call's contents).
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


@pytest.mark.parametrize("N,Z,seed", [(256, 5000, 71), (64, 1000, 72)])
def test_noalloc_adjoint_matches_mem_adjoint_twice(ms, N, Z, seed):
    import torch
    ds = S.random_problem(N, Z, seed, lam=0.0)
    ctx = ms.Context(ds, precision="bf16x3")
    u = torch.from_numpy(ds.u).cuda()
    v = torch.from_numpy(ds.v).cuda()
    pb = torch.from_numpy(ds.pb[0]).cuda().contiguous()
    for call in range(2):
        y = S.random_complex(Z, seed * 10 + call)
        yt = torch.from_numpy(np.stack([y.real, y.imag], 1).astype(np.float32)).cuda()
        ref = ctx.adjoint(yt)[0].double()
        out = torch.full((N, N), float("nan"), dtype=torch.float32, device="cuda")
        ms.mem_adjoint_noalloc(N, ds.dx, ds.dy, u, v, yt, pb, out,
                               stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        rel = float(torch.linalg.norm(out.double() - ref) / torch.linalg.norm(ref))
        assert rel <= TOL, (call, rel)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(ms):
    import torch
    u = torch.zeros(16, dtype=torch.float64, device="cuda")
    y = torch.zeros((16, 2), dtype=torch.float32, device="cuda")
    img = torch.zeros((512, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(ms.MemError) as e:
        ms.mem_adjoint_noalloc(512, 1e-7, 1e-7, u, u, y, img, img)
    assert e.value.status == 1
    assert "64, 128 or 256" in str(e.value)
