"""Failure detection without a GPU fault: every device-side wait in the
tensor-core kernels is bounded by mem_config.spin_limit.  With a limit of one
poll the waits give up at once; the kernels unwind (releasing tensor memory,
letting in-flight copies and MMAs land) and the call returns MEM_ETIMEOUT.
The device stays usable: a fresh context right after computes correctly."""
import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_device_stays_usable(oracle_mod):
    import torch
    from paper_1703_02920_gb300 import memsynth as ms
    ds = S.random_problem(128, 2000, 81, lam=1.0)
    img = torch.from_numpy(ds.truth).cuda()
    bad = ms.Context(ds, precision="bf16x3", spin_limit=1)
    with pytest.raises(ms.MemError) as e:
        bad.objective_grad(img)
    assert e.value.status == 4
    bad.close()
    good = ms.Context(ds, precision="bf16x3")
    phi, chi, S_, g = good.objective_grad(img)
    P = oracle_mod.Problem.from_dataset(ds)
    rphi = oracle_mod.objective(P, ds.truth.astype(np.float64))[0]
    assert abs(phi - rphi) <= 1e-5 * abs(rphi)
    good.close()


@pytest.mark.parametrize("form", ["fp16x3", "bf16x3"])
def test_streaming_kernels_time_out_cleanly(oracle_mod, form):
    """The same at N = 256, where the streaming forward (its copy warp's
    event loop drains the image chunks still in flight) and the split-K
    adjoint run; then a fresh context on the same device computes
    correctly."""
    import torch
    from paper_1703_02920_gb300 import memsynth as ms
    ds = S.random_problem(256, 3000, 85, lam=1.0)
    img = torch.from_numpy(ds.truth).cuda()
    bad = ms.Context(ds, precision=form, spin_limit=1)
    assert bad.tiling()[0] == "stream"
    with pytest.raises(ms.MemError) as e:
        bad.objective_grad(img)
    assert e.value.status == 4
    bad.close()
    good = ms.Context(ds, precision=form)
    phi, chi, S_, g = good.objective_grad(img)
    P = oracle_mod.Problem.from_dataset(ds)
    rphi = oracle_mod.objective(P, ds.truth.astype(np.float64))[0]
    assert abs(phi - rphi) <= 1e-5 * abs(rphi)
    good.close()


def test_allocation_cap_is_enforced_on_the_host(monkeypatch):
    """MEMSYNTH_MAX_BYTES caps the context's device allocations (host-side
    failure injection): creation fails cleanly with MEM_ENOMEM."""
    from paper_1703_02920_gb300 import memsynth as ms
    monkeypatch.setenv("MEMSYNTH_MAX_BYTES", "4096")
    ds = S.random_problem(64, 500, 82)
    with pytest.raises(ms.MemError) as e:
        ms.Context(ds, precision="bf16x3")
    assert e.value.status == 2
