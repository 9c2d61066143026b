"""The MEM solve run to convergence on config 1, in every form, against the
minimiser of Eq. minproblem.

For lambda > 0, Phi = chi^2 - lambda S is strictly convex on I >= G, so the
minimiser is unique and the objective bound applies as written: at
convergence the solve's final objective is within 1e-6 of the minimum and its
image within 1e-3 (relative L2) of the minimiser.  The minimiser and its
objective come from tests/golden/config1_minimiser.txt, written by
make_config1_minimiser.py from the FP64 oracle's objective and gradient with
scipy's L-BFGS-B (two starts, agreeing to 8e-7).

The paper's projected Polak-Ribiere CG converges slowly on this problem
(Phi is within 1e-6 of the minimum after about 2000 iterations, the image
within 1e-3 after about 3000), so the split and FP32 forms run 4000
iterations from I = G (or until their line search finds no decrease); the
FP64 form, about 100x slower, continues for 100 iterations from the FP16x3
form's final image.

BF16x3 splits each operand into 8 + 8 significant bits (up to 3 * 2^-18 per
product), so its evaluations carry errors of order 1e-6: its line search
stops finding decrease within its 3e-6 evaluation bound of the minimum (it
ends at about 2.8e-6), and where along the nearly flat directions of Phi it
stops sets its image, 6e-3 to 1.4e-2 from the FP64 minimiser in the runs
measured.  BF16x3 therefore does not meet the 1e-3 image bound at
convergence (FP16x3, the default form, does); its objective is held to its
3e-6 evaluation bound and its image only to a sanity bound of 5e-2.
"""
import os

import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config1_minimiser.txt")
ITERS = {"fp16x3": 4000, "bf16x3": 8000, "fp32_direct": 4000}
TOL_IMG = {"fp16x3": 1e-3, "bf16x3": 5e-2, "fp32_direct": 1e-3, "fp64_direct": 1e-3}
TOL_OWN = {"fp16x3": 1e-6, "bf16x3": 3e-6, "fp32_direct": 1e-6, "fp64_direct": 1e-6}
TOL_CONV = TOL_OWN  # the final objective (oracle-evaluated) above the minimum


def _golden(N, G):
    x = np.full((1, N, N), G)
    phi = None
    for line in open(GOLD):
        if line.startswith("# phi "):
            phi = float(line.split()[2])
        elif line[0].isdigit():
            n, m, v = line.split()
            x[0, int(n), int(m)] = float(v)
    return x, phi


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1703_02920_gb300 import memsynth
    memsynth.load()
    return memsynth


@pytest.fixture(scope="module")
def problem(oracle_mod):
    ds = S.make(1)
    P = oracle_mod.Problem.from_dataset(ds)
    x_star, phi_star = _golden(ds.N, ds.G)
    # the fixture is the oracle's: its objective there is the recorded one
    assert abs(oracle_mod.objective(P, x_star)[0] - phi_star) <= 1e-12 * phi_star
    return ds, P, x_star, phi_star, {}


def _check(oracle_mod, P, form, img, rep, x_star, phi_star):
    own = oracle_mod.objective(P, img)[0]
    # converged: the objective at the final image is the minimum (to 1e-6;
    # BF16x3 to its evaluation bound)
    assert own - phi_star <= TOL_CONV[form] * phi_star, (form, own, phi_star)
    assert own - phi_star >= -1e-6 * phi_star, (form, own, phi_star)
    # the form's own reported objective (the bound as written for the exact forms)
    assert abs(rep.phi - phi_star) <= TOL_OWN[form] * phi_star, (form, rep.phi, phi_star)
    assert abs(rep.phi - own) <= TOL_OWN[form] * own, (form, rep.phi, own)
    rel = np.linalg.norm(img - x_star) / np.linalg.norm(x_star)
    assert rel <= TOL_IMG[form], (form, rel)
    assert img.min() >= np.float32(P.G) * (1 - 1e-7)


def _solve(ms, problem, form):
    """The form's converged solve from I = G (cached for the module)."""
    import torch
    ds, P, x_star, phi_star, finals = problem
    if form not in finals:
        ctx = ms.Context(ds, precision=form)
        I0 = torch.full((1, ds.N, ds.N), float(ds.G), dtype=torch.float32, device="cuda")
        img, rep, hist = ctx.solve(I0, ITERS[form])
        ctx.close()
        # non-increasing up to the rounding of the recorded objective: each
        # history entry is a fresh evaluation of Phi with the form's own error
        # (at most TOL_OWN), while near the minimum a step lowers Phi by ~1e-9
        # relative (the line search itself compares differences, evaluated
        # from the image change, whose rounding scales with the step)
        phis = hist[0, : rep.iterations + 1, 0]
        assert np.all(np.diff(phis) <= 2 * TOL_OWN[form] * np.abs(phis[:-1]))
        finals[form] = (img.cpu().numpy().astype(np.float64), rep)
    return finals[form]


@pytest.mark.parametrize("form", ["fp16x3", "bf16x3", "fp32_direct"])
def test_converged_solve_reaches_the_minimiser(ms, oracle_mod, problem, form):
    ds, P, x_star, phi_star, _ = problem
    x, rep = _solve(ms, problem, form)
    _check(oracle_mod, P, form, x, rep, x_star, phi_star)


def test_converged_fp64_form_continues_from_the_split_form(ms, oracle_mod, problem):
    import torch
    ds, P, x_star, phi_star, _ = problem
    start, _ = _solve(ms, problem, "fp16x3")
    ctx = ms.Context(ds, precision="fp64_direct")
    img, rep, hist = ctx.solve(torch.from_numpy(start.astype(np.float32)).cuda(), 100)
    ctx.close()
    x = img.cpu().numpy().astype(np.float64)
    _check(oracle_mod, P, "fp64_direct", x, rep, x_star, phi_star)
