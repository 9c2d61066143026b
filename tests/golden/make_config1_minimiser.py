"""Write config1_minimiser.txt: the minimiser of Eq. minproblem (Phi =
chi^2 - lambda S over I >= G) for the 64 x 64 config-1 data set, computed from
the FP64 oracle's objective and gradient alone.

Phi is strictly convex on I >= G for lambda > 0, so the minimiser is unique.
It is found with scipy's L-BFGS-B under the same bounds, from two different
starts (I = G everywhere, and the sky image clipped at G), run to
L-BFGS-B's own convergence test; the two results must agree to 1e-6
(relative L2) before the file is written.  Pixels at the bound are not
listed.  Run from the repository root:

    python tests/golden/make_config1_minimiser.py
"""
import os
import sys

import numpy as np
from scipy.optimize import minimize

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1703_02920_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_minimiser.txt")


def minimise(P, x0):
    N = P.N

    def fg(x):
        phi, _, _, g = oracle.objective_grad(P, x.reshape(1, N, N))
        return phi, g.ravel()

    r = minimize(fg, x0.ravel(), jac=True, method="L-BFGS-B", bounds=[(P.G, None)] * (N * N),
                 options=dict(maxiter=50000, maxfun=100000, ftol=1e-16, gtol=1e-10, maxcor=30))
    return r.x.reshape(1, N, N), float(r.fun)


def main():
    ds = synth.make(1)
    P = oracle.Problem.from_dataset(ds)
    a, fa = minimise(P, np.full((1, ds.N, ds.N), ds.G))
    b, fb = minimise(P, np.maximum(ds.truth.astype(np.float64), ds.G))
    rel = float(np.linalg.norm(a - b) / np.linalg.norm(a))
    if rel > 1e-6:
        raise SystemExit(f"the two L-BFGS-B runs disagree: {rel:.3e}")
    x, f = (a, fa) if fa <= fb else (b, fb)
    phi, chi, S = oracle.objective(P, x)
    _, _, _, g = oracle.objective_grad(P, x)
    with open(OUT, "w") as out:
        out.write("# Minimiser of Eq. minproblem (Phi = chi^2 - lambda S, I >= G) for the config-1 data set\n")
        out.write(f"# (64x64, 10,260 visibilities, G = {ds.G!r}, lambda = {ds.lam!r}); oracle objective,\n")
        out.write("# scipy L-BFGS-B from two starts (written by make_config1_minimiser.py)\n")
        out.write(f"# phi {phi!r}\n# chi2 {chi!r}\n# entropy {S!r}\n")
        out.write(f"# starts_agree_rel_l2 {rel:.3e}\n# kkt_residual {oracle.kkt_residual(x, g, P.G):.6e}\n")
        out.write("# pixels above G: row column value (every other pixel equals G)\n")
        for n, m in zip(*np.nonzero(x[0] > P.G)):
            out.write(f"{n} {m} {float(x[0, n, m])!r}\n")
    print(OUT, phi, rel)


if __name__ == "__main__":
    main()
