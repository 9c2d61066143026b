"""The seeded synthetic inputs shared by the oracle and the GPU tests: the same
seed gives the same arrays bit for bit, the arrays have the documented
shapes, and config 1 appends the Hermitian conjugate of every sample."""
import numpy as np

from paper_1703_02920_gb300 import synth as S


def _same(a, b):
    for k in ("u", "v", "vo", "sigma", "pb", "offsets", "truth"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert (a.N, a.dx, a.dy, a.G, a.lam) == (b.N, b.dx, b.dy, b.G, b.lam)


def test_data_sets_are_reproducible_and_well_formed():
    a, b = S.make(1), S.make(1)
    _same(a, b)
    for ds in (a, S.random_problem(64, 0, seed=7, C=3, z_list=[50, 0, 20])):
        C = len(ds.offsets) - 1
        assert ds.offsets[0] == 0 and np.all(np.diff(ds.offsets) >= 0)
        Z = int(ds.offsets[-1])
        assert ds.u.shape == ds.v.shape == ds.vo.shape == ds.sigma.shape == (Z,)
        assert ds.pb.shape == (C, ds.N, ds.N)
        assert np.all(ds.sigma > 0) and np.all(ds.pb > 0) and np.all(ds.pb <= 1)
    _same(S.random_problem(64, 100, seed=5), S.random_problem(64, 100, seed=5))
    assert not np.array_equal(S.random_problem(64, 100, seed=5).u, S.random_problem(64, 100, seed=6).u)


def test_config1_appends_hermitian_conjugates():
    ds = S.make(1)
    h = ds.Z // 2
    assert ds.Z == 2 * h == 10260
    assert np.array_equal(ds.u[h:], -ds.u[:h]) and np.array_equal(ds.v[h:], -ds.v[:h])
    assert np.array_equal(ds.sigma[h:], ds.sigma[:h])
    assert np.array_equal(ds.vo[h:], np.conj(ds.vo[:h]))
