"""The library's host-side beam fit (Appendix A) against the oracle's: the
same main-lobe selection and log-quadratic least squares, so they agree to
float32 rounding of the PSF (no GPU)."""
import numpy as np
import pytest

from paper_1703_02920_gb300 import synth as S


@pytest.fixture(scope="module")
def lib():
    from paper_1703_02920_gb300 import memsynth
    return memsynth


def test_beam_fit_matches_oracle_on_gaussian_and_on_a_psf(lib, oracle_mod):
    N, dx, dy = 64, 0.05e-6, 0.07e-6
    n, m = np.mgrid[0:N, 0:N]
    x, y = (m - N // 2) * dx, (n - N // 2) * dy
    t = np.radians(25.0)
    a, b = x * np.sin(t) + y * np.cos(t), x * np.cos(t) - y * np.sin(t)
    s2 = 1 / (8 * np.log(2))
    g = np.exp(-(a ** 2 / (s2 * (9e-7) ** 2) + b ** 2 / (s2 * (5e-7) ** 2)) / 2).astype(np.float32)
    ds = S.make(1)
    P = oracle_mod.Problem.from_dataset(ds)
    psf = oracle_mod.dirty_image(P, psf=True)[0].astype(np.float32)
    for img, ddx, ddy in [(g, dx, dy), (psf, ds.dx, ds.dy)]:
        got = lib.mem_beam_fit(img, ddx, ddy)
        ref = oracle_mod.beam_fit(img.astype(np.float64), ddx, ddy)
        assert got[0] == pytest.approx(ref[0], rel=1e-6)
        assert got[1] == pytest.approx(ref[1], rel=1e-6)
        assert (got[2] - ref[2] + 90) % 180 - 90 == pytest.approx(0.0, abs=1e-4)
        assert got[3] == pytest.approx(ref[3], rel=1e-6)


def test_beam_fit_rejects_bad_input(lib):
    with pytest.raises(lib.MemError):
        lib.mem_beam_fit(np.zeros((16, 16), np.float32), 1e-6, 1e-6)


def test_phase_rotation_is_the_unit_modulus_factor(lib):
    """mem_phase_rotate multiplies by exp(-2 pi i (u x_p + v y_p)); a rotation
    and its inverse return the data."""
    rng = np.random.default_rng(7)
    u, v = rng.uniform(-2e6, 2e6, 300), rng.uniform(-2e6, 2e6, 300)
    V = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    xp, yp = 3.3e-6, -1.7e-6
    got = lib.mem_phase_rotate(u, v, V, xp, yp)
    ref = V * np.exp(-2j * np.pi * (u * xp + v * yp))
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(V))
    back = lib.mem_phase_rotate(u, v, got, -xp, -yp)
    assert np.max(np.abs(back - V)) <= 1e-12 * np.max(np.abs(V))
