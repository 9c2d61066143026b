"""Seeded synthetic interferometer data shaped like the paper's ALMA workloads.

This module is the only code shared by the FP64 oracle and the CUDA path: it
draws inputs (antenna layouts, Earth-rotation (u,v) tracks, a Gaussian primary
beam, a sky of elliptical Gaussians and point sources, thermal noise) and holds
none of the imaging method's arithmetic.  Observed visibilities are the
continuous Fourier transform of the beam-attenuated sky (closed forms for
Gaussians and points), i.e. a simulated measurement of Eq. (1), not the
discrete direct sum the method evaluates.

Conventions (Section 2, "Data description"): u, v in wavelengths, pixel sizes
in radians, images row-major [y][x] with x_m = (m - N/2) dx, y_n = (n - N/2) dy,
visibilities complex with per-sample deviation sigma (real and imaginary parts
each N(0, sigma^2)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ARCSEC = math.pi / 648000.0
C_LIGHT = 299792458.0
FWHM_TO_SIGMA = 1.0 / math.sqrt(8.0 * math.log(2.0))


def rng_for(config: int, stream: int) -> np.random.Generator:
    """Seed convention: 1000*config + stream (1 array, 2 sky, 3 noise, 4 subsets)."""
    return np.random.Generator(np.random.PCG64(1000 * config + stream))


# ----------------------------------------------------------------------------
# array geometry and (u,v) tracks
# ----------------------------------------------------------------------------
def antennas_in_disk(rng: np.random.Generator, n_ant: int, diameter_m: float) -> np.ndarray:
    """East/North positions uniform by area in a disk of the given diameter."""
    r = 0.5 * diameter_m * np.sqrt(rng.random(n_ant))
    phi = 2.0 * math.pi * rng.random(n_ant)
    return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)


def earth_rotation_uv(enu: np.ndarray, n_dumps: int, wavelength_m: float,
                      lat_deg: float = -23.03, dec_deg: float = -30.0,
                      ha_span_h: float = 3.0):
    """(u,v) in wavelengths for all baselines p<q over hour angles in [-span, +span].

    Textbook local-horizon -> equatorial -> (u,v,w) rotation with the w term
    dropped (coplanar array).  Output is ordered [dump][baseline].
    """
    n = enu.shape[0]
    p, q = np.triu_indices(n, k=1)
    east = enu[q, 0] - enu[p, 0]
    north = enu[q, 1] - enu[p, 1]
    lat = math.radians(lat_deg)
    dec = math.radians(dec_deg)
    X = -math.sin(lat) * north
    Y = east
    Zc = math.cos(lat) * north
    if n_dumps == 1:
        ha = np.zeros(1)
    else:
        ha = np.linspace(-ha_span_h, ha_span_h, n_dumps) * (math.pi / 12.0)
    sh = np.sin(ha)[:, None]
    ch = np.cos(ha)[:, None]
    u = sh * X[None, :] + ch * Y[None, :]
    v = -math.sin(dec) * ch * X[None, :] + math.sin(dec) * sh * Y[None, :] + math.cos(dec) * Zc[None, :]
    return (u / wavelength_m).ravel(), (v / wavelength_m).ravel()


# ----------------------------------------------------------------------------
# primary beam and sky
# ----------------------------------------------------------------------------
def pixel_coords(N: int, d: float) -> np.ndarray:
    return (np.arange(N, dtype=np.float64) - N // 2) * d


def gaussian_beam(N: int, dx: float, dy: float, fwhm_rad: float,
                  centre=(0.0, 0.0)) -> np.ndarray:
    """Gaussian primary beam A (peak 1) sampled on the pixel grid, float32."""
    s = fwhm_rad * FWHM_TO_SIGMA
    x = pixel_coords(N, dx) - centre[0]
    y = pixel_coords(N, dy) - centre[1]
    a = np.exp(-0.5 * (y[:, None] ** 2 + x[None, :] ** 2) / (s * s))
    return a.astype(np.float32)


@dataclass
class Gaussian:
    flux: float        # Jy (integral over the sky)
    x0: float          # radians
    y0: float
    fwhm_maj: float    # radians
    fwhm_min: float
    pa: float          # radians, rotation of the major axis from +y towards +x

    def cov(self) -> np.ndarray:
        smaj = self.fwhm_maj * FWHM_TO_SIGMA
        smin = self.fwhm_min * FWHM_TO_SIGMA
        c, s = math.cos(self.pa), math.sin(self.pa)
        # major axis along (sin pa, cos pa) in (x, y)
        R = np.array([[s, c], [c, -s]])
        return R @ np.diag([smaj * smaj, smin * smin]) @ R.T


@dataclass
class Point:
    flux: float
    x0: float
    y0: float


def sky_image(comps, N: int, dx: float, dy: float) -> np.ndarray:
    """Pixelised sky in Jy/pixel (brightness x pixel solid angle), float64."""
    x = pixel_coords(N, dx)
    y = pixel_coords(N, dy)
    img = np.zeros((N, N))
    for c in comps:
        if isinstance(c, Point):
            m = int(round(c.x0 / dx)) + N // 2
            n = int(round(c.y0 / dy)) + N // 2
            if 0 <= m < N and 0 <= n < N:
                img[n, m] += c.flux
        else:
            S = c.cov()
            Si = np.linalg.inv(S)
            ddx = x[None, :] - c.x0
            ddy = y[:, None] - c.y0
            q = Si[0, 0] * ddx * ddx + 2 * Si[0, 1] * ddx * ddy + Si[1, 1] * ddy * ddy
            img += c.flux / (2 * math.pi * math.sqrt(np.linalg.det(S))) * np.exp(-0.5 * q) * dx * dy
    return img


def sky_visibilities(comps, u: np.ndarray, v: np.ndarray, beam_fwhm: float,
                     beam_centre=(0.0, 0.0)) -> np.ndarray:
    """Continuous Fourier transform of (Gaussian beam) x (sky) at (u, v).

    Product of Gaussians is a Gaussian; its transform is closed-form.  Points
    give flux * beam(x0) * exp(-2 pi i (u x0 + v y0)).
    """
    sb2 = (beam_fwhm * FWHM_TO_SIGMA) ** 2
    bc = np.asarray(beam_centre, dtype=np.float64)
    out = np.zeros(u.shape, dtype=np.complex128)
    for c in comps:
        if isinstance(c, Point):
            d2 = (c.x0 - bc[0]) ** 2 + (c.y0 - bc[1]) ** 2
            amp = c.flux * math.exp(-0.5 * d2 / sb2)
            out += amp * np.exp(-2j * math.pi * (u * c.x0 + v * c.y0))
        else:
            S = c.cov()
            Si = np.linalg.inv(S)
            Bi = np.eye(2) / sb2
            P = Si + Bi
            Pi = np.linalg.inv(P)
            mu = np.array([c.x0, c.y0])
            h = Si @ mu + Bi @ bc
            mup = Pi @ h
            logK = (math.log(c.flux / (2 * math.pi * math.sqrt(np.linalg.det(S))))
                    + 0.5 * h @ Pi @ h - 0.5 * mu @ Si @ mu - 0.5 * bc @ Bi @ bc)
            amp = math.exp(logK) * 2 * math.pi / math.sqrt(np.linalg.det(P))
            quad = Pi[0, 0] * u * u + 2 * Pi[0, 1] * u * v + Pi[1, 1] * v * v
            out += amp * np.exp(-2 * math.pi ** 2 * quad - 2j * math.pi * (u * mup[0] + v * mup[1]))
    return out


def continuum_sky(rng: np.random.Generator, n_gauss: int = 3, n_points: int = 2,
                  flux_gauss: float = 0.7, flux_points: float = 0.3):
    """3 elliptical Gaussians + 2 point sources on a 0.2" lattice, 1 Jy total."""
    wg = rng.uniform(0.2, 1.0, n_gauss)
    wp = rng.uniform(0.2, 1.0, n_points)
    comps = []
    for i in range(n_gauss):
        fmaj = rng.uniform(0.8, 2.5) * ARCSEC
        ratio = rng.uniform(0.4, 1.0)
        comps.append(Gaussian(flux=flux_gauss * wg[i] / wg.sum(),
                              x0=rng.uniform(-4, 4) * ARCSEC, y0=rng.uniform(-4, 4) * ARCSEC,
                              fwhm_maj=fmaj, fwhm_min=fmaj * ratio,
                              pa=rng.uniform(0, math.pi)))
    for i in range(n_points):
        kx, ky = rng.integers(-20, 21, 2)
        comps.append(Point(flux=flux_points * wp[i] / wp.sum(),
                           x0=0.2 * kx * ARCSEC, y0=0.2 * ky * ARCSEC))
    return comps


# ----------------------------------------------------------------------------
# data sets
# ----------------------------------------------------------------------------
@dataclass
class Dataset:
    name: str
    N: int
    dx: float
    dy: float
    u: np.ndarray            # float64, all channels concatenated
    v: np.ndarray
    vo: np.ndarray           # complex128
    sigma: np.ndarray        # float64
    pb: np.ndarray           # float32, (C, N, N)
    offsets: np.ndarray      # int64, C+1
    truth: np.ndarray        # float32, (C, N, N)
    G: float
    lam: float
    n_iter: int
    shared_image: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def C(self) -> int:
        return len(self.offsets) - 1

    @property
    def Z(self) -> int:
        return int(self.offsets[-1])

    def channel(self, c: int):
        a, b = int(self.offsets[c]), int(self.offsets[c + 1])
        return self.u[a:b], self.v[a:b], self.vo[a:b], self.sigma[a:b]

    def subset(self, channels) -> "Dataset":
        """The data set restricted to the listed channels (in that order)."""
        channels = list(channels)
        sl = [slice(int(self.offsets[c]), int(self.offsets[c + 1])) for c in channels]
        offs = np.concatenate([[0], np.cumsum([s.stop - s.start for s in sl])]).astype(np.int64)
        cat = lambda a: np.concatenate([a[s] for s in sl])
        truth = self.truth[:1] if self.shared_image else self.truth[channels]
        return Dataset(name=f"{self.name}[{channels}]", N=self.N, dx=self.dx, dy=self.dy, u=cat(self.u),
                       v=cat(self.v), vo=cat(self.vo), sigma=cat(self.sigma), pb=self.pb[channels],
                       offsets=offs, truth=truth, G=self.G, lam=self.lam, n_iter=self.n_iter,
                       shared_image=self.shared_image, meta=dict(self.meta))


# Section 4 workloads are ALMA data sets; these stand-ins follow their shapes.
CONFIGS = {
    1: dict(N=64, cell=0.2, n_ant=20, diam=300.0, dumps=27, conj=True, G=1e-4, n_iter=50),
    2: dict(N=256, cell=0.05, n_ant=50, diam=1000.0, dumps=816, conj=False, G=6.25e-6, n_iter=50),
    3: dict(N=512, cell=0.025, n_ant=50, diam=2000.0, dumps=8164, conj=False, G=1.5625e-6, n_iter=200),
    5: dict(N=1024, cell=0.0125, n_ant=64, diam=3000.0, dumps=9920, conj=False, G=3.90625e-7, n_iter=100),
}
WAVELENGTH = 0.87e-3          # 345 GHz
BEAM_FWHM_345 = 18.0 * ARCSEC  # 12 m dish, scales with wavelength
SIGMA_NOISE = 5e-3            # Jy per real/imaginary component
LAMBDA_PAPER = 0.1            # entropy weight in the (I/G) log(I/G) convention


def make_continuum(config: int, dumps: int | None = None) -> Dataset:
    """Single-channel data set for configs 1, 2, 3, 5 (optionally fewer dumps)."""
    p = CONFIGS[config]
    N, dx = p["N"], p["cell"] * ARCSEC
    enu = antennas_in_disk(rng_for(config, 1), p["n_ant"], p["diam"])
    u, v = earth_rotation_uv(enu, dumps or p["dumps"], WAVELENGTH)
    comps = continuum_sky(rng_for(config, 2))
    vis = sky_visibilities(comps, u, v, BEAM_FWHM_345)
    nrng = rng_for(config, 3)
    noise = SIGMA_NOISE * (nrng.standard_normal(u.size) + 1j * nrng.standard_normal(u.size))
    vo = vis + noise
    if p["conj"]:
        u = np.concatenate([u, -u])
        v = np.concatenate([v, -v])
        vo = np.concatenate([vo, np.conj(vo)])
    sigma = np.full(u.size, SIGMA_NOISE)
    pb = gaussian_beam(N, dx, dx, BEAM_FWHM_345)[None]
    truth = sky_image(comps, N, dx, dx).astype(np.float32)[None]
    G = p["G"]
    return Dataset(name=f"continuum{config}", N=N, dx=dx, dy=dx, u=u, v=v, vo=vo, sigma=sigma,
                   pb=pb, offsets=np.array([0, u.size], dtype=np.int64), truth=truth,
                   G=G, lam=LAMBDA_PAPER / G, n_iter=p["n_iter"])


def make_cube(n_channels: int = 64, N: int = 256, cell: float = 0.05, dumps: int = 1633,
              z_min: float = 2e5, z_max: float = 2e6, config: int = 4,
              n_clouds: int = 64) -> Dataset:
    """Spectral-line cube: rotating Gaussian disk, per-channel (u,v) scaled by nu/nu0,
    per-channel beam, uneven per-channel visibility counts (log-uniform)."""
    dx = cell * ARCSEC
    nu0 = 690e9
    dnu = 1e9 / 64
    nus = 689.5e9 + (np.arange(n_channels) + 0.5) * dnu
    enu = antennas_in_disk(rng_for(config, 1), 50, 500.0)
    u0, v0 = earth_rotation_uv(enu, dumps, C_LIGHT / nu0)
    srng = rng_for(config, 4)
    zc = np.exp(srng.uniform(math.log(z_min), math.log(z_max), n_channels)).astype(np.int64)
    zc = np.minimum(zc, u0.size)
    # disk: clouds on rings, Keplerian line-of-sight velocities
    fwhm_disk, incl, pa = 5.0 * ARCSEC, math.radians(45.0), math.radians(30.0)
    crng = rng_for(config, 2)
    r = np.abs(crng.normal(0.0, fwhm_disk * FWHM_TO_SIGMA, n_clouds)) + 0.05 * ARCSEC
    az = crng.uniform(0, 2 * math.pi, n_clouds)
    xd, yd = r * np.cos(az), r * np.sin(az) * math.cos(incl)
    ca, sa = math.cos(pa), math.sin(pa)
    xs, ys = xd * ca + yd * sa, -xd * sa + yd * ca
    rs = 0.3 * ARCSEC
    vkep = 150e3 * (np.sqrt(rs) / np.sqrt(np.maximum(r, rs)))
    vlos = vkep * np.cos(az)
    vchan = C_LIGHT * (nu0 - nus) / nu0
    sig_v = 2.0 * C_LIGHT * dnu / nu0
    prof = np.exp(-0.5 * ((vchan[:, None] - vlos[None, :]) / sig_v) ** 2)  # (C, clouds)
    prof /= prof.sum(axis=1).max()
    us, vs, vos, sgs, pbs, truths, offs = [], [], [], [], [], [], [0]
    nrng = rng_for(config, 3)
    for c in range(n_channels):
        scale = nus[c] / nu0
        keep = np.sort(srng.choice(u0.size, size=int(zc[c]), replace=False))
        u, v = u0[keep] * scale, v0[keep] * scale
        fwhm_b = BEAM_FWHM_345 * (345e9 / nus[c])
        comps = [Gaussian(flux=float(prof[c, k]), x0=float(xs[k]), y0=float(ys[k]),
                          fwhm_maj=0.6 * ARCSEC, fwhm_min=0.6 * ARCSEC, pa=0.0)
                 for k in range(n_clouds) if prof[c, k] > 1e-6]
        vis = sky_visibilities(comps, u, v, fwhm_b)
        vo = vis + SIGMA_NOISE * (nrng.standard_normal(u.size) + 1j * nrng.standard_normal(u.size))
        us.append(u); vs.append(v); vos.append(vo); sgs.append(np.full(u.size, SIGMA_NOISE))
        pbs.append(gaussian_beam(N, dx, dx, fwhm_b))
        truths.append(sky_image(comps, N, dx, dx).astype(np.float32))
        offs.append(offs[-1] + u.size)
    G = 6.25e-6
    return Dataset(name=f"cube{n_channels}", N=N, dx=dx, dy=dx, u=np.concatenate(us),
                   v=np.concatenate(vs), vo=np.concatenate(vos), sigma=np.concatenate(sgs),
                   pb=np.stack(pbs), offsets=np.array(offs, dtype=np.int64),
                   truth=np.stack(truths), G=G, lam=LAMBDA_PAPER / G, n_iter=50,
                   meta=dict(nu=nus))


def make(config: int, **kw) -> Dataset:
    if config == 4:
        return make_cube(**kw)
    return make_continuum(config, **kw)


# ----------------------------------------------------------------------------
# random problems for parity tests
# ----------------------------------------------------------------------------
def random_problem(N: int, Z: int, seed: int, C: int = 1, shared_image: bool = False,
                   cell_arcsec: float = 0.1, uv_frac: float = 0.45, G: float = 1e-4,
                   lam: float | None = None, z_list=None) -> Dataset:
    """Random (u,v) inside the Nyquist disk |u| dx <= uv_frac, random beams and
    positive images; visibilities are random complex data with random sigma."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = cell_arcsec * ARCSEC
    umax = uv_frac / dx
    if z_list is None:
        z_list = [Z] * C
    us, vs, vos, sgs, pbs, imgs, offs = [], [], [], [], [], [], [0]
    for c in range(C):
        z = int(z_list[c])
        r = umax * np.sqrt(rng.random(z))
        t = 2 * math.pi * rng.random(z)
        us.append(r * np.cos(t)); vs.append(r * np.sin(t))
        vos.append(rng.standard_normal(z) * 0.3 + 1j * rng.standard_normal(z) * 0.3)
        sgs.append(rng.uniform(0.5, 2.0, z) * 0.05)
        fw = rng.uniform(0.6, 1.5) * N * dx
        pbs.append(gaussian_beam(N, dx, dx, fw, centre=tuple(rng.uniform(-0.05, 0.05, 2) * N * dx)))
        imgs.append((G + rng.random((N, N)) ** 4 * 0.02).astype(np.float32))
        offs.append(offs[-1] + z)
    truth = np.stack(imgs)
    if shared_image:
        truth = truth[:1]
    return Dataset(name=f"random{N}x{Z}s{seed}", N=N, dx=dx, dy=dx, u=np.concatenate(us),
                   v=np.concatenate(vs), vo=np.concatenate(vos), sigma=np.concatenate(sgs),
                   pb=np.stack(pbs), offsets=np.array(offs, dtype=np.int64), truth=truth,
                   G=G, lam=(1.0 if lam is None else lam), n_iter=10, shared_image=shared_image)


def random_complex(Z: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(Z) + 1j * rng.standard_normal(Z)


def random_image(N: int, seed: int, C: int = 1, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, (C, N, N)).astype(np.float32)
