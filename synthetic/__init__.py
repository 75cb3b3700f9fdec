"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, ``bench.py`` and the oracle-side checks.
It holds no arithmetic of the method (no lens equation, no shooting region,
no tree, no mapping): only a counter-based random generator, point-mass star
fields drawn uniformly in a disk with a chosen mass spectrum, and the named
workload recipes.

Random numbers: SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based
generator, ``u = (mix(seed_stream + (k+1) * golden) >> 11) * 2**-53``.
"""
import math
from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from stream ``stream`` of seed ``seed``."""
    base = _mix64(np.array([(seed & 0xFFFFFFFF) | ((stream & 0xFFFFFFFF) << 32)],
                           dtype=np.uint64))[0]
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(base + k * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# mass spectra
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class MassFunction:
    """Piecewise power law dN/dm = c_k m^-alpha_k on [edges[k], edges[k+1]),
    continuous at the inner edges."""
    name: str
    edges: Tuple[float, ...]
    alphas: Tuple[float, ...]

    def _segment_weights(self):
        # unnormalised segment integrals of c_k m^-alpha_k, c chosen continuous
        c = [1.0]
        for k in range(1, len(self.alphas)):
            e = self.edges[k]
            c.append(c[-1] * e ** (-self.alphas[k - 1]) / e ** (-self.alphas[k]))
        return c

    def moment(self, q: int) -> float:
        """Unnormalised integral of m^q dN/dm."""
        c = self._segment_weights()
        tot = 0.0
        for k, a in enumerate(self.alphas):
            lo, hi = self.edges[k], self.edges[k + 1]
            e = q + 1 - a
            tot += c[k] * (math.log(hi / lo) if abs(e) < 1e-12 else (hi ** e - lo ** e) / e)
        return tot

    @property
    def mean(self) -> float:
        if self.edges[0] == self.edges[-1]:
            return self.edges[0]
        return self.moment(1) / self.moment(0)

    @property
    def m2_over_m(self) -> float:
        if self.edges[0] == self.edges[-1]:
            return self.edges[0]
        return self.moment(2) / self.moment(1)

    def sample(self, u_seg: np.ndarray, u: np.ndarray) -> np.ndarray:
        """Inverse-CDF sampling: segment by u_seg, position within it by u."""
        c = self._segment_weights()
        w = []
        for k, a in enumerate(self.alphas):
            lo, hi = self.edges[k], self.edges[k + 1]
            e = 1 - a
            w.append(c[k] * (math.log(hi / lo) if abs(e) < 1e-12 else (hi ** e - lo ** e) / e))
        cw = np.cumsum(w) / sum(w)
        seg = np.searchsorted(cw, u_seg, side="right").clip(0, len(w) - 1)
        out = np.empty_like(u)
        for k, a in enumerate(self.alphas):
            sel = seg == k
            lo, hi = self.edges[k], self.edges[k + 1]
            e = 1 - a
            if abs(e) < 1e-12:
                out[sel] = lo * (hi / lo) ** u[sel]
            else:
                out[sel] = (lo ** e + u[sel] * (hi ** e - lo ** e)) ** (1.0 / e)
        return out


EQUAL = MassFunction("equal", (1.0, 1.0), (0.0,))
SALPETER_01_1 = MassFunction("salpeter_0.1_1", (0.1, 1.0), (2.35,))
SALPETER_01_2 = MassFunction("salpeter_0.1_2", (0.1, 2.0), (2.35,))
KROUPA_008_15 = MassFunction("kroupa_0.08_1.5", (0.08, 0.5, 1.5), (1.3, 2.3))


def star_field(seed: int, n_stars: int, radius: float, mass_fn: MassFunction = EQUAL,
               center=(0.0, 0.0)):
    """n_stars point masses uniform in a disk of the given radius.

    Returns (masses (n,), positions (n, 2)) as float64 numpy arrays."""
    u1 = uniform(seed, 0, n_stars)
    u2 = uniform(seed, 1, n_stars)
    r = radius * np.sqrt(u1)
    phi = 2.0 * math.pi * u2
    pos = np.stack([center[0] + r * np.cos(phi), center[1] + r * np.sin(phi)], axis=1)
    if mass_fn.name == "equal":
        m = np.ones(n_stars)
    else:
        m = mass_fn.sample(uniform(seed, 2, n_stars), uniform(seed, 3, n_stars))
    return m, pos


def star_field_rect(seed: int, n_stars: int, half_widths, mass_fn: MassFunction = EQUAL):
    """n_stars point masses uniform in the rectangle |x| <= c1, |y| <= c2
    (half_widths = (c1, c2)).  Returns (masses, positions) like star_field."""
    c1, c2 = float(half_widths[0]), float(half_widths[1])
    x = c1 * (2.0 * uniform(seed, 0, n_stars) - 1.0)
    y = c2 * (2.0 * uniform(seed, 1, n_stars) - 1.0)
    pos = np.stack([x, y], axis=1)
    if mass_fn.name == "equal":
        m = np.ones(n_stars)
    else:
        m = mass_fn.sample(uniform(seed, 2, n_stars), uniform(seed, 3, n_stars))
    return m, pos


def n_stars_for_rect(kappa_star: float, half_widths, mass_fn: MassFunction) -> int:
    """Star count giving surface density kappa_star/pi per unit area in the
    rectangle of the given half-widths."""
    return int(round(kappa_star * 4.0 * half_widths[0] * half_widths[1] / (math.pi * mass_fn.mean)))


def n_stars_for(kappa_star: float, radius: float, mass_fn: MassFunction) -> int:
    """Star count giving surface density kappa_star/pi per unit area (theta_E
    units) in a disk of the given radius."""
    return int(round(kappa_star * radius * radius / mass_fn.mean))


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    kappa: float
    gamma: float
    s: float
    mass_fn: MassFunction
    radius: float
    n_stars: int
    npix: int
    half_length: float
    rays_per_pixel: float = 0.0   # rays per pixel in the absence of lensing
    fmm_order: int = 0
    leaf_size: int = 0
    seed: int = 0
    img_half: Optional[Tuple[float, float]] = None
    ray_grid: Optional[Tuple[int, int]] = None
    npix_y: int = 0                # rows of square pixels (0: npix, a square map)
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def stars(self):
        return star_field(self.seed, self.n_stars, self.radius, self.mass_fn)


def workload(name: str) -> Workload:
    """The five workloads.  Radii, star counts and rays per pixel are fixed
    numbers here: a disk radius of 1.1 x the shooting region's half-diagonal
    (or the radius that holds a fixed star count at kappa_star), and rays per
    pixel ~100 / |mu_macro| so that ~100 rays land per pixel.  Seeds are
    1000 + index."""
    if name == "plain_fp64_160":
        # 160 equal stars in a disk of radius 20; kappa=0.4, gamma=0.3, s=0;
        # explicit 700 x 2000 ray grid over image half-widths (16/3, 16);
        # 256^2 pixel map of half-width 4.
        return Workload(name, 0.4, 0.3, 0.0, EQUAL, 20.0, 160, 256, 4.0,
                        seed=1001, img_half=(16.0 / 3.0, 16.0), ray_grid=(700, 2000))
    if name == "fmm_fp32_salpeter_2000":
        # kappa=0.5, gamma=0.4, s=0.5; Salpeter 0.1-1; disk radius 212 covers
        # the shooting region; 9 rays/px unlensed = ~100 rays landing per px.
        mf = SALPETER_01_1
        R = 212.0
        return Workload(name, 0.5, 0.4, 0.5, mf, R, n_stars_for(0.25, R, mf), 2000, 10.0,
                        rays_per_pixel=9.0, fmm_order=25, seed=1002)
    if name == "near_critical_5000":
        R = math.sqrt(5e5 / 0.8)
        return Workload(name, 0.8, 0.25, 0.0, EQUAL, R, 500000, 5000, 10.0,
                        rays_per_pixel=2.25, fmm_order=30, seed=1003)
    if name == "large_kroupa_10000":
        mf = KROUPA_008_15
        R = math.sqrt(1e6 * mf.mean / 0.1)
        return Workload(name, 0.5, 0.45, 0.8, mf, R, 1000000, 10000, 25.0,
                        rays_per_pixel=4.75, fmm_order=40, seed=1005)
    if name == "extreme_mu_10000x1000":
        # Sec. 5's extreme magnification: (1-k+g)^-1 = 1.5, (1-k-g)^-1 = -1000
        # (mu_macro = -1500), s = 1 - 5e-5, Salpeter 0.1-2 stars, a source
        # plane of 100 x 10 theta_E as 10000 x 1000 square pixels of 0.01,
        # ~100 rays landing per pixel; the disk radius is 1.1 x the shooting
        # region's half-diagonal (75.2 x 5110.5 theta_E at f = 1e-3)
        kappa, gamma, s = 0.66717, 0.33383, 1 - 5e-5
        mf = SALPETER_01_2
        R = 1.1 * math.hypot(75.2, 5110.5)
        mu = 1.0 / abs((1 - kappa) ** 2 - gamma ** 2)
        return Workload(name, kappa, gamma, s, mf, R, n_stars_for((1 - s) * kappa, R, mf),
                        10000, 50.0, rays_per_pixel=100.0 / mu, fmm_order=25, seed=1006,
                        npix_y=1000)
    raise KeyError(name)


def batch_draws(seed: int, n: int):
    """Candidate (kappa, gamma, s, npix, half_length) draws for the batched
    sweep: kappa in U[0.2, 0.9], gamma in U[0.1, 0.8] rejecting
    ||1-kappa| - gamma| < 0.05, s in {0, 0.3, 0.6, 0.9}, npix in U{500..2000},
    half_length in U[5, 20].  Yields dicts; the caller sizes the star disk."""
    k = 0
    while True:
        u = uniform(seed, 100 + k, 6)
        k += 1
        kappa = 0.2 + 0.7 * u[0]
        gamma = 0.1 + 0.7 * u[1]
        if abs(abs(1.0 - kappa) - gamma) < 0.05:
            continue
        s = (0.0, 0.3, 0.6, 0.9)[min(3, int(u[2] * 4))]
        npix = 500 + min(1500, int(u[3] * 1501))
        hl = 5.0 + 15.0 * u[4]
        yield {"kappa": kappa, "gamma": gamma, "s": s, "npix": npix,
               "half_length": hl, "seed": 40000 + k, "u_extra": float(u[5])}
