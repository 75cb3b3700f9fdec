"""Maps drawn like the batched sweep, scaled down for the tests (test
infrastructure shared by the GPU tests and the golden-value script).

Each draw takes kappa, gamma, s and the map size from
``synthetic.batch_draws`` and shrinks them so that a test stays quick: npix
64-160, half-length 1.5-4, ~20 rays landing per pixel, Salpeter stars in a
disk of radius 1.1 x the shooting region's half-diagonal, 20-20 000 of them.
A draw whose stars do not cover the ray grid is skipped: the stars must span
the grid's bounding box, and every grid corner must lie within the disk the
stars fill (radius max |z_i| about the origin), where the circular sheet's
interior form -kappa_star z holds (Sec. 3.1)."""
import math

import numpy as np

import synthetic

F_FLUX = 0.01   # App. A flux fraction of these maps


def grid_covered(p, pos):
    """Whether the stars cover the ray grid of derived parameters p (an
    oracle or library Params): bounding box and star disk."""
    lo = [p.x0[k] for k in (0, 1)]
    hi = [p.x0[k] + (p.n[k] - 1) * p.h[k] for k in (0, 1)]
    if any(pos[:, k].min() > lo[k] or pos[:, k].max() < hi[k] for k in (0, 1)):
        return False
    r_disk = float(np.sqrt((pos * pos).sum(axis=1)).max())
    corner = max(math.hypot(x, y) for x in (lo[0], hi[0]) for y in (lo[1], hi[1]))
    return corner <= r_disk


def batch_maps(oracle_mod, n_maps, seed=7):
    """Up to n_maps dicts (kappa, gamma, s, npix, hl, rpp, m, pos, draw)."""
    out = []
    for d in synthetic.batch_draws(seed, n_maps):
        kappa, gamma, s = d["kappa"], d["gamma"], d["s"]
        npix = 64 + (d["npix"] - 500) // 16
        hl = 1.5 + (d["half_length"] - 5.0) / 6.0
        rpp = 20.0 * abs((1 - kappa) ** 2 - gamma ** 2)
        ks = (1 - s) * kappa
        p0 = oracle_mod.derive_params(kappa, gamma, s, np.ones(4), hl, npix, rays_per_pixel=rpp,
                                      flux_fraction_f=F_FLUX)
        R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
        n = synthetic.n_stars_for(ks, R, synthetic.SALPETER_01_1)
        if n < 20 or n > 20000:
            continue
        m, pos = synthetic.star_field(d["seed"], n, R, synthetic.SALPETER_01_1)
        p = oracle_mod.derive_params(kappa, gamma, s, m, hl, npix, rays_per_pixel=rpp,
                                     flux_fraction_f=F_FLUX)
        if not grid_covered(p, pos):
            continue
        out.append(dict(kappa=kappa, gamma=gamma, s=s, npix=npix, hl=hl, rpp=rpp, m=m, pos=pos,
                        draw=d["seed"]))
        if len(out) == n_maps:
            return out
    return out


def oracle_params(oracle_mod, w):
    return oracle_mod.derive_params(w["kappa"], w["gamma"], w["s"], w["m"], w["hl"], w["npix"],
                                    rays_per_pixel=w["rpp"], flux_fraction_f=F_FLUX)


def pick_spread(maps, n_pick):
    """Indices of n_pick maps spread over the sweep: the extremes of N_star,
    |mu_macro| and the oracle's cost (rays x stars), the cheapest map of
    every s value, then the cheapest of the rest.  Chosen from the draws
    alone (no map values)."""
    def mu(w):
        return 1.0 / abs((1 - w["kappa"]) ** 2 - w["gamma"] ** 2)

    def cost(w):
        # rays ~ (rays landing per pixel) x pixels, independent of mu
        return len(w["m"]) * w["npix"] ** 2
    idx = list(range(len(maps)))
    chosen = []

    def take(k):
        if k not in chosen:
            chosen.append(k)
    take(min(idx, key=lambda i: len(maps[i]["m"])))
    take(max(idx, key=lambda i: len(maps[i]["m"])))
    take(min(idx, key=lambda i: mu(maps[i])))
    take(max(idx, key=lambda i: mu(maps[i])))
    take(max(idx, key=lambda i: cost(maps[i])))
    for s in sorted({w["s"] for w in maps}):
        take(min((i for i in idx if maps[i]["s"] == s), key=lambda i: cost(maps[i])))
    for i in sorted(idx, key=lambda i: cost(maps[i])):
        if len(chosen) >= n_pick:
            break
        take(i)
    return chosen[:n_pick]
