"""Comparison metrics shared by the GPU parity tests (test infrastructure).

Tolerances restate the targets for this path: deflection max relative error
<= 2e-6 (denominator max(|alpha_ref|, sqrt(kappa_star)), alpha the net
microlens deflection alpha_* + alpha_s); map 99.9th-percentile per-pixel
relative error <= 1e-3 over pixels with mu_ref > 0, and mu <= 1e-6 |mu_macro|
where mu_ref = 0; mean magnification relative error <= 1e-5."""
import numpy as np

DEFLECTION_TOL = 2e-6
MAP_P999_TOL = 1e-3
MEAN_TOL = 1e-5


def deflection_rel_error(params, z, w, w_ref):
    z = np.asarray(z).reshape(-1, 2)
    kappa, gamma, ks = params.kappa, params.gamma, params.kappa_star
    macro = np.stack([(1 - kappa + gamma) * z[:, 0], (1 - kappa - gamma) * z[:, 1]], 1)
    alpha_ref = macro - w_ref                       # alpha_* + alpha_s
    den = np.maximum(np.hypot(alpha_ref[:, 0], alpha_ref[:, 1]), np.sqrt(max(ks, 1e-30)))
    return np.hypot(*(np.asarray(w) - w_ref).T) / den


def map_errors(mu, mu_ref, mu_macro):
    mu = np.asarray(mu, dtype=np.float64)
    pos = mu_ref > 0
    rel = np.abs(mu[pos] - mu_ref[pos]) / mu_ref[pos]
    out = {
        "p999": float(np.quantile(rel, 0.999)) if rel.size else 0.0,
        "max": float(rel.max()) if rel.size else 0.0,
        "zero_max": float(np.abs(mu[~pos]).max()) / abs(mu_macro) if (~pos).any() else 0.0,
        "mean_rel": float(abs(mu.mean() - mu_ref.mean()) / mu_ref.mean()) if mu_ref.mean() else 0.0,
    }
    return out


def assert_map_parity(mu, mu_ref, mu_macro, p999=MAP_P999_TOL, mean=MEAN_TOL):
    e = map_errors(mu, mu_ref, mu_macro)
    assert e["p999"] <= p999, e
    assert e["zero_max"] <= 1e-6, e
    assert e["mean_rel"] <= mean, e
    return e


def band_errors(mu, mu_ref, mu_macro):
    """Errors of a partial (row-band) map: per-pixel |mu - mu_ref| relative to
    max(mu_ref, |mu_macro|), over pixels the band reaches."""
    mu = np.asarray(mu, dtype=np.float64)
    pos = (mu_ref > 0) | (mu > 0)
    rel = np.abs(mu[pos] - mu_ref[pos]) / np.maximum(mu_ref[pos], abs(mu_macro))
    return {"p999": float(np.quantile(rel, 0.999)), "max": float(rel.max()),
            "mean_rel": float(abs(mu.sum() - mu_ref.sum()) / mu_ref.sum())}
