"""Helpers shared by the GPU tests: device ensembles and the parity comparison."""
import numpy as np

# FP64 parity bar: relative 1e-10 on the final time and on the spin and L-hat
# components (components are scaled by their vector's magnitude, since a single
# component can be arbitrarily close to zero); 1e-10 absolute on the scalar
# products, which lie in [-1, 1].
FP64_TOL = 1e-10


def decided_alike(g, o):
    """Binaries whose accept/reject/landing decision counts agree on both sides."""
    return (g["n_acc"] == o["n_acc"]) & (g["n_rej"] == o["n_rej"]) & (g["n_land"] == o["n_land"])


def parity_errors(g, o, mask=None):
    """Max scaled deviations of the GPU outputs g from the oracle outputs o (numpy dicts)."""
    m = np.ones_like(o["t"], dtype=bool) if mask is None else mask
    e = {}
    e["t"] = np.max(np.abs(g["t"][m] - o["t"][m]) / np.abs(o["t"][m]), initial=0.0)
    e["omega"] = np.max(np.abs(g["omega"][m] - o["omega"][m]) / np.abs(o["omega"][m]), initial=0.0)
    for k in ("S1", "S2", "Lhat"):
        scale = np.linalg.norm(o[k][:, m], axis=0)
        d = np.max(np.abs(g[k][:, m] - o[k][:, m]), axis=0)
        ok = scale > 0
        e[k] = max(np.max(d[ok] / scale[ok], initial=0.0), np.max(d[~ok], initial=0.0))
    for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
        a, b = g[k][m], o[k][m]
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin), k
        e[k] = np.max(np.abs(a[fin] - b[fin]), initial=0.0)
    return e


def assert_fp64_parity(g, o, max_divergent=0, tol=FP64_TOL):
    assert np.array_equal(g["status"], o["status"]), "status differs"
    same = decided_alike(g, o)
    nd = int((~same).sum())
    assert nd <= max_divergent, f"{nd} binaries took different step decisions"
    e = parity_errors(g, o, same)
    bad = {k: v for k, v in e.items() if not v <= tol}
    assert not bad, f"FP64 parity exceeded {tol}: {bad}"
    return e


def per_binary_errors(g, o):
    """Per-binary scaled deviations (same scaling as parity_errors), one array per output."""
    e = {"t": np.abs(g["t"] - o["t"]) / np.abs(o["t"]),
         "omega": np.abs(g["omega"] - o["omega"]) / np.abs(o["omega"])}
    for k in ("S1", "S2", "Lhat"):
        scale = np.linalg.norm(o[k], axis=0)
        d = np.max(np.abs(g[k] - o[k]), axis=0)
        e[k] = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), d)
    for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
        e[k] = np.nan_to_num(np.abs(g[k] - o[k]), nan=0.0)
    return e


def ulp_response(orc, ens):
    """Per-binary largest change of the oracle's outputs (default parameters) when one input (omega0,
    m1 with m2 = 1 - m1, a component of each spin direction, chi2) or h0 moves by one ulp: the conditioning of each
    binary's result under roundoff-sized perturbations.  Binaries whose perturbed run takes other step
    decisions are left out of that run's maximum."""
    o = orc.integrate(ens)
    runs = []
    for key, comp in (("omega0", None), ("m1", None), ("s1hat", 0), ("s2hat", 2), ("chi2", None)):
        e2 = {k: v.copy() for k, v in ens.items()}
        a = e2[key] if comp is None else e2[key][comp]
        a[:] = np.nextafter(a, np.inf)
        if key == "m1":
            e2["m2"] = 1.0 - e2["m1"]
        runs.append(orc.integrate(e2))
    for h in (np.nextafter(10.0, np.inf), np.nextafter(10.0, 0.0)):
        runs.append(orc.integrate(ens, orc.params(h0=float(h))))
    resp = None
    for p in runs:
        e = per_binary_errors(p, o)
        same = decided_alike(p, o)
        for k in e:
            e[k] = np.where(same, e[k], 0.0)
        resp = e if resp is None else {k: np.maximum(resp[k], e[k]) for k in e}
    return o, resp


def assert_fp64_parity_conditioned(g, o, resp, max_relaxed, max_divergent=1):
    """FP64 parity where some binaries are ill-conditioned: each binary is held to max(1e-10, 10x its own
    one-ulp response ``resp`` (from ulp_response)), and at most ``max_relaxed`` binaries may use the
    relaxed bound.  Statuses must agree; at most ``max_divergent`` binaries may take other step decisions."""
    assert np.array_equal(g["status"], o["status"]), "status differs"
    same = decided_alike(g, o)
    assert int((~same).sum()) <= max_divergent, int((~same).sum())
    e = per_binary_errors(g, o)
    relaxed = np.zeros(o["t"].shape[0], dtype=bool)
    for k, v in e.items():
        bound = np.maximum(FP64_TOL, 10 * resp[k])
        assert np.all(v[same] <= bound[same]), (k, float(v[same].max()))
        relaxed |= same & (v > FP64_TOL)
    assert int(relaxed.sum()) <= max_relaxed, int(relaxed.sum())
    return e
