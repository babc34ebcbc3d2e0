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
