"""Seeded synthetic input ensembles shaped like the paper's workloads.

This module only draws inputs; it holds none of the integration method's
arithmetic, and both the CUDA path's tests and the CPU oracle's tests take
their inputs from it.  Random numbers come from NumPy's counter-based Philox
bit generator (``random_raw`` output, which NumPy keeps stable across
releases), turned into 53-bit uniforms here.  Spin directions are drawn
isotropically with the cylinder-projection construction (z uniform in
[-1, 1], azimuth uniform in [0, 2 pi)); this is deliberately not the paper's
Marsaglia draw, which the library implements as its own sampler.

Layout of an ensemble: a dict of float64 arrays; scalars have shape (n,),
vectors ("s1hat", "s2hat", "lhat") shape (3, n), component-major, which is the
structure-of-arrays order the library reads.

Ensembles (paper sections in brackets):
  C0  1,024 binaries, m1 = m2 = 0.5, chi = 1, isotropic spins, L-hat = z,
      M omega 0.025 -> 0.05.
  C1  1,048,576 binaries, equal mass, chi_i ~ U[0, 1], isotropic spins,
      M omega 0.01 -> 0.05.
  C2  4,194,304 binaries of uneven length: q = m1/m2 log-uniform in [1, 10],
      chi_i ~ U[0, 1], isotropic, M omega_0 ~ U[0.005, 0.02], omega_f = 0.05.
  C3  C1's ensemble (run in mixed precision).
  C4  65,536 binaries, q ~ U[1, 4], chi = 1, isotropic, M omega 0.01 -> 0.05.
  SCIENCE  equal mass, chi = 1, isotropic, omega 0.00395 -> 0.05 [Sec. V A].
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x0908_3889_0000

SIZES = {"C0": 1024, "C1": 1_048_576, "C2": 4_194_304, "C3": 1_048_576, "C4": 65_536}


def _uniforms(seed: int, shape) -> np.ndarray:
    bg = np.random.Philox(key=seed)
    raw = bg.random_raw(int(np.prod(shape)))
    return ((raw >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)).reshape(shape)


def _isotropic(u_z: np.ndarray, u_phi: np.ndarray) -> np.ndarray:
    z = 2.0 * u_z - 1.0
    phi = 2.0 * np.pi * u_phi
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z])


def ensemble(n: int, seed: int, *, q=(1.0, 1.0), q_dist: str = "fixed", chi=(1.0, 1.0),
             chi_dist: str = "fixed", omega0=(0.01, 0.01), omega_f: float = 0.05) -> dict:
    """Draw n binaries.  q = m1/m2 with m1 + m2 = 1; chi and omega0 fixed or uniform."""
    u = _uniforms(seed, (8, n))
    if q_dist == "fixed":
        qv = np.full(n, float(q[0]))
    elif q_dist == "uniform":
        qv = q[0] + (q[1] - q[0]) * u[0]
    elif q_dist == "loguniform":
        qv = q[0] * np.exp(u[0] * np.log(q[1] / q[0]))
    else:
        raise ValueError(q_dist)
    m1 = qv / (1.0 + qv)
    m2 = 1.0 / (1.0 + qv)
    if chi_dist == "fixed":
        c1 = np.full(n, float(chi[0]))
        c2 = np.full(n, float(chi[0]))
    elif chi_dist == "uniform":
        c1 = chi[0] + (chi[1] - chi[0]) * u[1]
        c2 = chi[0] + (chi[1] - chi[0]) * u[2]
    else:
        raise ValueError(chi_dist)
    w0 = omega0[0] + (omega0[1] - omega0[0]) * u[3]
    lhat = np.zeros((3, n))
    lhat[2] = 1.0
    return {"m1": m1, "m2": m2, "chi1": c1, "chi2": c2, "s1hat": _isotropic(u[4], u[5]),
            "s2hat": _isotropic(u[6], u[7]), "lhat": lhat, "omega0": w0, "omega_f": np.full(n, float(omega_f))}


def config(name: str, n: int | None = None, seed: int | None = None) -> dict:
    """Ensemble of a named workload; ``n`` truncates/extends the size, ``seed`` overrides."""
    k = {"C0": 0, "C1": 1, "C2": 2, "C3": 1, "C4": 4, "SCIENCE": 5, "PAPER_PERF": 6}[name]
    seed = SEED_BASE + k if seed is None else seed
    n = SIZES.get(name, 100_000) if n is None else n
    if name == "C0":
        return ensemble(n, seed, omega0=(0.025, 0.025))
    if name in ("C1", "C3"):
        return ensemble(n, seed, chi=(0.0, 1.0), chi_dist="uniform")
    if name == "C2":
        return ensemble(n, seed, q=(1.0, 10.0), q_dist="loguniform", chi=(0.0, 1.0), chi_dist="uniform",
                        omega0=(0.005, 0.02))
    if name == "C4":
        return ensemble(n, seed, q=(1.0, 4.0), q_dist="uniform")
    if name == "SCIENCE":
        return ensemble(n, seed, omega0=(0.00395, 0.00395))
    if name == "PAPER_PERF":
        # Sec. IV: one test inspiral, omega 0.004 -> 0.1, replicated n times (lock-step).
        one = ensemble(1, seed, omega0=(0.004, 0.004), omega_f=0.1)
        return {k: np.repeat(v, n, axis=-1) for k, v in one.items()}
    raise KeyError(name)


def paper_sweeps(n: int = 100_000) -> list:
    """The parameter sweeps of Sec. V, each ensemble n binaries, isotropic spins, omega 0.00395 -> 0.05:
    r vs chi at equal mass (Sec. V C: chi = 0.1 .. 0.9), the m1 = 0.4, chi = 0.05 ring (Sec. V D) and
    r vs m1 at chi = 1 (Sec. V B, Fig. 5: m1 = 0.5 .. 0.3).  Returns (kind, value, ensemble) triples."""
    out = []
    for chi in (0.1, 0.3, 0.5, 0.7, 0.9):
        out.append(("chi", chi, ensemble(n, 600 + int(chi * 10), chi=(chi, chi), omega0=(0.00395, 0.00395))))
    out.append(("ring", 0.4, ensemble(n, 77, q=(0.4 / 0.6, 0.4 / 0.6), chi=(0.05, 0.05), omega0=(0.00395, 0.00395))))
    for m1 in (0.5, 0.45, 0.4, 0.3):
        q = m1 / (1 - m1)
        out.append(("m1", m1, ensemble(n, 700 + int(m1 * 100), q=(q, q), omega0=(0.00395, 0.00395))))
    return out


def states(n: int, seed: int, omega_range: tuple = (0.003, 0.2)) -> dict:
    """n random points of the state space, for checking right-hand sides point by point: q = m1/m2
    log-uniform in [1, 10], M omega log-uniform in omega_range (default [0.003, 0.2]), spin vectors of
    isotropic direction and magnitude uniform in [0, m_i^2], L-hat isotropic.  Returns m1, m2 (n,) and
    y (10, n), component-major (omega, S1, S2, L-hat)."""
    u = _uniforms(seed, (9, n))
    qv = np.exp(u[0] * np.log(10.0))
    m1 = qv / (1.0 + qv)
    m2 = 1.0 / (1.0 + qv)
    y = np.empty((10, n))
    lo, hi = omega_range
    y[0] = lo * np.exp(u[1] * np.log(hi / lo))
    y[1:4] = _isotropic(u[2], u[3]) * (u[4] * m1 * m1)
    y[4:7] = _isotropic(u[5], u[6]) * (u[7] * m2 * m2)
    y[7:10] = _isotropic(u[8], _uniforms(seed + 1, (n,)))
    return {"m1": m1, "m2": m2, "y": y}


def subsample(n_total: int, k: int, seed: int) -> np.ndarray:
    """k distinct sorted indices of range(n_total), seeded."""
    u = _uniforms(seed, (n_total,))
    return np.sort(np.argsort(u, kind="stable")[:k])


def take(ens: dict, idx: np.ndarray) -> dict:
    return {key: np.ascontiguousarray(v[..., idx]) for key, v in ens.items()}
