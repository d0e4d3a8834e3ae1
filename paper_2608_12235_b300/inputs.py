"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds input synthesis only -- none of the method's arithmetic.
Diameters are the deterministic equal-probability inverse-CDF quantiles at
cumulative probabilities (i + 1/2)/N (Sec. II) of the paper's three
distribution families:

* truncated lognormal, Eq. lognormal and Eq. S (Sec. III.A):
  D = exp(alpha z), |z| <= a, S = exp(2 a alpha);
* truncated power law (Sec. III.B): P(D) ~ D^p on [1, S];
* truncated Weibull, Eq. weibull (Sec. III.C): P(D) ~ (D/lambda)^(k-1)
  exp(-(D/lambda)^k) on [1/sqrt(S), sqrt(S)], lambda = sqrt(S).

Positions are not drawn here: both sides generate them from the seed with
SplitMix64 (each side its own implementation of the published generator).
"""
from __future__ import annotations

import numpy as np
from scipy.special import ndtr, ndtri


def _u(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def lognormal(n: int, sigma_ln: float, S: float) -> np.ndarray:
    """Truncated lognormal quantiles with width alpha = sigma_ln and truncation
    a = ln(S) / (2 alpha), so that D_max / D_min -> S (Eq. S)."""
    alpha = float(sigma_ln)
    a = np.log(S) / (2.0 * alpha)
    lo, hi = ndtr(-a), ndtr(a)
    z = ndtri(lo + _u(n) * (hi - lo))
    return np.exp(alpha * z)


def power_law(n: int, p: float, S: float) -> np.ndarray:
    """Truncated power law P(D) ~ D^p on [1, S] (p != -1)."""
    q = p + 1.0
    return (1.0 + _u(n) * (S ** q - 1.0)) ** (1.0 / q)


def weibull(n: int, k: float, S: float) -> np.ndarray:
    """Truncated Weibull on [1/sqrt(S), sqrt(S)] with scale lambda = sqrt(S)."""
    lam = np.sqrt(S)
    a, b = 1.0 / np.sqrt(S), np.sqrt(S)
    ta, tb = np.exp(-((a / lam) ** k)), np.exp(-((b / lam) ** k))
    surv = ta - _u(n) * (ta - tb)
    return lam * (-np.log(surv)) ** (1.0 / k)


def monodisperse(n: int) -> np.ndarray:
    return np.ones(n)


# Named workloads (sizes and shapes of the paper's 3D periodic tests).
def workload(name: str) -> dict:
    """Diameters and run settings of a named synthetic workload."""
    if name == "lognormal-n1e3-s10":
        return dict(D0=lognormal(1000, 0.5, 10.0), seed=0, phi0=0.05)
    if name == "powerlaw-n1e5-s20":
        return dict(D0=power_law(100_000, -3.0, 20.0), seed=0, phi0=0.05)
    if name == "weibull-n2e5-s100":
        return dict(D0=weibull(200_000, 1.5, 100.0), seed=0, phi0=0.6)
    if name == "lognormal-n1e6-s5e5":
        return dict(D0=lognormal(1_000_000, 2.0, 5e5), seed=0, phi0=0.05)
    raise KeyError(name)


def batch_specs(count: int = 64, master_seed: int = 0, n_lo: float = 1e3, n_hi: float = 1e5):
    """Independent packings of uneven size: N log-uniform in [n_lo, n_hi],
    lognormal sigma_ln uniform in [0.2, 1.0], S log-uniform in [5, 200]."""
    rng = np.random.Generator(np.random.PCG64(master_seed))
    out = []
    for b in range(count):
        n = int(10 ** rng.uniform(np.log10(n_lo), np.log10(n_hi)))
        sig = float(rng.uniform(0.2, 1.0))
        S = float(10 ** rng.uniform(np.log10(5.0), np.log10(200.0)))
        seed = int(rng.integers(0, 2**63 - 1))
        out.append(dict(N=n, sigma_ln=sig, S=S, seed=seed, D0=lognormal(n, sig, S)))
    return out
