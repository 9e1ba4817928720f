"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic. The workloads stand in for the SK spin-glass instances the
paper measures on (Fig. 3 and Fig. 4: Sherrington-Kirkpatrick couplings with
standard-normal parameters), whose data set is not available here.

Draw order for one SK instance (numpy PCG64 ``default_rng``): first J as an
n x n matrix of standard normals divided by sqrt(n), of which only the strict
upper triangle is kept (the rest is zeroed), then the n fields h.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def sk_instance(n: int, seed: int, h_dist: str = "normal"):
    """Seeded SK couplings: J_ij ~ N(0,1)/sqrt(n) for i<j, h_i ~ N(0,1) or U(-1,1)."""
    rng = np.random.default_rng(seed)
    J = rng.standard_normal((n, n)) / np.sqrt(n)
    J = np.triu(J, k=1)
    if h_dist == "normal":
        h = rng.standard_normal(n)
    elif h_dist == "uniform":
        h = rng.uniform(-1.0, 1.0, n)
    else:
        raise ValueError(h_dist)
    return np.ascontiguousarray(h), np.ascontiguousarray(J)


def uniform_state(n: int, dtype=np.complex128) -> np.ndarray:
    """psi0 = 2^(-n/2) on every basis state."""
    return np.full(1 << n, 2.0 ** (-n / 2.0), dtype=dtype)


def random_state(n: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """A normalised random complex state (real and imaginary parts standard normal)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    v /= np.linalg.norm(v)
    return v.astype(dtype)


def basis_state(n: int, z: int = 0, dtype=np.complex128) -> np.ndarray:
    v = np.zeros(1 << n, dtype=dtype)
    v[z] = 1.0
    return v


@dataclass
class Single:
    name: str
    n: int
    h: np.ndarray
    J: np.ndarray
    gamma: float
    t: float


def config_n10() -> Single:
    """n=10, seed 0, h ~ N(0,1), gamma = 1, t = 1 (tol 1e-12, complex128)."""
    h, J = sk_instance(10, 0, "normal")
    return Single("sk_n10_g1.0_t1", 10, h, J, 1.0, 1.0)


def config_n24() -> Single:
    """n=24, seed 0, h ~ N(0,1), gamma = 0.8, t = 10."""
    h, J = sk_instance(24, 0, "normal")
    return Single("sk_n24_g0.8_t10", 24, h, J, 0.8, 10.0)


def config_n30() -> Single:
    """n=30, seed 0, h ~ U(-1,1), gamma = 1, t = 20."""
    h, J = sk_instance(30, 0, "uniform")
    return Single("sk_n30_g1.0_t20", 30, h, J, 1.0, 20.0)


def config_family(n: int, gamma: float, t: float, seed: int = 0, h_dist: str = "uniform") -> Single:
    """Same SK family at another size (used for bounded samples and parity sizes)."""
    h, J = sk_instance(n, seed, h_dist)
    return Single(f"sk_n{n}_g{gamma}_t{t}_s{seed}", n, h, J, gamma, t)


@dataclass
class Batch:
    ns: list
    hs: list
    Js: list
    gammas: np.ndarray
    ts: np.ndarray


def config_batch(B: int = 512, n_lo: int = 12, n_hi: int = 20, seed: int = 0) -> Batch:
    """Independent instances: master rng draws (n ~ U{n_lo..n_hi}, gamma ~ U(0.2,2),
    t ~ U(0.5,20)) per instance in that order; instance i's couplings come from
    default_rng(1000 + i) with h ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    ns, gs, ts = [], [], []
    for _ in range(B):
        ns.append(int(rng.integers(n_lo, n_hi + 1)))
        gs.append(float(rng.uniform(0.2, 2.0)))
        ts.append(float(rng.uniform(0.5, 20.0)))
    hs, Js = [], []
    for i, n in enumerate(ns):
        h, J = sk_instance(n, 1000 + i, "normal")
        hs.append(h)
        Js.append(J)
    return Batch(ns, hs, Js, np.array(gs), np.array(ts))


@dataclass
class Anneal:
    n: int
    h: np.ndarray
    J: np.ndarray
    gammas: np.ndarray
    ts: np.ndarray


def config_anneal(n: int = 22, S: int = 64, seed: int = 0) -> Anneal:
    """Piecewise-constant schedule: gamma_s = linspace(2.0, 0.05, S) + N(0, 0.05)
    jitter from default_rng(1), t_s = 0.5; SK couplings from default_rng(seed)."""
    h, J = sk_instance(n, seed, "normal")
    gam = np.linspace(2.0, 0.05, S) + np.random.default_rng(1).normal(0.0, 0.05, S)
    return Anneal(n, h, J, gam, np.full(S, 0.5))


def monomial_polynomial(degree: int = 50, seed: int = 0) -> np.ndarray:
    """Coefficients a_0..a_degree of a polynomial in the monomial basis, standard normal
    draws from default_rng(seed) (the random polynomials of the paper's Fig. 4 and
    Fig. 6 runtime workloads)."""
    return np.random.default_rng(seed).standard_normal(degree + 1)
