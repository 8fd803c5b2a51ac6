"""Seeded synthetic inputs shared by the CUDA path (tests, bench) and the oracle.

This module holds none of the solver's arithmetic: it only draws seeded random
numbers and evaluates given right-hand-side functions at coordinates the caller
supplies (each side computes its own node coordinates and its own weak
right-hand side from these values).

Workload shapes follow the paper's experiments (Section 4): periodic boxes,
equidistant meshes, a smooth periodic manufactured solution, random initial
guesses in [-1, 1], and the random right-hand sides and request streams of the
synthetic benchmark configurations.
"""
import math

import numpy as np


def gaussian(n, seed, out=None):
    """n i.i.d. N(0, 1) values (nodal right-hand side, element-blocked order);
    written into `out` (float64, n values) when given."""
    rng = np.random.default_rng(seed)
    if out is None:
        return rng.standard_normal(int(n))
    assert out.shape == (int(n),) and out.dtype == np.float64
    return rng.standard_normal(out=out)


def uniform_guess(n, seed):
    """n i.i.d. U[-1, 1] values: the random initial guess of Section 4."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, int(n))


def sines(x, y, z, lengths=(1.0, 1.0, 1.0)):
    """Manufactured periodic solution u = sin(2 pi x/lx) sin(2 pi y/ly) sin(2 pi z/lz)
    and its source f = -lap u.  Returns (u, f) at the given points."""
    lx, ly, lz = lengths
    u = np.sin(2 * math.pi * x / lx) * np.sin(2 * math.pi * y / ly) * np.sin(2 * math.pi * z / lz)
    k2 = (2 * math.pi) ** 2 * (1 / lx ** 2 + 1 / ly ** 2 + 1 / lz ** 2)
    return u, k2 * u


def fourier_modes(seed, n_modes=8, kmax=8):
    """Random periodic Fourier modes: integer wave vectors k with |k|_inf <= kmax
    (k != 0), amplitudes a ~ N(0, 1) and phases phi ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if np.any(k != 0):
            ks.append(k)
    a = rng.standard_normal(n_modes)
    phi = rng.uniform(0.0, 2 * math.pi, n_modes)
    return np.array(ks), a, phi


def eval_fourier(modes, x, y, z, lengths=(1.0, 1.0, 1.0)):
    """sum_m a_m sin(2 pi (k_m . (x/lx, y/ly, z/lz)) + phi_m) at the given points."""
    ks, a, phi = modes
    lx, ly, lz = lengths
    out = np.zeros_like(np.asarray(x, dtype=np.float64))
    for k, am, pm in zip(ks, a, phi):
        out += am * np.sin(2 * math.pi * (k[0] * x / lx + k[1] * y / ly + k[2] * z / lz) + pm)
    return out


def request_stream(seed, n_requests=512, rate=200.0, sizes=(4, 8, 16, 24, 32), orders=(2, 4, 8, 16),
                   aspect=(1.0, 8.0)):
    """Serving workload: Poisson arrivals at ``rate`` per second; each request a
    periodic box [0, AR] x [0, 1] x [0, 1] with n^3 elements, order P and a
    Gaussian right-hand-side seed.  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    out = []
    for i in range(n_requests):
        out.append({
            "arrival": float(t[i]),
            "n": int(rng.choice(sizes)),
            "P": int(rng.choice(orders)),
            "aspect": float(rng.uniform(*aspect)),
            "seed": int(rng.integers(0, 2 ** 31 - 1)),
        })
    return out
