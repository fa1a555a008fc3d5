"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Holds no arithmetic of the method: only random numbers and parameter draws.
Every draw is keyed by an explicit seed (numpy PCG64 via ``default_rng``).
"""

from __future__ import annotations

import numpy as np

BASE_SEED = 20090119


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def random_q5(shape, amp: float, seed: int) -> np.ndarray:
    """Five independent Q components [xx, xy, xz, yy, yz] at every site of a
    (nz, ny, nx) lattice, uniform in [-amp, amp)."""
    return rng(seed).uniform(-amp, amp, size=(5,) + tuple(shape))


def smooth_q5(shape, amp: float, seed: int, modes: int = 3) -> np.ndarray:
    """A sum of a few random lattice Fourier modes per component (smooth field)."""
    g = rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.zeros((5,) + tuple(shape))
    for c in range(5):
        for _ in range(modes):
            kx = 2 * np.pi * g.integers(0, max(nx, 1)) / nx
            ky = 2 * np.pi * g.integers(0, max(ny, 1)) / ny
            kz = 2 * np.pi * g.integers(0, max(nz, 1)) / nz
            out[c] += g.uniform(-1, 1) * np.cos(kx * x + ky * y + kz * z + g.uniform(0, 2 * np.pi))
    return amp * out / modes


def random_velocity(shape, amp: float, seed: int) -> np.ndarray:
    """u[3, z, y, x] uniform in [-amp, amp)."""
    return rng(seed).uniform(-amp, amp, size=(3,) + tuple(shape))


def random_moment_inputs(n: int, seed: int):
    """rho in [0.5, 1.5), u in [-0.1, 0.1)^3, symmetric traceless sigma with
    entries O(1e-2), b in [-1e-2, 1e-2)^3: n independent samples."""
    g = rng(seed)
    rho = g.uniform(0.5, 1.5, size=n)
    u = g.uniform(-0.1, 0.1, size=(n, 3))
    s = g.uniform(-1e-2, 1e-2, size=(n, 3, 3))
    s = 0.5 * (s + np.swapaxes(s, 1, 2))
    s -= np.trace(s, axis1=1, axis2=2)[:, None, None] * np.eye(3) / 3.0
    b = g.uniform(-1e-2, 1e-2, size=(n, 3))
    return rho, u, s, b


def random_distributions(shape, seed: int, base: np.ndarray | None = None,
                         amp: float = 1e-3) -> np.ndarray:
    """f[15, z, y, x]: ``base`` (per-direction weights, default the rest-state
    weights of a unit-density D3Q15 fluid at T = 1/3) plus uniform noise."""
    if base is None:
        base = np.array([8 / 15] + [1 / 30] * 6 + [1 / 30] * 8)
    g = rng(seed)
    return base[:, None, None, None] + g.uniform(-amp, amp, size=(15,) + tuple(shape))


def replica_sweep(R: int, seed: int = BASE_SEED):
    """Per-replica draws of a chirality/temperature sweep: replica r gets
    dims 32^3 (r even) or 48^3 (r odd), kappa ~ U[0.3, 2], tau ~ U[-1, 0.5],
    initial kind r mod 3 (0 BPII, 1 cholesteric along z, 2 isotropic noise)
    and seed + r as its noise seed."""
    out = []
    for r in range(R):
        g = rng(seed + r)
        n = 32 if r % 2 == 0 else 48
        out.append({
            "dims": (n, n, n),
            "kappa": float(g.uniform(0.3, 2.0)),
            "tau": float(g.uniform(-1.0, 0.5)),
            "kind": r % 3,
            "seed": seed + r,
        })
    return out
