"""Initial order-parameter fields for the FP64 oracle (TEST INFRASTRUCTURE ONLY).

Restated from their definitions; shares no code with the CUDA path.

* BPII seed: the simple-cubic O2 structure of the blue-phase literature the
  paper cites for its initial states (Sec. 3: "BPII structure, previously
  equilibrated").  With amplitude A and wavenumber 2 q0:
    Q_xx = A[cos 2q0z - cos 2q0y], Q_yy = A[cos 2q0x - cos 2q0z],
    Q_zz = A[cos 2q0y - cos 2q0x], Q_xy = A sin 2q0z, Q_xz = A sin 2q0y,
    Q_yz = A sin 2q0x.
  Its handedness is the one favoured by the chiral term of Eq. (free_energy)
  with q0 > 0 (pinned in the tests by comparing with the mirror image).
* Cholesteric helix: Q = S (n n - I/3) with n rotating about the helix axis,
  n = (0, cos q0 x, sin q0 x) for axis x, (sin q0 y, 0, cos q0 y) for y,
  (cos q0 z, sin q0 z, 0) for z.
* Noise: U[-amp, amp) added to each of the five independent components
  [xx, xy, xz, yy, yz] (Q_zz = -Q_xx - Q_yy), drawn from the k-th output of a
  SplitMix64 generator seeded with ``seed`` (Steele, Lea, Flood, OOPSLA 2014),
  k = 5 * site + component, site = (z * Ny + y) * Nx + x; the 64-bit output z
  maps to the double (z >> 11) * 2^-53 in [0, 1).
"""

from __future__ import annotations

import numpy as np

from .lbq import q5_to_q9

_MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, k: int) -> int:
    """k-th output (k = 0, 1, ...) of SplitMix64 seeded with ``seed``
    (Python integers, for single values)."""
    z = (seed + (k + 1) * GOLDEN) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def splitmix64_array(seed: int, k: np.ndarray) -> np.ndarray:
    """Vectorised :func:`splitmix64` over an array of counters (uint64 wraparound)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (k.astype(np.uint64) + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, k: np.ndarray) -> np.ndarray:
    return (splitmix64_array(seed, k) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def _coords(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def noise5(shape, amp: float, seed: int) -> np.ndarray:
    """q5-layout noise [5, z, y, x], U[-amp, amp)."""
    n = int(np.prod(shape))
    site = np.arange(n, dtype=np.uint64)
    out = np.empty((5, n))
    for c in range(5):
        out[c] = amp * (2.0 * uniform01(seed, site * np.uint64(5) + np.uint64(c)) - 1.0)
    return out.reshape((5,) + tuple(shape))


def bpii5(shape, q0: float, A: float) -> np.ndarray:
    x, y, z = _coords(shape)
    k = 2.0 * q0
    xx = A * (np.cos(k * z) - np.cos(k * y))
    yy = A * (np.cos(k * x) - np.cos(k * z))
    return np.stack([xx, A * np.sin(k * z), A * np.sin(k * y), yy, A * np.sin(k * x)])


def director_helix(shape, q0: float, axis: str) -> np.ndarray:
    x, y, z = _coords(shape)
    if axis == "x":
        n = (np.zeros_like(x), np.cos(q0 * x), np.sin(q0 * x))
    elif axis == "y":
        n = (np.sin(q0 * y), np.zeros_like(y), np.cos(q0 * y))
    elif axis == "z":
        n = (np.cos(q0 * z), np.sin(q0 * z), np.zeros_like(z))
    else:
        raise ValueError(axis)
    return np.stack(n, axis=-1)


def cholesteric5(shape, q0: float, S: float, axis: str) -> np.ndarray:
    n = director_helix(shape, q0, axis)
    Q = S * (np.einsum("...a,...b->...ab", n, n) - np.eye(3) / 3.0)
    return np.stack([Q[..., 0, 0], Q[..., 0, 1], Q[..., 0, 2], Q[..., 1, 1], Q[..., 1, 2]])


def s_eq(gamma: float) -> float:
    """Uniaxial bulk equilibrium order 1/4 + 3/4 sqrt(1 - 8/(3 gamma)) of the
    bulk part of Eq. (free_energy)."""
    return 0.25 + 0.75 * np.sqrt(1.0 - 8.0 / (3.0 * gamma))


# kinds, numbered as at the library boundary
BPII, CHOL_X, CHOL_Y, CHOL_Z, ISO_NOISE, SLAB_BPII_IN_CHOL, SLAB_BPII_IN_ISO, SLAB_BPII_IN_CHOL_Z = range(8)


def init_q5(shape, kind: int, q0: float, amplitude: float, noise: float, seed: int,
            z0: int = 0, s_helix: float = 0.0) -> np.ndarray:
    """Initial Q in q5 layout.  amplitude is A for BPII, S for the helices and
    unused for ISO_NOISE (zero mean); the slab kinds put BPII with
    A = amplitude for z < z0 and, elsewhere, an x-helix (SLAB_BPII_IN_CHOL) or a
    z-helix (SLAB_BPII_IN_CHOL_Z) with S = s_helix, or the isotropic phase
    (SLAB_BPII_IN_ISO, noise only)."""
    shape = tuple(int(v) for v in shape)
    if kind == BPII:
        q = bpii5(shape, q0, amplitude)
    elif kind in (CHOL_X, CHOL_Y, CHOL_Z):
        q = cholesteric5(shape, q0, amplitude, "xyz"[kind - CHOL_X])
    elif kind == ISO_NOISE:
        q = np.zeros((5,) + shape)
    elif kind in (SLAB_BPII_IN_CHOL, SLAB_BPII_IN_ISO, SLAB_BPII_IN_CHOL_Z):
        # Sec. 3: a BPII seed slab next to a cholesteric (helix in the wall
        # plane, along x, or normal to it, along z) or an isotropic phase
        zz = np.arange(shape[0])[None, :, None, None]
        if kind == SLAB_BPII_IN_ISO:
            other = np.zeros((5,) + shape)
        else:
            other = cholesteric5(shape, q0, s_helix, "x" if kind == SLAB_BPII_IN_CHOL else "z")
        q = np.where(zz < z0, bpii5(shape, q0, amplitude), other)
    else:
        raise ValueError(kind)
    if noise != 0.0:
        q = q + noise5(shape, noise, seed)
    return q


def init_q9(shape, kind, q0, amplitude, noise, seed, z0=0, s_helix=0.0) -> np.ndarray:
    return q5_to_q9(init_q5(shape, kind, q0, amplitude, noise, seed, z0, s_helix))
