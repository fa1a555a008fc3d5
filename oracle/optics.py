"""FP64 CPU oracle of the polarised-light texture (TEST INFRASTRUCTURE ONLY).

Restated from the paper's Sec. 2.3 (rendering of the optical pattern); shares
no code with the CUDA path.  Light travels along +z through the lattice
planes k = 0 .. Nz-1, each plane a uniaxial retarder of thickness h:

* director d(r): unit eigenvector of the largest eigenvalue q(r) of Q(r)
  (q is the local scalar order parameter of the section);
* alpha = arccos(d_z), beta = arctan(d_x / d_y) (taken as atan2(d_x, d_y)),
  delta = (2 pi q h / lambda) (n_o n_e / sqrt(n_o^2 sin^2 alpha + n_e^2 cos^2 alpha) - n_o);
* Mueller matrix of a plane, the section's first display equation, with
  c_b = cos 2 beta, s_b = sin 2 beta, c_d = cos delta, s_d = sin delta;
* polariser at angle phi, the section's second matrix with the double angle
  (cos 2 phi, sin 2 phi in place of cos phi, sin phi: the standard Mueller
  matrix of a linear polariser at angle phi; as printed, phi_out = pi / 2
  would be an analyser at 45 degrees, which is not the crossed set-up the
  text describes and would not extinguish an isotropic sample);
  polariser phi_in = 0, analyser phi_out = pi / 2;
* S_out = P_out M(Nz-1) ... M(0) P_in S_in per column (x, y), the first plane
  met by the beam applied first; S_in = (1, 0, 0, 0) (unpolarised light);
* the image is the weighted sum of S_out[0] over lambda = 16, 18, 20 lattice
  units with weights 0.2, 0.6, 0.2; n_o = 1.5, n_e = 2.0, h = 1.

The per-column product is done plainly, one 4x4 matrix at a time.
"""

from __future__ import annotations

import numpy as np

LAMBDAS = (16.0, 18.0, 20.0)
WEIGHTS = (0.2, 0.6, 0.2)
N_O, N_E = 1.5, 2.0


def director_and_order(Q9: np.ndarray):
    """Largest eigenvalue q and its unit eigenvector d of each symmetric 3x3 Q
    (library eigen-solver; Q9 [..., 3, 3])."""
    w, v = np.linalg.eigh(Q9)
    return w[..., 2], v[..., :, 2]


def retardance(d: np.ndarray, q: np.ndarray, lam: float, h: float = 1.0,
               n_o: float = N_O, n_e: float = N_E) -> np.ndarray:
    """delta of a plane: optical path difference of the extraordinary ray."""
    cos2 = d[..., 2] ** 2
    sin2 = 1.0 - cos2
    n_eff = n_o * n_e / np.sqrt(n_o ** 2 * sin2 + n_e ** 2 * cos2)
    return 2.0 * np.pi * q * h / lam * (n_eff - n_o)


def mueller(beta: float, delta: float) -> np.ndarray:
    """Mueller matrix of one retarding plane (Sec. 2.3, first matrix)."""
    cb, sb = np.cos(2 * beta), np.sin(2 * beta)
    cd, sd = np.cos(delta), np.sin(delta)
    return np.array([
        [1.0, 0.0, 0.0, 0.0],
        [0.0, cb * cb + sb * sb * cd, cb * sb * (1 - cd), -sb * sd],
        [0.0, cb * sb * (1 - cd), sb * sb + cb * cb * cd, cb * sd],
        [0.0, sb * sd, -cb * sd, cd]])


def polariser(phi: float) -> np.ndarray:
    """Mueller matrix of an ideal linear polariser at angle phi (Sec. 2.3, second
    matrix, read with the double angle 2 phi)."""
    c, s = np.cos(2 * phi), np.sin(2 * phi)
    return 0.5 * np.array([
        [1.0, c, s, 0.0],
        [c, c * c, c * s, 0.0],
        [s, s * c, s * s, 0.0],
        [0.0, 0.0, 0.0, 0.0]])


def column_s0(d_col: np.ndarray, q_col: np.ndarray, lam: float, phi_in: float = 0.0,
              phi_out: float = np.pi / 2) -> float:
    """S_out[0] of one column: d_col [Nz, 3], q_col [Nz]."""
    S = polariser(phi_in) @ np.array([1.0, 0.0, 0.0, 0.0])
    for k in range(len(q_col)):
        beta = np.arctan2(d_col[k, 0], d_col[k, 1])
        delta = retardance(d_col[k], q_col[k], lam)
        S = mueller(beta, delta) @ S
    return float((polariser(phi_out) @ S)[0])


def texture(Q9: np.ndarray, lambdas=LAMBDAS, weights=WEIGHTS) -> np.ndarray:
    """Weighted transmitted intensity image [Ny, Nx] of Q9 [Nz, Ny, Nx, 3, 3]."""
    q, d = director_and_order(Q9)
    nz, ny, nx = q.shape
    img = np.zeros((ny, nx))
    for y in range(ny):
        for x in range(nx):
            img[y, x] = sum(w * column_s0(d[:, y, x], q[:, y, x], lam) for lam, w in zip(lambdas, weights))
    return img
