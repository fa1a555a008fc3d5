"""Pins of the energy exactly as printed (L2 = 0) and of a general L2: the
printed chiral square equals the one-constant energy minus (K/2)(div Q)^2 up
to a divergence, which the lattice form keeps with a central-difference
divergence whose exact gradient enters H."""

import numpy as np
import pytest

from oracle import initial, lbq
from paper_0901_3293_gb300 import synth


def fourier_field(shape, seed, kmax=2):
    """A smooth periodic symmetric traceless field from a few Fourier modes,
    with its exact spatial derivatives (lattice units)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    Q = np.zeros(shape + (3, 3))
    dQ = np.zeros(shape + (3, 3, 3))  # [..., g, a, b] = d_g Q_ab
    for _ in range(4):
        kv = np.array([rng.integers(-kmax, kmax + 1) * 2 * np.pi / nx, rng.integers(-kmax, kmax + 1) * 2 * np.pi / ny,
                       rng.integers(-kmax, kmax + 1) * 2 * np.pi / nz])
        A = rng.normal(size=(3, 3)) * 0.1
        A = A + A.T
        A -= np.trace(A) / 3 * np.eye(3)
        ph = rng.uniform(0, 2 * np.pi)
        arg = kv[0] * x + kv[1] * y + kv[2] * z + ph
        Q += np.cos(arg)[..., None, None] * A
        dQ += (-np.sin(arg))[..., None, None, None] * kv[:, None, None] * A[None]
    return Q, dQ


def _printed_vs_lattice(N):
    p = lbq.Params(L2=0.0, q0=2 * np.pi / 32)
    Q, dQ = fourier_field((N, N, N), 1, kmax=1)
    epsdQ = np.einsum("agd,...gdb->...ab", lbq.EPS, dQ)
    printed = 0.5 * p.K * np.sum((epsdQ + 2 * p.q0 * Q) ** 2)
    bulk = float(np.sum(lbq.bulk_free_energy_density(Q, p)))
    lattice = lbq.free_energy(Q, p) - bulk
    onec = lbq.free_energy(Q, p.with_(L2=None)) - bulk
    div = np.einsum("...bab->...a", dQ)
    return printed, lattice, onec - lattice, 0.5 * p.K * np.sum(div * div)


def test_printed_energy_matches_the_continuum_square():
    """sum_x (K/2)(eps dQ + 2 q0 Q)^2 from exact derivatives of a smooth field
    equals the lattice gradient + chiral energy with L2 = 0, and the
    one-constant energy exceeds it by (K/2) sum (div Q)^2, both converging at
    second order in the lattice spacing."""
    pr16, la16, d16, dv16 = _printed_vs_lattice(16)
    pr32, la32, d32, dv32 = _printed_vs_lattice(32)
    assert abs(la32 - pr32) < 2e-3 * abs(pr32)
    assert abs(d32 - dv32) < 0.02 * dv32
    e16, e32 = abs(d16 / dv16 - 1), abs(d32 / dv32 - 1)
    assert e16 / e32 > 3.5


@pytest.mark.parametrize("L2", [0.0, 0.003])
def test_molecular_field_is_exact_gradient_with_l2(L2):
    p = lbq.Params(L2=L2)
    shape = (4, 5, 3)
    q5 = synth.random_q5(shape, 0.2, 41)
    H = lbq.molecular_field(lbq.q5_to_q9(q5), p)
    h = 1e-6
    comp_to_H = {0: lambda M: -(M[0, 0] - M[2, 2]), 1: lambda M: -2 * M[0, 1],
                 2: lambda M: -2 * M[0, 2], 3: lambda M: -(M[1, 1] - M[2, 2]),
                 4: lambda M: -2 * M[1, 2]}
    rng = np.random.default_rng(3)
    for _ in range(5):
        z, y, x = (int(rng.integers(0, n)) for n in shape)
        for c in range(5):
            qp, qm = q5.copy(), q5.copy()
            qp[c, z, y, x] += h
            qm[c, z, y, x] -= h
            dF = (lbq.free_energy(lbq.q5_to_q9(qp), p) - lbq.free_energy(lbq.q5_to_q9(qm), p)) / (2 * h)
            assert abs(dF - comp_to_H[c](H[z, y, x])) < 1e-8


def test_helix_is_divergence_free_so_l2_drops_out():
    p0, p1 = lbq.Params(), lbq.Params(L2=0.0)
    for axis, kind in (("x", initial.CHOL_X), ("y", initial.CHOL_Y), ("z", initial.CHOL_Z)):
        Q = initial.init_q9((16, 16, 16), kind, p0.q0, 0.4, 0.0, 0)
        assert np.abs(lbq.divergence(Q)).max() < 1e-15
        assert abs(lbq.free_energy(Q, p0) - lbq.free_energy(Q, p1)) < 1e-12
        assert np.abs(lbq.molecular_field(Q, p0) - lbq.molecular_field(Q, p1)).max() < 1e-15


def test_free_energy_decreases_with_printed_energy_flow_off():
    p = lbq.Params(L2=0.0, flow_on=False)
    shape = (6, 6, 6)
    Q = lbq.q5_to_q9(synth.smooth_q5(shape, 0.3, 5) + synth.random_q5(shape, 0.05, 6))
    f = np.zeros(shape + (15,))
    F = [lbq.free_energy(Q, p)]
    for _ in range(200):
        f, Q = lbq.step(f, Q, p)
        F.append(lbq.free_energy(Q, p))
    assert np.all(np.diff(F) <= 1e-14 * abs(F[0])) and F[-1] < F[0]
