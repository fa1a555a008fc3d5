"""Pins of the oracle's solid walls in z (half-way bounce-back, strong Q
anchoring on ghost planes, no-slip ghost velocity)."""

import numpy as np
import pytest

from oracle import initial, lbq
from paper_0901_3293_gb300 import synth

PLANAR = (0.3 * 2 / 3, 0.0, 0.0, -0.3 / 3, 0.0)  # S (x x - I/3) with S = 0.3


def test_bond_form_equals_site_form_on_the_periodic_lattice():
    p = lbq.Params()
    for seed, shape in ((1, (5, 4, 6)), (2, (3, 7, 2))):
        Q = lbq.q5_to_q9(synth.smooth_q5(shape, 0.3, seed) + synth.random_q5(shape, 0.05, seed + 1))
        F_site = lbq.free_energy(Q, p)
        F_bond = lbq.free_energy_bonds(Q, p)
        assert abs(F_site - F_bond) < 1e-12 * max(1.0, abs(F_site))


@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 4, 4)])
def test_walled_molecular_field_is_exact_gradient(shape):
    """With fixed ghost planes the energy of every bond touching the lattice
    is a function of the interior Q only through those bonds, so H from the
    ghosted stencils is -dF/dQ exactly (brute force on every site of z = 0,
    z = Nz-1 and an interior plane)."""
    p = lbq.Params(walls_z=True, q_wall=PLANAR)
    q5 = synth.random_q5(shape, 0.2, 31)
    H = lbq.molecular_field(lbq.q5_to_q9(q5), p)
    h = 1e-6
    comp_to_H = {0: lambda M: -(M[0, 0] - M[2, 2]), 1: lambda M: -2 * M[0, 1],
                 2: lambda M: -2 * M[0, 2], 3: lambda M: -(M[1, 1] - M[2, 2]),
                 4: lambda M: -2 * M[1, 2]}
    nz, ny, nx = shape
    for z in (0, nz - 1, nz // 2):
        for (y, x) in ((0, 0), (ny - 1, nx // 2)):
            for c in range(5):
                qp, qm = q5.copy(), q5.copy()
                qp[c, z, y, x] += h
                qm[c, z, y, x] -= h
                dF = (lbq.free_energy(lbq.q5_to_q9(qp), p) - lbq.free_energy(lbq.q5_to_q9(qm), p)) / (2 * h)
                assert abs(dF - comp_to_H[c](H[z, y, x])) < 1e-8, (z, y, x, c)


def test_anchoring_enters_only_through_the_wall_planes():
    """Changing q_wall changes H on z = 0 and z = Nz-1 only."""
    shape = (5, 3, 4)
    Q = lbq.q5_to_q9(synth.random_q5(shape, 0.2, 3))
    H0 = lbq.molecular_field(Q, lbq.Params(walls_z=True))
    H1 = lbq.molecular_field(Q, lbq.Params(walls_z=True, q_wall=PLANAR))
    d = np.abs(H1 - H0).max(axis=(1, 2, 3, 4))
    assert d[0] > 1e-4 and d[-1] > 1e-4 and d[1:-1].max() == 0.0


def test_free_energy_decreases_with_walls_flow_off():
    p = lbq.Params(walls_z=True, q_wall=PLANAR, flow_on=False)
    shape = (8, 4, 4)
    Q = initial.init_q9(shape, initial.BPII, p.q0, 0.3, 1e-3, 5)
    f = np.zeros(shape + (15,))
    F = [lbq.free_energy(Q, p)]
    for _ in range(300):
        f, Q = lbq.step(f, Q, p)
        F.append(lbq.free_energy(Q, p))
    assert np.all(np.diff(F) <= 1e-14 * abs(F[0]))
    assert F[-1] < F[0]


def test_mass_conserved_and_symmetric_traceless_with_walls():
    p = lbq.Params(walls_z=True, q_wall=PLANAR)
    shape = (6, 4, 5)
    Q = lbq.q5_to_q9(synth.smooth_q5(shape, 0.3, 7) + synth.random_q5(shape, 0.01, 8))
    f = lbq.init_f_equilibrium(Q, p)
    m0, _ = lbq.totals(f)
    for _ in range(40):
        f, Q = lbq.step(f, Q, p)
    m1, _ = lbq.totals(f)
    assert abs(m1 - m0) < 1e-13 * m0
    assert np.abs(Q - np.swapaxes(Q, -1, -2)).max() < 1e-15
    assert np.abs(np.trace(Q, axis1=-2, axis2=-1)).max() < 1e-15


def test_coupled_step_with_walls_reduces_to_poiseuille_lb():
    """Q = 0, xi = 0 and a uniform external force: the coupled step with walls is
    the walled LB of the Poiseuille pin (Q stays 0, sigma = b_LC = 0)."""
    p = lbq.Params(walls_z=True, xi=0.0)
    shape = (8, 1, 1)
    g = np.zeros(shape + (3,))
    g[..., 0] = 1e-6
    Q = np.zeros(shape + (3, 3))
    f = lbq.init_f_equilibrium(Q, p)
    f2 = f.copy()
    for _ in range(50):
        f, Q = lbq.step(f, Q, p, b_ext=g)
        f2 = lbq.lb_step(f2, np.zeros(shape + (3, 3)), g, p.tau_f, walls_z=True)
    assert np.abs(Q).max() == 0.0
    assert np.abs(f - f2).max() < 1e-17


def test_walled_step_is_local():
    """One coupled step at a site depends on the state within 4 sites: a cube
    of 9 planes cut at a wall (with a second, artificial wall 5 or more planes
    away) or, away from the walls, a periodic 9^3 cube reproduces the full
    walled lattice's step at its sample site.  This is what the full-size
    sampled parity of the GPU path rests on."""
    p = lbq.Params(q0=2 * np.pi / 32)
    pw = lbq.Params(q0=2 * np.pi / 32, walls_z=True, q_wall=PLANAR)
    nz, n, r = 14, 9, 4
    shape = (nz, n, n)
    q5 = synth.smooth_q5(shape, 0.3, 1) + synth.random_q5(shape, 1e-2, 2)
    f15 = synth.random_distributions(shape, 3, amp=2e-3)
    f, Q = lbq.step(lbq.f_from_soa(f15), lbq.q5_to_q9(q5), pw)
    qf, uf = lbq.q9_to_q5(Q), np.moveaxis(lbq.moments(f)[1], -1, 0)
    for z, y, x in [(0, 3, 7), (2, 0, 0), (4, 8, 1), (6, 4, 4), (9, 2, 5), (11, 6, 8), (13, 1, 3)]:
        iy, ix = (np.arange(c - r, c + r + 1) % n for c in (y, x))
        if z < r:
            iz, cz, pp = np.arange(0, 2 * r + 1), z, pw
        elif z > nz - 1 - r:
            iz, cz, pp = np.arange(nz - 1 - 2 * r, nz), z - (nz - 1 - 2 * r), pw
        else:
            iz, cz, pp = np.arange(z - r, z + r + 1), r, p
        cube = np.ix_(iz, iy, ix)
        fo, Qo = lbq.step(lbq.f_from_soa(f15[(slice(None),) + cube]), lbq.q5_to_q9(q5[(slice(None),) + cube]), pp)
        assert np.abs(qf[:, z, y, x] - lbq.q9_to_q5(Qo)[:, cz, r, r]).max() < 1e-15
        assert np.abs(uf[:, z, y, x] - np.moveaxis(lbq.moments(fo)[1], -1, 0)[:, cz, r, r]).max() < 1e-15
