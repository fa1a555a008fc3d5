"""Pins of the polarised-light texture oracle (Sec. 2.3): closed forms of
crossed polarisers, extinction cases, and an independent Jones-calculus
computation of twisted stacks."""

import numpy as np

from oracle import lbq, optics


def uniaxial(n, S):
    n = np.asarray(n, dtype=float)
    n = n / np.linalg.norm(n)
    return S * (np.outer(n, n) - np.eye(3) / 3.0)


def test_director_and_order_of_uniaxial_q():
    rng = np.random.default_rng(0)
    for _ in range(5):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        q, d = optics.director_and_order(uniaxial(n, 0.4))
        assert abs(q - 2 * 0.4 / 3) < 1e-14
        assert abs(abs(d @ n) - 1.0) < 1e-12


def test_isotropic_and_homeotropic_columns_are_dark():
    Q = np.zeros((6, 2, 3, 3, 3))
    assert np.abs(optics.texture(Q)).max() < 1e-15
    Q[:] = uniaxial([0, 0, 1], 0.5)  # director along the beam: no retardation
    assert np.abs(optics.texture(Q)).max() < 1e-15


def test_uniform_planar_slab_matches_crossed_polariser_formula():
    """In-plane director at angle t to x, N planes: transmitted fraction of
    unpolarised light I = (1/2) sin^2(2 t) sin^2(Gamma / 2), Gamma = N delta,
    delta = 2 pi q (n_e - n_o) / lambda."""
    N, S = 7, 0.3
    q = 2 * S / 3
    for t in (0.0, np.pi / 8, np.pi / 4, np.pi / 3, 0.9):
        Q = np.broadcast_to(uniaxial([np.cos(t), np.sin(t), 0], S), (N, 1, 1, 3, 3)).copy()
        for lam in optics.LAMBDAS:
            got = optics.texture(Q, lambdas=(lam,), weights=(1.0,))[0, 0]
            Gamma = N * 2 * np.pi * q * (optics.N_E - optics.N_O) / lam
            want = 0.5 * np.sin(2 * t) ** 2 * np.sin(Gamma / 2) ** 2
            assert abs(got - want) < 1e-13, (t, lam, got, want)


def test_tilted_director_uses_the_effective_index():
    """Director tilted by alpha from the beam: delta uses n_o n_e / sqrt(n_o^2 sin^2 + n_e^2 cos^2) - n_o."""
    a, S, N, lam = 0.6, 0.5, 5, 18.0
    n = [np.sin(a) * np.cos(np.pi / 4), np.sin(a) * np.sin(np.pi / 4), np.cos(a)]
    Q = np.broadcast_to(uniaxial(n, S), (N, 1, 1, 3, 3)).copy()
    got = optics.texture(Q, lambdas=(lam,), weights=(1.0,))[0, 0]
    n_eff = optics.N_O * optics.N_E / np.sqrt(optics.N_O ** 2 * np.sin(a) ** 2 + optics.N_E ** 2 * np.cos(a) ** 2)
    Gamma = N * 2 * np.pi * (2 * S / 3) * (n_eff - optics.N_O) / lam
    assert abs(got - 0.5 * np.sin(Gamma / 2) ** 2) < 1e-13


def jones_intensity(d_col, q_col, lam):
    """Independent method: Jones calculus of the same stack between crossed
    linear polarisers (x then y), unpolarised input of unit intensity."""
    E = np.array([1.0, 0.0], dtype=complex) / np.sqrt(2.0)
    for d, q in zip(d_col, q_col):
        th = np.arctan2(d[0], d[1])  # axis angle as in the section's beta
        delta = optics.retardance(d, q, lam)
        R = np.array([[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]])
        J = R.T @ np.diag([1.0, np.exp(1j * delta)]) @ R
        E = J @ E
    return abs(E[1]) ** 2


def test_twisted_stacks_match_jones_calculus():
    rng = np.random.default_rng(1)
    for trial in range(6):
        N = 9
        Q9 = np.zeros((N, 1, 1, 3, 3))
        for k in range(N):
            n = rng.normal(size=3)
            Q9[k, 0, 0] = uniaxial(n, rng.uniform(0.1, 0.6))
            Q9[k, 0, 0] += 0.02 * lbq.q5_to_q9(rng.normal(size=(5, 1, 1, 1)))[0, 0, 0]  # slightly biaxial
        q, d = optics.director_and_order(Q9)
        for lam in optics.LAMBDAS:
            got = optics.texture(Q9, lambdas=(lam,), weights=(1.0,))[0, 0]
            want = jones_intensity(d[:, 0, 0], q[:, 0, 0], lam)
            assert abs(got - want) < 1e-13, (trial, lam, got, want)


def test_wavelength_weighting():
    rng = np.random.default_rng(2)
    Q9 = lbq.q5_to_q9(rng.normal(size=(5, 4, 2, 3)) * 0.2)
    parts = [optics.texture(Q9, lambdas=(lam,), weights=(1.0,)) for lam in optics.LAMBDAS]
    assert np.allclose(optics.texture(Q9), sum(w * p for w, p in zip(optics.WEIGHTS, parts)), atol=1e-15)
