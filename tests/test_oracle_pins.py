"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: exact
moment identities, conservation laws, closed forms, convergence to known
continuum limits, brute-force derivatives and published generator outputs.
"""

import os

import numpy as np
import pytest

from oracle import initial, lbq
from paper_0901_3293_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EF = lbq.E.astype(np.float64)


def sym_traceless(M):
    M = 0.5 * (M + np.swapaxes(M, -1, -2))
    return M - np.trace(M, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3.0


# ---------------------------------------------------------------------------
# Generators and parameters
# ---------------------------------------------------------------------------
def test_splitmix64_published_outputs():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    for k, v in rows:
        assert initial.splitmix64(0, int(k)) == int(v, 16)
    ks = np.arange(1000, dtype=np.uint64)
    vec = initial.splitmix64_array(12345, ks)
    assert all(int(vec[i]) == initial.splitmix64(12345, i) for i in range(0, 1000, 37))


def test_noise_range_and_independence():
    q = initial.noise5((6, 5, 4), 1e-4, 7)
    assert q.shape == (5, 6, 5, 4)
    assert q.min() >= -1e-4 and q.max() < 1e-4
    assert abs(q.mean()) < 2e-5
    assert not np.allclose(q, initial.noise5((6, 5, 4), 1e-4, 8))


def test_reduced_variables_golden():
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "config1_reduced_variables.txt"))
                if l.strip() and not l.startswith("#"))
    kappa, tau = lbq.kappa_tau(0.01, 3.1, 0.01, 2 * np.pi / 16)
    assert abs(kappa - float(vals["kappa"])) < 1e-4
    assert abs(tau - float(vals["tau"])) < 1e-5
    g, K = lbq.gamma_K_from_kappa_tau(0.01, 2 * np.pi / 16, kappa, tau)
    assert abs(g - 3.1) < 1e-12 and abs(K - 0.01) < 1e-12


# ---------------------------------------------------------------------------
# (b) moments of f_eq and p_i, Eq. (eq6a), (eq6b), (eq7a), (eq7b)
# ---------------------------------------------------------------------------
def test_d3q15_velocity_set():
    assert lbq.E.shape == (15, 3)
    sq = (lbq.E ** 2).sum(1)
    assert list(sq) == [0] + [1] * 6 + [3] * 8
    assert len({tuple(e) for e in lbq.E}) == 15
    assert (lbq.E[lbq.OPPOSITE] == -lbq.E).all()


def test_equilibrium_moments_exact():
    rho, u, s, b = synth.random_moment_inputs(50, 1)
    feq = lbq.equilibrium(rho, u, s)
    d = np.eye(3)
    m0 = feq.sum(-1)
    m1 = feq @ EF
    m2 = np.einsum("ni,ia,ib->nab", feq, EF, EF)
    m3 = np.einsum("ni,ia,ib,ic->nabc", feq, EF, EF, EF)
    assert np.allclose(m0, rho, atol=1e-14, rtol=0)
    assert np.allclose(m1, rho[:, None] * u, atol=1e-15, rtol=0)
    want2 = (rho[:, None, None] / 3.0 * d - s + rho[:, None, None] * np.einsum("na,nb->nab", u, u))
    assert np.allclose(m2, want2, atol=1e-15, rtol=0)
    want3 = rho[:, None, None, None] / 3.0 * (np.einsum("na,bc->nabc", u, d)
                                              + np.einsum("nb,ac->nabc", u, d)
                                              + np.einsum("nc,ab->nabc", u, d))
    assert np.allclose(m3, want3, atol=1e-15, rtol=0)
    p = lbq.forcing(b)
    assert np.allclose(p.sum(-1), 0, atol=1e-16)
    assert np.allclose(p @ EF, b, atol=1e-16)
    assert np.allclose(np.einsum("ni,ia,ib->nab", p, EF, EF), 0, atol=1e-16)


def test_uniform_rest_state_is_fixed_point():
    shape = (3, 4, 5)
    f = lbq.equilibrium(np.ones(shape), np.zeros(shape + (3,)), np.zeros(shape + (3, 3)))
    f1 = lbq.lb_step(f, np.zeros(shape + (3, 3)), np.zeros(shape + (3,)), 2.0)
    assert np.abs(f1 - f).max() < 1e-16


# ---------------------------------------------------------------------------
# (a) mass and momentum bookkeeping
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("coupling", ["jacobi", "gauss_seidel"])
def test_mass_and_momentum_bookkeeping(coupling):
    p = lbq.Params(coupling=coupling)
    shape = (6, 5, 4)
    Q = lbq.q5_to_q9(initial.bpii5(shape, p.q0, 0.3) + synth.random_q5(shape, 1e-2, 3))
    f = lbq.f_from_soa(synth.random_distributions(shape, 4))
    m0, P0 = lbq.totals(f)
    for _ in range(10):
        H = lbq.molecular_field(Q, p)
        _, tau = lbq.lc_stress(Q, H, p)
        bsum = lbq.body_force(Q, H, tau).reshape(-1, 3).sum(0)
        f, Q = lbq.step(f, Q, p)
        m1, P1 = lbq.totals(f)
        assert abs(m1 - m0) < 1e-13 * m0
        assert np.abs(P1 - P0 - bsum).max() < 1e-14
        m0, P0 = m1, P1


def test_momentum_conserved_without_order_parameter():
    # xi = 0: flow cannot create order from Q = 0 (S(W, 0) = 2 xi D / 3)
    p = lbq.Params(xi=0.0)
    shape = (5, 6, 7)
    Q = np.zeros(shape + (3, 3))
    f = lbq.f_from_soa(synth.random_distributions(shape, 5, amp=1e-2))
    _, P0 = lbq.totals(f)
    f, Q = lbq.run(f, Q, p, 20)
    _, P1 = lbq.totals(f)
    assert np.abs(P1 - P0).max() < 1e-14


# ---------------------------------------------------------------------------
# (c) flow: viscosity eta = rho tau_f / 3 (second-order scheme), Kolmogorov,
#     forced Poiseuille between half-way bounce-back walls
# ---------------------------------------------------------------------------
TAU_F = 2.0
NU = TAU_F / 3.0


def _shear_wave_nu(L):
    shape = (L, 1, 1)
    z = np.arange(L)[:, None, None] * 1.0
    k = 2 * np.pi / L
    u = np.zeros(shape + (3,))
    u[..., 0] = 1e-3 * np.sin(k * z)
    sig, b = np.zeros(shape + (3, 3)), np.zeros(shape + (3,))
    f = lbq.equilibrium(np.ones(shape), u, sig)
    T1, T2 = 2 * L, 6 * L
    amps = {}
    for t in range(T2 + 1):
        if t in (T1, T2):
            amps[t] = 2 * np.mean(lbq.moments(f)[1][..., 0] * np.sin(k * z))
        f = lbq.lb_step(f, sig, b, TAU_F)
    return -np.log(amps[T2] / amps[T1]) / (k * k * (T2 - T1))


def test_shear_wave_viscosity_converges_to_tau_over_3():
    nus = {L: _shear_wave_nu(L) for L in (16, 32, 64)}
    d = {L: NU - nus[L] for L in nus}
    # second-order approach (error ratio 4 per halving of k) ...
    assert 3.6 < d[16] / d[32] < 4.4 and 3.6 < d[32] / d[64] < 4.4
    # ... to eta = rho tau_f / 3 (plain BGK would give (tau_f - 1/2) / 3 = 0.5)
    rich = nus[64] + (nus[64] - nus[32]) / 3.0
    assert abs(rich - NU) < 2e-3 * NU


def _kolmogorov_ratio(L, F0=1e-6):
    shape = (L, 1, 1)
    z = np.arange(L)[:, None, None] * 1.0
    k = 2 * np.pi / L
    b = np.zeros(shape + (3,))
    b[..., 0] = F0 * np.sin(k * z)
    sig = np.zeros(shape + (3, 3))
    f = lbq.equilibrium(np.ones(shape), np.zeros(shape + (3,)), sig)
    for _ in range(int(14 / (NU * k * k))):
        f = lbq.lb_step(f, sig, b, TAU_F)
    amp = 2 * np.mean(lbq.moments(f)[1][..., 0] * np.sin(k * z))
    return amp / (F0 / (NU * k * k))


def test_kolmogorov_steady_amplitude():
    r = {L: _kolmogorov_ratio(L) for L in (16, 32, 64)}
    assert 3.6 < (r[16] - 1) / (r[32] - 1) < 4.4
    rich = r[64] + (r[64] - r[32]) / 3.0
    assert abs(rich - 1.0) < 2e-3


def _poiseuille(Hh, g=1e-6):
    shape = (Hh, 1, 1)
    zc = np.arange(Hh) + 0.5
    b = np.zeros(shape + (3,))
    b[..., 0] = g
    sig = np.zeros(shape + (3, 3))
    u0 = np.zeros(shape + (3,))
    u0[:, 0, 0, 0] = g / (2 * NU) * zc * (Hh - zc)
    f = lbq.equilibrium(np.ones(shape), u0, sig)
    for _ in range(int(15 * Hh * Hh / (np.pi ** 2 * NU))):
        f = lbq.lb_step(f, sig, b, TAU_F, walls_z=True)
    u = lbq.moments(f)[1][:, 0, 0, 0]
    umax = g * Hh * Hh / (8 * NU)
    curvature = np.polyfit(zc, u, 2)[0]
    return u.max() / umax - 1.0, curvature / (-g / (2 * NU)) - 1.0


def test_forced_poiseuille_between_walls():
    """Walls half a spacing outside z = 0 and z = H-1, uniform force g:
    u_max -> g H^2 / (8 eta) at second order and u'' -> -g / eta."""
    e8, c8 = _poiseuille(8)
    e16, c16 = _poiseuille(16)
    e32, c32 = _poiseuille(32)
    assert 3.6 < e8 / e16 < 4.4 and 3.6 < e16 / e32 < 4.4   # second order
    assert abs(e32 + (e32 - e16) / 3.0) < 2e-3              # -> g H^2 / (8 eta)
    assert e32 < 0.03
    assert abs(c32) < 5e-3 and abs(c32) < abs(c16) < abs(c8)


# ---------------------------------------------------------------------------
# (d) cholesteric helix: closed-form energy, pitch of the minimum, stationarity
# ---------------------------------------------------------------------------
def _helix_energy_per_site(q, S, p):
    """Closed form of F_h per site for a uniaxial helix of wavenumber q on the
    lattice: bulk + K S^2 sin^2 q - K q0 S^2 sin 2q + (4/3) K q0^2 S^2
    (forward-difference gradient energy gives 4 sin^2 q per unit amplitude^2,
    the central-difference chiral term gives sin 2q in place of 2q)."""
    bulk = p.A0 * ((1 - p.gamma / 3) * S ** 2 / 3 - 2 * p.gamma * S ** 3 / 27 + p.gamma * S ** 4 / 9)
    return (bulk + p.K * S ** 2 * np.sin(q) ** 2 - p.K * p.q0 * S ** 2 * np.sin(2 * q)
            + 4.0 / 3.0 * p.K * p.q0 ** 2 * S ** 2)


@pytest.mark.parametrize("axis,kind", [("x", initial.CHOL_X), ("y", initial.CHOL_Y), ("z", initial.CHOL_Z)])
def test_helix_energy_closed_form(axis, kind):
    p = lbq.Params()
    S = 0.4
    for L in (12, 16, 20):
        shape = {"x": (1, 1, L), "y": (1, L, 1), "z": (L, 1, 1)}[axis]
        qq = 2 * np.pi / L
        Q = initial.init_q9(shape, kind, qq, S, 0.0, 0)
        assert abs(lbq.free_energy(Q, p) / L - _helix_energy_per_site(qq, S, p)) < 1e-15
        # the mirror-image helix costs more (handedness fixed by q0 > 0)
        Qm = initial.init_q9(shape, kind, -qq, S, 0.0, 0)
        assert lbq.free_energy(Qm, p) > lbq.free_energy(Q, p)


def _relax_flow_off(Q, p, tol=1e-12, nmax=5000):
    for n in range(nmax):
        if np.abs(lbq.molecular_field(Q, p)).max() < tol:
            return Q, n
        Q = lbq.heun_step(Q, np.zeros(Q.shape[:3] + (3,)), p)
    raise AssertionError("did not relax")


def _fast_params(kappa, q0, **kw):
    A0 = 0.1
    g, K = lbq.gamma_K_from_kappa_tau(A0, q0, kappa, -0.5)
    return lbq.Params(A0=A0, gamma=g, K=K, q0=q0, Gamma=1.0, **kw)


def test_helix_free_energy_minimum_at_pitch_2pi_over_q0():
    q0 = 2 * np.pi / 64
    p = _fast_params(0.5, q0, flow_on=False)
    S = initial.s_eq(p.gamma)
    Ls = list(range(56, 74, 2))
    closed = [_helix_energy_per_site(2 * np.pi / L, S, p) for L in Ls]
    assert Ls[int(np.argmin(closed))] == 64
    # lattice optimum of the closed form: tan 2q* = 2 q0, pitch 64.81 at q0 = 2 pi / 64
    qstar = 0.5 * np.arctan(2 * q0)
    assert abs(2 * np.pi / qstar - 64.81) < 0.01
    relaxed = []
    for L in Ls:
        Q = initial.init_q9((L, 1, 1), initial.CHOL_Z, 2 * np.pi / L, S, 0.0, 0)
        Q, _ = _relax_flow_off(Q, p, tol=1e-11)
        relaxed.append(lbq.free_energy(Q, p) / L)
    assert Ls[int(np.argmin(relaxed))] == 64


def _rotating_frame_spread(Q, q0):
    """max over z of |R(-q0 z) Q(z) R(-q0 z)^T - (the same at z = 0)| on a column."""
    ref, worst = None, 0.0
    for z in range(Q.shape[0]):
        c, s = np.cos(-q0 * z), np.sin(-q0 * z)
        R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
        M = R @ Q[z, 0, 0] @ R.T
        ref = M if ref is None else ref
        worst = max(worst, float(np.abs(M - ref).max()))
    return worst


def test_relaxed_helix_is_stationary_with_flow_on():
    """A helix relaxed with flow off stays put for 1000 coupled steps with flow
    on: its sigma^LC and body force vanish, so no velocity develops (|u| below
    1e-14 throughout), Q keeps its rotating-frame form, and Q follows the
    flow-off trajectory from the same state (the residual relaxation of
    max |H| ~ 1e-12, the same with and without flow)."""
    q0 = 2 * np.pi / 16
    p = _fast_params(0.5, q0, flow_on=False)
    L = 16
    Q = initial.init_q9((L, 1, 1), initial.CHOL_Z, q0, initial.s_eq(p.gamma), 0.0, 0)
    Q, _ = _relax_flow_off(Q, p)
    # rotating frame: R(-q0 z) Q(z) R(-q0 z)^T is z-independent
    assert _rotating_frame_spread(Q, q0) < 1e-12
    Q_relaxed = Q.copy()
    pf = p.with_(flow_on=True)
    f = lbq.init_f_equilibrium(Q, pf)
    for _ in range(10):
        f, Q = lbq.run(f, Q, pf, 100)
        assert np.abs(lbq.moments(f)[1]).max() < 1e-14
    assert _rotating_frame_spread(Q, q0) < 1e-12
    Q_off = Q_relaxed
    for _ in range(1000):
        Q_off = lbq.heun_step(Q_off, np.zeros(Q_off.shape[:3] + (3,)), p)
    assert np.abs(Q - Q_off).max() < 1e-14


# ---------------------------------------------------------------------------
# (e) symmetric and traceless; (f) monotone free energy with flow off
# ---------------------------------------------------------------------------
def test_q_stays_symmetric_and_traceless():
    p = lbq.Params()
    shape = (6, 6, 6)
    Q = initial.init_q9(shape, initial.BPII, p.q0, 0.3, 1e-2, 11)
    f = lbq.init_f_equilibrium(Q, p)
    f, Q = lbq.run(f, Q, p, 100)
    assert np.abs(Q - np.swapaxes(Q, -1, -2)).max() <= 1e-14
    assert np.abs(np.trace(Q, axis1=-2, axis2=-1)).max() <= 1e-14
    assert np.abs(lbq.moments(f)[1]).max() > 1e-7  # flow actually developed


def test_free_energy_never_increases_with_flow_off():
    p = lbq.Params(flow_on=False)
    shape = (8, 8, 8)
    Q = initial.init_q9(shape, initial.BPII, p.q0, 0.3, 1e-2, 12)
    F = [lbq.free_energy(Q, p)]
    for _ in range(600):
        Q = lbq.heun_step(Q, np.zeros(shape + (3,)), p)
        F.append(lbq.free_energy(Q, p))
    dF = np.diff(F)
    assert (dF <= 1e-15 * abs(F[0])).all()
    assert F[-1] < F[0]


# ---------------------------------------------------------------------------
# (g) brute-force gradients of F_h against the molecular field
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 5)])
def test_molecular_field_is_exact_lattice_gradient(shape):
    p = lbq.Params()
    q5 = synth.random_q5(shape, 0.2, 21)
    H = lbq.molecular_field(lbq.q5_to_q9(q5), p)
    h = 1e-6
    rng = np.random.default_rng(2)
    sites = [tuple(rng.integers(0, n) for n in shape) for _ in range(6)]
    comp_to_H = {0: lambda M: -(M[0, 0] - M[2, 2]), 1: lambda M: -2 * M[0, 1],
                 2: lambda M: -2 * M[0, 2], 3: lambda M: -(M[1, 1] - M[2, 2]),
                 4: lambda M: -2 * M[1, 2]}
    for (z, y, x) in sites:
        for c in range(5):
            qp, qm = q5.copy(), q5.copy()
            qp[c, z, y, x] += h
            qm[c, z, y, x] -= h
            dF = (lbq.free_energy(lbq.q5_to_q9(qp), p) - lbq.free_energy(lbq.q5_to_q9(qm), p)) / (2 * h)
            assert abs(dF - comp_to_H[c](H[z, y, x])) < 1e-8


# ---------------------------------------------------------------------------
# Closed forms for the order-parameter update
# ---------------------------------------------------------------------------
def test_uniform_uniaxial_relaxes_to_S_eq():
    p = lbq.Params(q0=0.0, flow_on=False, Gamma=1.0, A0=0.1)
    n = np.array([1.0, 2.0, 2.0]) / 3.0
    Q = (0.3 * (np.outer(n, n) - np.eye(3) / 3.0))[None, None, None]
    for _ in range(3000):
        Q = lbq.heun_step(Q, np.zeros((1, 1, 1, 3)), p)
    lam = np.linalg.eigvalsh(Q[0, 0, 0])
    S = initial.s_eq(p.gamma)
    assert abs(lam[-1] - 2 * S / 3) < 1e-10 and abs(lam[0] + S / 3) < 1e-10


def test_heun_is_second_order_in_time():
    from scipy.integrate import solve_ivp
    p0 = lbq.Params(q0=0.0, flow_on=False, Gamma=1.0, A0=0.1)
    Q0 = lbq.q5_to_q9(np.array([0.05, 0.02, -0.03, 0.01, 0.04]).reshape(5, 1, 1, 1))
    T = 20.0

    def rhs(t, y):
        return (p0.Gamma * lbq.molecular_field(y.reshape(1, 1, 1, 3, 3), p0)).ravel()

    exact = solve_ivp(rhs, (0, T), Q0.ravel(), rtol=1e-12, atol=1e-14).y[:, -1]
    errs = []
    for h in (1.0, 0.5, 0.25):
        p = p0.with_(Gamma=p0.Gamma * h)  # Gamma * dt with dt = h
        Q = Q0.copy()
        for _ in range(int(round(T / h))):
            Q = lbq.heun_step(Q, np.zeros((1, 1, 1, 3)), p)
        errs.append(np.abs(Q.ravel() - exact).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_advection_of_a_fourier_mode():
    """Gamma = 0, uniform u: one Heun step with central differences multiplies a
    mode exp(i k x) by g = 1 + z + z^2/2 with z = -i u sin k."""
    p = lbq.Params(Gamma=0.0)
    L, m, ux = 16, 3, 0.2
    k = 2 * np.pi * m / L
    x = np.arange(L)
    Q = np.zeros((1, 1, L, 3, 3))
    Q[0, 0, :, 0, 1] = Q[0, 0, :, 1, 0] = np.cos(k * x)
    u = np.zeros((1, 1, L, 3))
    u[..., 0] = ux
    zz = -1j * ux * np.sin(k)
    g = 1 + zz + zz * zz / 2
    nsteps = 7
    for _ in range(nsteps):
        Q = lbq.heun_step(Q, u, p)
    want = np.real(g ** nsteps * np.exp(1j * k * x))
    assert np.abs(Q[0, 0, :, 0, 1] - want).max() < 1e-14
    assert np.abs(Q[0, 0, :, 0, 0]).max() < 1e-15


def test_corotational_term_under_shear():
    """Uniform diagonal Q, u_x = U sin(k z): only the xz entry of dQ/dt is
    non-zero and equals (gdot/2) [xi (p1 + p3) + p3 - p1] with
    gdot = D0_z u_x = U sin k cos(k z), p = diag(Q + I/3)."""
    xi = 0.7
    p = lbq.Params(Gamma=0.0, xi=xi)
    L, U = 16, 0.01
    k = 2 * np.pi / L
    d = np.array([0.2, -0.05, -0.15])
    Q = np.zeros((L, 1, 1, 3, 3))
    Q[..., :, :] = np.diag(d)
    u = np.zeros((L, 1, 1, 3))
    z = np.arange(L)
    u[:, 0, 0, 0] = U * np.sin(k * z)
    R = lbq.be_rhs(Q, u, p)
    p1, p3 = d[0] + 1 / 3, d[2] + 1 / 3
    want = 0.5 * U * np.sin(k) * np.cos(k * z) * (xi * (p1 + p3) + p3 - p1)
    assert np.abs(R[:, 0, 0, 0, 2] - want).max() < 1e-16
    assert np.abs(R[:, 0, 0, 2, 0] - want).max() < 1e-16
    mask = np.ones((3, 3), bool)
    mask[0, 2] = mask[2, 0] = False
    assert np.abs(R[:, 0, 0][:, mask]).max() < 1e-17


def test_reactive_couplings_balance_energy():
    """Continuum Beris-Edwards energy balance, exact on the lattice:
    sigma_LC : D + H : S_xi(W) = (2 xi / 3) Tr(QH) Tr D pointwise, and
    sum_x [u . (D0 . tau) - H : S_omega(W)] = 0 with W = D0 u (summation by
    parts), which fixes the signs of sigma_LC, tau and the rotation term."""
    p = lbq.Params()
    shape = (6, 5, 4)
    Q = lbq.q5_to_q9(synth.smooth_q5(shape, 0.3, 31))
    u = np.moveaxis(synth.random_velocity(shape, 0.05, 32), 0, -1)
    H = lbq.molecular_field(Q, p)
    sigma, tau = lbq.lc_stress(Q, H, p)
    W = lbq.velocity_gradient(u)
    D = 0.5 * (W + np.swapaxes(W, -1, -2))
    S_om = lbq.corotational(Q, W, 0.0)
    S_xi = lbq.corotational(Q, W, p.xi) - S_om
    lhs = lbq.ddot(sigma, D) + lbq.ddot(H, S_xi)
    rhs = 2 * p.xi / 3 * lbq.ddot(Q, H) * np.trace(D, axis1=-2, axis2=-1)
    assert np.abs(lhs - rhs).max() < 1e-15
    assert np.abs(lbq.ddot(sigma, D)).max() > 1e-5
    div_tau = np.zeros(shape + (3,))
    for a in range(3):
        for bb in range(3):
            div_tau[..., a] += lbq.d0(tau[..., a, bb], bb)
    total = np.sum(np.einsum("...a,...a->...", u, div_tau) - lbq.ddot(H, S_om))
    assert abs(total) < 1e-15
    assert np.abs(lbq.ddot(H, S_om)).max() > 1e-6
    # the -H:D0Q part of b cancels the advection power H:(u.D0 Q) pointwise
    b = lbq.body_force(Q, H, tau) - div_tau
    adv = sum(u[..., g][..., None, None] * lbq.d0(Q, g) for g in range(3))
    assert np.abs(np.einsum("...a,...a->...", u, b) + lbq.ddot(H, adv)).max() < 1e-16


def test_body_force_vanishes_when_H_vanishes():
    p = lbq.Params()
    shape = (4, 4, 4)
    Q = lbq.q5_to_q9(synth.smooth_q5(shape, 0.2, 40))
    H = np.zeros_like(Q)
    sigma, tau = lbq.lc_stress(Q, H, p)
    assert np.abs(sigma).max() == 0 and np.abs(lbq.body_force(Q, H, tau)).max() == 0


# ---------------------------------------------------------------------------
# Initial states and diagnostics
# ---------------------------------------------------------------------------
def test_bpii_formula_properties():
    q0 = 2 * np.pi / 16
    shape = (16, 16, 16)
    Q = initial.init_q9(shape, initial.BPII, q0, 0.3, 0.0, 0)
    assert np.abs(Q - np.swapaxes(Q, -1, -2)).max() == 0
    assert np.abs(np.trace(Q, axis1=-2, axis2=-1)).max() < 1e-15
    period = int(round(np.pi / q0))  # 8 sites at pitch 16
    for ax in range(3):
        assert np.abs(np.roll(Q, period, axis=ax) - Q).max() < 1e-14
        assert np.abs(np.roll(Q, period // 2, axis=ax) - Q).max() > 0.1
    # the chiral term favours this handedness over the mirror image x -> -x
    p = lbq.Params()
    Qm = np.roll(Q[:, :, ::-1], 1, axis=2).copy()
    for a, b in ((0, 1), (1, 0), (0, 2), (2, 0)):
        Qm[..., a, b] *= -1
    assert lbq.free_energy(Q, p) < 0.5 * lbq.free_energy(Qm, p)


def test_cholesteric_and_slab_initial_states():
    q0 = 2 * np.pi / 16
    S = 0.5
    Q = initial.init_q9((4, 5, 16), initial.CHOL_X, q0, S, 0.0, 0)
    lam = np.linalg.eigvalsh(Q)
    assert np.abs(lam[..., -1] - 2 * S / 3).max() < 1e-14
    assert np.abs(lam[..., 0] + S / 3).max() < 1e-14
    q = initial.init_q5((8, 4, 4), initial.SLAB_BPII_IN_CHOL, q0, 0.3, 0.0, 0, z0=3, s_helix=S)
    assert np.allclose(q[:, :3], initial.bpii5((8, 4, 4), q0, 0.3)[:, :3])
    assert np.allclose(q[:, 3:], initial.cholesteric5((8, 4, 4), q0, S, "x")[:, 3:])
    # BPII next to the isotropic phase (Sec. 3, Fig. 3): Q vanishes beyond the seed
    q = initial.init_q5((8, 4, 4), initial.SLAB_BPII_IN_ISO, q0, 0.3, 0.0, 0, z0=3, s_helix=S)
    assert np.allclose(q[:, :3], initial.bpii5((8, 4, 4), q0, 0.3)[:, :3]) and not q[:, 3:].any()
    # helix normal to the wall: the director turns in the x-y plane along z,
    # n = (cos q0 z, sin q0 z, 0), uniaxial with eigenvalues 2S/3, -S/3, -S/3
    q = initial.init_q5((8, 4, 4), initial.SLAB_BPII_IN_CHOL_Z, q0, 0.3, 0.0, 0, z0=3, s_helix=S)
    Q = initial.q5_to_q9(q)[3:]
    z = np.arange(3, 8)[:, None, None]
    n = np.stack([np.cos(q0 * z) * np.ones((1, 4, 4)), np.sin(q0 * z) * np.ones((1, 4, 4)), np.zeros((5, 4, 4))], -1)
    assert np.abs(np.einsum("...ab,...b->...a", Q, n) - 2 * S / 3 * n).max() < 1e-14
    assert np.abs(Q[..., 2, 2] + S / 3).max() < 1e-14


def test_s_eq_is_bulk_minimum():
    from scipy.optimize import minimize_scalar
    p = lbq.Params(gamma=3.1)
    n = np.array([0.0, 0.0, 1.0])

    def fb(S):
        Q = (S * (np.outer(n, n) - np.eye(3) / 3))[None, None, None]
        return float(lbq.bulk_free_energy_density(Q, p)[0, 0, 0])

    res = minimize_scalar(fb, bounds=(0.3, 0.9), method="bounded", options={"xatol": 1e-12})
    assert abs(res.x - initial.s_eq(3.1)) < 1e-6
    assert abs(initial.s_eq(3.1) - 0.53041) < 1e-5  # 1/4 + 3/4 sqrt(0.139785)


def test_defect_fraction_closed_form():
    n = np.array([0.0, 0.6, 0.8])
    Quni = lambda S: S * (np.outer(n, n) - np.eye(3) / 3)
    Q = np.zeros((2, 2, 2, 3, 3))
    Q[0] = Quni(0.2)   # q = 2S/3 = 0.133 < 0.19: disclination
    Q[1] = Quni(0.5)   # q = 0.333
    assert np.allclose(lbq.scalar_order(Q)[1], 2 * 0.5 / 3)
    assert lbq.defect_fraction(Q) == 0.5
    assert lbq.defect_fraction(np.zeros((2, 2, 2, 3, 3))) == 1.0
