"""Plain FP64 CPU oracle for the coupled hybrid LB + Beris-Edwards step.

TEST INFRASTRUCTURE ONLY.  This module is the correctness reference for the
CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it; the product library never does.
It shares no code with the CUDA path: every formula is restated here from the
paper (Henrich, Marenduzzo, Stratford, Cates, arXiv:0901.3293):

* Sec. 2.1, Eq. (free_energy): chiral Landau-de Gennes free energy density.
* Sec. 2.1, Eq. (Qevolution): Beris-Edwards equation D_t Q = Gamma H.
* Sec. 2.1, Eq. (mat_der): material derivative and co-rotational term S(W,Q).
* Sec. 2.1, Eq. (BEstress): symmetric LC stress sigma and antisymmetric tau.
* Sec. 2.2, Eq. (latvects): D3Q15 velocity set.
* Sec. 2.2, Eq. (eq1), (eq2), (eq4): moments, predictor-corrector LB, BGK + forcing.
* Sec. 2.2, Eq. (eq6a/b), (eq7a/b), (spurious), (feq), (coeff): equilibrium
  and forcing polynomials and the spurious-velocity-free body force.

Deliberately naive storage: Q is a full 3x3 matrix per site (9 doubles) so
that symmetry and tracelessness are *tested*, not assumed; f is
``f[z, y, x, i]``.  All arrays are indexed ``[z, y, x, ...]``; vector
components are ordered (x, y, z).  Lattice units: dx = dt = 1.

Readings of points the paper leaves open (each shared with the CUDA path only
through this written specification, never through code):

* Gradient terms (Eq. free_energy + "one-constant approximation"): the
  one-constant energy (K/2)|grad Q|^2 + 2 K q0 Q:(eps grad Q) + 2 K q0^2 |Q|^2,
  i.e. the printed chiral square plus (K/2)(d_b Q_ab)^2, up to a divergence.
  Discretised as F_h below; H is the exact lattice gradient of F_h.
* T = 1/3 in A_2 = rho T / 10 (Eq. coeff).
* P_s b.e_i is the forcing p_i of Eq. (eq4), not part of f_eq.
* E_2 = -sigma_LC / 16 with sigma_LC the symmetric traceless LC stress.
* sigma_LC and b are held at step n inside the LB predictor-corrector.
* The order-parameter predictor-corrector is Heun (explicit trapezoid), with
  central differences; Tr S (= 2 xi div(u) / 3) is removed.
* Coupling order "Jacobi" (default): LB and Q both read step-n fields.
  "Gauss-Seidel": LB first, then Q with u^{n+1}.
* u = sum_i f_i e_i / rho, with no half-force shift (Eq. eq1).
"""

from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

# ---------------------------------------------------------------------------
# D3Q15 velocity set, Sec. 2.2 Eq. (latvects).  The paper fixes only the
# groups: 0 rest, 1..6 the |e|^2 = 1 set, 7..14 the |e|^2 = 3 set.  Order
# chosen here: +x,-x,+y,-y,+z,-z, then (+-1,+-1,+-1) lexicographic, + first.
# ---------------------------------------------------------------------------
E = np.array(
    [[0, 0, 0],
     [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
     [1, 1, 1], [1, 1, -1], [1, -1, 1], [1, -1, -1],
     [-1, 1, 1], [-1, 1, -1], [-1, -1, 1], [-1, -1, -1]], dtype=np.int64)
NVEL = 15
# speed class s of each direction: |e|^2 in {0, 1, 3}  <->  s in {0, 1, 2}
CLASS = np.array([0] + [1] * 6 + [2] * 8)
OPPOSITE = np.array([int(np.where((E == -E[i]).all(axis=1))[0][0]) for i in range(NVEL)])

EYE = np.eye(3)
# Levi-Civita symbol eps[a, b, c]
EPS = np.zeros((3, 3, 3))
for _a, _b, _c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
    EPS[_a, _b, _c] = 1.0
    EPS[_a, _c, _b] = -1.0

T_LATTICE = 1.0 / 3.0  # temperature in A_2 = rho T / 10 (reading, see header)


@dataclass(frozen=True)
class Params:
    """Model parameters (Sec. 2.1, Eq. free_energy and the kinetic parameters).

    A0, gamma, K, q0: Landau-de Gennes free energy.  Gamma: rotational
    diffusion constant.  xi: flow-aligning parameter.  tau_f: LB relaxation
    time (viscosity eta = rho tau_f / 3).  flow_on: 0 imposes u = 0 (Sec. 2.1,
    last paragraph before the kappa/tau definitions).  coupling: "jacobi" or
    "gauss_seidel".
    """

    A0: float = 0.01
    gamma: float = 3.1
    K: float = 0.01
    q0: float = 2.0 * np.pi / 16.0
    Gamma: float = 0.3
    xi: float = 0.7
    tau_f: float = 2.0
    flow_on: bool = True
    coupling: str = "jacobi"
    # solid walls half a spacing below z = 0 and above z = Nz-1 (see the
    # "Solid walls" section below); q_wall = the anchored Q in q5 order
    walls_z: bool = False
    q_wall: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)
    # coefficient of (1/2)(d_b Q_ab)^2 beside the printed chiral square: None =
    # K (the one-constant energy, default); 0 = the energy exactly as printed
    L2: float | None = None

    @property
    def c_div(self) -> float:
        """(K - L2) / 2: weight of -(d_b Q_ab)^2 relative to the one-constant energy."""
        return 0.0 if self.L2 is None else 0.5 * (self.K - self.L2)

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


def kappa_tau(A0: float, gamma: float, K: float, q0: float) -> tuple[float, float]:
    """Reduced chirality and temperature, Sec. 2.1 (kappa, tau definitions; L1 = K)."""
    kappa = np.sqrt(108.0 * K * q0 * q0 / (A0 * gamma))
    tau = 27.0 * (1.0 - gamma / 3.0) / gamma
    return float(kappa), float(tau)


def gamma_K_from_kappa_tau(A0: float, q0: float, kappa: float, tau: float) -> tuple[float, float]:
    """Inverse of :func:`kappa_tau`: gamma = 27/(9+tau), K = kappa^2 A0 gamma/(108 q0^2)."""
    gamma = 27.0 / (9.0 + tau)
    K = kappa * kappa * A0 * gamma / (108.0 * q0 * q0)
    return float(gamma), float(K)


# ---------------------------------------------------------------------------
# Periodic lattice calculus.  axis 0 = z, 1 = y, 2 = x.
# ---------------------------------------------------------------------------
_AXIS = {0: 2, 1: 1, 2: 0}  # Cartesian direction -> array axis


def shift(A: np.ndarray, d) -> np.ndarray:
    """Return B with B(r) = A(r + d) on the periodic lattice (d = (dx, dy, dz))."""
    dx, dy, dz = (int(v) for v in d)
    return np.roll(A, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def unit(g: int, s: int = 1):
    d = [0, 0, 0]
    d[g] = s
    return d


def d0(A: np.ndarray, g: int) -> np.ndarray:
    """Central difference (A(r+e_g) - A(r-e_g)) / 2."""
    return 0.5 * (shift(A, unit(g, 1)) - shift(A, unit(g, -1)))


def dplus(A: np.ndarray, g: int) -> np.ndarray:
    """Forward difference A(r+e_g) - A(r)."""
    return shift(A, unit(g, 1)) - A


def laplacian7(A: np.ndarray) -> np.ndarray:
    """Compact 7-point Laplacian sum_g A(r+e_g) - 2 A(r) + A(r-e_g)."""
    out = np.zeros_like(A)
    for g in range(3):
        out += shift(A, unit(g, 1)) - 2.0 * A + shift(A, unit(g, -1))
    return out


def grad_central(A: np.ndarray) -> np.ndarray:
    """dA[..., g, <A's trailing axes>] = D0_g A."""
    return np.stack([d0(A, g) for g in range(3)], axis=3)


def trace(M: np.ndarray) -> np.ndarray:
    return np.einsum("...aa->...", M)


def ddot(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A_ab B_ab."""
    return np.einsum("...ab,...ab->...", A, B)


def transpose(M: np.ndarray) -> np.ndarray:
    return np.swapaxes(M, -1, -2)


# ---------------------------------------------------------------------------
# Solid walls (a reading: the paper's slab is periodic; walls are an option).
# Walls sit half a lattice spacing below z = 0 and above z = Nz-1:
#  * LB: half-way bounce-back, a population that would arrive from beyond a
#    wall is the reflected one of the same site (see stream);
#  * Q: strong anchoring, ghost planes z = -1 and z = Nz hold Q = q_wall;
#  * u: no slip at the wall, ghost u = -u of the adjacent plane;
#  * tau and H: zero on the ghost planes (the wall carries no molecular field).
# Field operators act on arrays padded with these ghost planes; the energy
# counts every bond with at least one end inside, so H stays its exact gradient.
# ---------------------------------------------------------------------------
def _pad_z(A: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    return np.concatenate([lo[None], A, hi[None]], axis=0)


def q_wall9(Q: np.ndarray, p: "Params") -> np.ndarray:
    """The anchored Q as a ghost plane shaped like one z-plane of Q."""
    qw = np.asarray(p.q_wall, dtype=np.float64).reshape(5, 1, 1, 1)
    plane = q5_to_q9(np.broadcast_to(qw, (5, 1) + Q.shape[1:3]))[0]
    return plane


def _pad_q(Q: np.ndarray, p: "Params") -> np.ndarray:
    w = q_wall9(Q, p)
    return _pad_z(Q, w, w)


def _no_walls(p: "Params") -> "Params":
    return replace(p, walls_z=False)


# ---------------------------------------------------------------------------
# Free energy and molecular field, Sec. 2.1 Eq. (free_energy), Eq. (Qevolution)
# ---------------------------------------------------------------------------
def curl_term(Q: np.ndarray) -> np.ndarray:
    """(eps D0 Q)_ab = eps_{a g d} D0_g Q_{d b}: the lattice form of the
    epsilon_{alpha gamma delta} d_gamma Q_{delta beta} term of Eq. (free_energy)."""
    dQ = grad_central(Q)  # [..., g, d, b]
    return np.einsum("agd,...gdb->...ab", EPS, dQ)


def divergence(Q: np.ndarray) -> np.ndarray:
    """div_a = sum_b D0_b Q_ab (central differences)."""
    d = np.zeros(Q.shape[:3] + (3,))
    for a in range(3):
        for b in range(3):
            d[..., a] += d0(Q[..., a, b], b)
    return d


def bulk_free_energy_density(Q: np.ndarray, p: Params) -> np.ndarray:
    """Bulk part of Eq. (free_energy):
    A0/2 (1 - gamma/3) Q_ab^2 - A0 gamma/3 Q_ab Q_bc Q_ca + A0 gamma/4 (Q_ab^2)^2."""
    q2 = ddot(Q, Q)
    q3 = np.einsum("...ab,...bc,...ca->...", Q, Q, Q)
    return (0.5 * p.A0 * (1.0 - p.gamma / 3.0) * q2
            - p.A0 * p.gamma / 3.0 * q3
            + 0.25 * p.A0 * p.gamma * q2 * q2)


def free_energy_density(Q: np.ndarray, p: Params) -> np.ndarray:
    """Lattice free-energy density f_h(r) whose sum F_h is the discrete energy.

    Bulk terms of Eq. (free_energy) plus the one-constant gradient energy
    (K/2) sum_g |D+_g Q|^2 + 2 K q0 Q:(eps D0 Q) + 2 K q0^2 |Q|^2, which expands
    the printed chiral square (K/2)(eps dQ + 2 q0 Q)^2 together with
    (K/2)(d_b Q_ab)^2 (one-constant approximation) up to a divergence.
    """
    grad2 = np.zeros(Q.shape[:3])
    for g in range(3):
        dq = dplus(Q, g)
        grad2 += ddot(dq, dq)
    chiral = ddot(Q, curl_term(Q))
    out = (bulk_free_energy_density(Q, p)
           + 0.5 * p.K * grad2
           + 2.0 * p.K * p.q0 * chiral
           + 2.0 * p.K * p.q0 * p.q0 * ddot(Q, Q))
    if p.c_div != 0.0:
        # (K/2)(eps dQ + 2 q0 Q)^2 = one-constant energy - (K/2)(d_b Q_ab)^2 up to a
        # divergence; a general L2 keeps -((K - L2)/2)(div Q)^2 of that difference
        dv = divergence(Q)
        out = out - p.c_div * np.sum(dv * dv, axis=-1)
    return out


def bond_energy(A: np.ndarray, B: np.ndarray, g: int, p: Params) -> np.ndarray:
    """Energy of the bond from A (at r) to B (at r + e_g):
    (K/2)|B - A|^2 + K q0 (A_ab eps_agd B_db - B_ab eps_agd A_db).  Summed over
    all bonds it equals the gradient and chiral parts of free_energy_density
    (the chiral site term 2 K q0 Q:(eps D0 Q) splits into these bond halves)."""
    e = EPS[:, g, :]
    dQ = B - A
    chiral = np.einsum("...ab,ad,...db->...", A, e, B) - np.einsum("...ab,ad,...db->...", B, e, A)
    return 0.5 * p.K * ddot(dQ, dQ) + p.K * p.q0 * chiral


def free_energy_bonds(Q: np.ndarray, p: Params) -> float:
    """F_h in bond form: site terms (bulk + 2 K q0^2 |Q|^2) plus every bond with
    at least one end on the lattice; with walls the bonds to the anchored ghost
    planes are included (periodic in x, y)."""
    site = bulk_free_energy_density(Q, p) + 2.0 * p.K * p.q0 * p.q0 * ddot(Q, Q)
    F = float(np.sum(site))
    for g in (0, 1):  # x, y: periodic bonds
        F += float(np.sum(bond_energy(Q, shift(Q, unit(g, 1)), g, p)))
    if p.walls_z:
        Qp = _pad_q(Q, p)
        F += float(np.sum(bond_energy(Qp[:-1], Qp[1:], 2, p)))
    else:
        F += float(np.sum(bond_energy(Q, shift(Q, unit(2, 1)), 2, p)))
    return F


def free_energy(Q: np.ndarray, p: Params) -> float:
    """F_h = sum over sites of :func:`free_energy_density` (FP64); with walls the
    bond form :func:`free_energy_bonds`."""
    if p.walls_z:
        return free_energy_bonds(Q, p)
    return float(np.sum(free_energy_density(Q, p)))


def dF_dQ(Q: np.ndarray, p: Params) -> np.ndarray:
    """delta F_h / delta Q for a symmetric Q field (symmetrised derivative).

    Bulk: A0(1-gamma/3) Q - A0 gamma Q.Q + A0 gamma Tr(Q^2) Q.
    Gradient: -K Lap7 Q + 2 K q0 (C + C^T) + 4 K q0^2 Q with C = eps D0 Q.
    """
    if p.walls_z:
        if p.c_div != 0.0:
            raise ValueError("walls with L2 != K are not supported")
        return dF_dQ(_pad_q(Q, p), _no_walls(p))[1:-1]
    q2 = ddot(Q, Q)[..., None, None]
    QQ = Q @ Q
    C = curl_term(Q)
    G = (p.A0 * (1.0 - p.gamma / 3.0) * Q
         - p.A0 * p.gamma * QQ
         + p.A0 * p.gamma * q2 * Q
         - p.K * laplacian7(Q)
         + 2.0 * p.K * p.q0 * (C + transpose(C))
         + 4.0 * p.K * p.q0 * p.q0 * Q)
    if p.c_div != 0.0:
        # d/dQ_ab of -c sum_x |div|^2 (summation by parts: the adjoint of D0 is -D0),
        # symmetrised: c (D0_b div_a + D0_a div_b)
        dv = divergence(Q)
        M = np.zeros_like(Q)
        for a in range(3):
            for b in range(3):
                M[..., a, b] = d0(dv[..., a], b)
        G = G + p.c_div * (M + transpose(M))
    return G


def molecular_field(Q: np.ndarray, p: Params) -> np.ndarray:
    """H = -dF/dQ + (1/3) Tr(dF/dQ) I, Sec. 2.1 Eq. (Qevolution)."""
    G = dF_dQ(Q, p)
    return -G + (trace(G) / 3.0)[..., None, None] * EYE


# ---------------------------------------------------------------------------
# Stress and body force, Sec. 2.1 Eq. (BEstress); Sec. 2.2 Eq. (eq7a), (spurious)
# ---------------------------------------------------------------------------
def lc_stress(Q: np.ndarray, H: np.ndarray, p: Params) -> tuple[np.ndarray, np.ndarray]:
    """Return (sigma_LC, tau).

    sigma_LC = 2 xi (Q + I/3) Tr(QH) - xi H (Q + I/3) - xi (Q + I/3) H: the part
    of sigma in Eq. (BEstress) that enters the second moment of f_eq
    (Eq. eq6a), i.e. without -P0 delta and without the double-gradient term,
    which act through the body force.  tau = Q H - H Q.
    """
    P = Q + EYE / 3.0
    qh = ddot(Q, H)[..., None, None]
    sigma = 2.0 * p.xi * P * qh - p.xi * (H @ P) - p.xi * (P @ H)
    tau = Q @ H - H @ Q
    return sigma, tau


def body_force(Q: np.ndarray, H: np.ndarray, tau: np.ndarray, p: Params | None = None) -> np.ndarray:
    """b_a = D0_b tau_ab - H_gn D0_a Q_gn, Sec. 2.2 Eq. (eq7a) with the last two
    terms rewritten through Eq. (spurious); the sum runs over all 9 (g, n).
    With walls (p.walls_z) the ghost planes hold Q = q_wall, H = tau = 0."""
    if p is not None and p.walls_z:
        z = np.zeros_like(H[:1])
        return body_force(_pad_q(Q, p), _pad_z(H, z[0], z[0]), _pad_z(tau, z[0], z[0]))[1:-1]
    b = np.zeros(Q.shape[:3] + (3,))
    for a in range(3):
        for bb in range(3):
            b[..., a] += d0(tau[..., a, bb], bb)
        b[..., a] -= ddot(H, d0(Q, a))
    return b


# ---------------------------------------------------------------------------
# Lattice Boltzmann, Sec. 2.2 Eq. (eq1)-(coeff)
# ---------------------------------------------------------------------------
def moments(f: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """rho = sum_i f_i, rho u = sum_i f_i e_i (Eq. eq1)."""
    rho = f.sum(axis=-1)
    u = (f @ E.astype(np.float64)) / rho[..., None]
    return rho, u


def equilibrium(rho: np.ndarray, u: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """f_i^eq = A_s + B_s u.e + C_s u^2 + D_s (u.e)^2 + e.E_s.e (Eq. feq, coeff).

    A_2 = A_1 = rho T/10, A_0 = rho - 14 A_2; B_2 = rho/24, B_1 = 8 B_2;
    C_2 = -rho/24, C_1 = 2 C_2, C_0 = -2 rho/3; D_2 = rho/16, D_1 = 8 D_2;
    E_2 = -sigma/16, E_1 = 8 E_2 (E_0 = 0, B_0 = D_0 = 0).
    """
    Ef = E.astype(np.float64)
    ue = u @ Ef.T                      # [..., i]
    usq = np.einsum("...a,...a->...", u, u)[..., None]
    eSe = np.einsum("ia,ib,...ab->...i", Ef, Ef, sigma)
    r = rho[..., None]
    A2 = r * T_LATTICE / 10.0
    A = np.where(CLASS == 0, r - 14.0 * A2, A2)
    B = np.where(CLASS == 1, r / 3.0, np.where(CLASS == 2, r / 24.0, 0.0))
    C = np.where(CLASS == 0, -2.0 * r / 3.0, np.where(CLASS == 1, -r / 12.0, -r / 24.0))
    D = np.where(CLASS == 1, r / 2.0, np.where(CLASS == 2, r / 16.0, 0.0))
    Efac = np.where(CLASS == 1, -0.5, np.where(CLASS == 2, -1.0 / 16.0, 0.0))
    return A + B * ue + C * usq + D * ue * ue + Efac * eSe


def forcing(b: np.ndarray) -> np.ndarray:
    """p_i = P_s b.e_i with P_2 = 1/24, P_1 = 8 P_2, P_0 = 0 (Eq. coeff)."""
    Ps = np.where(CLASS == 1, 1.0 / 3.0, np.where(CLASS == 2, 1.0 / 24.0, 0.0))
    return Ps * (b @ E.astype(np.float64).T)


def collision(f: np.ndarray, sigma: np.ndarray, b: np.ndarray, tau_f: float) -> np.ndarray:
    """C_i = -(f_i - f_i^eq)/tau_f + p_i, Eq. (eq4), f^eq from the moments of f."""
    rho, u = moments(f)
    return -(f - equilibrium(rho, u, sigma)) / tau_f + forcing(b)


def stream(g: np.ndarray, walls_z: bool = False) -> np.ndarray:
    """out_i(y) = g_i(y - e_i) on the periodic lattice.

    walls_z (oracle-only option for the Poiseuille check): solid walls half a
    lattice spacing below z = 0 and above z = Nz-1; a population that would
    arrive from beyond a wall is the reflected one, out_i(y) = g_opp(i)(y).
    """
    out = np.empty_like(g)
    nz = g.shape[0]
    for i in range(NVEL):
        out[..., i] = shift(g[..., i], -E[i])
        if walls_z and E[i][2] != 0:
            src_plane = 0 if E[i][2] > 0 else nz - 1  # plane whose upstream is the wall
            out[src_plane, :, :, i] = g[src_plane, :, :, OPPOSITE[i]]
    return out


def lb_step(f: np.ndarray, sigma: np.ndarray, b: np.ndarray, tau_f: float,
            walls_z: bool = False) -> np.ndarray:
    """Predictor-corrector LB update, Sec. 2.2 Eq. (eq2).

    f_i(x + e_i, t+1) - f_i(x, t) = 1/2 [C_i(x, t, {f}) + C_i(x + e_i, t+1, {f*})]
    with the predictor f*_i(x + e_i) = f_i(x) + C_i(x, t, {f}).  sigma and b are
    held at their step-n values in both collision evaluations.
    """
    C = collision(f, sigma, b, tau_f)
    fstar = stream(f + C, walls_z)
    Cstar = collision(fstar, sigma, b, tau_f)
    return stream(f + 0.5 * C, walls_z) + 0.5 * Cstar


# ---------------------------------------------------------------------------
# Beris-Edwards update, Sec. 2.1 Eq. (Qevolution), (mat_der)
# ---------------------------------------------------------------------------
def corotational(Q: np.ndarray, W: np.ndarray, xi: float) -> np.ndarray:
    """S(W, Q) of Eq. (mat_der) with W_ab = d_b u_a, D = sym W, omega = antisym W.

    S = (xi D + omega)(Q + I/3) + (Q + I/3)(xi D - omega) - 2 xi (Q + I/3) Tr(Q W)
    """
    D = 0.5 * (W + transpose(W))
    Om = 0.5 * (W - transpose(W))
    P = Q + EYE / 3.0
    trQW = np.einsum("...ab,...ba->...", Q, W)[..., None, None]
    return (xi * D + Om) @ P + P @ (xi * D - Om) - 2.0 * xi * P * trQW


def velocity_gradient(u: np.ndarray) -> np.ndarray:
    """W_ab = D0_b u_a."""
    W = np.zeros(u.shape[:3] + (3, 3))
    for a in range(3):
        for bb in range(3):
            W[..., a, bb] = d0(u[..., a], bb)
    return W


def be_rhs(Q: np.ndarray, u: np.ndarray, p: Params) -> np.ndarray:
    """dQ/dt = Gamma H + S(W, Q) - u.grad Q  (Eq. Qevolution with Eq. mat_der).

    Central differences for grad u and the advection; the trace of S is removed.
    With walls the ghost planes hold Q = q_wall and u = -u (no slip).
    """
    if p.walls_z:
        up = _pad_z(u, -u[0], -u[-1])
        return be_rhs(_pad_q(Q, p), up, _no_walls(p))[1:-1]
    H = molecular_field(Q, p)
    S = corotational(Q, velocity_gradient(u), p.xi)
    S = S - (trace(S) / 3.0)[..., None, None] * EYE
    adv = np.zeros_like(Q)
    for g in range(3):
        adv += u[..., g][..., None, None] * d0(Q, g)
    return p.Gamma * H + S - adv


def heun_step(Q: np.ndarray, u: np.ndarray, p: Params) -> np.ndarray:
    """Finite-difference predictor-corrector for Q (Sec. 2.2, first paragraph):
    Q* = Q + R(Q), Q_new = Q + (R(Q) + R(Q*)) / 2, with u held fixed."""
    R0 = be_rhs(Q, u, p)
    Qs = Q + R0
    R1 = be_rhs(Qs, u, p)
    return Q + 0.5 * (R0 + R1)


# ---------------------------------------------------------------------------
# One coupled step, Sec. 2.2 (hybrid scheme)
# ---------------------------------------------------------------------------
def step(f: np.ndarray, Q: np.ndarray, p: Params,
         b_ext: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Advance (f, Q) by one time step.

    flow_on: rho, u from f; H(Q), sigma_LC, tau, b; LB predictor-corrector;
    Heun update of Q with u^n (Jacobi) or u^{n+1} (Gauss-Seidel).
    b_ext (optional) is an external body force added to b (Sec. 2.2 remark on
    external forces).  flow off: f untouched, Q relaxes with u = 0.
    """
    if not p.flow_on:
        return f, heun_step(Q, np.zeros(Q.shape[:3] + (3,)), p)
    _, u = moments(f)
    H = molecular_field(Q, p)
    sigma, tau = lc_stress(Q, H, p)
    b = body_force(Q, H, tau, p)
    if b_ext is not None:
        b = b + b_ext
    f_new = lb_step(f, sigma, b, p.tau_f, walls_z=p.walls_z)
    if p.coupling == "gauss_seidel":
        _, u = moments(f_new)
    elif p.coupling != "jacobi":
        raise ValueError(p.coupling)
    return f_new, heun_step(Q, u, p)


def run(f: np.ndarray, Q: np.ndarray, p: Params, nsteps: int, b_ext=None):
    for _ in range(nsteps):
        f, Q = step(f, Q, p, b_ext)
    return f, Q


def init_f_equilibrium(Q: np.ndarray, p: Params, rho0: float = 1.0,
                       u0: np.ndarray | None = None) -> np.ndarray:
    """f^0 = f^eq(rho0, u0, sigma_LC(Q^0)), no forcing term."""
    shape = Q.shape[:3]
    rho = np.full(shape, float(rho0))
    u = np.zeros(shape + (3,)) if u0 is None else np.asarray(u0, dtype=np.float64)
    sigma, _ = lc_stress(Q, molecular_field(Q, p), p)
    return equilibrium(rho, u, sigma)


# ---------------------------------------------------------------------------
# Diagnostics, Sec. 2.1 (scalar order parameter and disclination threshold)
# ---------------------------------------------------------------------------
def totals(f: np.ndarray) -> tuple[float, np.ndarray]:
    """(sum rho, sum rho u) over the lattice."""
    return float(f.sum()), (f.reshape(-1, NVEL) @ E.astype(np.float64)).sum(axis=0)


def scalar_order(Q: np.ndarray) -> np.ndarray:
    """q(r) = largest eigenvalue of Q (Sec. 2.1)."""
    return np.linalg.eigvalsh(0.5 * (Q + transpose(Q)))[..., -1]


def defect_fraction(Q: np.ndarray, threshold: float = 0.19) -> float:
    """Fraction of sites with q(r) below the disclination threshold."""
    return float(np.mean(scalar_order(Q) < threshold))


# ---------------------------------------------------------------------------
# Five-component packing used at the library boundary: [xx, xy, xz, yy, yz]
# ---------------------------------------------------------------------------
def q5_to_q9(q5: np.ndarray) -> np.ndarray:
    """q5[c, z, y, x] -> Q[z, y, x, 3, 3] with Q_zz = -Q_xx - Q_yy."""
    xx, xy, xz, yy, yz = (np.asarray(q5[c], dtype=np.float64) for c in range(5))
    Q = np.empty(xx.shape + (3, 3))
    Q[..., 0, 0] = xx
    Q[..., 0, 1] = Q[..., 1, 0] = xy
    Q[..., 0, 2] = Q[..., 2, 0] = xz
    Q[..., 1, 1] = yy
    Q[..., 1, 2] = Q[..., 2, 1] = yz
    Q[..., 2, 2] = -xx - yy
    return Q


def q9_to_q5(Q: np.ndarray) -> np.ndarray:
    return np.stack([Q[..., 0, 0], Q[..., 0, 1], Q[..., 0, 2], Q[..., 1, 1], Q[..., 1, 2]])


def f_to_soa(f: np.ndarray) -> np.ndarray:
    """f[z, y, x, i] -> f[i, z, y, x]."""
    return np.moveaxis(f, -1, 0)


def f_from_soa(f: np.ndarray) -> np.ndarray:
    return np.moveaxis(np.asarray(f, dtype=np.float64), 0, -1)
