"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 state: agreement to rounding (<= 1e-12 after 100 steps).
FP32 state: max |dQ|, max |du| <= 1e-4 after 100 steps of the 32^3 BPII run
(the tolerance the hot path is specified to); per-component errors are
printed.  Shapes include odd and ragged sizes, one-site-wide columns and
several tiles with a ragged tail.
"""

import os

import numpy as np
import pytest

from oracle import initial, lbq
from paper_0901_3293_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = synth.BASE_SEED


@pytest.fixture(scope="module")
def lcbp():
    import torch
    from paper_0901_3293_gb300 import build
    build.build()
    from paper_0901_3293_gb300 import lcbp as L
    torch.cuda.set_device(0)
    return L


def make(L, shape, dtype, p: lbq.Params, memory="torch"):
    nz, ny, nx = shape
    lat = L.Lattice(nx, ny, nz, dtype=dtype, memory=memory)
    lat.set_ldg(p.A0, p.gamma, p.K, p.q0)
    lat.set_flow(p.tau_f, p.xi, p.Gamma, p.flow_on, L.GAUSS_SEIDEL if p.coupling == "gauss_seidel" else L.JACOBI)
    return lat


def oracle_u(f):
    return np.moveaxis(lbq.moments(f)[1], -1, 0)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-15), ("f32", 2e-7)])
@pytest.mark.parametrize("kind", [initial.BPII, initial.CHOL_X, initial.CHOL_Y, initial.CHOL_Z,
                                  initial.ISO_NOISE, initial.SLAB_BPII_IN_CHOL, initial.SLAB_BPII_IN_ISO,
                                  initial.SLAB_BPII_IN_CHOL_Z])
def test_init_q_matches_oracle(lcbp, kind, dtype, tol):
    p = lbq.Params()
    shape = (9, 6, 7)
    lat = make(lcbp, shape, dtype, p)
    slab = kind >= initial.SLAB_BPII_IN_CHOL
    amp = 0.3 if kind == initial.BPII or slab else 0.45
    lat.init_q(kind, amp, noise=1e-3, seed=SEED + kind, z0=4 if slab else None)
    want = initial.init_q5(shape, kind, p.q0, amp, 1e-3, SEED + kind, z0=4, s_helix=initial.s_eq(p.gamma))
    assert np.abs(lat.read_q() - want).max() <= tol


# ---------------------------------------------------------------------------
# (nz, ny, nx): odd and ragged sizes; nx % 4 == 0 selects the fast z-marching
# TMA kernels (tiles of 32 x TY columns; 36 = one full tile + a ragged tail)
SHAPES = [(5, 6, 7), (4, 4, 4), (64, 1, 1), (3, 5, 33), (1, 9, 2), (5, 6, 8), (3, 9, 36), (7, 3, 12),
          (2, 1, 4), (9, 17, 64)]


@pytest.mark.parametrize("path", ["auto", "generic"])
@pytest.mark.parametrize("shape", SHAPES)
def test_one_coupled_step_f64(lcbp, shape, path):
    p = lbq.Params()
    q5 = synth.smooth_q5(shape, 0.3, 1) + synth.random_q5(shape, 1e-2, 2)
    f15 = synth.random_distributions(shape, 3, amp=2e-3)
    lat = make(lcbp, shape, "f64", p)
    if path == "generic":
        lat.set_path(lcbp.PATH_GENERIC)
    lat.set_q(q5).set_f(f15).step(1)
    assert lat.path()[0] == (path == "auto" and shape[2] % 4 == 0)
    f, Q = lbq.step(lbq.f_from_soa(f15), lbq.q5_to_q9(q5), p)
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 1e-14
    assert np.abs(lat.read_f() - lbq.f_to_soa(f)).max() < 1e-14
    assert np.abs(lat.read_u() - oracle_u(f)).max() < 1e-14


@pytest.mark.parametrize("kind", [initial.SLAB_BPII_IN_ISO, initial.SLAB_BPII_IN_CHOL_Z])
def test_slab_growth_states_step_f64(lcbp, kind):
    """Ten coupled steps from the growth states of Sec. 3: a BPII seed next to
    the isotropic phase, and next to a helix whose axis is normal to the wall."""
    p = lbq.Params()
    shape = (16, 8, 8)
    lat = make(lcbp, shape, "f64", p)
    lat.init_q(kind, 0.3, noise=1e-4, seed=SEED, z0=8).init_f_equilibrium(1.0).step(10)
    Q = initial.init_q9(shape, kind, p.q0, 0.3, 1e-4, SEED, z0=8, s_helix=initial.s_eq(p.gamma))
    f, Q = lbq.run(lbq.init_f_equilibrium(Q, p), Q, p, 10)
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 1e-13
    assert np.abs(lat.read_u() - oracle_u(f)).max() < 1e-14


@pytest.mark.parametrize("mode", ["flow", "no_flow", "l2", "walls"])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-15), ("f32", 3e-8)])
def test_rate_matches_oracle(lcbp, mode, dtype, tol):
    """lcbp_read_rate: the Beris-Edwards rate R(Q, u) with u from the stored
    moments (Sec. 2.1 Eq. Qevolution, mat_der) against the oracle's be_rhs, with
    flow, without flow (u = 0), with L2 != K, and between walls."""
    shape = (7, 6, 8)
    kw = {}
    if mode == "no_flow":
        kw["flow_on"] = False
    if mode == "l2":
        kw["L2"] = 0.004
    if mode == "walls":
        kw["walls_z"] = True
    p = lbq.Params(**kw)
    q5 = synth.smooth_q5(shape, 0.3, 1) + synth.random_q5(shape, 1e-2, 2)
    f15 = synth.random_distributions(shape, 3, amp=2e-3)
    lat = make(lcbp, shape, dtype, p)
    if mode == "l2":
        lat.set_l2(p.L2)
    if mode == "walls":
        lat.set_walls(True)
    lat.set_q(q5).set_f(f15)
    f = lbq.f_from_soa(f15)
    u = lbq.moments(f)[1] if p.flow_on else np.zeros(shape + (3,))
    # the lattice holds Q in its state type: the oracle takes that Q
    Q9 = lbq.q5_to_q9(lat.read_q())
    want = lbq.q9_to_q5(lbq.be_rhs(Q9, np.asarray(u, dtype=np.float64), p))
    got = lat.read_rate()
    # FP32: the rate carries the rounding of u (from FP32 populations) and of its own
    # arithmetic; the bound is half an ulp of the Q values (O(0.3)) it is added to
    assert np.abs(want).max() > 1e-6
    assert np.abs(got - want).max() < tol, np.abs(got - want).max()


FAST_PATHS = {"fast1": "PATH_FAST1", "fast2": "PATH_FAST2", "generic": "PATH_GENERIC"}


@pytest.mark.parametrize("path", list(FAST_PATHS))
@pytest.mark.parametrize("shape", SHAPES)
def test_one_coupled_step_f32(lcbp, shape, path):
    """FP32 state, both fast builds (one and two sites per thread) and the generic
    kernels against the FP64 oracle.  Bounds: Q and f are O(1/2) in FP32 (ulp
    2^-24 = 6e-8) after ~10^2 rounded operations of O(1e-3) increments, so a few
    ulp; u is O(1e-3) and carries the rounding of O(1e-3) deviations."""
    p = lbq.Params()
    q5 = synth.smooth_q5(shape, 0.3, 1) + synth.random_q5(shape, 1e-2, 2)
    f15 = synth.random_distributions(shape, 3, amp=2e-3)
    lat = make(lcbp, shape, "f32", p)
    lat.set_path(getattr(lcbp, FAST_PATHS[path]))
    lat.set_q(q5).set_f(f15).step(1)
    fast, _, spt = lat.path()
    assert fast == (path != "generic" and shape[2] % 4 == 0)
    if fast:
        assert spt == (1 if path == "fast1" else 2)
    f, Q = lbq.step(lbq.f_from_soa(f15.astype(np.float32).astype(np.float64)),
                    lbq.q5_to_q9(q5.astype(np.float32).astype(np.float64)), p)
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 2.5e-7
    assert np.abs(lat.read_f() - lbq.f_to_soa(f)).max() < 2.5e-7
    assert np.abs(lat.read_u() - oracle_u(f)).max() < 1e-8


@pytest.mark.parametrize("coupling", ["jacobi", "gauss_seidel"])
@pytest.mark.parametrize("flow_on", [True, False])
def test_ten_steps_f64_modes(lcbp, coupling, flow_on):
    p = lbq.Params(coupling=coupling, flow_on=flow_on)
    shape = (6, 7, 8)
    q5 = initial.init_q5(shape, initial.BPII, p.q0, 0.3, 1e-2, 5)
    f15 = synth.random_distributions(shape, 6, amp=2e-3)
    lat = make(lcbp, shape, "f64", p)
    lat.set_q(q5).set_f(f15).step(10)
    f, Q = lbq.run(lbq.f_from_soa(f15), lbq.q5_to_q9(q5), p, 10)
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 1e-13
    assert np.abs(lat.read_f() - lbq.f_to_soa(f)).max() < 1e-14


def _config1(lcbp, dtype, nsteps=100):
    p = lbq.Params()  # A0 0.01, gamma 3.1, K 0.01, q0 2 pi/16, Gamma 0.3, xi 0.7, tau_f 2
    shape = (32, 32, 32)
    lat = make(lcbp, shape, dtype, p)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=SEED)
    lat.init_f_equilibrium(1.0)
    lat.step(nsteps)
    Q = initial.init_q9(shape, initial.BPII, p.q0, 0.3, 1e-4, SEED)
    f = lbq.init_f_equilibrium(Q, p)
    f, Q = lbq.run(f, Q, p, nsteps)
    return lat, f, Q, p


@pytest.fixture(scope="module")
def config1_f32(lcbp):
    return _config1(lcbp, "f32")


def test_config1_f32_within_1e_4_after_100_steps(config1_f32):
    lat, f, Q, p = config1_f32
    dq = np.abs(lat.read_q() - lbq.q9_to_q5(Q)).reshape(5, -1).max(axis=1)
    du = np.abs(lat.read_u() - oracle_u(f)).reshape(3, -1).max(axis=1)
    print("config-1 FP32 max|dQ| per component [xx xy xz yy yz]:", dq)
    print("config-1 FP32 max|du| per component [x y z]:", du, " max|u| =", np.abs(oracle_u(f)).max())
    assert dq.max() <= 1e-4 and du.max() <= 1e-4


def test_config1_f64_matches_to_rounding(lcbp):
    lat, f, Q, p = _config1(lcbp, "f64")
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 1e-12
    assert np.abs(lat.read_u() - oracle_u(f)).max() < 1e-13
    F = lat.free_energy()
    assert abs(F - lbq.free_energy(Q, p)) < 1e-11 * abs(F)
    mass, mom = lat.totals()
    m_o, P_o = lbq.totals(f)
    assert abs(mass - m_o) < 1e-10 and np.abs(mom - P_o).max() < 1e-12
    assert lat.defect_fraction(0.19) == lbq.defect_fraction(Q, 0.19)


def test_diagnostics_f32(config1_f32):
    lat, f, Q, p = config1_f32
    F = lat.free_energy()
    assert abs(F - lbq.free_energy(Q, p)) < 1e-4 * abs(F)
    mass, mom = lat.totals()
    m_o, P_o = lbq.totals(f)
    print("config-1 FP32 relative mass error after 100 steps:", abs(mass - m_o) / m_o)
    assert abs(mass - m_o) < 1e-7 * m_o and np.abs(mom - P_o).max() < 1e-4
    # sites near the threshold may flip in FP32: compare within a few sites
    assert abs(lat.defect_fraction(0.19) - lbq.defect_fraction(Q, 0.19)) * 32 ** 3 <= 3


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-14), ("f32", 5e-7)])
def test_external_force_kolmogorov(lcbp, dtype, tol):
    """Q = 0 and xi = 0 leave pure forced LB: a Kolmogorov force along x."""
    p = lbq.Params(xi=0.0)
    L_ = 32
    shape = (L_, 2, 3)
    z = np.arange(L_)[:, None, None] * np.ones(shape)
    b = np.zeros((3,) + shape)
    b[0] = 1e-5 * np.sin(2 * np.pi * z / L_)
    lat = make(lcbp, shape, dtype, p)
    lat.set_q(np.zeros((5,) + shape)).init_f_equilibrium(1.0).set_body_force(b).step(200)
    f = lbq.equilibrium(np.ones(shape), np.zeros(shape + (3,)), np.zeros(shape + (3, 3)))
    f, _ = lbq.run(f, np.zeros(shape + (3, 3)), p, 200, b_ext=np.moveaxis(b, 0, -1))
    assert np.abs(lat.read_u() - oracle_u(f)).max() < tol
    assert np.abs(lat.read_u()).max() > 1e-5


# (nz, ny, nx): cubes, and ragged tiles in x (36 and 68: 4 lanes of the last
# column tile in the lattice) and in y (13, 9) over several z-chunks, so that
# edge tiles of every kind patch their periodic frames through many planes
@pytest.mark.parametrize("fast", ["PATH_FAST1", "PATH_FAST2"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (6, 10, 36), (64, 64, 64), (45, 13, 36), (20, 9, 68)])
def test_fast_path_matches_generic_f32(lcbp, shape, fast):
    """Both kernel sets compute the same FP32 step (op order differs slightly)."""
    p = lbq.Params()
    a = make(lcbp, shape, "f32", p)
    b = make(lcbp, shape, "f32", p)
    a.set_path(getattr(lcbp, fast))
    b.set_path(lcbp.PATH_GENERIC)
    for lat in (a, b):
        lat.init_q(lcbp.BPII, 0.3, noise=1e-3, seed=4).init_f_equilibrium(1.0).step(20)
    assert a.path()[0] and not b.path()[0] and a.path()[1] >= 1
    assert np.abs(a.read_q() - b.read_q()).max() < 1e-6
    assert np.abs(a.read_u() - b.read_u()).max() < 1e-8
    # read_f rebuilds f = w + df in FP32: one ulp of a population in [1/2, 1) is 2^-24
    assert np.abs(a.read_f() - b.read_f()).max() <= 2.0 ** -23


def test_fast_path_external_force_f64(lcbp):
    p = lbq.Params(xi=0.0)
    shape = (32, 2, 4)
    z = np.arange(32)[:, None, None] * np.ones(shape)
    b = np.zeros((3,) + shape)
    b[0] = 1e-5 * np.sin(2 * np.pi * z / 32)
    lat = make(lcbp, shape, "f64", p)
    lat.set_q(np.zeros((5,) + shape)).init_f_equilibrium(1.0).set_body_force(b).step(100)
    assert lat.path()[0]
    f = lbq.equilibrium(np.ones(shape), np.zeros(shape + (3,)), np.zeros(shape + (3, 3)))
    f, _ = lbq.run(f, np.zeros(shape + (3, 3)), p, 100, b_ext=np.moveaxis(b, 0, -1))
    assert np.abs(lat.read_u() - oracle_u(f)).max() < 1e-14


def test_graph_replay_equals_eager_steps(lcbp):
    p = lbq.Params()
    shape = (8, 8, 8)
    a = make(lcbp, shape, "f32", p)
    b = make(lcbp, shape, "f32", p, memory="library")
    for lat in (a, b):
        lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=1).init_f_equilibrium(1.0)
    a.step(11)
    for _ in range(11):
        b.step(1)
    assert np.array_equal(a.read_f(), b.read_f()) and np.array_equal(a.read_q(), b.read_q())
    assert a.info()[2] == 11 and b.info()[2] == 11


def test_checkpoint_resume_is_bitwise(lcbp, tmp_path):
    p = lbq.Params()
    shape = (6, 8, 10)
    a = make(lcbp, shape, "f32", p)
    a.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=2).init_f_equilibrium(1.0).step(20)
    b = make(lcbp, shape, "f32", p)
    b.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=2).init_f_equilibrium(1.0).step(9)
    path = str(tmp_path / "ck.bin")
    b.save(path)
    c = make(lcbp, shape, "f32", lbq.Params(A0=0.5))
    c.load(path)
    assert c.info()[2] == 9
    c.step(11)
    assert np.array_equal(a.read_f(), c.read_f()) and np.array_equal(a.read_q(), c.read_q())


def test_errors_are_status_codes(lcbp):
    L = lcbp
    with pytest.raises(L.LcbpError) as e:
        L.Lattice(0, 4, 4)
    assert e.value.code == L.EINVAL
    lat = L.Lattice(4, 4, 4)
    with pytest.raises(L.LcbpError) as e:
        lat.step(1)  # f not initialised, flow on
    assert e.value.code == L.ESTATE
    with pytest.raises(L.LcbpError) as e:
        lat.set_flow(tau_f=-1.0)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.LcbpError) as e:
        lat.init_q(99, 0.3)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.LcbpError) as e:
        lat.set_path(7)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.LcbpError) as e:
        L.Lattice(4, 4, 4, dtype="f64").set_path(L.PATH_FAST2)  # packed lanes are FP32 only
    assert e.value.code == L.EINVAL
    with pytest.raises(L.LcbpError) as e:
        lat.set_flow(rho0=0.0)
    assert e.value.code == L.EINVAL
    # a NaN planted in a host-uploaded Q (or f) is refused, and the state keeps its values
    q_ok = initial.init_q5((4, 4, 4), initial.BPII, 2 * np.pi / 16, 0.3, 1e-3, 3)
    lat.set_q(q_ok).init_f_equilibrium(1.0)
    f_ok = lat.read_f()
    q = q_ok.copy()
    q[2, 1, 2, 3] = np.nan
    with pytest.raises(L.LcbpError) as e:
        lat.set_q(q)
    assert e.value.code == L.ENONFINITE
    assert np.array_equal(lat.read_q(dtype=np.float32), q_ok.astype(np.float32))
    f = f_ok.copy()
    f[7, 0, 1, 2] = np.inf
    with pytest.raises(L.LcbpError) as e:
        lat.set_f(f)
    assert e.value.code == L.ENONFINITE
    assert np.array_equal(lat.read_f(), f_ok)
    # a state that blows up (an explicit step far past its stability bound,
    # Gamma K 12 >> 2) is reported by the FP64 diagnostics
    bad = L.Lattice(4, 4, 4, dtype="f32")
    bad.set_ldg(0.01, 3.1, 1e5, 2 * np.pi / 16).set_q(q_ok).init_f_equilibrium(1.0).step(40)
    with pytest.raises(L.LcbpError) as e:
        bad.free_energy()
    assert e.value.code == L.ENONFINITE
    # the lattice stays usable afterwards
    lat.set_q(np.zeros((5, 4, 4, 4))).init_f_equilibrium(1.0).step(3)
    assert lat.free_energy() == 0.0
    # rho0 = 0 takes the reference density of set_flow
    lat.set_flow(rho0=1.25).init_f_equilibrium(0.0)
    assert np.allclose(lat.read_rho(), 1.25, rtol=0, atol=1e-6)


def test_bounded_wait_gives_up_and_reports(lcbp):
    """Failure detection without a fault: the bounded barrier wait of the
    fast kernels, on a barrier that nothing arrives on, gives up after its
    limit, reports it to the host, and leaves the context usable."""
    import time
    L = lcbp
    with pytest.raises(L.LcbpError) as e:
        L.check_wait_timeout(0.0)
    assert e.value.code == L.EINVAL
    assert L.check_wait_timeout(1.0)  # also brings up the context, untimed
    t0 = time.perf_counter()
    assert L.check_wait_timeout(50.0)
    dt = time.perf_counter() - t0
    assert 0.05 <= dt < 2.0, dt
    lat = make(L, (8, 8, 8), "f32", lbq.Params())
    lat.init_q(L.BPII, 0.3, noise=1e-4, seed=1).init_f_equilibrium(1.0).step(4)
    assert lat.path()[0] and np.isfinite(lat.free_energy())


def test_torch_device_buffers(lcbp):
    import torch
    p = lbq.Params()
    shape = (4, 5, 6)
    q5 = torch.tensor(synth.random_q5(shape, 0.1, 9), device="cuda", dtype=torch.float32)
    lat = make(lcbp, shape, "f32", p)
    lat.set_q(q5).init_f_equilibrium(1.0)
    out = torch.empty_like(q5)
    lat.read_q(out=out)
    assert torch.equal(out, q5)
    out64 = lat.read_q()
    assert np.abs(out64 - q5.double().cpu().numpy()).max() == 0


# ---------------------------------------------------------------------------
# Full-size sampled parity: 256^3 BPII (pitch 32), one step, in the launch
# configuration the benchmark times.  One coupled step at a site depends on Q
# within 3 sites and f within 2 sites, so the oracle run on a periodic 9^3
# cube cut around a sampled site reproduces that site exactly.
# ---------------------------------------------------------------------------
def test_full_size_sampled_parity_256(lcbp):
    p = lbq.Params(q0=2 * np.pi / 32)
    n = 256
    lat = make(lcbp, (n, n, n), "f32", p)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=SEED)
    lat.init_f_equilibrium(1.0)
    lat.step(2)  # develop some flow first
    q0 = lat.read_q(dtype=np.float32)
    f0 = lat.read_f(dtype=np.float32)
    m0, _ = lat.totals()
    lat.step(1)
    q1 = lat.read_q(dtype=np.float32)
    u1 = lat.read_u(dtype=np.float32)
    m1, _ = lat.totals()
    rng = np.random.default_rng(7)
    sites = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(12)] + [(0, 0, 0), (255, 255, 255)]
    r = 4
    for (z, y, x) in sites:
        idx = [np.arange(c - r, c + r + 1) % n for c in (z, y, x)]
        cube = np.ix_(idx[0], idx[1], idx[2])
        Qc = lbq.q5_to_q9(q0[(slice(None),) + cube].astype(np.float64))
        fc = lbq.f_from_soa(f0[(slice(None),) + cube].astype(np.float64))
        fo, Qo = lbq.step(fc, Qc, p)
        dq = np.abs(q1[:, z, y, x] - lbq.q9_to_q5(Qo)[:, r, r, r]).max()
        du = np.abs(u1[:, z, y, x] - np.moveaxis(lbq.moments(fo)[1], -1, 0)[:, r, r, r]).max()
        assert dq < 1e-6 and du < 1e-6, ((z, y, x), dq, du)
    assert abs(m1 - m0) < 1e-6 * m0


def test_full_size_sampled_parity_256_walls(lcbp):
    """The same at 256^3 between walls in z (the walled fast kernels, as the
    benchmark's walled line runs them).  A site within 4 planes of a wall is
    compared with the walled oracle on a cube cut at that wall (the cube's
    other, artificial wall lies beyond the step's reach); other sites with
    the periodic oracle as above."""
    qw = (0.2, 0.0, 0.0, -0.1, 0.0)
    p = lbq.Params(q0=2 * np.pi / 32)
    pw = lbq.Params(q0=2 * np.pi / 32, walls_z=True, q_wall=qw)
    n = 256
    lat = make(lcbp, (n, n, n), "f32", p)
    lat.set_walls(True, qw)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=SEED)
    lat.init_f_equilibrium(1.0)
    lat.step(2)
    assert lat.path()[0]
    q0 = lat.read_q(dtype=np.float32)
    f0 = lat.read_f(dtype=np.float32)
    lat.step(1)
    q1 = lat.read_q(dtype=np.float32)
    u1 = lat.read_u(dtype=np.float32)
    rng = np.random.default_rng(11)
    sites = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(6)]
    sites += [(0, 0, 0), (1, 17, 200), (3, 255, 31), (255, 255, 255), (254, 3, 128), (252, 100, 0)]
    r = 4
    for (z, y, x) in sites:
        iy, ix = (np.arange(c - r, c + r + 1) % n for c in (y, x))
        if z < r:
            iz, cz, pp = np.arange(0, 2 * r + 1), z, pw
        elif z > n - 1 - r:
            iz, cz, pp = np.arange(n - 1 - 2 * r, n), z - (n - 1 - 2 * r), pw
        else:
            iz, cz, pp = np.arange(z - r, z + r + 1), r, p
        cube = np.ix_(iz, iy, ix)
        Qc = lbq.q5_to_q9(q0[(slice(None),) + cube].astype(np.float64))
        fc = lbq.f_from_soa(f0[(slice(None),) + cube].astype(np.float64))
        fo, Qo = lbq.step(fc, Qc, pp)
        dq = np.abs(q1[:, z, y, x] - lbq.q9_to_q5(Qo)[:, cz, r, r]).max()
        du = np.abs(u1[:, z, y, x] - np.moveaxis(lbq.moments(fo)[1], -1, 0)[:, cz, r, r]).max()
        assert dq < 1e-6 and du < 1e-6, ((z, y, x), dq, du)


# ---------------------------------------------------------------------------
# Largest lattice of the fast path: its kernels index every field of a lattice
# with 32-bit offsets and the host takes the path only where those fit
# (15 population planes, the 16-value scratch and the Q mirror within 2^31 - 1
# elements).  512 x 512 x 506 is the last nz that fits at 512 x 512; one step
# there, compared site by site with the oracle as above (the far corner, where
# the offsets are largest, among the sites), and nz = 507 leaves the path.
# ---------------------------------------------------------------------------
def test_largest_fast_path_lattice_sampled(lcbp):
    p = lbq.Params(q0=2 * np.pi / 32)
    nx, ny, nz = 512, 512, 506
    lat = make(lcbp, (nz, ny, nx), "f32", p)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=SEED)
    lat.init_f_equilibrium(1.0)
    lat.step(1)
    assert lat.path()[0]
    q0 = lat.read_q(dtype=np.float32)
    f0 = lat.read_f(dtype=np.float32)
    lat.step(1)
    q1 = lat.read_q(dtype=np.float32)
    u1 = lat.read_u(dtype=np.float32)
    lat.close()
    rng = np.random.default_rng(13)
    sites = [(int(rng.integers(0, nz)), int(rng.integers(0, ny)), int(rng.integers(0, nx))) for _ in range(6)]
    sites += [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz - 1, 0, nx - 1), (nz // 2, ny - 1, 0)]
    r = 4
    for (z, y, x) in sites:
        idx = [np.arange(c - r, c + r + 1) % m for c, m in ((z, nz), (y, ny), (x, nx))]
        cube = np.ix_(idx[0], idx[1], idx[2])
        Qc = lbq.q5_to_q9(q0[(slice(None),) + cube].astype(np.float64))
        fc = lbq.f_from_soa(f0[(slice(None),) + cube].astype(np.float64))
        fo, Qo = lbq.step(fc, Qc, p)
        dq = np.abs(q1[:, z, y, x] - lbq.q9_to_q5(Qo)[:, r, r, r]).max()
        du = np.abs(u1[:, z, y, x] - oracle_u(fo)[:, r, r, r]).max()
        assert dq < 1e-6 and du < 1e-6, ((z, y, x), dq, du)
    big = make(lcbp, (nz + 1, ny, nx), "f32", p)
    assert not big.path()[0]
    big.close()
