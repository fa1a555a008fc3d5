"""Solid walls in z on the GPU (bounce-back, strong anchoring) against the
walled oracle, on both kernel sets: the fast z-marching kernels (flow on,
Jacobi coupling, nx % 4 == 0) and the generic ones."""

import numpy as np
import pytest

from oracle import initial, lbq
from paper_0901_3293_gb300 import synth

pytestmark = pytest.mark.gpu
PLANAR = (0.2, 0.0, 0.0, -0.1, 0.0)  # S (x x - I/3), S = 0.3


@pytest.fixture(scope="module")
def lcbp():
    import torch
    from paper_0901_3293_gb300 import build
    build.build()
    from paper_0901_3293_gb300 import lcbp as L
    torch.cuda.set_device(0)
    return L


def make(L, shape, dtype, p, path="auto"):
    nz, ny, nx = shape
    lat = L.Lattice(nx, ny, nz, dtype=dtype)
    if path == "generic":
        lat.set_path(L.PATH_GENERIC)
    lat.set_ldg(p.A0, p.gamma, p.K, p.q0)
    lat.set_flow(p.tau_f, p.xi, p.Gamma, p.flow_on, L.GAUSS_SEIDEL if p.coupling == "gauss_seidel" else L.JACOBI)
    if p.walls_z:
        lat.set_walls(True, p.q_wall)
    return lat


def oracle_u(f):
    return np.moveaxis(lbq.moments(f)[1], -1, 0)


# (nz, ny, nx): nz = 1 puts both walls beside the same plane; 36 and 13 give
# ragged column tiles; nx % 4 != 0 runs the generic kernels under either path
@pytest.mark.parametrize("path", ["auto", "generic"])
@pytest.mark.parametrize("shape", [(6, 5, 8), (5, 3, 7), (2, 4, 4), (1, 4, 8), (9, 13, 36)])
def test_one_step_with_walls_f64(lcbp, shape, path):
    p = lbq.Params(walls_z=True, q_wall=PLANAR)
    q5 = synth.smooth_q5(shape, 0.3, 1) + synth.random_q5(shape, 1e-2, 2)
    f15 = synth.random_distributions(shape, 3, amp=2e-3)
    lat = make(lcbp, shape, "f64", p, path)
    lat.set_q(q5).set_f(f15).step(1)
    assert lat.path()[0] == (path == "auto" and shape[2] % 4 == 0)
    f, Q = lbq.step(lbq.f_from_soa(f15), lbq.q5_to_q9(q5), p)
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 1e-14
    assert np.abs(lat.read_f() - lbq.f_to_soa(f)).max() < 1e-14
    assert np.abs(lat.read_u() - oracle_u(f)).max() < 1e-14


@pytest.mark.parametrize("coupling", ["jacobi", "gauss_seidel"])
@pytest.mark.parametrize("flow_on", [True, False])
@pytest.mark.parametrize("shape", [(7, 4, 6), (7, 4, 8)])
def test_ten_steps_with_walls_f64(lcbp, coupling, flow_on, shape):
    p = lbq.Params(walls_z=True, q_wall=PLANAR, coupling=coupling, flow_on=flow_on)
    q5 = initial.init_q5(shape, initial.BPII, p.q0, 0.3, 1e-2, 5)
    f15 = synth.random_distributions(shape, 6, amp=2e-3)
    lat = make(lcbp, shape, "f64", p)
    lat.set_q(q5).set_f(f15).step(10)
    assert lat.path()[0] == (flow_on and coupling == "jacobi" and shape[2] % 4 == 0)
    f, Q = lbq.run(lbq.f_from_soa(f15), lbq.q5_to_q9(q5), p, 10)
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 1e-13
    assert np.abs(lat.read_f() - lbq.f_to_soa(f)).max() < 1e-14


def test_free_energy_and_mass_with_walls(lcbp):
    p = lbq.Params(walls_z=True, q_wall=PLANAR)
    shape = (6, 5, 4)
    q5 = synth.smooth_q5(shape, 0.3, 7) + synth.random_q5(shape, 0.02, 8)
    lat = make(lcbp, shape, "f64", p)
    lat.set_q(q5).init_f_equilibrium(1.0)
    F = lbq.free_energy(lbq.q5_to_q9(q5), p)
    assert abs(lat.free_energy() - F) < 1e-12 * max(1.0, abs(F))
    m0 = lat.totals()[0]
    lat.step(50)
    assert abs(lat.totals()[0] - m0) < 1e-12 * m0


@pytest.mark.parametrize("path", ["auto", "generic"])
def test_poiseuille_between_walls_f64(lcbp, path):
    """Q = 0, xi = 0, uniform force g along x between the walls: the GPU run
    follows the oracle step by step and approaches g H^2 / (8 eta)."""
    p = lbq.Params(walls_z=True, xi=0.0)
    H, g = 16, 1e-6
    shape = (H, 1, 4)
    b = np.zeros((3,) + shape)
    b[0] = g
    lat = make(lcbp, shape, "f64", p, path)
    lat.set_q(np.zeros((5,) + shape)).init_f_equilibrium(1.0).set_body_force(b)
    nsteps = 1500
    lat.step(nsteps)
    assert lat.path()[0] == (path == "auto")
    Q = np.zeros(shape + (3, 3))
    f = lbq.init_f_equilibrium(Q, p)
    f, Q = lbq.run(f, Q, p, nsteps, b_ext=np.moveaxis(b, 0, -1))
    u = lat.read_u()
    assert np.abs(u - oracle_u(f)).max() < 1e-15
    # half-way bounce-back converges at second order; at H = 16 the peak sits
    # 9.1 % above g H^2 / (8 eta) (2.4 % at H = 32, 0.6 % at H = 64 in the oracle pin)
    umax = g * H * H / (8 * p.tau_f / 3)
    assert 0.0 < u[0].max() / umax - 1.0 < 0.1


# (nz, ny, nx): 70 and 130 planes are more than one CTA marches through (at
# most 64), so z-chunks start and end at the walls and inside the lattice;
# ragged tiles in x (36, 68) and y (13)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape", [(70, 13, 36), (130, 8, 8), (33, 9, 68)])
def test_fast_walls_match_generic(lcbp, shape, dtype):
    """The two kernel sets compute the same walled step: bitwise-close in FP64,
    within FP32 rounding of the operation order otherwise."""
    p = lbq.Params(walls_z=True, q_wall=PLANAR)
    a = make(lcbp, shape, dtype, p)
    b = make(lcbp, shape, dtype, p, "generic")
    for lat in (a, b):
        lat.init_q(lcbp.BPII, 0.3, noise=1e-3, seed=4).init_f_equilibrium(1.0).step(20)
    assert a.path()[0] and not b.path()[0] and a.path()[2] == 1
    tq, tu, tf = (1e-13, 1e-15, 1e-15) if dtype == "f64" else (1e-6, 1e-8, 2.0 ** -23)
    assert np.abs(a.read_q() - b.read_q()).max() < tq
    assert np.abs(a.read_u() - b.read_u()).max() < tu
    assert np.abs(a.read_f() - b.read_f()).max() <= tf


def test_fast_walls_follow_a_new_q_wall(lcbp):
    """q_wall is a launch argument of the fast kernels: changing it after a
    captured step takes effect on the next step."""
    p = lbq.Params(walls_z=True, q_wall=PLANAR)
    shape = (8, 4, 8)
    other = (0.0, 0.1, 0.0, 0.1, 0.0)
    a = make(lcbp, shape, "f64", p)
    b = make(lcbp, shape, "f64", p, "generic")
    for lat in (a, b):
        lat.init_q(lcbp.BPII, 0.3, noise=1e-3, seed=9).init_f_equilibrium(1.0).step(4)
        lat.set_walls(True, other)
        lat.step(4)
    assert a.path()[0]
    assert np.abs(a.read_q() - b.read_q()).max() < 1e-13


def test_checkpoint_keeps_walls(lcbp, tmp_path):
    p = lbq.Params(walls_z=True, q_wall=PLANAR)
    shape = (6, 4, 4)
    a = make(lcbp, shape, "f32", p)
    a.init_q(lcbp.BPII, 0.3, noise=1e-3, seed=2).init_f_equilibrium(1.0).step(3)
    path = str(tmp_path / "w.bin")
    a.save(path)
    c = make(lcbp, shape, "f32", lbq.Params())  # periodic until the checkpoint says otherwise
    c.load(path)
    a.step(5)
    c.step(5)
    assert np.array_equal(a.read_q(), c.read_q()) and np.array_equal(a.read_f(), c.read_f())


def test_surrogate_refuses_walls(lcbp):
    lat = lcbp.Lattice(8, 8, 8).set_walls(True)
    lat.init_q(lcbp.BPII, 0.3).init_f_equilibrium(1.0)
    sur = lcbp.Surrogate(8, 8, 8)
    with pytest.raises(lcbp.LcbpError) as e:
        sur.step(lat, 1.0, -0.5, 1)
    assert e.value.code == lcbp.EINVAL
