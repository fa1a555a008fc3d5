"""The energy exactly as printed (L2 = 0) and a general L2 on the GPU against the oracle."""

import numpy as np
import pytest

from oracle import initial, lbq
from paper_0901_3293_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lcbp():
    import torch
    from paper_0901_3293_gb300 import build
    build.build()
    from paper_0901_3293_gb300 import lcbp as L
    torch.cuda.set_device(0)
    return L


def make(L, shape, dtype, p):
    nz, ny, nx = shape
    lat = L.Lattice(nx, ny, nz, dtype=dtype)
    lat.set_ldg(p.A0, p.gamma, p.K, p.q0)
    lat.set_flow(p.tau_f, p.xi, p.Gamma, p.flow_on, L.GAUSS_SEIDEL if p.coupling == "gauss_seidel" else L.JACOBI)
    lat.set_l2(p.L2)
    return lat


def oracle_u(f):
    return np.moveaxis(lbq.moments(f)[1], -1, 0)


@pytest.mark.parametrize("L2", [0.0, 0.004])
@pytest.mark.parametrize("shape", [(6, 5, 8), (3, 7, 4)])
def test_one_step_with_l2_f64(lcbp, shape, L2):
    p = lbq.Params(L2=L2)
    q5 = synth.smooth_q5(shape, 0.3, 1) + synth.random_q5(shape, 1e-2, 2)
    f15 = synth.random_distributions(shape, 3, amp=2e-3)
    lat = make(lcbp, shape, "f64", p)
    lat.set_q(q5).set_f(f15).step(1)
    assert not lat.path()[0]
    f, Q = lbq.step(lbq.f_from_soa(f15), lbq.q5_to_q9(q5), p)
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 1e-14
    assert np.abs(lat.read_f() - lbq.f_to_soa(f)).max() < 1e-14
    assert np.abs(lat.read_u() - oracle_u(f)).max() < 1e-14


@pytest.mark.parametrize("coupling,flow_on", [("jacobi", True), ("gauss_seidel", True), ("jacobi", False)])
def test_ten_steps_printed_energy_f64(lcbp, coupling, flow_on):
    p = lbq.Params(L2=0.0, coupling=coupling, flow_on=flow_on)
    shape = (8, 6, 5)
    q5 = initial.init_q5(shape, initial.BPII, p.q0, 0.3, 1e-2, 9)
    f15 = synth.random_distributions(shape, 8, amp=2e-3)
    lat = make(lcbp, shape, "f64", p)
    lat.set_q(q5).set_f(f15).step(10)
    f, Q = lbq.run(lbq.f_from_soa(f15), lbq.q5_to_q9(q5), p, 10)
    assert np.abs(lat.read_q() - lbq.q9_to_q5(Q)).max() < 1e-13
    assert np.abs(lat.read_f() - lbq.f_to_soa(f)).max() < 1e-14


def test_free_energy_with_l2(lcbp):
    shape = (6, 5, 7)
    q5 = synth.smooth_q5(shape, 0.3, 4) + synth.random_q5(shape, 0.05, 5)
    for L2 in (0.0, 0.004, None):
        p = lbq.Params(L2=L2)
        lat = make(lcbp, shape, "f64", p)
        lat.set_q(q5)
        F = lbq.free_energy(lbq.q5_to_q9(q5), p)
        assert abs(lat.free_energy() - F) < 1e-12 * max(1.0, abs(F))


def test_l2_and_walls_exclude_each_other(lcbp):
    lat = lcbp.Lattice(4, 4, 4).set_l2(0.0)
    with pytest.raises(lcbp.LcbpError):
        lat.set_walls(True)
    lat = lcbp.Lattice(4, 4, 4).set_walls(True)
    with pytest.raises(lcbp.LcbpError):
        lat.set_l2(0.0)
