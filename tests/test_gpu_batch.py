"""Batched replicas: every replica of a batch equals the oracle (FP64) and
equals the same lattice stepped alone (FP32, bitwise)."""

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


def replica_params(kappa, tau, q0=2 * np.pi / 16, A0=0.01):
    gamma, K = lbq.gamma_K_from_kappa_tau(A0, q0, kappa, tau)
    return dict(A0=A0, gamma=gamma, K=K, q0=q0, tau_f=2.0, xi=0.7, Gamma=0.3)


# (nx, ny, nz), kappa, tau, kind
MIXED = [((8, 8, 8), 0.5, -0.5, initial.BPII), ((12, 10, 6), 1.0, 0.0, initial.CHOL_Z),
         ((7, 5, 9), 2.0, -1.0, initial.ISO_NOISE), ((16, 16, 16), 1.5, 0.3, initial.CHOL_X),
         ((6, 6, 6), 0.3, 0.5, initial.BPII)]


def test_batch_replicas_match_oracle_f64(lcbp):
    dims = [d for d, *_ in MIXED]
    params = [replica_params(k, t) for _, k, t, _ in MIXED]
    b = lcbp.Batch(dims, params, dtype="f64")
    for r, (d, k, t, kind) in enumerate(MIXED):
        amp = 0.3 if kind == initial.BPII else 0.4
        b.init_q(r, kind, amp, noise=1e-2, seed=100 + r)
    b.init_f_equilibrium(1.0).step(10)
    info = b.info()
    assert info["R"] == 5 and info["step"] == 10 and info["persistent_ctas"] >= 1
    for r, (d, k, t, kind) in enumerate(MIXED):
        nx, ny, nz = d
        p = lbq.Params(**{kk: v for kk, v in params[r].items()})
        amp = 0.3 if kind == initial.BPII else 0.4
        Q = initial.init_q9((nz, ny, nx), kind, p.q0, amp, 1e-2, 100 + r)
        f = lbq.init_f_equilibrium(Q, p)
        f, Q = lbq.run(f, Q, p, 10)
        assert np.abs(b.read_q(r) - lbq.q9_to_q5(Q)).max() < 1e-13, r
        assert np.abs(b.read_u(r) - np.moveaxis(lbq.moments(f)[1], -1, 0)).max() < 1e-14, r
        F = b.free_energy(r)
        assert abs(F - lbq.free_energy(Q, p)) < 1e-12 * max(1.0, abs(F)), r
        m, P = b.totals(r)
        m_o, P_o = lbq.totals(f)
        assert abs(m - m_o) < 1e-10 and np.abs(P - P_o).max() < 1e-12


def test_batch_equals_single_lattices_bitwise_f32(lcbp):
    sweep = synth.replica_sweep(6)
    sweep[1]["dims"] = (20, 12, 8)  # a ragged replica among the cubes
    dims = [s["dims"] for s in sweep]
    params = [replica_params(s["kappa"], s["tau"]) for s in sweep]
    kinds = [initial.BPII, initial.CHOL_Z, initial.ISO_NOISE]
    b = lcbp.Batch(dims, params, dtype="f32")
    for r, s in enumerate(sweep):
        b.init_q(r, kinds[s["kind"]], 0.3 if s["kind"] == 0 else 0.4, noise=1e-3, seed=s["seed"])
    b.init_f_equilibrium(1.0).step(25)
    for r, s in enumerate(sweep):
        nx, ny, nz = s["dims"]
        p = params[r]
        lat = lcbp.Lattice(nx, ny, nz, dtype="f32")
        lat.set_path(lcbp.PATH_GENERIC)
        lat.set_ldg(p["A0"], p["gamma"], p["K"], p["q0"]).set_flow(p["tau_f"], p["xi"], p["Gamma"])
        lat.init_q(kinds[s["kind"]], 0.3 if s["kind"] == 0 else 0.4, noise=1e-3, seed=s["seed"])
        lat.init_f_equilibrium(1.0).step(25)
        assert np.array_equal(b.read_q(r, np.float32), lat.read_q(dtype=np.float32)), r
        assert np.array_equal(b.read_u(r, np.float32), lat.read_u(dtype=np.float32)), r
        lat.close()


def test_sweep_of_48_replicas(lcbp):
    """The 48-replica sweep: 32^3 and 48^3 lattices, kappa ~ U[0.3, 2],
    tau ~ U[-1, 0.5], kinds BPII / cholesteric / isotropic noise."""
    sweep = synth.replica_sweep(48)
    dims = [s["dims"] for s in sweep]
    params = [replica_params(s["kappa"], s["tau"]) for s in sweep]
    kinds = [initial.BPII, initial.CHOL_Z, initial.ISO_NOISE]
    b = lcbp.Batch(dims, params, dtype="f32")
    for r, s in enumerate(sweep):
        b.init_q(r, kinds[s["kind"]], 0.3 if s["kind"] == 0 else 0.4, noise=1e-2, seed=s["seed"])
    b.init_f_equilibrium(1.0)
    m0 = [b.totals(r)[0] for r in range(48)]
    b.step(40)
    info = b.info()
    assert info["sites"] == 24 * 32 ** 3 + 24 * 48 ** 3
    for r in range(48):
        m, _ = b.totals(r)
        assert abs(m - m0[r]) < 1e-6 * m0[r]
        assert np.isfinite(b.free_energy(r))
    with pytest.raises(lcbp.LcbpError):
        b.read_q(48)
