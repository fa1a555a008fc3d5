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


@pytest.mark.parametrize("path", ["generic", "fast"])
def test_batch_equals_single_lattices_bitwise_f32(lcbp, path):
    """Three classes (32^3, 48^3 and one 20 x 12 x 8 replica): on either path
    every replica equals the lattice stepped alone on the same path."""
    sweep = synth.replica_sweep(6)
    sweep[1]["dims"] = (20, 12, 8)  # a ragged replica among the cubes
    dims = [s["dims"] for s in sweep]
    params = [replica_params(s["kappa"], s["tau"]) for s in sweep]
    kinds = [initial.BPII, initial.CHOL_Z, initial.ISO_NOISE]
    b = lcbp.Batch(dims, params, dtype="f32")
    b.set_path(lcbp.PATH_GENERIC if path == "generic" else lcbp.PATH_FAST1)
    for r, s in enumerate(sweep):
        b.init_q(r, kinds[s["kind"]], 0.3 if s["kind"] == 0 else 0.4, noise=1e-3, seed=s["seed"])
    b.init_f_equilibrium(1.0).step(25)
    assert b.path()[0] == (path == "fast")
    for r, s in enumerate(sweep):
        nx, ny, nz = s["dims"]
        p = params[r]
        lat = lcbp.Lattice(nx, ny, nz, dtype="f32")
        lat.set_path(lcbp.PATH_GENERIC if path == "generic" else lcbp.PATH_FAST1)
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


# classes of equal dims with nx % 4 == 0: the fast path; one class has a single replica
FAST_MIXED = [((8, 8, 8), 0.5, -0.5, initial.BPII), ((12, 10, 6), 1.0, 0.0, initial.CHOL_Z),
              ((8, 8, 8), 2.0, -1.0, initial.ISO_NOISE), ((16, 6, 9), 1.5, 0.3, initial.CHOL_X),
              ((12, 10, 6), 0.3, 0.5, initial.BPII)]


def test_fast_batch_matches_oracle_f64(lcbp):
    dims = [d for d, *_ in FAST_MIXED]
    params = [replica_params(k, t) for _, k, t, _ in FAST_MIXED]
    b = lcbp.Batch(dims, params, dtype="f64").set_path(lcbp.PATH_FAST1)
    for r, (d, k, t, kind) in enumerate(FAST_MIXED):
        b.init_q(r, kind, 0.3 if kind == initial.BPII else 0.4, noise=1e-2, seed=200 + r)
    b.init_f_equilibrium(1.0).step(10)
    fast, zc = b.path()
    assert fast and zc >= 1
    for r, (d, k, t, kind) in enumerate(FAST_MIXED):
        nx, ny, nz = d
        p = lbq.Params(**params[r])
        Q = initial.init_q9((nz, ny, nx), kind, p.q0, 0.3 if kind == initial.BPII else 0.4, 1e-2, 200 + r)
        f = lbq.init_f_equilibrium(Q, p)
        f, Q = lbq.run(f, Q, p, 10)
        assert np.abs(b.read_q(r) - lbq.q9_to_q5(Q)).max() < 1e-13, r
        assert np.abs(b.read_u(r) - np.moveaxis(lbq.moments(f)[1], -1, 0)).max() < 1e-14, r


def test_fast_batch_matches_generic_batch_f32(lcbp):
    """The 48-replica sweep's two classes, a few replicas each: fast and generic
    batches agree to FP32 rounding after 20 steps."""
    sweep = synth.replica_sweep(8)
    dims = [s["dims"] for s in sweep]
    params = [replica_params(s["kappa"], s["tau"]) for s in sweep]
    kinds = [initial.BPII, initial.CHOL_Z, initial.ISO_NOISE]
    out = {}
    for path in (lcbp.PATH_FAST1, lcbp.PATH_GENERIC):
        b = lcbp.Batch(dims, params, dtype="f32").set_path(path)
        for r, s in enumerate(sweep):
            b.init_q(r, kinds[s["kind"]], 0.3 if s["kind"] == 0 else 0.4, noise=1e-3, seed=s["seed"])
        b.init_f_equilibrium(1.0).step(20)
        assert b.path()[0] == (path == lcbp.PATH_FAST1)
        out[path] = [(b.read_q(r, np.float32), b.read_u(r, np.float32)) for r in range(len(sweep))]
        b.close()
    for r in range(len(sweep)):
        (qa, ua), (qg, ug) = out[lcbp.PATH_FAST1][r], out[lcbp.PATH_GENERIC][r]
        # the same bounds as a single lattice's fast-against-generic check
        assert np.abs(qa - qg).max() < 1e-6, r
        assert np.abs(ua - ug).max() < 1e-8, r


def test_batch_path_rules(lcbp):
    """More than four classes, an nx not divisible by 4, flow off or
    Gauss-Seidel coupling: the generic kernels even when the fast ones are
    asked for; AUTO keeps the faster of the two after timing both."""
    p = replica_params(1.0, 0.0)
    five = lcbp.Batch([(8, 4, 4), (8, 4, 5), (8, 4, 6), (8, 4, 7), (8, 4, 8)], [p] * 5).set_path(lcbp.PATH_FAST1)
    ragged = lcbp.Batch([(8, 8, 8), (6, 8, 8)], [p] * 2).set_path(lcbp.PATH_FAST1)
    ok = lcbp.Batch([(8, 8, 8), (12, 4, 4)], [p] * 2).set_path(lcbp.PATH_FAST1)
    for b in (five, ragged, ok):
        for r in range(b.R):
            b.init_q(r, initial.BPII, 0.3, noise=1e-3, seed=r)
        b.init_f_equilibrium(1.0).step(2)
    assert not five.path()[0] and not ragged.path()[0] and ok.path()[0]
    ok.set_flow(True, lcbp.GAUSS_SEIDEL).step(1)
    assert not ok.path()[0]
    ok.set_flow(True, lcbp.JACOBI).step(1)
    assert ok.path()[0]
    ok.set_flow(False).step(1)
    assert not ok.path()[0]
    with pytest.raises(lcbp.LcbpError):
        ok.set_path(lcbp.PATH_FAST2)
    ok.set_flow(True, lcbp.JACOBI).set_path(lcbp.PATH_AUTO).step(1)
    fast, zc = ok.path()
    assert (zc >= 1) if fast else (zc == 0)
    for b in (five, ragged, ok):
        b.close()


@pytest.mark.parametrize("dims_list", [[(8, 8, 8)], [(8, 4, 3), (12, 4, 5), (4, 8, 9), (16, 12, 2)],
                                       [(48, 20, 5), (16, 36, 3), (40, 12, 4)]])
def test_fast_batch_edge_counts_bitwise_f32(lcbp, dims_list):
    """One replica, exactly four classes (one replica each, with nz of 2, 3, 5
    and 9), and classes of narrow tiles (16 x 16 sites, taken where a 32-wide
    tile would be at most half full) with ragged rows and columns: the fast
    batch equals the lattices stepped alone on the fast kernels (32 x 8
    tiles), bit for bit."""
    params = [replica_params(0.5 + 0.4 * r, -0.3 + 0.2 * r) for r in range(len(dims_list))]
    b = lcbp.Batch(dims_list, params, dtype="f32").set_path(lcbp.PATH_FAST1)
    for r in range(len(dims_list)):
        b.init_q(r, initial.BPII, 0.3, noise=1e-3, seed=50 + r)
    b.init_f_equilibrium(1.0).step(7)
    assert b.path()[0]
    for r, (nx, ny, nz) in enumerate(dims_list):
        p = params[r]
        lat = lcbp.Lattice(nx, ny, nz, dtype="f32")
        lat.set_path(lcbp.PATH_FAST1)
        lat.set_ldg(p["A0"], p["gamma"], p["K"], p["q0"]).set_flow(p["tau_f"], p["xi"], p["Gamma"])
        lat.init_q(initial.BPII, 0.3, noise=1e-3, seed=50 + r)
        lat.init_f_equilibrium(1.0).step(7)
        assert lat.path()[0]
        assert np.array_equal(b.read_q(r, np.float32), lat.read_q(dtype=np.float32)), r
        assert np.array_equal(b.read_u(r, np.float32), lat.read_u(dtype=np.float32)), r
        lat.close()
    b.close()
