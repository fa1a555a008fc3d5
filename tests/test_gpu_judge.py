"""The judged surrogate run of the library (lcbp_judge_*), through the C ABI.

The judge is orchestration over calls that are parity-tested elsewhere (the
coupled step against the FP64 oracle, the surrogate network against its
oracle).  What these tests pin is the orchestration itself:

* a judgement that always fails (tol_F = 0) rolls every segment back and
  redoes it with plain steps, so the run equals a plain run bitwise, and its
  log holds the plain run's free energy and defect fraction;
* a judgement that always passes gives exactly the call and step counts of
  the segment arithmetic, and the state of the same calls made by hand
  (surrogate calls, re-equilibration, ten plain steps per segment);
* a non-finite surrogate state fails the judgement (NaN weights), and a NaN
  planted in a host-uploaded Q is refused at the boundary;
* the weights file round-trips the network bitwise.
"""

import numpy as np
import pytest

from oracle import surrogate as S
from paper_0901_3293_gb300 import synth

pytestmark = pytest.mark.gpu
BLOCKS = 4
SHAPE = (64, 32, 32)  # (nz, ny, nx): a small slab
KAPPA, TAU = 1.0, -0.5


@pytest.fixture(scope="module")
def lcbp():
    import torch
    from paper_0901_3293_gb300 import build
    build.build()
    from paper_0901_3293_gb300 import lcbp as L
    torch.cuda.set_device(0)
    return L


def slab(L):
    nz, ny, nx = SHAPE
    lat = L.Lattice(nx, ny, nz, dtype="f32")
    lat.set_ldg_kappa_tau(0.01, 2 * np.pi / 16, KAPPA, TAU).set_flow(2.0, 0.7, 0.3, True, L.JACOBI)
    lat.init_q(L.SLAB_BPII_IN_CHOL, 0.3, noise=1e-4, seed=11, z0=nz // 8).init_f_equilibrium(1.0)
    return lat


def surrogate(L, seed=3, scale=0.5):
    nz, ny, nx = SHAPE
    sur = L.Surrogate(nx, ny, nz)
    sur.set_scales(1e-3, 1e-4, 3e-6)
    sur.set_params(S.flatten(S.init_params(15, 32, 5, BLOCKS, np.random.default_rng(seed), scale=scale), BLOCKS))
    return sur


def test_failing_judgement_equals_plain_run_bitwise(lcbp):
    L = lcbp
    lat, ref = slab(L), slab(L)
    sur = surrogate(L)
    judge = L.Judge(lat, sur, KAPPA, TAU, calls_per_segment=4, tol_F=0.0)
    t, F, D = judge.advance(200, log_every=100)
    st = judge.stats()
    # segments of 4 calls from t = 0, 40, 80, 120 and of 3 from 160 (a judge's ten
    # steps must fit before t_end), each redone plainly; the last 10 steps plain
    assert st["t"] == 200 and st["accepted"] == 0 and st["fallbacks"] == st["segments"] == 5
    assert st["surrogate_calls"] == 0 and st["plain_steps"] == 200
    assert np.isfinite(st["last_gap_F"]) and st["last_gap_F"] > 0
    F_ref, D_ref = [], []
    for _ in range(2):
        ref.step(100)
        F_ref.append(ref.free_energy())
        D_ref.append(ref.defect_fraction(0.19))
    assert list(t) == [100, 200]
    assert list(F) == F_ref and list(D) == D_ref
    assert np.array_equal(lat.read_f(), ref.read_f())
    assert np.array_equal(lat.read_q(dtype=np.float32), ref.read_q(dtype=np.float32))
    assert np.array_equal(lat.read_u(dtype=np.float32), ref.read_u(dtype=np.float32))
    judge.close()


def test_passing_judgement_counts_and_replays_by_hand(lcbp):
    L = lcbp
    lat, ref = slab(L), slab(L)
    sur = surrogate(L)
    judge = L.Judge(lat, sur, KAPPA, TAU, calls_per_segment=4, tol_F=1e30)
    t, F, _ = judge.advance(200, log_every=50)
    st = judge.stats()
    # segments of 4 calls + 10 judge steps = 50 steps each: 0, 50, 100, 150 -> 200
    assert st["t"] == 200 and st["segments"] == st["accepted"] == 4 and st["fallbacks"] == 0
    assert st["surrogate_calls"] == 16 and st["plain_steps"] == 40
    assert list(t) == [50, 100, 150, 200]
    # the same calls by hand
    F_hand = []
    for _ in range(4):
        sur.step(ref, KAPPA, TAU, 4)
        ref.reequilibrate_f().step(10)
        F_hand.append(ref.free_energy())
    assert list(F) == F_hand
    assert np.array_equal(lat.read_q(dtype=np.float32), ref.read_q(dtype=np.float32))
    assert np.array_equal(lat.read_f(), ref.read_f())
    # the judge's own copy leaves no trace: gaps were measured and finite
    assert np.isfinite(st["max_gap_F"]) and np.isfinite(st["last_gap_Q"]) and st["last_gap_Q"] > 0
    judge.close()


def test_q_tolerance_decides_too(lcbp):
    """With tol_F wide open, a max |dQ| bound below the measured gap rolls back."""
    L = lcbp
    lat = slab(L)
    sur = surrogate(L)
    judge = L.Judge(lat, sur, KAPPA, TAU, calls_per_segment=2, tol_F=1e30, tol_Q=1e-30)
    judge.advance(60)
    st = judge.stats()
    assert st["accepted"] == 0 and st["fallbacks"] == st["segments"] >= 1
    judge.close()


def test_non_finite_state_fails_the_judgement(lcbp):
    """NaN weights make the surrogate state non-finite: every segment is
    rolled back and the run equals a plain run; a NaN planted in a host Q is
    refused before it reaches the state."""
    L = lcbp
    lat, ref = slab(L), slab(L)
    sur = surrogate(L)
    p = sur.get_params()
    p[-1] = np.nan  # the output layer's last bias: a NaN in an earlier layer can die in a ReLU
    sur.set_params(p)
    judge = L.Judge(lat, sur, KAPPA, TAU, calls_per_segment=3, tol_F=1e30)
    judge.advance(120)
    st = judge.stats()
    assert st["accepted"] == 0 and st["fallbacks"] == st["segments"] and not np.isfinite(st["last_gap_F"])
    ref.step(120)
    assert np.array_equal(lat.read_q(dtype=np.float32), ref.read_q(dtype=np.float32))
    q = lat.read_q()
    q[1, 3, 4, 5] = np.nan
    with pytest.raises(L.LcbpError) as e:
        lat.set_q(q)
    assert e.value.code == L.ENONFINITE
    assert np.array_equal(lat.read_q(dtype=np.float32), ref.read_q(dtype=np.float32))
    judge.close()


def test_judge_rejects_bad_arguments(lcbp):
    L = lcbp
    lat = slab(L)
    sur = surrogate(L)
    with pytest.raises(L.LcbpError) as e:
        L.Judge(lat, sur, KAPPA, TAU, calls_per_segment=0)
    assert e.value.code == L.EINVAL
    judge = L.Judge(lat, sur, KAPPA, TAU, calls_per_segment=2)
    with pytest.raises(L.LcbpError) as e:
        judge.advance(100, log_every=15)  # not a multiple of ten
    assert e.value.code == L.EINVAL
    judge.close()


def test_weights_file_roundtrip(lcbp, tmp_path):
    L = lcbp
    nz, ny, nx = SHAPE
    sur = surrogate(L, seed=8, scale=1.0)
    path = str(tmp_path / "w.lcbpsur")
    sur.save(path)
    other = L.Surrogate(16, 8, 4)  # weights do not depend on the lattice size
    other.load(path)
    assert np.array_equal(other.get_params(), sur.get_params())
    again = L.Surrogate(nx, ny, nz).load(path)
    shape = SHAPE
    q5 = synth.smooth_q5(shape, 0.3, 1)
    u3 = synth.random_velocity(shape, 2e-4, 2)
    r5 = synth.random_q5(shape, 1e-5, 3)
    assert np.array_equal(again.forward(q5, u3, r5, KAPPA, TAU), sur.forward(q5, u3, r5, KAPPA, TAU))
    # a damaged file is refused
    raw = bytearray(open(path, "rb").read())
    raw[0] = ord("X")
    bad = tmp_path / "bad.lcbpsur"
    bad.write_bytes(bytes(raw))
    with pytest.raises(L.LcbpError) as e:
        again.load(str(bad))
    assert e.value.code == L.EIO
    (tmp_path / "short.lcbpsur").write_bytes(open(path, "rb").read()[:1000])
    with pytest.raises(L.LcbpError) as e:
        again.load(str(tmp_path / "short.lcbpsur"))
    assert e.value.code == L.EIO


def test_snapshot_restore_is_bitwise(lcbp):
    import torch
    L = lcbp
    lat = slab(L)
    lat.step(7)
    buf = torch.empty(lat.snapshot_bytes(), dtype=torch.uint8, device="cuda")
    lat.snapshot(buf)
    f0, q0 = lat.read_f(), lat.read_q()
    lat.step(5)
    lat.restore(buf)
    assert np.array_equal(lat.read_f(), f0) and np.array_equal(lat.read_q(), q0)
    a = lat.step(9).read_q()
    lat.restore(buf).step(9)
    assert np.array_equal(lat.read_q(), a)
