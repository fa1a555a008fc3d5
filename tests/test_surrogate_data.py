"""The quarter-turn augmentation of the surrogate's training data, on the CPU.

Training crops are rotated by quarter turns about z (surrogate_train.rotate_z
and its device twin rotate_z_device).  A rotated state is only a valid
training pair if the rotation is a proper rotation of the whole problem:
the oracle's free energy must be unchanged and its Beris-Edwards rate must
rotate with the fields.  A sign error in any component would make the map a
reflection, which flips the chiral term and fails both.
"""

import numpy as np
import pytest

from oracle import lbq
from paper_0901_3293_gb300 import surrogate_train as T
from paper_0901_3293_gb300 import synth

SHAPE = (6, 8, 8)  # (nz, ny, nx), square x-y planes


def fields(seed):
    q5 = synth.smooth_q5(SHAPE, 0.3, seed) + synth.random_q5(SHAPE, 0.02, seed + 1)
    u3 = synth.random_velocity(SHAPE, 1e-3, seed + 2)
    return q5, u3


def test_four_quarter_turns_are_the_identity():
    q5, u3 = fields(1)
    q4, u4 = T.rotate_z(q5, u3, 4)
    assert np.array_equal(q4, q5) and np.array_equal(u4, u3)
    q2, u2 = T.rotate_z(*T.rotate_z(q5, u3, 1), 1)
    q2b, u2b = T.rotate_z(q5, u3, 2)
    assert np.array_equal(q2, q2b) and np.array_equal(u2, u2b)


@pytest.mark.parametrize("turns", [1, 2, 3])
def test_free_energy_is_invariant(turns):
    p = lbq.Params()
    q5, u3 = fields(5)
    F = lbq.free_energy(lbq.q5_to_q9(q5), p)
    qr, _ = T.rotate_z(q5, u3, turns)
    assert abs(lbq.free_energy(lbq.q5_to_q9(qr), p) - F) <= 1e-12 * abs(F)


@pytest.mark.parametrize("turns", [1, 3])
def test_beris_edwards_rate_rotates_with_the_fields(turns):
    """R(rot Q, rot u) = rot R(Q, u) for the oracle's rate (flow coupling on)."""
    p = lbq.Params()
    q5, u3 = fields(9)
    R = lbq.q9_to_q5(lbq.be_rhs(lbq.q5_to_q9(q5), np.moveaxis(u3, 0, -1), p))
    qr, ur = T.rotate_z(q5, u3, turns)
    R_rot, _ = T.rotate_z(R, None, turns)
    R_of_rot = lbq.q9_to_q5(lbq.be_rhs(lbq.q5_to_q9(qr), np.moveaxis(ur, 0, -1), p))
    assert np.abs(R_of_rot - R_rot).max() <= 1e-13 * np.abs(R).max()


def test_device_twin_matches():
    torch = pytest.importorskip("torch")
    q5, u3 = fields(3)
    for turns in range(4):
        qa, ua = T.rotate_z(q5, u3, turns)
        qb, ub = T.rotate_z_device(torch.from_numpy(q5), torch.from_numpy(u3), turns)
        assert np.array_equal(qa, qb.numpy()) and np.array_equal(ua, ub.numpy())
