"""Polarised-light texture kernel (Sec. 2.3) against the FP64 optics oracle."""

import numpy as np
import pytest

from oracle import initial, lbq, optics
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


def nematic_field(shape, seed, S=0.4):
    """Smoothly varying uniaxial Q plus a little biaxial noise: the largest
    eigenvalue stays well separated, so the director is well conditioned."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    th = 2 * np.pi * (x / 23.0 + y / 31.0) + rng.uniform(0, 2 * np.pi)
    ph = 0.3 + 1.2 * np.sin(2 * np.pi * z / 17.0 + y / 9.0)
    n = np.stack([np.sin(ph) * np.cos(th), np.sin(ph) * np.sin(th), np.cos(ph)], axis=-1)
    Q9 = S * (n[..., :, None] * n[..., None, :] - np.eye(3) / 3.0)
    Q9 += lbq.q5_to_q9(synth.random_q5(shape, 0.01, seed + 1))
    return lbq.q9_to_q5(Q9)


# (nz, ny, nx): ragged x tiles, z not a multiple of the 8 chunks, fewer planes than
# chunks; the last two have so few columns that each column's planes are split
# between several CTAs (4 and 3 ranges) and the range products combined after
SHAPES = [(12, 5, 40), (3, 4, 7), (33, 2, 32), (1, 3, 70), (128, 4, 8), (100, 3, 40)]


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-5), ("f64", 2e-5)])
@pytest.mark.parametrize("shape", SHAPES)
def test_texture_matches_oracle(lcbp, shape, dtype, tol):
    nz, ny, nx = shape
    q5 = nematic_field(shape, 7)
    lat = lcbp.Lattice(nx, ny, nz, dtype=dtype)
    lat.set_q(q5)
    img = lat.texture()
    want = optics.texture(lbq.q5_to_q9(lat.read_q()))
    assert img.shape == (ny, nx)
    assert np.abs(img - want).max() < tol, np.abs(img - want).max()


def test_texture_single_wavelength_and_angles(lcbp):
    shape = (10, 3, 9)
    q5 = nematic_field(shape, 3)
    lat = lcbp.Lattice(9, 3, 10)
    lat.set_q(q5)
    o = lcbp.Optics.default()
    o.nlambda = 1
    o.lambda_[0] = 12.0
    o.weight[0] = 1.0
    img = lat.texture(o)
    Q9 = lbq.q5_to_q9(lat.read_q())
    want = optics.texture(Q9, lambdas=(12.0,), weights=(1.0,))
    assert np.abs(img - want).max() < 2e-5


def test_homeotropic_and_isotropic_are_dark(lcbp):
    lat = lcbp.Lattice(8, 4, 6)
    lat.set_q(np.zeros((5, 6, 4, 8)))
    assert np.abs(lat.texture()).max() < 1e-7
    q5 = np.zeros((5, 6, 4, 8))
    q5[0] = q5[3] = -0.4 / 3  # n = z: Q_xx = Q_yy = -S/3
    lat.set_q(q5)
    assert np.abs(lat.texture()).max() < 1e-6


def test_texture_errors(lcbp):
    lat = lcbp.Lattice(4, 4, 4)
    o = lcbp.Optics.default()
    o.nlambda = 0
    with pytest.raises(lcbp.LcbpError) as e:
        lat.texture(o)
    assert e.value.code == lcbp.EINVAL
    o = lcbp.Optics.default()
    o.lambda_[1] = -1.0
    with pytest.raises(lcbp.LcbpError):
        lat.texture(o)


def test_slab_texture_sampled_columns(lcbp):
    """The 64 x 64 x 256 slab (BPII seed in a helix) after some growth, at the
    size the bench renders: the oracle on 48 sampled columns of 256 planes."""
    from paper_0901_3293_gb300 import surrogate_train as st
    lat = st.slab_lattice(1.0)
    lat.step(200)
    img = lat.texture()
    Q9 = lbq.q5_to_q9(lat.read_q())
    rng = np.random.default_rng(0)
    ys, xs = rng.integers(0, 64, size=48), rng.integers(0, 64, size=48)
    got = img[ys, xs]
    want = np.array([optics.texture(Q9[:, y:y + 1, x:x + 1])[0, 0] for y, x in zip(ys, xs)])
    err = np.abs(got - want)
    print("median", np.median(err), "max", err.max(), "mean |img|", np.abs(img).mean())
    assert err.max() < 2e-5
    # intensities lie in [0, 1/2]; FP32 rounding over 256 planes leaves ~1e-6 below 0
    assert -1e-5 <= img.min() and img.max() <= 0.5 + 1e-5
