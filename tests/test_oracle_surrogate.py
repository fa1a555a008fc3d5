"""Pins of the surrogate oracle: library correlation, adjointness, finite differences."""

import numpy as np
import pytest

from oracle import surrogate as S


def test_conv_matches_library_periodic_correlation():
    from scipy import ndimage
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 5, 6, 7))
    W = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=2)
    y = S.conv(x, W, b)
    for co in range(2):
        want = np.full(x.shape[1:], b[co])
        for ci in range(3):
            # kernel k[dz+1, dy+1, dx+1] = W[t, ci, co]; correlate: out(r) = sum k(o) x(r + o)
            k = np.zeros((3, 3, 3))
            for t, (dx, dy, dz) in enumerate(S.OFFSETS):
                k[dz + 1, dy + 1, dx + 1] = W[t, ci, co]
            want += ndimage.correlate(x[ci], k, mode="wrap")
        assert np.abs(y[co] - want).max() < 1e-12


def test_conv_backward_is_adjoint_and_matches_fd():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 4, 5, 3))
    W = rng.normal(size=(27, 4, 3))
    b = np.zeros(3)
    dy = rng.normal(size=(3, 4, 5, 3))
    dx, dW, db = S.conv_backward(x, W, dy)
    # adjointness <conv(x), dy> = <x, dx>
    assert abs(np.sum(S.conv(x, W, b) * dy) - np.sum(x * dx)) < 1e-10
    # dW by central differences of L = <conv(x, W), dy>
    h = 1e-6
    for (t, i, o) in [(0, 0, 0), (13, 2, 1), (26, 3, 2), (5, 1, 0)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[t, i, o] += h
        Wm[t, i, o] -= h
        fd = (np.sum(S.conv(x, Wp, b) * dy) - np.sum(S.conv(x, Wm, b) * dy)) / (2 * h)
        assert abs(fd - dW[t, i, o]) < 1e-6
    assert np.allclose(db, dy.sum(axis=(1, 2, 3)))


def test_network_gradients_by_finite_differences():
    """2 residual blocks, 4 channels, 6^3 lattice: every parameter group and the
    input gradient against central differences of the masked MSE."""
    rng = np.random.default_rng(2)
    blocks = 2
    P = S.init_params(3, 4, 2, blocks, rng, scale=1.5)
    x = rng.normal(size=(3, 6, 6, 6))
    target = rng.normal(size=(2, 6, 6, 6)) * 0.1
    mask = (rng.uniform(size=(6, 6, 6)) > 0.3).astype(float)

    def loss(P_, x_):
        y, _ = S.forward(P_, x_, blocks)
        return S.masked_mse(y, target, mask)[0]

    y, acts = S.forward(P, x, blocks)
    _, dout = S.masked_mse(y, target, mask)
    G, dx = S.backward(P, acts, dout, blocks)
    h = 1e-6
    for name in S.layer_names(blocks):
        W, b = P[name]
        for idx in [(0, 0, 0), (13, W.shape[1] - 1, W.shape[2] - 1), (20, 1, 0)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            fd = (loss({**P, name: (Wp, b)}, x) - loss({**P, name: (Wm, b)}, x)) / (2 * h)
            assert abs(fd - G[name][0][idx]) < 1e-7 + 1e-5 * abs(fd), (name, idx)
        bp, bm = b.copy(), b.copy()
        bp[0] += h
        bm[0] -= h
        fd = (loss({**P, name: (W, bp)}, x) - loss({**P, name: (W, bm)}, x)) / (2 * h)
        assert abs(fd - G[name][1][0]) < 1e-7 + 1e-5 * abs(fd), name
    for idx in [(0, 1, 2, 3), (2, 5, 0, 4)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss(P, xp) - loss(P, xm)) / (2 * h)
        assert abs(fd - dx[idx]) < 1e-7 + 1e-5 * abs(fd)


def test_adam_first_step_moves_by_lr():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 2.0])
    w1, m, v = S.adam_update(w, g, np.zeros(3), np.zeros(3), 1, lr=1e-2)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step = lr * sign(g)
    assert np.allclose(w1, w - 1e-2 * np.sign(g), atol=1e-7)


def test_bf16_rounding_matches_library():
    import torch
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-6, 6, size=1000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16(x), want)


def test_flatten_roundtrip_and_count():
    rng = np.random.default_rng(4)
    P = S.init_params(10, 32, 5, 4, rng)
    v = S.flatten(P, 4)
    assert v.size == 27 * 10 * 32 + 32 + 8 * (27 * 32 * 32 + 32) + 27 * 32 * 5 + 5 == 234437
    Q = S.unflatten(v, P, 4)
    assert all(np.array_equal(P[k][0], Q[k][0]) and np.array_equal(P[k][1], Q[k][1]) for k in P)
