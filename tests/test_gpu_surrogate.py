"""Tensor-core surrogate kernels against the FP64 oracle of the network.

The oracle rounds weights, inputs and stored activations / gradients to BF16
exactly where the GPU stores them (the arithmetic stays FP64), so the
comparison measures accumulation-order and FP32-epilogue differences only.
"""

import numpy as np
import pytest

from oracle import initial, lbq
from oracle import surrogate as S
from paper_0901_3293_gb300 import synth

pytestmark = pytest.mark.gpu
BLOCKS = 4


@pytest.fixture(scope="module")
def lcbp():
    import torch
    from paper_0901_3293_gb300 import build
    build.build()
    from paper_0901_3293_gb300 import lcbp as L
    torch.cuda.set_device(0)
    return L


S_U, S_R, S_DQ = 1e-3, 1e-3, 1e-3


def net_input(q5, u3, r5, kappa, tau):
    """Channels of the network input (the surrogate's definition)."""
    x = np.zeros((15,) + q5.shape[1:])
    x[:5] = q5
    x[5:8] = u3 / S_U
    x[8] = kappa - 1.0
    x[9] = tau
    x[10:15] = r5 / S_R
    return x


def random_params(seed, scale=1.5):
    return S.init_params(15, 32, 5, BLOCKS, np.random.default_rng(seed), scale=scale)


KERNELS = ["CONV_TAPS", "CONV_WINDOW"]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("dims", [(16, 8, 6), (40, 12, 5), (32, 4, 1), (6, 70, 3)])
def test_forward_matches_oracle(lcbp, dims, kernel):
    """Both convolution kernels: one shifted tile per tap, and one staged
    window per plane (tiles of 128 linear positions of the padded plane that
    straddle rows, with ghost rows discarded)."""
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    P = random_params(10)
    q5 = synth.smooth_q5(shape, 0.3, 11) + synth.random_q5(shape, 0.05, 12)
    u3 = synth.random_velocity(shape, 2e-4, 13)
    r5 = synth.random_q5(shape, 1e-3, 14)
    sur = lcbp.Surrogate(nx, ny, nz)
    sur.set_conv_kernel(getattr(lcbp, kernel))
    sur.set_params(S.flatten(P, BLOCKS))
    y = sur.forward(q5, u3, r5, 1.3, -0.4)
    x = net_input(q5, u3, r5, 1.3, -0.4)
    y_q, _ = S.forward(P, x, BLOCKS, quant=S.bf16)
    y_e, _ = S.forward(P, x, BLOCKS)
    scale = np.abs(y_e).max()
    err_q = np.abs(y - y_q).max() / scale
    err_e = np.abs(y - y_e).max() / scale
    print(f"{dims}: max|y| {scale:.3e}, rel err vs BF16-rounding oracle {err_q:.2e}, vs FP64 {err_e:.2e}")
    assert err_q < 1e-2 and err_e < 5e-2


# (conv kernel, dims): the weight gradients run on the tensor cores (plane
# windows staged in shared memory; three stages for the 32-wide planes, two
# for the 144-wide ones), and on the CUDA-core kernel for the 200-wide plane,
# whose windows do not fit
@pytest.mark.parametrize("kernel,dims", [("CONV_TAPS", (32, 8, 6)), ("CONV_WINDOW", (32, 8, 6)),
                                         ("CONV_TAPS", (144, 4, 2)), ("CONV_TAPS", (200, 4, 2))])
def test_training_gradients_match_oracle(lcbp, kernel, dims):
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    P = random_params(20)
    q5 = synth.smooth_q5(shape, 0.3, 21)
    u3 = synth.random_velocity(shape, 2e-4, 22)
    r5 = synth.random_q5(shape, 1e-3, 24)
    # a realistic target: ten Euler steps of the rate plus a small correction
    dq = 10.0 * r5 + synth.random_q5(shape, 5e-4, 23)
    mask = (np.arange(nz)[:, None, None] * np.ones(shape) >= 1).astype(np.float64)
    sur = lcbp.Surrogate(nx, ny, nz, training=True)
    sur.set_conv_kernel(getattr(lcbp, kernel))
    sur.set_params(S.flatten(P, BLOCKS))
    loss = sur.train_step(q5, u3, r5, 0.9, 0.2, dq, mask, lr=1e-6)
    g = S.unflatten(sur.get_grads().astype(np.float64), P, BLOCKS)
    x = net_input(q5, u3, r5, 0.9, 0.2)
    y, acts = S.forward(P, x, BLOCKS, quant=S.bf16)
    # the network learns the correction to ten Euler steps of the rate
    loss_o, dout = S.masked_mse(y, (dq - 10.0 * r5) / S_DQ, mask)
    G, _ = S.backward(P, acts, dout, BLOCKS, quant=S.bf16)
    # the same gradients with no BF16 rounding anywhere (plain FP64 network)
    y_e, acts_e = S.forward(P, x, BLOCKS)
    _, dout_e = S.masked_mse(y_e, (dq - 10.0 * r5) / S_DQ, mask)
    G_e, _ = S.backward(P, acts_e, dout_e, BLOCKS)
    assert abs(loss - loss_o) < 1e-3 * loss_o
    # Element-wise bounds, per layer, relative to the layer's largest gradient.
    # BF16 keeps 8 significant bits (unit roundoff u = 2^-8).  Against the
    # oracle that rounds where the kernels store, only the FP32 accumulation
    # order differs: a stored activation or gradient can land one BF16 ulp
    # (2u) away, and a weight gradient sums products of several such stored
    # tensors, so its worst element can sit a few ulps off: 5e-2 (about six
    # ulps) bounds every element, while a wrong tap or channel is off by O(1).
    # Against the unrounded FP64 network the gradient of each weight passes
    # through about twenty BF16 roundings (ten stored activations, ten stored
    # gradients); to first order that is 20u = 8e-2, so 1e-1 bounds every element.
    for name in S.layer_names(BLOCKS):
        for k in (0, 1):
            got, ref, ref_e = g[name][k], G[name][k], G_e[name][k]
            err_q = np.abs(got - ref).max() / np.abs(ref).max()
            err_e = np.abs(got - ref_e).max() / np.abs(ref_e).max()
            print(name, "W" if k == 0 else "b", f"max err / max|g|: vs BF16 oracle {err_q:.2e}, vs FP64 {err_e:.2e}")
            assert err_q < 5e-2, (name, k, err_q)
            assert err_e < 1e-1, (name, k, err_e)
    # Adam moved the parameters by about lr
    step = sur.get_params().astype(np.float64) - S.flatten(P, BLOCKS)
    assert 0 < np.abs(step).max() < 1.5e-6


def test_tensor_core_weight_gradients_match_cuda_cores_over_many_items(lcbp):
    """32 x 32 x 72: 648 items of 128 plane positions, so each of the (up to
    152) CTAs of the tensor-core kernel takes four or five and its ring of
    three stages wraps.  The same training step with the weight gradients on
    the CUDA-core kernel (FP32 atomics) gives the same loss bitwise (the
    forward pass is the same) and the same gradients up to the FP32
    accumulation order: 1e-3 of each layer's largest gradient bounds every
    element, while a dropped item, a wrong stage or a stale tile is off by
    O(1)."""
    nx, ny, nz = 32, 32, 72
    shape = (nz, ny, nx)
    P = random_params(30)
    q5 = synth.smooth_q5(shape, 0.3, 31)
    u3 = synth.random_velocity(shape, 2e-4, 32)
    r5 = synth.random_q5(shape, 1e-3, 33)
    dq = 10.0 * r5 + synth.random_q5(shape, 5e-4, 34)
    mask = np.ones(shape)
    out = {}
    for name, kind in (("tc", lcbp.CONV_WINDOW), ("cc", lcbp.CONV_WINDOW | lcbp.CONV_DW_CUDA_CORES)):
        sur = lcbp.Surrogate(nx, ny, nz, training=True)
        sur.set_conv_kernel(kind)
        sur.set_params(S.flatten(P, BLOCKS))
        loss = sur.train_step(q5, u3, r5, 0.9, 0.2, dq, mask, lr=1e-6)
        out[name] = (loss, S.unflatten(sur.get_grads().astype(np.float64), P, BLOCKS))
        sur.close()
    assert out["tc"][0] == out["cc"][0]
    for layer in S.layer_names(BLOCKS):
        for k in (0, 1):
            a, b = out["tc"][1][layer][k], out["cc"][1][layer][k]
            err = np.abs(a - b).max() / np.abs(b).max()
            print(layer, "W" if k == 0 else "b", f"max |tc - cc| / max|g| {err:.2e}")
            assert err < 1e-3, (layer, k, err)


def test_surrogate_step_applies_prediction(lcbp):
    nx, ny, nz = 32, 8, 8
    p = lbq.Params()
    lat = lcbp.Lattice(nx, ny, nz)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-3, seed=3).init_f_equilibrium(1.0).step(5)
    q0 = lat.read_q(dtype=np.float32)
    u0 = lat.read_u(dtype=np.float32)
    r0 = lat.read_rate(dtype=np.float32)
    # the rate is the Beris-Edwards right-hand side of the oracle
    Q9 = lbq.q5_to_q9(q0.astype(np.float64))
    R9 = lbq.be_rhs(Q9, np.moveaxis(u0.astype(np.float64), 0, -1), p)
    assert np.abs(r0 - lbq.q9_to_q5(R9)).max() < 1e-6
    sur = lcbp.Surrogate(nx, ny, nz)
    sur.set_params(S.flatten(random_params(30, scale=1.0), BLOCKS))
    y = sur.forward(q0, u0, r0, 1.0, -0.5)
    sur.step(lat, 1.0, -0.5, 1)
    q1 = lat.read_q(dtype=np.float32)
    assert np.abs(q1 - (q0 + 10.0 * r0 + S_DQ * y)).max() < 1e-6
    lat.reequilibrate_f().step(2)  # plain stepping resumes
    assert np.isfinite(lat.free_energy())


def test_window_and_tap_kernels_agree_on_slab(lcbp):
    """The two kernels on a 64 x 64 x 16 slab section (the window kernel's
    production shape): same sums, FP32 accumulation in a different order."""
    nx, ny, nz = 64, 64, 16
    shape = (nz, ny, nx)
    q5 = initial.init_q5(shape, initial.SLAB_BPII_IN_CHOL, 2 * np.pi / 16, 0.3, 1e-4, 5, z0=4)
    u3 = synth.random_velocity(shape, 2e-4, 6)
    r5 = synth.random_q5(shape, 1e-3, 7)
    params = S.flatten(random_params(40, scale=1.0), BLOCKS)
    out = {}
    for kernel in KERNELS:
        sur = lcbp.Surrogate(nx, ny, nz)
        sur.set_conv_kernel(getattr(lcbp, kernel)).set_params(params)
        out[kernel] = sur.forward(q5, u3, r5, 1.0, -0.5)
        sur.close()
    a, b = out["CONV_TAPS"], out["CONV_WINDOW"]
    # the window kernel sums the taps of two output planes in another order
    # (input plane by input plane), so the FP32 accumulations round differently
    print("bitwise equal:", np.array_equal(a, b), "max diff", np.abs(a - b).max())
    assert np.abs(a - b).max() <= 1e-2 * np.abs(a).max()
    assert np.mean(np.abs(a - b)) <= 1e-3 * np.mean(np.abs(a))


def test_window_kernel_rejected_where_it_does_not_fit(lcbp):
    sur = lcbp.Surrogate(256, 4, 2)
    with pytest.raises(lcbp.LcbpError) as e:
        sur.set_conv_kernel(lcbp.CONV_WINDOW)
    assert e.value.code == lcbp.EINVAL
    with pytest.raises(lcbp.LcbpError):
        sur.set_conv_kernel(7)
