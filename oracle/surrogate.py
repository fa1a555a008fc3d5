"""FP64 CPU oracle of the convolutional surrogate (TEST INFRASTRUCTURE ONLY).

The surrogate is not in the paper; it is the learned part that advances Q by
k = 10 solver steps.  Its definition, restated plainly here:

* periodic 3x3x3 convolution (cross-correlation form), tap t <-> offset
  o_t = (dx, dy, dz) with t = 9 (dz+1) + 3 (dy+1) + (dx+1):
      y[co](r) = b[co] + sum_t sum_ci W[t, ci, co] x[ci](r + o_t)
* network: h = relu(conv_in(x)); 4 residual blocks h = h + conv_b2(relu(conv_b1(h)));
  out = conv_out(h)  (no activation)
* backward of one convolution:
      dx[ci](r) = sum_t sum_co W[t, ci, co] dy[co](r - o_t)
      dW[t, ci, co] = sum_r x[ci](r + o_t) dy[co](r),   db[co] = sum_r dy[co](r)

Arrays are channel-first [C, z, y, x]; shares no code with the CUDA path.
"""

from __future__ import annotations

import numpy as np

OFFSETS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shifted(x: np.ndarray, o) -> np.ndarray:
    """x(r + o) on the periodic lattice for x of shape [C, z, y, x]."""
    dx, dy, dz = o
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(1, 2, 3))


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y = b + sum_t W_t^T x(r + o_t); W: [27, C_in, C_out], b: [C_out]."""
    y = np.zeros((W.shape[2],) + x.shape[1:])
    for t, o in enumerate(OFFSETS):
        y += np.einsum("io,izyx->ozyx", W[t], shifted(x, o))
    return y + b[:, None, None, None]


def conv_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """(dx, dW, db) of conv for upstream gradient dy."""
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t, o in enumerate(OFFSETS):
        dx += np.einsum("io,ozyx->izyx", W[t], shifted(dy, tuple(-v for v in o)))
        dW[t] = np.einsum("izyx,ozyx->io", shifted(x, o), dy)
    return dx, dW, dy.sum(axis=(1, 2, 3))


def relu(v):
    return np.maximum(v, 0.0)


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64: the
    storage precision of weights and activations on the tensor-core path."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return a


def layer_names(blocks: int):
    names = ["in"]
    for k in range(blocks):
        names += [f"b{k}a", f"b{k}b"]
    return names + ["out"]


def init_params(c_in: int, width: int, c_out: int, blocks: int, rng: np.random.Generator, scale: float = 1.0):
    """He-style random weights {name: (W, b)}; the last layer starts small."""
    P = {}
    dims = {"in": (c_in, width), "out": (width, c_out)}
    for name in layer_names(blocks):
        ci, co = dims.get(name, (width, width))
        std = scale * np.sqrt(2.0 / (27 * ci))
        if name == "out" or name.endswith("b"):
            std *= 0.1
        P[name] = (rng.normal(0.0, std, size=(27, ci, co)), rng.normal(0.0, 0.01, size=co))
    return P


def forward(P, x: np.ndarray, blocks: int, quant=None):
    """Network output and the activations the backward pass needs.

    quant (e.g. :func:`bf16`) rounds the weights, the input and every stored
    activation, as a reduced-precision implementation stores them; the
    arithmetic itself stays FP64."""
    q = quant or _ident
    Wq = {k: (q(W), b) for k, (W, b) in P.items()}
    x = q(x)
    acts = {"x": x}
    h = q(relu(conv(x, *Wq["in"])))
    acts["h0"] = h
    for k in range(blocks):
        a = q(relu(conv(h, *Wq[f"b{k}a"])))
        acts[f"a{k}"] = a
        h = q(h + conv(a, *Wq[f"b{k}b"]))
        acts[f"h{k + 1}"] = h
    return conv(h, *Wq["out"]), acts


def backward(P, acts, dout: np.ndarray, blocks: int, quant=None):
    """Gradients {name: (dW, db)} and d(loss)/d(input) for upstream dout.

    quant rounds the weights and every stored gradient tensor (see forward)."""
    q = quant or _ident
    Wq = {k: q(W) for k, (W, b) in P.items()}
    G = {}
    dout = q(dout)
    h = acts[f"h{blocks}"]
    dh, dW, db = conv_backward(h, Wq["out"], dout)
    dh = q(dh)
    G["out"] = (dW, db)
    for k in reversed(range(blocks)):
        a = acts[f"a{k}"]
        da, dW, db = conv_backward(a, Wq[f"b{k}b"], dh)
        G[f"b{k}b"] = (dW, db)
        dpre = q(da * (a > 0))
        dh_in, dW, db = conv_backward(acts[f"h{k}"], Wq[f"b{k}a"], dpre)
        G[f"b{k}a"] = (dW, db)
        dh = q(dh + dh_in) if k > 0 else dh + dh_in
    dpre = q(dh * (acts["h0"] > 0))
    dx, dW, db = conv_backward(acts["x"], Wq["in"], dpre)
    G["in"] = (dW, db)
    return G, dx


def flatten(P, blocks: int) -> np.ndarray:
    """Parameter vector: per layer (in, b0a, b0b, ..., out) W[t][ci][co] then b[co]."""
    return np.concatenate([np.concatenate([P[n][0].ravel(), P[n][1]]) for n in layer_names(blocks)])


def unflatten(v: np.ndarray, like, blocks: int):
    out, off = {}, 0
    for n in layer_names(blocks):
        W, b = like[n]
        out[n] = (v[off:off + W.size].reshape(W.shape), v[off + W.size:off + W.size + b.size])
        off += W.size + b.size
    return out


def masked_mse(y: np.ndarray, target: np.ndarray, mask: np.ndarray):
    """Loss sum(mask (y - t)^2) / sum(mask) over all channels and its gradient."""
    w = mask[None] * np.ones_like(y)
    den = w.sum()
    d = y - target
    return float((w * d * d).sum() / den), 2.0 * w * d / den


def adam_update(w, g, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
