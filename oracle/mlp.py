"""Small multilayer perceptron used as the initial guess of the Newton solve (FP64 reference).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Not in the paper: the learned guess is an extension beyond it.  The network maps
x = (u_x, u_y, T/T0 - 1) to the 8 Lagrange multipliers of Eq. exponential through
    h1 = tanh(W1 x + b1)   (64)
    h2 = tanh(W2 h1 + b2)  (64)
    y  = W3 h2 + b3        (8),     lambda = m + s * y
with a fixed per-output offset m and scale s (taken from the training targets).  Weights are
used rounded to bfloat16 (round to nearest even), arithmetic here is FP64.  Loss: half the mean
over samples of ||y - (lambda_target - m)/s||^2.  Optimiser: Adam (beta1 0.9, beta2 0.999,
eps 1e-8) on FP32-representable master weights.

Tensor-core form (``bf16_act=True``): the kernels that run the matrix products of 64-wide
layers on BF16 tensor cores round the operands of those products to bfloat16 and accumulate in
FP32.  This form rounds exactly those operands: the layer-1 output h1 entering layer 2, h2
entering layer 3; in the backward pass dL/dy entering dW3 and dL/dh2, h2 entering dW3, the
layer-2 delta d2 entering dW2 and dL/dh1, and h1 entering dW2.  Layer 1 (three inputs), its
gradient dW1, the biases, tanh and its derivative 1 - h^2 use unrounded values.
"""
from __future__ import annotations

import numpy as np

SHAPES = {"w1": (64, 3), "b1": (64,), "w2": (64, 64), "b2": (64,), "w3": (8, 64), "b3": (8,)}
ORDER = ["w1", "b1", "w2", "b2", "w3", "b3"]


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = x.view(np.uint32).astype(np.uint64)
    bias = ((bits >> np.uint64(16)) & np.uint64(1)) + np.uint64(0x7FFF)
    r = ((bits + bias) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).reshape(x.shape)


def compute_weights(params: dict, rounded: bool = True) -> dict:
    """Weights as used by the network: bf16-rounded weight matrices, biases as given."""
    out = {}
    for k in ORDER:
        v = np.asarray(params[k], dtype=np.float64)
        out[k] = bf16_round(v).astype(np.float64) if (rounded and k.startswith("w")) else v
    return out


def _op(a, bf16_act: bool):
    """A matrix-product operand as the tensor cores see it (bfloat16 of its FP32 value)."""
    return bf16_round(a).astype(np.float64) if bf16_act else a


def forward(params: dict, x: np.ndarray, rounded: bool = True, bf16_act: bool = False):
    """x (n, 3) -> (y (n, 8), cache)."""
    W = compute_weights(params, rounded)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(x @ W["w1"].T + W["b1"])
    h2 = np.tanh(_op(h1, bf16_act) @ W["w2"].T + W["b2"])
    y = _op(h2, bf16_act) @ W["w3"].T + W["b3"]
    return y, (W, x, h1, h2)


def loss_and_grads(params: dict, x: np.ndarray, t: np.ndarray, rounded: bool = True, bf16_act: bool = False):
    """Loss 1/(2n) sum ||y - t||^2 and its gradients with respect to every parameter."""
    y, (W, x, h1, h2) = forward(params, x, rounded, bf16_act)
    n = x.shape[0]
    d3 = (y - t) / n                                   # dL/dy
    g = {"w3": _op(d3, bf16_act).T @ _op(h2, bf16_act), "b3": d3.sum(axis=0)}
    d2 = (_op(d3, bf16_act) @ W["w3"]) * (1.0 - h2 * h2)
    g["w2"] = _op(d2, bf16_act).T @ _op(h1, bf16_act)
    g["b2"] = d2.sum(axis=0)
    d1 = (_op(d2, bf16_act) @ W["w2"]) * (1.0 - h1 * h1)
    g["w1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    loss = 0.5 * ((y - t) ** 2).sum() / n
    return loss, g


def adam_step(params: dict, grads: dict, state: dict, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place (state holds m, v and the step count t)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in ORDER:
        m = state.setdefault("m_" + k, np.zeros(SHAPES[k]))
        v = state.setdefault("v_" + k, np.zeros(SHAPES[k]))
        m[...] = b1 * m + (1 - b1) * grads[k]
        v[...] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)


def features(u: np.ndarray, T: np.ndarray, T0: float) -> np.ndarray:
    """Network input (n, 3) from velocity (2, n) and temperature (n,)."""
    return np.stack([u[0], u[1], T / T0 - 1.0], axis=1)


def guess(params: dict, m: np.ndarray, s: np.ndarray, T0: float):
    """Newton guess function lambda0(u, T) for the oracle solver (returns (8, n))."""
    def fn(u, T):
        y, _ = forward(params, features(u, T, T0))
        return (m[None, :] + s[None, :] * y).T
    return fn
