"""Pins of the Newton-guess network reference (oracle/mlp.py) to things other than itself:
bfloat16 rounding against torch's own conversion, gradients against central finite differences
and against torch autograd, the Adam first step against its closed form, special weights that
reduce the network to a hand-computable function, and the fact that Newton from the network's
guess reaches the same root as Newton from the polynomial guess."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import lattices as L
from oracle import mlp
from oracle import numerical as nm


def random_params(seed: int, scale: float = 1.0) -> dict:
    rng = np.random.default_rng(seed)
    p = {}
    for k, sh in mlp.SHAPES.items():
        fan = sh[1] if len(sh) == 2 else 4
        p[k] = (scale * rng.standard_normal(sh) / np.sqrt(fan)).astype(np.float32).astype(np.float64)
    return p


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(4096).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 4096),
                        np.array([0.0, -0.0, 1.0, -1.0, 1.00390625, 1.01171875, 3.0e-39, -2.5e-40,
                                  np.inf, -np.inf, 3.3895314e38], np.float32)])
    # exact ties: low 16 bits 0x8000 with even and odd bit 16
    ties = (np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x40498000], np.uint32)).view(np.float32)
    x = np.concatenate([x.astype(np.float32), ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = mlp.bf16_round(x)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_special_weights_reduce_to_closed_form():
    p = {k: np.zeros(sh) for k, sh in mlp.SHAPES.items()}
    p["b3"] = np.arange(8, dtype=np.float64)
    x = np.random.default_rng(2).standard_normal((5, 3))
    y, _ = mlp.forward(p, x)
    assert np.array_equal(y, np.tile(np.arange(8.0), (5, 1)))
    # one path: unit 0 of layer 1 sees x_1, unit 0 of layer 2 sees unit 0, output 3 sees unit 0
    p["w1"][0, 1] = 0.5
    p["w2"][0, 0] = 2.0
    p["w3"][3, 0] = -1.5
    y, _ = mlp.forward(p, x)
    want = np.tile(np.arange(8.0), (5, 1))
    want[:, 3] += -1.5 * np.tanh(2.0 * np.tanh(0.5 * x[:, 1]))
    assert np.allclose(y, want, rtol=0, atol=1e-15)


def test_gradients_match_finite_differences():
    p = random_params(3)
    rng = np.random.default_rng(4)
    x = rng.uniform(-0.6, 0.6, (37, 3))
    t = rng.standard_normal((37, 8))
    _, g = mlp.loss_and_grads(p, x, t, rounded=False)
    h = 1e-6
    for k in mlp.ORDER:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(p, x, t, rounded=False)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(p, x, t, rounded=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 + 1e-6 * abs(an), (k, idx, fd, an)


def test_gradients_match_autograd_with_rounded_weights():
    p = random_params(5)
    rng = np.random.default_rng(6)
    x = rng.uniform(-0.6, 0.6, (50, 3))
    t = rng.standard_normal((50, 8))
    loss, g = mlp.loss_and_grads(p, x, t, rounded=True)
    W = {k: torch.tensor(mlp.bf16_round(p[k]).astype(np.float64) if k.startswith("w") else p[k],
                         dtype=torch.float64, requires_grad=True) for k in mlp.ORDER}
    xt = torch.tensor(x)
    h1 = torch.tanh(xt @ W["w1"].T + W["b1"])
    h2 = torch.tanh(h1 @ W["w2"].T + W["b2"])
    y = h2 @ W["w3"].T + W["b3"]
    lt = 0.5 * ((y - torch.tensor(t)) ** 2).sum() / x.shape[0]
    lt.backward()
    assert abs(float(lt.detach()) - loss) < 1e-13
    for k in mlp.ORDER:
        assert np.allclose(g[k], W[k].grad.numpy(), rtol=1e-12, atol=1e-15), k


class _RoundFwd(torch.autograd.Function):
    """bfloat16 of the value going forward (torch's own conversion), gradient passed unchanged."""
    @staticmethod
    def forward(ctx, a):
        return a.to(torch.float32).to(torch.bfloat16).to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        return g


class _RoundBwd(torch.autograd.Function):
    """Value passed unchanged, bfloat16 of the gradient going back."""
    @staticmethod
    def forward(ctx, a):
        return a.clone()

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def test_tensor_core_form_matches_autograd_with_bf16_operands():
    """The bf16-operand gradients equal autograd of the network in which every operand of the
    two 64-wide products is cast to bfloat16 by torch: activations on the way forward, the
    gradient entering each product on the way back (biases and layer 1 unrounded)."""
    p = random_params(15)
    rng = np.random.default_rng(16)
    x = rng.uniform(-0.6, 0.6, (40, 3))
    t = rng.standard_normal((40, 8))
    loss, g = mlp.loss_and_grads(p, x, t, rounded=True, bf16_act=True)
    W = {k: torch.tensor(mlp.bf16_round(p[k]).astype(np.float64) if k.startswith("w") else p[k],
                         dtype=torch.float64, requires_grad=True) for k in mlp.ORDER}
    xt = torch.tensor(x)
    h1 = torch.tanh(xt @ W["w1"].T + W["b1"])
    h2 = torch.tanh(_RoundBwd.apply(_RoundFwd.apply(h1) @ W["w2"].T) + W["b2"])
    y = _RoundBwd.apply(_RoundFwd.apply(h2) @ W["w3"].T) + W["b3"]
    lt = 0.5 * ((y - torch.tensor(t)) ** 2).sum() / x.shape[0]
    lt.backward()
    assert abs(float(lt.detach()) - loss) < 1e-13
    for k in mlp.ORDER:
        assert np.allclose(g[k], W[k].grad.numpy(), rtol=1e-12, atol=1e-15), k
    # and the rounding is real: the form differs from the FP64 one by about the bf16 unit roundoff
    _, g64 = mlp.loss_and_grads(p, x, t, rounded=True)
    for k in ("w2", "w3", "b2"):
        d = np.linalg.norm(g[k] - g64[k]) / np.linalg.norm(g64[k])
        assert 1e-5 < d < 2e-2, (k, d)


def test_adam_first_step_closed_form():
    p = random_params(7)
    before = {k: v.copy() for k, v in p.items()}
    rng = np.random.default_rng(8)
    g = {k: rng.standard_normal(sh) for k, sh in mlp.SHAPES.items()}
    st = {}
    mlp.adam_step(p, g, st, lr=1e-2)
    # after one step both moments are bias-corrected to g and g^2: delta = -lr g / (|g| + eps)
    for k in mlp.ORDER:
        want = before[k] - 1e-2 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(p[k], want, rtol=1e-12, atol=1e-15), k
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    mlp.adam_step(p, g, st, lr=1e-2)
    for k in mlp.ORDER:
        want = before[k] - 2e-2 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(p[k], want, rtol=1e-12, atol=1e-14), k


def test_training_lowers_loss_and_newton_reaches_the_same_root():
    lat = L.LATTICES["D2Q21"]
    rng = np.random.default_rng(9)
    n = 2048
    u = rng.uniform(-0.4, 0.4, (2, n))
    T = rng.uniform(0.8, 1.0, n)
    T0 = 0.9
    lam, _, it_poly, conv = nm.newton(lat, u, T, nm.poly_guess(lat, u, T, 3), 1e-12, 50)
    assert conv.all()
    m = lam.mean(axis=1)
    s = lam.std(axis=1)
    x = mlp.features(u, T, T0)
    t = ((lam - m[:, None]) / s[:, None]).T
    p = random_params(10)
    st = {}
    l0, _ = mlp.loss_and_grads(p, x, t)
    for i in range(400):
        idx = rng.integers(0, n, 256)
        _, g = mlp.loss_and_grads(p, x[idx], t[idx])
        mlp.adam_step(p, g, st, 3e-3)
    l1, _ = mlp.loss_and_grads(p, x, t)
    assert l1 < 0.05 * l0, (l0, l1)
    lam0 = mlp.guess(p, m, s, T0)(u, T)
    lam_m, e_m, it_m, conv_m = nm.newton(lat, u, T, lam0, 1e-12, 50)
    assert conv_m.all()
    # the root does not depend on the starting point (strictly convex dual)
    assert np.abs(lam_m - lam).max() < 1e-9
    assert it_m.mean() < it_poly.mean()


@pytest.mark.parametrize("k", mlp.ORDER)
def test_shapes_and_order_cover_the_flat_layout(k):
    # the flat parameter vector of the library: [W1 (64x3), b1, W2 (64x64), b2, W3 (8x64), b3]
    sizes = {kk: int(np.prod(mlp.SHAPES[kk])) for kk in mlp.ORDER}
    assert sum(sizes.values()) == 4936
    off = sum(sizes[kk] for kk in mlp.ORDER[:mlp.ORDER.index(k)])
    assert off == {"w1": 0, "b1": 192, "w2": 256, "b2": 4352, "w3": 4416, "b3": 4928}[k]
