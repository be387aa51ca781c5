"""Newton-guess network on the GPU: forward, gradient and Adam kernels against the FP64 oracle
(oracle/mlp.py) on the same seeded parameters and samples; training on equilibria the solver
produced; Newton from the trained guess reaching the same root in fewer iterations; and the
solver run with the network guess against the oracle.

Tolerances: the kernels compute in FP32 with the same bf16-rounded weight matrices as the
oracle, so the forward pass agrees to FP32 rounding of 64-term sums (relative 1e-5 of the output
scale) and the gradients, accumulated in FP32 over the batch with atomics, to 1e-4 relative L2
per parameter tensor.  The BF16 tensor-core kernels are compared with the oracle's tensor-core
form (the same operands rounded to bfloat16); see their tests for the bounds."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import lattices as L
from oracle import mlp
from oracle import numerical as nm
from tests import harness as H
from tests.test_gpu_parity import SUP_SPEC

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def lt():
    from paper_2504_04465_b300 import lbmtree
    return lbmtree


def random_params(seed: int) -> dict:
    rng = np.random.default_rng(seed)
    return {k: (rng.standard_normal(sh) / np.sqrt(sh[1] if len(sh) == 2 else 4)).astype(np.float32).astype(np.float64)
            for k, sh in mlp.SHAPES.items()}


def flat(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float32).reshape(-1) for k in mlp.ORDER])


def unflat(v: np.ndarray) -> dict:
    out, o = {}, 0
    for k in mlp.ORDER:
        n = int(np.prod(mlp.SHAPES[k]))
        out[k] = np.asarray(v[o:o + n], np.float64).reshape(mlp.SHAPES[k])
        o += n
    return out


def dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("n", [1, 128, 1000])
def test_forward_matches_oracle(n):
    p = random_params(11)
    x = np.random.default_rng(12).uniform(-0.8, 0.8, (n, 3))
    d_p, d_x = dev(flat(p), torch.float32), dev(x, torch.float64)
    d_y = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    lt().mlp_forward(d_p.data_ptr(), d_x.data_ptr(), n, d_y.data_ptr())
    torch.cuda.synchronize()
    y, _ = mlp.forward(p, x)
    err = np.abs(d_y.cpu().numpy() - y).max() / np.abs(y).max()
    assert err < 1e-5, err


def test_gradients_and_adam_match_oracle():
    n = 1000                                   # several blocks of 64 samples and a ragged tail
    p = random_params(13)
    rng = np.random.default_rng(14)
    x = rng.uniform(-0.6, 0.6, (n, 3))
    t = rng.standard_normal((n, 8)).astype(np.float32).astype(np.float64)
    d_p, d_x, d_t = dev(flat(p), torch.float32), dev(x, torch.float64), dev(t, torch.float32)
    npar = lt().mlp_nparams()
    d_g = torch.empty(npar, dtype=torch.float32, device="cuda")
    d_l = torch.empty(1, dtype=torch.float32, device="cuda")
    lt().mlp_grad(d_p.data_ptr(), d_x.data_ptr(), d_t.data_ptr(), n, d_g.data_ptr(), d_l.data_ptr())
    torch.cuda.synchronize()
    loss, g = mlp.loss_and_grads(p, x, t)
    assert abs(float(d_l.item()) - loss) < 1e-5 * loss
    gg = unflat(d_g.cpu().numpy())
    for k in mlp.ORDER:
        assert H.rel_l2(gg[k], g[k]) < 1e-4, (k, H.rel_l2(gg[k], g[k]))
    # one Adam step from zero moments with the oracle's gradient on both sides
    d_g2 = dev(flat(g), torch.float32)
    d_m = torch.zeros(npar, dtype=torch.float32, device="cuda")
    d_v = torch.zeros(npar, dtype=torch.float32, device="cuda")
    for step in (1, 2):
        lt().mlp_adam(d_p.data_ptr(), d_g2.data_ptr(), d_m.data_ptr(), d_v.data_ptr(), step, 1e-3)
    torch.cuda.synchronize()
    q = {k: v.copy() for k, v in p.items()}
    st = {}
    g32 = unflat(flat(g))
    mlp.adam_step(q, g32, st, 1e-3)
    mlp.adam_step(q, g32, st, 1e-3)
    got = unflat(d_p.cpu().numpy())
    for k in mlp.ORDER:
        assert np.abs(got[k] - q[k]).max() < 1e-6, k


@pytest.mark.parametrize("n", [1, 100, 1000])
def test_tensor_core_forward_matches_oracle(n):
    """BF16 tensor-core forward pass against the oracle's tensor-core form (hidden activations
    rounded to bfloat16 where the kernel rounds them).  An activation whose FP32 value lies
    within FP32 rounding of a bfloat16 rounding boundary can round the other way on one side
    (about 3e-5 of them), moving its outputs by one bfloat16 step of that term: every output
    agrees to 2e-3 of the output scale, and all but a handful to 1e-5."""
    p = random_params(11)
    x = np.random.default_rng(12).uniform(-0.8, 0.8, (n, 3))
    d_p, d_x = dev(flat(p), torch.float32), dev(x, torch.float64)
    d_y = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    lt().mlp_forward(d_p.data_ptr(), d_x.data_ptr(), n, d_y.data_ptr(), tensor_cores=True)
    torch.cuda.synchronize()
    y, _ = mlp.forward(p, x, bf16_act=True)
    err = np.abs(d_y.cpu().numpy() - y) / np.abs(y).max()
    assert err.max() < 2e-3, err.max()
    assert (err > 1e-5).sum() <= max(2, n // 100), (err > 1e-5).sum()


def test_tensor_core_gradients_match_oracle():
    n = 1000                                   # several blocks of 64 samples and a ragged tail
    p = random_params(13)
    rng = np.random.default_rng(14)
    x = rng.uniform(-0.6, 0.6, (n, 3))
    t = rng.standard_normal((n, 8)).astype(np.float32).astype(np.float64)
    d_p, d_x, d_t = dev(flat(p), torch.float32), dev(x, torch.float64), dev(t, torch.float32)
    npar = lt().mlp_nparams()
    d_g = torch.empty(npar, dtype=torch.float32, device="cuda")
    d_l = torch.empty(1, dtype=torch.float32, device="cuda")
    lt().mlp_grad(d_p.data_ptr(), d_x.data_ptr(), d_t.data_ptr(), n, d_g.data_ptr(), d_l.data_ptr(),
                  tensor_cores=True)
    torch.cuda.synchronize()
    loss, g = mlp.loss_and_grads(p, x, t, bf16_act=True)
    _, g64 = mlp.loss_and_grads(p, x, t)
    assert abs(float(d_l.item()) - loss) < 1e-4 * loss
    gg = unflat(d_g.cpu().numpy())
    for k in mlp.ORDER:
        e = H.rel_l2(gg[k], g[k])
        print(k, "tensor-core form %.2e, FP64 form %.2e" % (e, H.rel_l2(gg[k], g64[k])))
        assert e < 1e-3, (k, e)


def sup_fields(level, coords, c):
    """Ma ~0.6 inflow over a periodic channel with a density pulse and transverse waves."""
    x, y = c[:, 0], c[:, 1]
    rho = 1 + 0.2 * np.exp(-((x - 64) ** 2 + (y - 16) ** 2) / 50)
    ux = 0.6 + 0.05 * np.sin(2 * np.pi * y / 32)
    uy = 0.05 * np.sin(2 * np.pi * x / 128)
    T = 0.9 + 0.05 * np.cos(2 * np.pi * y / 32)
    return rho, np.stack([ux, uy]), T


def solver_samples(steps: int = 40):
    """(u_x, u_y, T) and converged multipliers of every fluid cell of a D2Q21 supersonic run."""
    ctx = H.make_gpu(SUP_SPEC, "D2Q21", "num_ddf", "f64", sup_fields, nu0=0.01, T0=0.9, sensor_A=1.35, guess="poly")
    ctx.step_fine(steps)
    ctx.sync()
    rho, u, T = ctx.moments()
    lam = ctx.populations("lambda")
    lv, xyz, ty = ctx.cells()
    keep = ty == 1
    uT = np.stack([u[0, keep], u[1, keep], T[keep]], axis=1)
    return ctx, uT, lam[:, keep].T.copy()


def test_batched_newton_matches_oracle_and_trained_guess_saves_iterations():
    ctx, uT, lam_solver = solver_samples()
    n = uT.shape[0]
    d_uT = dev(uT, torch.float64)
    d_lam = torch.empty((n, 8), dtype=torch.float64, device="cuda")
    d_it = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.newton_batch(d_uT.data_ptr(), n, "poly", d_lam.data_ptr(), d_it.data_ptr())
    ctx.sync()
    lam_poly = d_lam.cpu().numpy()
    it_poly = d_it.cpu().numpy()
    lat = L.LATTICES["D2Q21"]
    sel = np.arange(0, n, 7)
    u, T = uT[sel, :2].T, uT[sel, 2]
    lam_o, _, it_o, conv_o = nm.newton(lat, u, T, nm.poly_guess(lat, u, T, 3), 1e-12, 50)
    assert conv_o.all() and (it_poly >= 0).all()
    assert np.abs(lam_poly[sel] - lam_o.T).max() < 1e-10
    assert abs(it_poly[sel].mean() - it_o.mean()) < 0.05
    # training on the solver's own equilibria, with the project's kernels
    loss = ctx.mlp_train(d_uT.data_ptr(), d_lam.data_ptr(), n, steps=2000, batch=1024, lr=3e-3, lr_final=3e-4)
    assert loss < 0.1, loss               # the mean predictor scores 4.0 on unit-variance targets
    ctx.newton_batch(d_uT.data_ptr(), n, "mlp", d_lam.data_ptr(), d_it.data_ptr())
    d_it_zero = torch.empty(n, dtype=torch.int32, device="cuda")
    d_lam_zero = torch.empty((n, 8), dtype=torch.float64, device="cuda")
    ctx.newton_batch(d_uT.data_ptr(), n, "zero", d_lam_zero.data_ptr(), d_it_zero.data_ptr())
    ctx.sync()
    it_mlp = d_it.cpu().numpy()
    it_zero = d_it_zero.cpu().numpy()
    assert (it_mlp >= 0).all()
    # Newton from the learned guess reaches the same root
    assert np.abs(d_lam.cpu().numpy() - lam_poly).max() < 1e-9
    print(f"mean Newton iterations: zero {it_zero.mean():.3f} poly {it_poly.mean():.3f} mlp {it_mlp.mean():.3f}")
    assert it_mlp.mean() <= it_poly.mean() - 1.0
    # the network read back equals the oracle's forward pass of the same parameters
    params, m, s = ctx.mlp_get()
    y, _ = mlp.forward(unflat(params), mlp.features(uT[:64, :2].T, uT[:64, 2], 0.9))
    d_y = torch.empty((64, 8), dtype=torch.float32, device="cuda")
    x = dev(mlp.features(uT[:64, :2].T, uT[:64, 2], 0.9), torch.float64)
    d_p = dev(params, torch.float32)
    lt().mlp_forward(d_p.data_ptr(), x.data_ptr(), 64, d_y.data_ptr())
    torch.cuda.synchronize()
    assert np.abs(d_y.cpu().numpy() - y).max() < 1e-5 * max(1.0, np.abs(y).max())
    ctx.close()


def test_tensor_core_training_saves_iterations():
    """Training with the BF16 tensor-core gradient reaches the same quality as the FP32-core
    training: loss below 0.1 and at least one Newton iteration saved against the polynomial
    guess, Newton from it reaching the same root."""
    import time
    ctx, uT, _ = solver_samples()
    n = uT.shape[0]
    d_uT = dev(uT, torch.float64)
    d_lam = torch.empty((n, 8), dtype=torch.float64, device="cuda")
    d_it = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.newton_batch(d_uT.data_ptr(), n, "poly", d_lam.data_ptr(), d_it.data_ptr())
    ctx.sync()
    lam_poly, it_poly = d_lam.cpu().numpy(), d_it.cpu().numpy()
    secs = {}
    for tc in (False, True):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = ctx.mlp_train(d_uT.data_ptr(), d_lam.data_ptr(), n, steps=2000, batch=1024, lr=3e-3, lr_final=3e-4,
                             tensor_cores=tc)
        secs[tc] = time.perf_counter() - t0
        assert loss < 0.1, (tc, loss)
    ctx.newton_batch(d_uT.data_ptr(), n, "mlp", d_lam.data_ptr(), d_it.data_ptr())
    ctx.sync()
    it_mlp = d_it.cpu().numpy()
    print(f"training 2000 steps of 1024: FP32 cores {secs[False]:.3f} s, tensor cores {secs[True]:.3f} s; "
          f"Newton iterations poly {it_poly.mean():.3f} mlp(tc) {it_mlp.mean():.3f}")
    assert (it_mlp >= 0).all()
    assert np.abs(d_lam.cpu().numpy() - lam_poly).max() < 1e-9
    assert it_mlp.mean() <= it_poly.mean() - 1.0
    ctx.close()


def test_solver_with_learned_guess_matches_oracle():
    ctx, uT, _ = solver_samples(20)
    n = uT.shape[0]
    d_uT = dev(uT, torch.float64)
    d_lam = torch.empty((n, 8), dtype=torch.float64, device="cuda")
    d_it = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.newton_batch(d_uT.data_ptr(), n, "zero", d_lam.data_ptr(), d_it.data_ptr())
    ctx.mlp_train(d_uT.data_ptr(), d_lam.data_ptr(), n, steps=1500, batch=1024)
    params, m, s = ctx.mlp_get()
    ctx.close()
    g = H.make_gpu(SUP_SPEC, "D2Q21", "num_ddf", "f64", sup_fields, nu0=0.01, T0=0.9, sensor_A=1.35, guess="mlp")
    g.mlp_set(params, m, s)
    g.step_fine(30)
    g.sync()
    st = g.stats()
    assert st.newton_nonconverged == 0
    sol_mlp = H.run_oracle(SUP_SPEC, "D2Q21", "num_ddf", sup_fields, 30, nu0=0.01, T0=0.9, sensor_A=1.35,
                           guess="mlp", mlp=mlp.guess(unflat(params), m, s, 0.9))
    err = H.compare_moments(sol_mlp, g)
    assert err["rho"] < 1e-12 and err["u"] < 1e-12 and err["T"] < 1e-12, err
    # same root as the polynomial-guess run of the oracle: a different starting point converges
    # to the root only within the Newton tolerance (1e-12 on the moment constraints), and that
    # difference accumulates over the 30 fine iterations (observed ~1e-12; bound 1e-11)
    sol_poly = H.run_oracle(SUP_SPEC, "D2Q21", "num_ddf", sup_fields, 30, nu0=0.01, T0=0.9, sensor_A=1.35,
                            guess="poly")
    err = H.compare_moments(sol_poly, g)
    assert err["rho"] < 1e-11 and err["u"] < 1e-11 and err["T"] < 1e-11, err
    gp = H.make_gpu(SUP_SPEC, "D2Q21", "num_ddf", "f64", sup_fields, nu0=0.01, T0=0.9, sensor_A=1.35, guess="poly")
    gp.step_fine(30)
    gp.sync()
    sp = gp.stats()
    it_mlp = st.newton_iter_sum / st.newton_updates
    it_poly = sp.newton_iter_sum / sp.newton_updates
    print(f"solver mean Newton iterations: poly {it_poly:.3f} mlp {it_mlp:.3f}")
    assert it_mlp < it_poly
    gp.close()
    g.close()


def test_network_guess_requires_a_network():
    from paper_2504_04465_b300.lbmtree import LbmError
    g = H.make_gpu(SUP_SPEC, "D2Q21", "num_ddf", "f64", sup_fields, nu0=0.01, T0=0.9, guess="mlp")
    with pytest.raises(LbmError):
        g.step_fine(1)
    g.close()
