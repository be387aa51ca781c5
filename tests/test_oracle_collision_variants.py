"""Pins of the oracle's collision variants beside BGK and RR (CPU only): the two-relaxation-time
collision (TRT), recursive regularization with the trace of the second-order moments
equilibrated (Appendix A, after Eq. a1Rec) and the far-field relaxation of Eq.
relaxation_pressure, checked against special cases that reduce to BGK/RR, conservation, the
moments the definitions fix, and closed-form decay rates."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import grid as G
from oracle import hermite as hm
from oracle import lattices as L
from oracle import solver as S
from paper_2504_04465_b300 import inputs as I


def _random_state(lat, n=64, seed=3):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, n)
    u = 0.1 * rng.uniform(-1, 1, (lat.D, n))
    feq = hm.feq_athermal(lat, rho, u)
    return feq * (1.0 + 0.05 * rng.uniform(-1, 1, feq.shape))


def _moments2(lat, f):
    """sum_i H2_ab f_i for a <= b (independent of the collision code)."""
    out = {}
    for a in range(lat.D):
        for b in range(a, lat.D):
            out[(a, b)] = hm.hermite_tensor(lat.xi, (a, b), lat.cs2) @ f
    return out


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_trt_with_equal_rates_is_bgk(name):
    """Lambda = (tau - 1/2)^2 gives tau- = tau+ and the TRT collision is BGK exactly."""
    lat = L.LATTICES[name]
    f = _random_state(lat)
    tau = 0.8
    rho, u = hm.macroscopic(lat, f)
    feq = hm.feq_athermal(lat, rho, u)
    trt = hm.collide_trt(lat, f, feq, tau, (tau - 0.5) ** 2)
    bgk = hm.collide_bgk(f, feq, tau)
    assert np.abs(trt - bgk).max() < 1e-15


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_trt_conserves_and_relaxes_even_and_odd_parts(name):
    lat = L.LATTICES[name]
    f = _random_state(lat)
    tau, magic = 0.7, 0.25
    rho, u = hm.macroscopic(lat, f)
    feq = hm.feq_athermal(lat, rho, u)
    fs = hm.collide_trt(lat, f, feq, tau, magic)
    rho2, u2 = hm.macroscopic(lat, fs)
    assert np.abs(rho2 - rho).max() < 1e-14 and np.abs(rho2 * u2 - rho * u).max() < 1e-14
    # second-order moments (even) relax at 1/tau+; the omega- of Lambda = 1/4 follows from
    # (tau+ - 1/2)(tau- - 1/2) = 1/4 with tau+ = 0.7: tau- = 1.75
    P0, P1 = _moments2(lat, f - feq), _moments2(lat, fs - feq)
    for k in P0:
        assert np.abs(P1[k] - (1 - 1 / tau) * P0[k]).max() < 1e-14
    assert abs(1.0 / hm.trt_omega_minus(tau, magic) - 1.75) < 1e-14
    # the third-order (odd) moment xxy relaxes at 1/tau-
    H3 = hm.hermite_tensor(lat.xi, (0, 0, 1), lat.cs2)
    assert np.abs(H3 @ (fs - feq) - (1 - 1 / 1.75) * (H3 @ (f - feq))).max() < 1e-14


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_trace_equilibration(name):
    """RR with the trace equilibrated: after the collision the non-equilibrium second-order
    moment is (1 - 1/tau) times the deviatoric part of Pi (no trace left); mass and momentum are
    kept; a state whose Pi is already traceless collides as in plain RR."""
    lat = L.LATTICES[name]
    f = _random_state(lat)
    tau = 0.9
    rho, u = hm.macroscopic(lat, f)
    feq = hm.feq_athermal(lat, rho, u)
    fs = hm.collide_rr(lat, f, tau, trace_eq=True)
    rho2, u2 = hm.macroscopic(lat, fs)
    assert np.abs(rho2 - rho).max() < 1e-14 and np.abs(rho2 * u2 - rho * u).max() < 1e-14
    P0, P1 = _moments2(lat, f - feq), _moments2(lat, fs - feq)
    tr = sum(P0[(a, a)] for a in range(lat.D)) / lat.D
    for (a, b), v in P0.items():
        want = (1 - 1 / tau) * (v - (tr if a == b else 0.0))
        assert np.abs(P1[(a, b)] - want).max() < 1e-14
    assert np.abs(sum(P1[(a, a)] for a in range(lat.D))).max() < 1e-14
    # a traceless Pi: same result as RR
    fneq = f - feq
    shift = np.zeros_like(fneq)
    H2tr = sum(hm.hermite_tensor(lat.xi, (a, a), lat.cs2) for a in range(lat.D))
    # remove the trace part with a population pattern carrying only trace: w_i H2tr_i / |.|^2
    pattern = lat.w * H2tr
    scale = (H2tr @ fneq) / (H2tr @ pattern)
    f0 = feq + fneq - pattern[:, None] * scale[None, :]
    assert np.abs(sum(_moments2(lat, f0 - feq)[(a, a)] for a in range(lat.D))).max() < 1e-14
    assert np.abs(hm.collide_rr(lat, f0, tau, trace_eq=True) - hm.collide_rr(lat, f0, tau)).max() < 1e-14


def _decay_rate(lat, model, kind, trace_eq=False, n=64, steps=(20, 120), magic=0.25, nu=0.02):
    """Fitted exponential rate of a shear wave (kind 'shear': u_y = U sin kx) or a standing
    density wave (kind 'sound': rho = 1 + A cos kx) on a uniform periodic D2Q9 grid."""
    spec = I.GridSpec(2, (n, 4), 1, [], (True, True))
    g = G.build(spec, lat)
    s = S.Solver(g, model, nu0=nu, trace_eq=trace_eq, trt_magic=magic)
    lv = g.levels[0]
    x = I.cell_centres(lv.coords, 0)[:, 0]
    k = 2 * np.pi / n
    if kind == "shear":
        rho = np.ones(x.size)
        u = np.stack([np.zeros(x.size), 1e-3 * np.sin(k * x)])
    else:
        rho = 1.0 + 1e-4 * np.cos(k * x)
        u = np.zeros((2, x.size))
    s.init_fields([(rho, u, None)])
    amps, ts = [], []
    for t in range(steps[1] + 1):
        if t >= steps[0] and t % 10 == 0:
            r, uu, _ = s.moments(0)
            if kind == "shear":
                amps.append(np.abs(uu[1] @ np.sin(k * x)))
            else:
                # amplitude of the standing wave's energy: density and velocity parts
                amps.append(np.sqrt((((r - 1) @ np.cos(k * x)) ** 2 + ((uu[0] @ np.sin(k * x)) / np.sqrt(lat.cs2)) ** 2)))
            ts.append(t)
        s.step_fine(1)
    return -np.polyfit(ts, np.log(amps), 1)[0], k


@pytest.mark.parametrize("model,trace", [("trt", False), ("rr", True)])
def test_shear_wave_decays_at_the_viscosity(model, trace):
    """The shear viscosity of TRT and of trace-equilibrated RR is the one of tau = nu/c_s^2 + 1/2:
    a shear wave decays as exp(-nu k^2 t)."""
    nu = 0.02
    rate, k = _decay_rate(L.D2Q9, model, "shear", trace_eq=trace, nu=nu)
    assert abs(rate / (nu * k * k) - 1) < 0.01


def test_trace_equilibration_adds_bulk_damping():
    """Sound damping Gamma = (1/2) [(2 - 2/D) nu + zeta] k^2.  Plain RR carries the lattice's
    bulk viscosity zeta = (2/D) nu (Gamma = nu k^2); equilibrating the trace relaxes the bulk part
    with tau_b = 1, zeta = (2/D)(tau_b - 1/2) c_s^2 = c_s^2 / 2 in 2D."""
    nu = 0.02
    lat = L.D2Q9
    r_rr, k = _decay_rate(lat, "rr", "sound", nu=nu)
    r_tr, _ = _decay_rate(lat, "rr", "sound", trace_eq=True, nu=nu)
    assert abs(r_rr / (nu * k * k) - 1) < 0.05
    want = 0.5 * ((2 - 2 / 2) * nu + (2 / 2) * 0.5 * lat.cs2) * k * k
    assert abs(r_tr / want - 1) < 0.03


def test_far_field_relaxation():
    """Eq. relaxation_pressure: sigma is 0 inside r0, sigma_max beyond r1 and linear between;
    rho moves to rho (1 - sigma) + sigma rho_inf, the velocity and the non-equilibrium second
    moments are kept, and cells inside r0 are untouched."""
    lat = L.D2Q9
    spec = I.GridSpec(2, (64, 64), 1, [], (True, True))
    g = G.build(spec, lat)
    sp = {"centre": (32.0, 32.0, 0.0), "r0": 10.0, "r1": 20.0, "sigma_max": 0.4, "rho_inf": 1.0}
    s = S.Solver(g, "rr", nu0=0.02, sponge=sp)
    lv = g.levels[0]
    f = _random_state(lat, lv.n, seed=11)
    cells = np.arange(lv.n)
    out = s._relax_far_field(0, cells, f)
    c = I.cell_centres(lv.coords, 0)
    r = np.hypot(c[:, 0] - 32, c[:, 1] - 32)
    sigma = np.where(r < 10, 0.0, np.where(r >= 20, 0.4, 0.4 * (r - 10) / 10))
    rho0, u0 = hm.macroscopic(lat, f)
    rho1, u1 = hm.macroscopic(lat, out)
    assert np.abs(rho1 - (rho0 * (1 - sigma) + sigma)).max() < 1e-14
    assert np.abs(u1 - u0).max() < 1e-14
    inside = r < 10
    assert np.array_equal(out[:, inside], f[:, inside])
    P0 = _moments2(lat, f - hm.feq_athermal(lat, rho0, u0))
    P1 = _moments2(lat, out - hm.feq_athermal(lat, rho1, u1))
    for key in P0:
        assert np.abs(P1[key] - P0[key]).max() < 1e-14
