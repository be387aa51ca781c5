"""Multi-level collide-and-stream time stepping with Rohde coalescence/explosion.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sources (arXiv 2504.04465):
  * Sec. 2, Eq. CollAndStream and Appendix A, Eqs. CollisionStep/StreamingStep: collide locally,
    then stream f*_i to x + xi_i.  Stored state = pre-collision populations; two buffers.
  * Sec. 4.5 (per-iteration schedule): for iLevel = depth..1, if iter % 2^iLevel == 0 then
    refinementCoupling(iLevel, iLevel-1) then collideAndStream(iLevel); finally
    collideAndStream(0).  Fine ghost cells only stream, they never collide.
  * Sec. 3.2, Eqs. coalescence / explosion_uniform and the lambda versions: before the coarse
    collision the unknown coarse-ghost populations are the mean of the fine-ghost children;
    after it, every fine-ghost child receives the coarse post-collision populations (and the
    multipliers).  Reading R2: the coarse ghost collides once per coarse step; the coupling's
    post-collision state is both exploded and streamed.
  * Sec. 3.2, Eq. tau_fine_to_coarse (reading R13): nu_c = nu_f / 2, tau = nu / theta + 1/2 in
    each level's own units, theta = c_s^2 (weakly compressible) or T0 (compressible, R4).
  * Appendix A: polyatomic DDF (Eqs. gEq, polyTemp), kinetic shock sensor (Eqs. DeltaAvg,
    shock_function; reading R10: alpha = 1 below 0.01, terms with f_eq <= 1e-300 skipped),
    boundary conditions (A.3; readings R11, R12; wall faces with Ladd's moving-wall term, R38).
  * Populations with no source (outside a non-periodic face, or a coarse cell covered by the
    finer level) are set to 0 by streaming; they are either overwritten (boundary layers,
    coalescence) or never reach a bulk cell.
"""
from __future__ import annotations

import numpy as np

from . import hermite as hm
from . import numerical as nm
from .grid import BC, CGHOST, FGHOST, FLUID, SOLID, Grid

WEAK_MODELS = ("bgk", "rr", "trt")
COMP_MODELS = ("poly_ddf", "num_ddf")


def sensor_alpha(eps: np.ndarray, tau, A: float) -> np.ndarray:
    """Eq. shock_function with alpha = 1 below 0.01 (reading R10)."""
    tau = np.broadcast_to(np.asarray(tau, dtype=np.float64), eps.shape)
    a = np.ones_like(eps)
    a = np.where((eps >= 0.01) & (eps < 0.10), 1.05, a)
    a = np.where((eps >= 0.10) & (eps < 1.00), A, a)
    a = np.where(eps >= 1.00, 1.0 / tau, a)
    return a


def sensor_eps(f: np.ndarray, feq: np.ndarray) -> np.ndarray:
    """Eq. DeltaAvg: eps = (1/V) sum_i |f_i - f_i^eq| / f_i^eq (f only)."""
    V = f.shape[0]
    ok = feq > 1e-300
    term = np.where(ok, np.abs(f - feq) / np.where(ok, feq, 1.0), 0.0)
    return term.sum(axis=0) / V


class Solver:
    def __init__(self, grid: Grid, model: str, nu0: float = 0.0, T0: float | None = None,
                 gamma: float = 1.4, sensor_A: float | None = None, newton_tol: float = 1e-12,
                 newton_max_iter: int = 50, guess: str = "warm", poly_order: int | None = None,
                 mlp=None, trace_eq: bool = False, trt_magic: float = 0.25, sponge=None):
        self.g = grid
        self.lat = grid.lat
        self.model = model
        if model not in WEAK_MODELS + COMP_MODELS:
            raise ValueError(model)
        self.comp = model in COMP_MODELS
        self.gamma = gamma
        self.Cv = 1.0 / (gamma - 1.0)
        self.T0 = T0 if T0 is not None else self.lat.cs2
        theta = self.T0 if self.comp else self.lat.cs2
        L = grid.n_levels
        self.nu = [nu0 / 2 ** i for i in range(L)]
        self.tau = [self.nu[i] / theta + 0.5 for i in range(L)]
        self.sensor_A = sensor_A
        self.tol = newton_tol
        self.max_iter = newton_max_iter
        self.guess = guess
        self.poly_order = poly_order if poly_order is not None else (4 if self.lat.Q >= 37 else 3)
        self.mlp = mlp
        self.trace_eq = bool(trace_eq)
        self.trt_magic = trt_magic
        if trace_eq and model != "rr":
            raise ValueError("trace equilibration applies to the recursive-regularized collision")
        self.sponge = sponge
        if self.comp and any(np.any(lv.wall_term != 0.0) for lv in grid.levels):
            raise ValueError("moving walls are built for the weakly compressible models")
        if sponge is not None and self.comp:
            raise ValueError("the far-field relaxation is built for the weakly compressible models")
        self.t = 0
        Q = self.lat.Q
        self.f = [np.zeros((Q, lv.n)) for lv in grid.levels]
        self.g_ = [np.zeros((Q, lv.n)) for lv in grid.levels] if self.comp else None
        self.lam = [np.zeros((nm.N_LAMBDA, lv.n)) for lv in grid.levels] if model == "num_ddf" else None
        self.iters = [np.zeros(lv.n, dtype=np.int64) for lv in grid.levels]
        self.nonconv = 0
        self._cg_post = [None] * L

    # ------------------------------------------------------------------ equilibria
    def _moments(self, f, g):
        lat = self.lat
        rho = f.sum(axis=0)
        u = (lat.xi.T.astype(np.float64) @ f) / rho
        if not self.comp:
            return rho, u, None
        xi2 = (lat.xi.astype(np.float64) ** 2).sum(axis=1)
        T = (xi2 @ f + g.sum(axis=0) - rho * (u * u).sum(axis=0)) / (2.0 * rho * self.Cv)
        return rho, u, T

    def _guess(self, u, T, lam_stored):
        if self.guess == "warm":
            return lam_stored.copy()
        if self.guess == "zero":
            return np.zeros_like(lam_stored)
        if self.guess == "poly":
            return nm.poly_guess(self.lat, u, T, self.poly_order)
        if self.guess == "mlp":
            return self.mlp(u, T)
        raise ValueError(self.guess)

    def _feq_comp(self, rho, u, T, lam0):
        """Compressible equilibrium -> (f_eq, lambda or None, iterations)."""
        if self.model == "poly_ddf":
            return hm.feq_thermal(self.lat, rho, u, T, self.poly_order), None, np.zeros(rho.size, np.int64)
        lam, e, it, conv = nm.newton(self.lat, u, T, lam0, self.tol, self.max_iter)
        self.nonconv += int((~conv).sum())
        return rho[None, :] * e, lam, it

    # ------------------------------------------------------------------ collision
    def _relax_far_field(self, lev: int, cells, f):
        """Eq. relaxation_pressure before the collision (weakly compressible, p = rho c_s^2):
        rho' = rho (1 - sigma) + sigma rho_inf with sigma ramping linearly from 0 at distance r0
        to sigma_max at r1 from the centre (finest units, cell centres) and sigma_max beyond; the
        populations become f + f_eq(rho', u) - f_eq(rho, u), the velocity and the
        non-equilibrium part kept (reading R37)."""
        sp = self.sponge
        lv = self.g.levels[lev]
        x = (lv.coords[cells] + 0.5) * float(2 ** lev)
        r = np.sqrt(((x - np.asarray(sp["centre"], float)[None, : self.lat.D]) ** 2).sum(axis=1))
        sigma = np.clip((r - sp["r0"]) / (sp["r1"] - sp["r0"]), 0.0, 1.0) * sp["sigma_max"]
        rho, u = hm.macroscopic(self.lat, f)
        rho_new = rho * (1.0 - sigma) + sigma * sp["rho_inf"]
        relaxed = f + hm.feq_athermal(self.lat, rho_new, u) - hm.feq_athermal(self.lat, rho, u)
        return np.where(sigma[None, :] > 0.0, relaxed, f)

    def _collide(self, lev: int, f, g, lam, cells=None):
        """Post-collision state of cells with pre-collision (f, g, lam) at level ``lev``
        (``cells``: their indices in the level, for position-dependent terms)."""
        tau = self.tau[lev]
        if not self.comp:
            if self.sponge is not None and cells is not None:
                f = self._relax_far_field(lev, cells, f)
            fs = hm.collide_weak(self.lat, f, tau, self.model, self.trace_eq, self.trt_magic)
            return fs, None, None, np.zeros(f.shape[1], np.int64)
        rho, u, T = self._moments(f, g)
        lam0 = self._guess(u, T, lam) if lam is not None else None
        feq, lam_new, it = self._feq_comp(rho, u, T, lam0)
        geq = (2.0 * self.Cv - self.lat.D) * T[None, :] * feq
        tau_eff = np.full(f.shape[1], tau)
        if self.sensor_A is not None:
            tau_eff = tau_eff * sensor_alpha(sensor_eps(f, feq), tau, self.sensor_A)
        fs = f - (f - feq) / tau_eff[None, :]
        gs = g - (g - geq) / tau_eff[None, :]
        return fs, gs, lam_new, it

    # ------------------------------------------------------------------ initialisation
    def init_fields(self, fields) -> None:
        """fields[level] = (rho (n,), u (D, n), T (n,) or None): equilibrium initialisation."""
        for lev, (rho, u, T) in enumerate(fields):
            rho = np.asarray(rho, dtype=np.float64)
            u = np.asarray(u, dtype=np.float64).reshape(self.lat.D, -1)
            if rho.size == 0:
                continue
            if not self.comp:
                self.f[lev] = hm.feq_athermal(self.lat, rho, u)
                continue
            T = np.asarray(T, dtype=np.float64)
            lam0 = None
            if self.model == "num_ddf":
                lam0 = nm.poly_guess(self.lat, u, T, self.poly_order)
            feq, lam, _ = self._feq_comp(rho, u, T, lam0)
            self.f[lev] = feq
            self.g_[lev] = (2.0 * self.Cv - self.lat.D) * T[None, :] * feq
            if lam is not None:
                self.lam[lev] = lam
        # the boundary layers hold their boundary values from the start (Appendix A.3: the
        # conditions are applied over the reach layers; here also to the initial state)
        for lev in range(self.g.n_levels):
            self._boundaries(lev)

    # ------------------------------------------------------------------ phases
    def _coalesced(self, lev: int):
        """Pre-collision populations of the coarse ghosts of ``lev`` with unknowns coalesced: the
        mean over the children of their streamed populations, a child whose history left the
        finer level standing in with the ghost's own streamed population (reading R33)."""
        lv = self.g.levels[lev]
        C, kids, unk = lv.cg_cells, lv.cg_children, lv.cg_unknown
        brk = lv.cg_broken
        f = self.f[lev][:, C].copy()
        fine_f = np.where(brk, f[:, :, None], self.f[lev - 1][:, kids])        # (Q, nc, nk), R33
        f[unk] = fine_f.mean(axis=2)[unk]
        g = lam = None
        if self.comp:
            g = self.g_[lev][:, C].copy()
            fine_g = np.where(brk, g[:, :, None], self.g_[lev - 1][:, kids])
            g[unk] = fine_g.mean(axis=2)[unk]
        if self.lam is not None:
            lam = self.lam[lev - 1][:, kids].mean(axis=2)
        return f, g, lam

    def coupling(self, lev: int) -> None:
        """refinementCoupling(lev, lev-1): coalescence, coarse collision, uniform explosion."""
        lv = self.g.levels[lev]
        C, kids = lv.cg_cells, lv.cg_children
        if C.size == 0:
            self._cg_post[lev] = None
            return
        f, g, lam = self._coalesced(lev)
        fs, gs, lam_new, it = self._collide(lev, f, g, lam, C)
        self._cg_post[lev] = (fs, gs, lam_new, it)
        nk = kids.shape[1]
        for k in range(nk):
            self.f[lev - 1][:, kids[:, k]] = fs
            if self.comp:
                self.g_[lev - 1][:, kids[:, k]] = gs
            if self.lam is not None:
                self.lam[lev - 1][:, kids[:, k]] = lam_new

    def collide_and_stream(self, lev: int) -> None:
        lv = self.g.levels[lev]
        lat = self.lat
        ct = lv.ctype
        f = self.f[lev]
        fs = f.copy()
        gs = self.g_[lev].copy() if self.comp else None
        lam = self.lam[lev] if self.lam is not None else None
        # bulk fluid and boundary cells collide; fine ghosts keep f* = f (pure streaming)
        coll = np.nonzero((ct == FLUID) | (ct == BC))[0]
        if coll.size:
            g_in = self.g_[lev][:, coll] if self.comp else None
            l_in = lam[:, coll] if lam is not None else None
            a, b, c, it = self._collide(lev, f[:, coll], g_in, l_in, coll)
            fs[:, coll] = a
            if self.comp:
                gs[:, coll] = b
            if lam is not None:
                lam[:, coll] = c
            self.iters[lev][coll] = it
        # coarse ghosts: the coupling's post-collision state (R2)
        if lev >= 1 and lv.cg_cells.size:
            a, b, c, it = self._cg_post[lev]
            fs[:, lv.cg_cells] = a
            if self.comp:
                gs[:, lv.cg_cells] = b
            if lam is not None:
                lam[:, lv.cg_cells] = c
            self.iters[lev][lv.cg_cells] = it
            self._cg_post[lev] = None
        fs[:, ct == SOLID] = 0.0
        if self.comp:
            gs[:, ct == SOLID] = 0.0
        # streaming: f_i(x, t+1) = f*_i(x - xi_i, t); blocked links bounce back
        self.f[lev] = self._stream(lv, fs)
        if self.comp:
            self.g_[lev] = self._stream(lv, gs, wall_terms=False)
        self._boundaries(lev)

    def _stream(self, lv, fs, wall_terms: bool = True):
        lat = self.lat
        new = np.zeros_like(fs)
        opp = lat.opp
        for q in range(lat.Q):
            src = lv.src[q]
            ok = (src >= 0) & ~lv.blocked[q]
            new[q, ok] = fs[q, src[ok]]
            b = lv.blocked[q]
            new[q, b] = fs[opp[q], b] + (lv.wall_term[q, b] if wall_terms else 0.0)
        new[:, lv.ctype == SOLID] = 0.0
        return new

    def _boundaries(self, lev: int) -> None:
        lv = self.g.levels[lev]
        if lv.bc_cells.size == 0:
            return
        from .grid import FACES
        cells, kinds, faces, part = lv.bc_cells, lv.bc_kind, lv.bc_face, lv.bc_partner
        neu = kinds == 3
        if neu.any():
            c, p = cells[neu], part[neu]
            self.f[lev][:, c] = self.f[lev][:, p]
            if self.comp:
                self.g_[lev][:, c] = self.g_[lev][:, p]
            if self.lam is not None:
                self.lam[lev][:, c] = self.lam[lev][:, p]
        dirm = ~neu
        if not dirm.any():
            return
        c, p = cells[dirm], part[dirm]
        n = c.size
        rho = np.empty(n)
        u = np.empty((self.lat.D, n))
        T = np.empty(n)
        for k in range(n):
            spec = self.g.faces[FACES[faces[dirm][k]]]
            _, r, uu, TT = spec[0], spec[1], spec[2], spec[3] if len(spec) > 3 else None
            rho[k] = r
            u[:, k] = uu[: self.lat.D]
            T[k] = TT if TT is not None else self.T0
        extrap = kinds[dirm] == 2
        rho[extrap] = self.f[lev][:, p[extrap]].sum(axis=0)
        if not self.comp:
            self.f[lev][:, c] = hm.feq_athermal(self.lat, rho, u)
            return
        lam0 = self.lam[lev][:, c] if self.lam is not None else None
        if lam0 is not None and self.guess != "warm":
            lam0 = self._guess(u, T, lam0)
        feq, lam, _ = self._feq_comp(rho, u, T, lam0)
        self.f[lev][:, c] = feq
        self.g_[lev][:, c] = (2.0 * self.Cv - self.lat.D) * T[None, :] * feq
        if lam is not None:
            self.lam[lev][:, c] = lam

    # ------------------------------------------------------------------ schedule
    def fine_iteration(self) -> None:
        """One iteration of the Sec. 4.5 schedule."""
        t = self.t
        for lev in range(self.g.n_levels - 1, 0, -1):
            if t % (2 ** lev) == 0:
                self.coupling(lev)
                self.collide_and_stream(lev)
        self.collide_and_stream(0)
        self.t += 1

    def step_fine(self, n: int) -> None:
        for _ in range(n):
            self.fine_iteration()

    def step_coarse(self, n: int) -> None:
        self.step_fine(n * 2 ** (self.g.n_levels - 1))

    # ------------------------------------------------------------------ outputs
    def moments(self, lev: int):
        """(rho, u, T) of every cell of ``lev`` from its current pre-collision populations."""
        g = self.g_[lev] if self.comp else None
        return self._moments(self.f[lev], g)

    def ledger(self) -> np.ndarray:
        """Conserved totals (R3): mass, momentum (D), energy, at a coarse synchronisation instant.

        Sum over bulk, boundary and coarse-ghost cells of every level (fine ghosts excluded)
        of the cell volume 2^(i D) times sum_i f_i, sum_i xi_i f_i and
        sum_i (|xi_i|^2 f_i + g_i)/2, the coarse ghosts' unknown populations replaced by their
        coalesced values.
        """
        if self.t % (2 ** (self.g.n_levels - 1)):
            raise ValueError("ledger is defined at coarse synchronisation instants only")
        lat = self.lat
        xi = lat.xi.astype(np.float64)
        xi2 = (xi ** 2).sum(axis=1)
        out = np.zeros(lat.D + 2)
        for lev, lv in enumerate(self.g.levels):
            V = float(2 ** (lev * lat.D))
            sel = np.nonzero((lv.ctype == FLUID) | (lv.ctype == BC))[0]
            parts = [(self.f[lev][:, sel], self.g_[lev][:, sel] if self.comp else None)]
            if lev >= 1 and lv.cg_cells.size:
                f, g, _ = self._coalesced(lev)
                parts.append((f, g))
            for f, g in parts:
                out[0] += V * f.sum()
                out[1:1 + lat.D] += V * (xi.T @ f).sum(axis=1)
                e = 0.5 * (xi2 @ f).sum()
                if g is not None:
                    e += 0.5 * g.sum()
                out[1 + lat.D] += V * e
        return out
