"""Max-entropy ("numerical") equilibrium by Newton-Raphson with a backtracking line search.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sources (arXiv 2504.04465, Appendix A):
  * Eq. exponential: f_i^eq = a exp[-(1 + sum_n lambda^(n) . M_i^(n))], with a = rho.
  * Eqs. G0_8mom .. G3yaa_8mom: eight constraints on the raw moments
        1, xi_x, xi_y, xi_x^2, xi_x xi_y, xi_y^2, xi_x |xi|^2, xi_y |xi|^2
    whose Maxwell-Boltzmann values are rho, rho u, rho(u_x^2 + T), rho u_x u_y,
    rho(u_y^2 + T), 2 rho u (E + T) with 2E = |u|^2 + D T (D = 2).
  * Newton-Raphson "coupled with a line search as in GSL"; tolerance 1e-12 in FP64.

Readings (design notes R7/R8): because a = rho, every constraint is rho times a function of
(lambda, u, T), so the multipliers are solved with rho = 1 and do not depend on rho.  The
Jacobian is J = -sum_i f_i M_i M_i^T, so the Newton step is d = (sum_i f_i M_i M_i^T)^{-1} G and
lambda <- lambda + t d.  The step length t starts at 1 and halves (at most 30 times) until
||G||_2 decreases; after the last halving the trial is accepted as is.  The iteration stops
when max_a |G_a| < tol, or after ``max_iter`` steps.  The iteration count of a cell is the
number of Newton steps it took.

The polynomial guess (R8) is the weighted least-squares fit, with the lattice weights, of
-1 - ln f_poly,i onto the eight basis functions over the populations where f_poly,i > 0,
f_poly being the thermal Hermite equilibrium of the lattice (rho = 1).
"""
from __future__ import annotations

import numpy as np

from .hermite import feq_thermal
from .lattices import Lattice

N_LAMBDA = 8


def moment_basis(lat: Lattice) -> np.ndarray:
    """M (8, Q): the raw monomials constrained by Eqs. G0..G3yaa."""
    x = lat.xi[:, 0].astype(np.float64)
    y = lat.xi[:, 1].astype(np.float64)
    r2 = x * x + y * y
    return np.stack([np.ones_like(x), x, y, x * x, x * y, y * y, x * r2, y * r2])


def mb_targets(u: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Maxwell-Boltzmann values of the 8 moments for rho = 1 -> (8, n)."""
    ux, uy = u[0], u[1]
    u2 = ux * ux + uy * uy
    two_e_plus_t = u2 + 4.0 * T          # 2(E + T) with 2E = |u|^2 + 2T
    return np.stack([np.ones_like(ux), ux, uy, ux * ux + T, ux * uy, uy * uy + T,
                     ux * two_e_plus_t, uy * two_e_plus_t])


def feq_exp(M: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """exp[-(1 + lambda . M_i)] for rho = 1 -> (Q, n)."""
    return np.exp(-(1.0 + M.T @ lam))


def residual(M: np.ndarray, lam: np.ndarray, target: np.ndarray):
    e = feq_exp(M, lam)
    return M @ e - target, e


def newton(lat: Lattice, u: np.ndarray, T: np.ndarray, lam0: np.ndarray, tol: float = 1e-12,
           max_iter: int = 50, max_halvings: int = 30):
    """Solve G(lambda) = 0 for every cell.  Returns (lambda, f_eq/rho, iterations, converged)."""
    M = moment_basis(lat)
    target = mb_targets(u, T)
    lam = np.array(lam0, dtype=np.float64, copy=True)
    n = lam.shape[1]
    iters = np.zeros(n, dtype=np.int64)
    done = np.zeros(n, dtype=bool)
    converged = np.zeros(n, dtype=bool)
    G, e = residual(M, lam, target)
    e_final = e.copy()
    for it in range(max_iter + 1):
        ok = (~done) & (np.abs(G).max(axis=0) < tol)
        converged |= ok
        e_final[:, ok] = e[:, ok]
        done |= ok
        if it == max_iter:
            e_final[:, ~done] = e[:, ~done]
            done[:] = True
        act = np.nonzero(~done)[0]
        if act.size == 0:
            break
        # Newton direction: (sum_i e_i M_i M_i^T) d = G
        Ea = e[:, act]
        A = np.einsum("ai,bi,in->nab", M, M, Ea)
        d = np.linalg.solve(A, G[:, act].T[:, :, None])[:, :, 0].T   # (8, na)
        g0 = (G[:, act] ** 2).sum(axis=0)
        t = np.ones(act.size)
        lam_a = lam[:, act]
        accepted = np.zeros(act.size, dtype=bool)
        lam_new = lam_a.copy()
        G_new = G[:, act].copy()
        e_new = Ea.copy()
        for h in range(max_halvings + 1):
            pend = np.nonzero(~accepted)[0]
            if pend.size == 0:
                break
            trial = lam_a[:, pend] + t[pend] * d[:, pend]
            Gt, et = residual(M, trial, target[:, act[pend]])
            better = (Gt ** 2).sum(axis=0) < g0[pend]
            take = better | (h == max_halvings)
            sel = pend[take]
            lam_new[:, sel] = trial[:, take]
            G_new[:, sel] = Gt[:, take]
            e_new[:, sel] = et[:, take]
            accepted[sel] = True
            t[pend[~take]] *= 0.5
        lam[:, act] = lam_new
        G[:, act] = G_new
        e[:, act] = e_new
        iters[act] += 1
    return lam, e_final, iters, converged


def poly_guess(lat: Lattice, u: np.ndarray, T: np.ndarray, order: int) -> np.ndarray:
    """Weighted least-squares fit of -1 - ln f_poly onto the 8 basis functions (R8).

    Only populations with f_poly > 0 take part (the truncated polynomial turns negative on
    the outer velocities at large |u| or T - theta); the weights are the lattice weights.
    """
    M = moment_basis(lat)
    rho1 = np.ones_like(T)
    fp = feq_thermal(lat, rho1, u, T, order)
    pos = fp > 0.0
    y = np.where(pos, -1.0 - np.log(np.where(pos, fp, 1.0)), 0.0)     # (Q, n)
    W = lat.w[:, None] * pos                                           # (Q, n)
    A = np.einsum("ai,bi,in->nab", M, M, W)                            # (n, 8, 8)
    b = np.einsum("ai,in->na", M, W * y)                               # (n, 8)
    return np.linalg.solve(A, b[:, :, None])[:, :, 0].T
