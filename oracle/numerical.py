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
Jacobian is J = -sum_i f_i M_i M_i^T, so the Newton step is d = (sum_i f_i M_i M_i^T)^{-1} G
(solved by Cholesky) and lambda <- lambda + t d.  The step length t starts at 1 and halves (at
most 30 times) until ||G||_2 decreases; after the last halving the trial is accepted if its
residual is finite.  A cell converges when its residual is finite and max_a |G_a| < tol.  A
cell stops unconverged, keeping its last finite iterate, when the Cholesky factorisation
meets a pivot that is not positive (singular Jacobian: exp underflow at extreme states), when
the last trial of the line search is not finite, or after ``max_iter`` steps.  The iteration
count of a cell is the number of Newton steps it took.

The polynomial guess (R8) is the weighted least-squares fit, with the lattice weights, of
-1 - ln f_poly,i onto the eight basis functions over the populations where f_poly,i > 0,
f_poly being the thermal Hermite equilibrium of the lattice (rho = 1), solved by Cholesky.
The fit is kept only where it is finite and its residual ||G||_2 is below that of
lambda = 0; elsewhere (large |u| or T far from the lattice temperature, where the truncated
polynomial is a poor model of the exponential) the guess is lambda = 0.
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


def cholesky_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x with A x = b for SPD A (n, m, m), b (n, m), by the Cholesky factorisation A = L L^T
    (column by column, inner sums in increasing index order).  Cells where a pivot is not
    positive get NaN."""
    n, m, _ = A.shape
    Lf = np.zeros_like(A)
    bad = np.zeros(n, dtype=bool)
    for j in range(m):
        s = A[:, j, j].copy()
        for k in range(j):
            s -= Lf[:, j, k] * Lf[:, j, k]
        bad |= ~(s > 0.0)
        djj = np.sqrt(np.where(s > 0.0, s, 1.0))
        Lf[:, j, j] = djj
        for i in range(j + 1, m):
            t = A[:, i, j].copy()
            for k in range(j):
                t -= Lf[:, i, k] * Lf[:, j, k]
            Lf[:, i, j] = t / djj
    y = np.zeros((n, m))
    for i in range(m):
        t = b[:, i].copy()
        for k in range(i):
            t -= Lf[:, i, k] * y[:, k]
        y[:, i] = t / Lf[:, i, i]
    x = np.zeros((n, m))
    for i in range(m - 1, -1, -1):
        t = y[:, i].copy()
        for k in range(i + 1, m):
            t -= Lf[:, k, i] * x[:, k]
        x[:, i] = t / Lf[:, i, i]
    x[bad] = np.nan
    return x


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
        finite = np.isfinite(G).all(axis=0)
        ok = (~done) & finite & (np.abs(G).max(axis=0) < tol)
        converged |= ok
        e_final[:, ok] = e[:, ok]
        done |= ok
        stop = (~done) & ~finite
        if it == max_iter:
            stop = ~done
        e_final[:, stop] = e[:, stop]
        done |= stop
        act = np.nonzero(~done)[0]
        if act.size == 0:
            break
        # Newton direction: (sum_i e_i M_i M_i^T) d = G; a singular system stops the cell
        Ea = e[:, act]
        A = np.einsum("ai,bi,in->nab", M, M, Ea)
        d = cholesky_solve(A, G[:, act].T).T                          # (8, na)
        sing = ~np.isfinite(d).all(axis=0)
        if sing.any():
            s_idx = act[sing]
            e_final[:, s_idx] = e[:, s_idx]
            done[s_idx] = True
            act, d, Ea = act[~sing], d[:, ~sing], Ea[:, ~sing]
            if act.size == 0:
                continue
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
            g1 = (Gt ** 2).sum(axis=0)
            take = (g1 < g0[pend]) | ((h == max_halvings) & np.isfinite(g1))
            sel = pend[take]
            lam_new[:, sel] = trial[:, take]
            G_new[:, sel] = Gt[:, take]
            e_new[:, sel] = et[:, take]
            accepted[sel] = True
            t[pend[~take]] *= 0.5
        # a line search that ends on a non-finite trial stops the cell at its current iterate
        rej = act[~accepted]
        e_final[:, rej] = e[:, rej]
        done[rej] = True
        acc = act[accepted]
        lam[:, acc] = lam_new[:, accepted]
        G[:, acc] = G_new[:, accepted]
        e[:, acc] = e_new[:, accepted]
        iters[acc] += 1
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
    fit = cholesky_solve(A, b).T                                       # (8, n)
    # keep the fit where it is finite and closer to the root than lambda = 0 (R8)
    target = mb_targets(u, T)
    zero = np.zeros_like(fit)
    with np.errstate(over="ignore", invalid="ignore"):
        G_fit, _ = residual(M, np.where(np.isfinite(fit), fit, 0.0), target)
        G_zero, _ = residual(M, zero, target)
        keep = np.isfinite(fit).all(axis=0) & ((G_fit ** 2).sum(axis=0) < (G_zero ** 2).sum(axis=0))
    return np.where(keep[None, :], fit, 0.0)
