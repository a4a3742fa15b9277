"""The alpha heuristic of Sec. 3.7 on the oracle: test infrastructure, like
the rest of ``oracle/``.

The paper searches the ACAP weight alpha upward from 1 at a fixed
activation, tallies the Newton iterations to convergence, and takes the
value just before a sharp increase of that count. Readings: the values are
alpha_rel = alpha0 * factor^k (decades by default, as in the paper's table
of alpha = 1e0 .. 1e5); "sharp" means more than ``jump`` times the previous
count (default 3); a solve that does not converge counts as a sharp
increase; with no increase the last value tried is taken.
"""
from __future__ import annotations

from .emu_oracle import EmuOracle, OracleParams


def pick_alpha(alphas, iters, jump=3.0):
    """The value before the first count above jump times its predecessor's
    (None counts as unbounded), else the last value; with its index."""
    for k in range(1, len(iters)):
        prev, cur = iters[k - 1], iters[k]
        if cur is None or (prev is not None and cur > jump * prev):
            return alphas[k - 1], k - 1
    return alphas[len(iters) - 1], len(iters) - 1


def alpha_sweep(mesh, activation, alpha0=1.0, factor=10.0, max_steps=6, jump=3.0, tol=1e-6, max_newton=2000,
                params: OracleParams | None = None):
    """Runs the sweep from the rest state; returns (alpha_rel, alphas, iters),
    iters[k] None where the solve did not converge."""
    base = params or OracleParams()
    alphas, iters = [], []
    for k in range(max_steps):
        ar = alpha0 * factor ** k
        p = OracleParams(**{**base.__dict__, "alpha_rel": ar})
        try:
            r = EmuOracle(mesh, p).solve(activation, tol=tol, max_newton=max_newton)
            it = r.iterations if r.rel_residual <= tol else None
        except RuntimeError:
            it = None
        alphas.append(ar)
        iters.append(it)
        if k > 0 and (it is None or (iters[k - 1] is not None and it > jump * iters[k - 1])):
            break
    a, _ = pick_alpha(alphas, iters, jump)
    return a, alphas, iters
