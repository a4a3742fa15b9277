"""Independent vertex-space solvers used to pin the oracle (test infrastructure).

1. ``envelope_solve``: Newton on positions q for
       E_hat(q) = sum_i min_F [V_i Psi(F) + alpha w_i / 2 ||G_i q - F||^2].
   Minimising Eq. 5 over F with q = q*(F) is the same as minimising the
   joint energy over (q, F), because the two minimisations commute. So
   E_hat has the same stationary positions as EMU (Sec. 3.1). The inner
   minimisation is a per-tet 9-variable Newton solve. The outer gradient
   follows from the envelope theorem. The outer Hessian is
   G^T [alpha W - alpha^2 W^2 (V Psi'' + alpha W)^-1] G. This is a
   different algorithm from Algorithm 1: no low-rank Hessian and no
   Woodbury step.

2. ``fem_solve``: plain finite elements, min_q sum_i V_i Psi(G_i q) - q^T f
   (f the mesh's constant per-vertex force, if any). This is the
   alpha -> infinity limit that Sec. 3.7 compares against.

Both reuse only the per-tet energy functions (themselves pinned by finite
differences) and the sparse G of Eq. 2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .emu_oracle import EmuOracle, d2psi, dpsi, psd_project, psi


def _prox_F(o: EmuOracle, A, a, F0=None, iters=60):
    """Per tet: argmin_F V Psi(F) + c/2 ||A - F||^2, c = alpha w (Newton)."""
    c = o.alpha * o.w
    ka = o.kappa * a
    F = A.copy() if F0 is None else F0.copy()
    # keep the start non-inverted
    bad = np.linalg.det(F) <= 0
    F[bad] = np.eye(3)

    def f(F):
        D = (F - A).reshape(o.m, 9)
        return o.V * psi(F, o.mu, o.lam, ka, o.u) + 0.5 * c * np.einsum("ij,ij->i", D, D)

    for _ in range(iters):
        g = (o.V[:, None, None] * dpsi(F, o.mu, o.lam, ka, o.u) + c[:, None, None] * (F - A)).reshape(o.m, 9)
        if np.max(np.abs(g)) < 1e-15 * np.max(o.V * o.mu):
            break
        H = psd_project(o.V[:, None, None] * d2psi(F, o.mu, o.lam, ka, o.u)) + c[:, None, None] * np.eye(9)
        d = -np.linalg.solve(H, g[..., None])[..., 0].reshape(o.m, 3, 3)
        f0 = f(F)
        step = np.ones(o.m)
        for _ in range(40):
            Ft = F + step[:, None, None] * d
            ok = f(Ft) <= f0 + 1e-4 * step * np.einsum("ij,ij->i", g, d.reshape(o.m, 9)) + 1e-14 * np.abs(f0)
            if np.all(ok):
                break
            step = np.where(ok, step, 0.5 * step)
        F = F + step[:, None, None] * d
    return F


def envelope_solve(o: EmuOracle, a, tol=1e-12, max_iter=100):
    """Newton on E_hat(q) over the free DOFs; returns positions (n, 3)."""
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), (o.m,)).copy()
    c = o.alpha * o.w
    ka = o.kappa * a
    q = o.acap_solve(np.broadcast_to(np.eye(3), (o.m, 3, 3)).copy())
    F = None
    g_ref = None
    for _ in range(max_iter):
        A = o.deformation_gradients(q)
        F = _prox_F(o, A, a, F)
        r = (c[:, None, None] * (A - F)).reshape(-1)
        grad = o.G_f.T @ r
        gn = np.linalg.norm(grad)
        if g_ref is None:
            g_ref = max(gn, 1e-300)
        if gn <= tol * g_ref:
            break
        Hel = o.V[:, None, None] * d2psi(F, o.mu, o.lam, ka, o.u)
        inner = np.linalg.inv(Hel + c[:, None, None] * np.eye(9))
        Hb = c[:, None, None] * np.eye(9) - (c**2)[:, None, None] * inner
        m = o.m
        rows = np.repeat(np.arange(9 * m).reshape(m, 9, 1), 9, axis=2)
        cols = np.repeat(np.arange(9 * m).reshape(m, 1, 9), 9, axis=1)
        Hbig = sp.csr_matrix((Hb.ravel(), (rows.ravel(), cols.ravel())), shape=(9 * m, 9 * m))
        Hq = (o.G_f.T @ Hbig @ o.G_f).tocsc()
        dq_f = spla.spsolve(Hq, -grad)
        dq = np.zeros_like(q)
        dq[o.free_dofs] = dq_f
        q = q + dq
    return q.reshape(o.n, 3)


def fem_solve(o: EmuOracle, a, tol=1e-12, max_iter=200):
    """Newton with backtracking on sum_i V_i Psi(G_i q) (plain FEM)."""
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), (o.m,)).copy()
    ka = o.kappa * a
    q = o.Q.reshape(-1).copy()
    q[o.fixed_dofs] = o.q_c

    f_ext = getattr(o.mesh, "f_ext", None)
    f_free = (np.zeros(o.free_dofs.size) if f_ext is None
              else np.asarray(f_ext, dtype=np.float64).reshape(-1)[o.free_dofs])

    def energy(q):
        return np.sum(o.V * psi(o.deformation_gradients(q), o.mu, o.lam, ka, o.u)) - float(q[o.free_dofs] @ f_free)

    g_ref = None
    for _ in range(max_iter):
        F = o.deformation_gradients(q)
        P = o.V[:, None, None] * dpsi(F, o.mu, o.lam, ka, o.u)
        grad = o.G_f.T @ P.reshape(-1) - f_free
        gn = np.linalg.norm(grad)
        if g_ref is None:
            g_ref = max(gn, 1e-300)
        if gn <= tol * g_ref:
            break
        Hb = psd_project(o.V[:, None, None] * d2psi(F, o.mu, o.lam, ka, o.u))
        m = o.m
        rows = np.repeat(np.arange(9 * m).reshape(m, 9, 1), 9, axis=2)
        cols = np.repeat(np.arange(9 * m).reshape(m, 1, 9), 9, axis=1)
        Hbig = sp.csr_matrix((Hb.ravel(), (rows.ravel(), cols.ravel())), shape=(9 * m, 9 * m))
        Hq = (o.G_f.T @ Hbig @ o.G_f).tocsc()
        d = spla.spsolve(Hq, -grad)
        e0 = energy(q)
        gtd = float(grad @ d)
        s = 1.0
        for _ in range(50):
            qt = q.copy()
            qt[o.free_dofs] += s * d
            if energy(qt) <= e0 + 1e-4 * s * gtd + 1e-15 * abs(e0):
                break
            s *= 0.5
        q[o.free_dofs] += s * d
    return q.reshape(o.n, 3)
