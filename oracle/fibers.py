"""Fiber directions from the heat equation (Sec. 3.6, "Modeling"): test
infrastructure, like the rest of ``oracle/`` (only the tests, the smoke
check and the benchmark's CPU leg call it).

For a muscle the paper solves the steady heat equation Delta f = 0 with
Dirichlet values +1 at the insertion and -1 at the origin and takes the
normalised gradient of f as the fiber direction. Here, with P1 elements on
the tets: f is the vertex field minimising sum_i V_i |grad f_i|^2 under the
Dirichlet values (the discrete Laplace equation), grad f_i = sum_{j<3}
(f_j - f_3) D_m^-T e_j on tet i, and u_i = grad f_i / |grad f_i| (zero where
the gradient vanishes).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .emu_oracle import rest_geometry


def scalar_gradient(n_verts, tets, Dinv):
    """Sparse (3m x n): (Gs f)_{3i+c} = sum_{j<3} (f_j - f_3) Dinv_i[j][c]."""
    T = np.asarray(tets, dtype=np.int64)
    m = T.shape[0]
    rows, cols, vals = [], [], []
    ii = np.arange(m)
    for c in range(3):
        row = 3 * ii + c
        for j in range(3):
            rows.append(row)
            cols.append(T[:, j])
            vals.append(Dinv[:, j, c])
        rows.append(row)
        cols.append(T[:, 3])
        vals.append(-(Dinv[:, 0, c] + Dinv[:, 1, c] + Dinv[:, 2, c]))
    Gs = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * m, n_verts))
    Gs.sum_duplicates()
    return Gs


def harmonic_field(rest_pos, tets, dirichlet_verts, dirichlet_vals):
    """The vertex field f minimising sum_i V_i |grad f_i|^2 with f fixed on
    ``dirichlet_verts``; vertices in no tet keep 0."""
    Q = np.asarray(rest_pos, dtype=np.float64)
    n = Q.shape[0]
    _, Dinv, V = rest_geometry(Q, tets)
    Gs = scalar_gradient(n, tets, Dinv)
    L = (Gs.T @ sp.diags(np.repeat(V, 3)) @ Gs).tocsr()
    dv = np.asarray(dirichlet_verts, dtype=np.int64)
    f = np.zeros(n)
    f[dv] = np.asarray(dirichlet_vals, dtype=np.float64)
    in_tet = np.zeros(n, dtype=bool)
    in_tet[np.asarray(tets, dtype=np.int64).ravel()] = True
    free = np.ones(n, dtype=bool)
    free[dv] = False
    free &= in_tet
    fi = np.nonzero(free)[0]
    di = np.nonzero(~free & in_tet)[0]
    rhs = -(L[fi][:, di] @ f[di])
    f[fi] = spla.spsolve(L[fi][:, fi].tocsc(), rhs)
    return f, Gs


def fiber_field(rest_pos, tets, origin, insertion):
    """Per-tet unit fiber directions (m, 3): the normalised gradient of the
    harmonic field that is -1 on ``origin`` and +1 on ``insertion``."""
    origin = np.asarray(origin, dtype=np.int64)
    insertion = np.asarray(insertion, dtype=np.int64)
    verts = np.concatenate([origin, insertion])
    vals = np.concatenate([-np.ones(origin.size), np.ones(insertion.size)])
    f, Gs = harmonic_field(rest_pos, tets, verts, vals)
    g = (Gs @ f).reshape(-1, 3)
    nrm = np.linalg.norm(g, axis=1)
    u = np.zeros_like(g)
    ok = nrm > 0.0
    u[ok] = g[ok] / nrm[ok, None]
    return u, f
