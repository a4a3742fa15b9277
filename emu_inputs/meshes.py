"""Synthetic tetrahedral meshes and workloads (seeded, NumPy only).

Stand-ins for the paper's musculoskeletal assets (Table 2 of the paper lists
meshes of 3k-600k tets built with TetWild; none are available here). Every
mesh is a grid of cubes of edge ``h`` split into six tets per cube along the
main diagonal (Kuhn/Freudenthal split), optionally masked to a cylinder.

Conventions shared by every consumer:

* ``rest_pos``  (n, 3) float64, metres.
* ``tets``      (m, 4) int32. Corner 3 is the paper's reference corner
  (Eq. 2 uses q_i4 as the origin of the edge matrix). The ordering makes the
  edge matrix [Q0-Q3, Q1-Q3, Q2-Q3] positively oriented; this is arranged
  from the permutation parity of the Kuhn split.
* ``material_id`` (m,) uint8 indexing ``youngs`` / ``poisson``.
* ``fiber_dir`` (m, 3) float64 unit vectors (muscle fiber direction u_i).
* ``fixed_verts`` int32 vertex indices held at their rest positions.
* ``activations`` (frames, m) float64, a_i(t) >= 0 per tet and frame.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

MUSCLE, TENDON, BONE = 0, 1, 2

# Permutations of the three axes and their parity. The Kuhn tet for
# permutation p is [c, c+e_p0, c+e_p0+e_p1, c+(1,1,1)].
_PERMS = list(itertools.permutations(range(3)))


def _perm_sign(p):
    s = 1
    p = list(p)
    for i in range(3):
        for j in range(i + 1, 3):
            if p[i] > p[j]:
                s = -s
    return s


@dataclasses.dataclass
class MeshSpec:
    name: str
    rest_pos: np.ndarray
    tets: np.ndarray
    youngs: np.ndarray
    poisson: np.ndarray
    material_id: np.ndarray
    fiber_dir: np.ndarray
    fixed_verts: np.ndarray
    activations: np.ndarray
    fixed_pos: np.ndarray | None = None
    bone_id: np.ndarray | None = None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_verts(self) -> int:
        return int(self.rest_pos.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    def with_activation(self, a) -> "MeshSpec":
        a = np.asarray(a, dtype=np.float64)
        if a.ndim == 0:
            a = np.full((1, self.n_tets), float(a))
        elif a.ndim == 1:
            a = a[None, :]
        return dataclasses.replace(self, activations=a)


def kuhn_grid(nx: int, ny: int, nz: int, h: float):
    """Vertices and Kuhn-split tets of an nx x ny x nz grid of cubes.

    Returns (rest_pos (n,3), tets (m,4), centroid (m,3)). Tets are ordered
    cell by cell (x fastest), six per cell.
    """
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    # vertex id = i + (nx+1)*(j + (ny+1)*k)
    vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)  # noqa: E731
    n = (nx + 1) * (ny + 1) * (nz + 1)
    rest = np.zeros((n, 3))
    flat = vid(ii, jj, kk).ravel()
    rest[flat, 0] = ii.ravel() * h
    rest[flat, 1] = jj.ravel() * h
    rest[flat, 2] = kk.ravel() * h

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci = ci.transpose(2, 1, 0).ravel()  # cell order: x fastest, then y, then z
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    ncell = ci.size
    tets = np.zeros((ncell, 6, 4), dtype=np.int64)
    for t, p in enumerate(_PERMS):
        corners = [np.zeros(3, dtype=np.int64)]
        e = np.zeros(3, dtype=np.int64)
        for ax in p:
            e = e.copy()
            e[ax] += 1
            corners.append(e)
        ids = [vid(ci + c[0], cj + c[1], ck + c[2]) for c in corners]
        # [Q0-Q3, Q1-Q3, Q2-Q3] has the sign of -sign(p) for this order; swap
        # corners 1 and 2 for even permutations so every tet is positive.
        if _perm_sign(p) > 0:
            ids[1], ids[2] = ids[2], ids[1]
        for c in range(4):
            tets[:, t, c] = ids[c]
    tets = tets.reshape(-1, 4)
    centroid = rest[tets].mean(axis=1)
    return rest, tets.astype(np.int32), centroid


def _compact(rest, tets, keep):
    tets = tets[keep]
    used = np.unique(tets)
    remap = -np.ones(rest.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    return rest[used].copy(), remap[tets].astype(np.int32), used


def box_beam(nx=4, ny=4, nz=16, h=0.01, youngs=6e5, poisson=0.45, activation=0.5, name=None):
    """Box beam of nx x ny x nz cubes, one muscle material, fibers along z,
    the z = 0 face pinned. The 4x4x16, h = 1 cm default has 1,536 tets and
    425 vertices."""
    rest, tets, _ = kuhn_grid(nx, ny, nz, h)
    m = tets.shape[0]
    fixed = np.nonzero(rest[:, 2] == 0.0)[0].astype(np.int32)
    fib = np.zeros((m, 3))
    fib[:, 2] = 1.0
    act = np.atleast_1d(np.asarray(activation, dtype=np.float64))
    acts = np.broadcast_to(act[:, None], (act.size, m)).copy()
    return MeshSpec(
        name=name or f"box_beam_{nx}x{ny}x{nz}",
        rest_pos=rest,
        tets=tets,
        youngs=np.array([youngs], dtype=np.float64),
        poisson=np.array([poisson], dtype=np.float64),
        material_id=np.zeros(m, dtype=np.uint8),
        fiber_dir=fib,
        fixed_verts=fixed,
        activations=acts,
        meta=dict(nx=nx, ny=ny, nz=nz, h=h),
    )


def single_tet():
    """One tet, corner 3 pinned and corners 0..2 free (brute-force tests)."""
    rest = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [0, 0, 0]]) * 0.01
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    return MeshSpec(
        name="single_tet",
        rest_pos=rest,
        tets=tets,
        youngs=np.array([6e5]),
        poisson=np.array([0.45]),
        material_id=np.zeros(1, dtype=np.uint8),
        fiber_dir=np.array([[0.0, 0.0, 1.0]]),
        fixed_verts=np.array([3], dtype=np.int32),
        activations=np.array([[0.5]]),
    )


def muscle_tendon_unit(nx=32, ny=32, nz=128, h=2.5e-3, radius_cells=12.9, tendon_frac=0.10,
                       frames=60, seed=1, youngs_muscle=6e5, youngs_tendon=1e8, poisson=0.45,
                       fiber_sigma_deg=5.0, a_max=1.0, name=None):
    """Muscle-tendon unit: a cube grid masked to a cylinder about the z axis.

    Tets whose centroid lies within ``radius_cells * h`` of the grid's axis
    are kept. Tets with centroid z below ``tendon_frac/2 * L`` or above
    ``(1 - tendon_frac/2) * L`` are tendon, the rest muscle. Fibers follow z
    with a seeded Gaussian tilt (|N(0, sigma)|, uniform azimuth). The
    activation ramps linearly from 0 to ``a_max`` over ``frames`` frames on
    muscle tets only. Vertices on z = 0 are pinned.
    """
    rest, tets, cen = kuhn_grid(nx, ny, nz, h)
    cx, cy = 0.5 * nx * h, 0.5 * ny * h
    r = np.hypot(cen[:, 0] - cx, cen[:, 1] - cy)
    keep = r <= radius_cells * h
    rest, tets, _ = _compact(rest, tets, keep)
    cen = cen[keep]
    m = tets.shape[0]
    L = nz * h
    half = 0.5 * tendon_frac
    is_tendon = (cen[:, 2] < half * L) | (cen[:, 2] > (1.0 - half) * L)
    mat = np.where(is_tendon, TENDON, MUSCLE).astype(np.uint8)
    rng = np.random.default_rng(seed)
    theta = np.abs(rng.normal(0.0, math.radians(fiber_sigma_deg), size=m))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=m)
    fib = np.stack([np.tan(theta) * np.cos(phi), np.tan(theta) * np.sin(phi), np.ones(m)], axis=1)
    fib /= np.linalg.norm(fib, axis=1, keepdims=True)
    if frames > 1:
        ramp = a_max * np.arange(frames) / (frames - 1)
    else:
        ramp = np.array([a_max])
    acts = np.where(is_tendon[None, :], 0.0, ramp[:, None])
    fixed = np.nonzero(rest[:, 2] == 0.0)[0].astype(np.int32)
    return MeshSpec(
        name=name or f"mtu_{nx}x{ny}x{nz}",
        rest_pos=rest,
        tets=tets,
        youngs=np.array([youngs_muscle, youngs_tendon], dtype=np.float64),
        poisson=np.array([poisson, poisson], dtype=np.float64),
        material_id=mat,
        fiber_dir=fib,
        fixed_verts=fixed,
        activations=acts,
        meta=dict(nx=nx, ny=ny, nz=nz, h=h, radius_cells=radius_cells, tendon_frac=tendon_frac),
    )


def mtu_for_tet_count(target_tets, tendon_frac=0.10, frames=1, seed=1, a_max=1.0, h=None):
    """Muscle-tendon unit with about ``target_tets`` tets: a c x c x 4c grid
    masked to radius 0.403c (the 32x32x128, r = 12.9h proportions)."""
    c = max(2, int(round((target_tets / 12.25) ** (1.0 / 3.0))))
    hh = h if h is not None else 0.08 / c
    return muscle_tendon_unit(nx=c, ny=c, nz=4 * c, h=hh, radius_cells=0.403 * c,
                              tendon_frac=tendon_frac, frames=frames, seed=seed, a_max=a_max)


def batch_set(count=256, seed=3, t_min=1e3, t_max=6e4, h=0.01):
    """Independent box beams with log-uniform tet counts in [t_min, t_max].

    Cross-section c x c with c = max(2, round((T/24)^(1/3))), length
    nz = max(1, round(T/(6c^2))); material, fibers and pins as the box beam;
    activation uniform in [0, 1] per mesh.
    """
    rng = np.random.default_rng(seed)
    T = np.exp(rng.uniform(math.log(t_min), math.log(t_max), size=count))
    acts = rng.uniform(0.0, 1.0, size=count)
    out = []
    for b in range(count):
        c = max(2, int(round((T[b] / 24.0) ** (1.0 / 3.0))))
        nz = max(1, int(round(T[b] / (6.0 * c * c))))
        out.append(box_beam(c, c, nz, h=h, activation=acts[b], name=f"batch{b}_{c}x{c}x{nz}"))
    return out


def request_stream(rate_hz=200.0, horizon_s=60.0, seed=4, t_min=1e3, t_max=2e5, max_frames=30,
                   max_requests=None):
    """Poisson request stream of quasi-static solves (descriptors only).

    Each request: arrival time, target tet count (log-uniform), tendon
    fraction U[0, 0.2], frame count U{1..max_frames}, and a_max U[0, 1]. The
    mesh itself is built on demand with ``mtu_for_tet_count``.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > horizon_s:
            break
        reqs.append(dict(
            id=len(reqs),
            arrival_s=t,
            tets=float(math.exp(rng.uniform(math.log(t_min), math.log(t_max)))),
            tendon_frac=float(rng.uniform(0.0, 0.2)),
            frames=int(rng.integers(1, max_frames + 1)),
            a_max=float(rng.uniform(0.0, 1.0)),
            seed=int(rng.integers(0, 2**31 - 1)),
        ))
        if max_requests is not None and len(reqs) >= max_requests:
            break
    return reqs
