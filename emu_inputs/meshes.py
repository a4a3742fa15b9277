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
    # joints between bones: dicts with "type" ("hinge" or "ball"), "bones"
    # (b1, b2), "point" (3,) metres, and for a hinge "axis" (3,) unit and
    # "half_length" (metres; the hinge's two points are point +- half_length axis)
    joints: list | None = None
    # constant external force per vertex (n, 3), newtons (e.g. gravity_forces)
    f_ext: np.ndarray | None = None
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


def arm_assembly(bone_w=12, bone_len=58, r0=32.0, gap_x=1, h=2.5e-3, frames=120, a_max=1.0,
                 youngs_muscle=6e5, youngs_tendon=1e8, youngs_bone=1e10, poisson=0.45,
                 poisson_bone=0.3, name=None):
    """Arm-like assembly: two box bones, a hinge between them, and a fusiform
    muscle spanning them (the setting of Sec. 3.3 of the paper).

    One cube grid of edge h, every size below in cells:

    * bone 1 occupies x in [0, bone_w), y in [y0, y0 + bone_w), z in
      [0, bone_len); bone 2 the same x, y range and z in [bone_len + 1,
      2 bone_len + 1): the bones are collinear along z with a one-cell gap,
      so they share no vertex;
    * the muscle is a spindle about the line x = bone_w + gap_x + r0,
      y = ny / 2, from z_a = bone_len / 2 (mid bone 1) to z_b = bone_len +
      1 + bone_len / 2 (mid bone 2), of radius r(t) = r0 (0.3 + 0.7 sin pi t),
      t = (z - z_a) / (z_b - z_a), by cell centres; it never touches a bone;
    * two tendon bars, two cells thick in z around z_a and z_b, join the
      spindle's ends to the bones' +x faces (shared vertices);
    * materials: muscle (E = 6e5), tendon (E = 1e8), bone (E = 1e10,
      nu = 0.3); bone_id 0 / 1 on the bones' tets, -1 elsewhere;
    * spindle fibers u = normalise(e_z + rho r'(z) / r(z) e_rho) (rho the
      distance to the spindle's axis, e_rho its direction); e_z elsewhere;
    * every vertex of bone 1 is pinned;
    * one hinge at the gap's centre on the bones' axis, along y, with
      half-length bone_w / 2;
    * activation a_max sin^2(pi f / frames), f = 0 .. frames - 1, on the
      spindle's tets (0 on tendon and bone).

    The defaults give about 800k tets with two 50,112-tet bones.
    """
    bw, L = int(bone_w), int(bone_len)
    nyc = max(bw, 2 * int(math.ceil(r0)) + 2)
    if (nyc - bw) % 2:
        nyc += 1
    y0 = (nyc - bw) // 2
    xc = bw + gap_x + r0
    yc = 0.5 * nyc
    nx = int(math.ceil(xc + r0)) + 1
    nz = 2 * L + 1
    rest, tets, cen = kuhn_grid(nx, nyc, nz, h)
    c = cen / h  # centroids in cell units
    # label each tet by its cell (the six tets of a cell share its centre)
    cell = np.floor(c).astype(np.int64)
    cc = cell + 0.5
    in_y = (cell[:, 1] >= y0) & (cell[:, 1] < y0 + bw)
    in_x = cell[:, 0] < bw
    bone1 = in_x & in_y & (cell[:, 2] < L)
    bone2 = in_x & in_y & (cell[:, 2] >= L + 1) & (cell[:, 2] < 2 * L + 1)
    za, zb = 0.5 * L, L + 1 + 0.5 * L
    t = (cc[:, 2] - za) / (zb - za)
    tt = np.clip(t, 0.0, 1.0)
    rt = r0 * (0.3 + 0.7 * np.sin(np.pi * tt))
    rho = np.hypot(cc[:, 0] - xc, cc[:, 1] - yc)
    spindle = (t >= 0.0) & (t <= 1.0) & (rho <= rt)
    bar_y = np.abs(cc[:, 1] - yc) <= max(0.3 * r0, 0.5)
    bar_x = (cc[:, 0] > bw) & (cc[:, 0] <= xc)
    bar_z = (np.abs(cc[:, 2] - za) <= 1.0) | (np.abs(cc[:, 2] - zb) <= 1.0)
    bar = bar_x & bar_y & bar_z
    bone = bone1 | bone2
    spindle &= ~bone
    bar &= ~(bone | spindle)
    keep = bone | spindle | bar
    rest, tets, _ = _compact(rest, tets, keep)
    bone1, bone2, spindle, bar = bone1[keep], bone2[keep], spindle[keep], bar[keep]
    cc, rho, tt = cc[keep], rho[keep], tt[keep]
    m = tets.shape[0]
    mat = np.full(m, MUSCLE, dtype=np.uint8)
    mat[bar] = TENDON
    mat[bone1 | bone2] = BONE
    bone_id = np.full(m, -1, dtype=np.int32)
    bone_id[bone1] = 0
    bone_id[bone2] = 1
    # spindle fibers: e_z plus the radial slope of the spindle's surface
    drdz = r0 * 0.7 * np.pi * np.cos(np.pi * tt) / (zb - za)
    er = np.stack([cc[:, 0] - xc, cc[:, 1] - yc, np.zeros(m)], axis=1)
    er /= np.maximum(rho, 1e-12)[:, None]
    slope = np.where(spindle, rho * drdz / np.maximum(r0 * (0.3 + 0.7 * np.sin(np.pi * tt)), 1e-12), 0.0)
    fib = np.zeros((m, 3))
    fib[:, 2] = 1.0
    fib += slope[:, None] * er
    fib /= np.linalg.norm(fib, axis=1, keepdims=True)
    f = np.arange(frames)
    ramp = a_max * np.sin(np.pi * f / frames) ** 2
    acts = np.where(spindle[None, :], ramp[:, None], 0.0)
    fixed = np.unique(tets[bone1]).astype(np.int32)
    hinge = dict(type="hinge", bones=(0, 1),
                 point=np.array([0.5 * bw, y0 + 0.5 * bw, L + 0.5]) * h,
                 axis=np.array([0.0, 1.0, 0.0]), half_length=0.5 * bw * h)
    return MeshSpec(
        name=name or f"arm_{bw}x{L}_r{r0:g}",
        rest_pos=rest,
        tets=tets,
        youngs=np.array([youngs_muscle, youngs_tendon, youngs_bone], dtype=np.float64),
        poisson=np.array([poisson, poisson, poisson_bone], dtype=np.float64),
        material_id=mat,
        fiber_dir=fib,
        fixed_verts=fixed,
        activations=acts,
        bone_id=bone_id,
        joints=[hinge],
        meta=dict(nx=nx, ny=nyc, nz=nz, h=h, bone_w=bw, bone_len=L, r0=r0, gap_x=gap_x),
    )


def gravity_forces(mesh: MeshSpec, density=1060.0, g=(0.0, 0.0, -9.81)) -> np.ndarray:
    """Per-vertex gravity on a Kuhn-grid mesh: every tet of a grid of cubes
    of edge h (``mesh.meta["h"]``) has the mass density * h^3 / 6, split
    equally over its four corners, times the acceleration g. (n, 3).
    Soft tissue density (1060 kg/m^3) by default."""
    h = float(mesh.meta["h"])
    T = np.asarray(mesh.tets, dtype=np.int64)
    mass = np.zeros(mesh.n_verts)
    np.add.at(mass, T.ravel(), density * h ** 3 / 24.0)
    return mass[:, None] * np.asarray(g, dtype=np.float64)[None, :]
