"""The seeded input generators: reproducible, and with the sizes and
structure the workloads are stated with (Kuhn grids, pins, tendon ends,
fiber tilt, activation ramps, the batch and the request stream)."""
import math

import numpy as np

from emu_inputs import (BONE, MUSCLE, TENDON, arm_assembly, batch_set, box_beam, muscle_tendon_unit,
                        request_stream)


def _same(a, b):
    for f in ("rest_pos", "tets", "youngs", "poisson", "material_id", "fiber_dir", "fixed_verts", "activations"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_generators_are_reproducible():
    _same(muscle_tendon_unit(8, 8, 32, h=0.01, radius_cells=3.2, frames=3, seed=5),
          muscle_tendon_unit(8, 8, 32, h=0.01, radius_cells=3.2, frames=3, seed=5))
    _same(arm_assembly(bone_w=2, bone_len=4, r0=2.0, frames=3), arm_assembly(bone_w=2, bone_len=4, r0=2.0, frames=3))
    a, b = batch_set(count=8, seed=3), batch_set(count=8, seed=3)
    for x, y in zip(a, b):
        _same(x, y)
    assert request_stream(seed=4, max_requests=20) == request_stream(seed=4, max_requests=20)


def test_box_beam_has_the_stated_size_and_pins():
    mesh = box_beam(4, 4, 16, h=0.01)
    assert (mesh.n_tets, mesh.n_verts) == (1536, 425)
    assert set(mesh.fixed_verts.tolist()) == set(np.nonzero(mesh.rest_pos[:, 2] == 0.0)[0].tolist())
    assert mesh.fixed_verts.size == 25


def test_muscle_tendon_unit_structure():
    mesh = muscle_tendon_unit(frames=60)
    assert (mesh.n_tets, mesh.n_verts) == (401920, 74929)
    cz = mesh.rest_pos[mesh.tets].mean(axis=1)[:, 2]
    L = 128 * 2.5e-3
    tendon = mesh.material_id == TENDON
    np.testing.assert_array_equal(tendon, (cz < 0.05 * L) | (cz > 0.95 * L))
    assert set(np.unique(mesh.material_id).tolist()) == {MUSCLE, TENDON}
    # fibers: unit vectors tilted from z by |N(0, 5 deg)|
    np.testing.assert_allclose(np.linalg.norm(mesh.fiber_dir, axis=1), 1.0, rtol=1e-12)
    tilt = np.degrees(np.arccos(mesh.fiber_dir[:, 2]))
    assert 3.5 < tilt.mean() < 4.5  # E|N(0, 5)| = 5 sqrt(2 / pi) = 3.99
    # ramp 0 -> 1 over 60 frames on muscle only
    np.testing.assert_array_equal(mesh.activations[:, tendon], 0.0)
    np.testing.assert_allclose(mesh.activations[:, ~tendon][:, 0], np.arange(60) / 59.0)


def test_batch_set_sizes_are_log_uniform_in_range():
    meshes = batch_set(count=256, seed=3)
    m = np.array([x.n_tets for x in meshes])
    assert m.sum() == 3548724
    assert m.min() >= 500 and m.max() <= 80000
    a = np.array([x.activations[0, 0] for x in meshes])
    assert 0.0 <= a.min() and a.max() <= 1.0


def test_request_stream_statistics():
    reqs = request_stream(seed=4, horizon_s=60.0)
    gaps = np.diff([r["arrival_s"] for r in reqs])
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0          # Poisson, 200 / s
    t = np.log([r["tets"] for r in reqs])
    assert math.log(1e3) <= t.min() and t.max() <= math.log(2e5)
    assert all(1 <= r["frames"] <= 30 for r in reqs)
    assert all(0.0 <= r["tendon_frac"] <= 0.2 for r in reqs)


def test_arm_assembly_materials_and_activation():
    mesh = arm_assembly(bone_w=2, bone_len=4, r0=2.0, frames=8)
    bone = mesh.bone_id >= 0
    np.testing.assert_array_equal(bone, mesh.material_id == BONE)
    assert mesh.youngs[BONE] == 1e10 and mesh.poisson[BONE] == 0.3
    active = mesh.activations.max(axis=0) > 0
    assert not np.any(active & bone) and not np.any(active & (mesh.material_id == TENDON))
    np.testing.assert_allclose(mesh.activations[:, active][:, 0], np.sin(np.pi * np.arange(8) / 8) ** 2)
