"""GPU parity of constant external forces (Sec. 3.4, Eq. external-forces)
against the FP64 oracle, through emu_set_external_forces.

Tolerances as for the other parity tests (positions relative to the rest
bounding-box diagonal): FP64 path 1e-9 with both sides at relative residual
1e-11; mixed path 1e-4 at 1e-6. Gravity is the lumped mass of the Kuhn grid
times g, strong enough here to bend the beams visibly; one case adds an
arbitrary per-vertex force field and one has no activation at all.
"""
import dataclasses

import numpy as np
import pytest

from emu_inputs import box_beam, gravity_forces, muscle_tendon_unit
from oracle import EmuOracle, OracleParams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def emu():
    import torch

    assert torch.cuda.is_available()
    from paper_2006_08821_gb300 import build as b

    b.build()
    import paper_2006_08821_gb300 as emu

    emu.load_library()
    return emu


def _diag(mesh):
    return float(np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0)))


def _oracle(mesh, a, tol=1e-11):
    o = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0))
    return o.solve(a, tol=tol)


def _gpu(emu, mesh, a, precision=0, tol=1e-11):
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=tol, precision=precision))  # picks up mesh.f_ext
    s.set_activation(a)
    st = s.solve()
    return s, st


def _beam(act=0.5, g=(0.0, -40.0, -20.0), extra=False, dims=(2, 2, 6)):
    mesh = box_beam(*dims, activation=act)
    f = gravity_forces(mesh, g=g)
    if extra:
        f = f + np.random.default_rng(5).normal(size=f.shape) * np.abs(f).max()
    return dataclasses.replace(mesh, f_ext=f)


@pytest.mark.parametrize("act,extra", [(0.5, False), (0.0, False), (0.3, True)])
def test_fp64_path_with_external_forces_matches_oracle(emu, act, extra):
    mesh = _beam(act, extra=extra)
    r = _oracle(mesh, act)
    s, st = _gpu(emu, mesh, act)
    assert st.status == 0 and st.rel_residual <= 1e-11
    q = s.positions()
    diag = _diag(mesh)
    assert np.abs(q - mesh.rest_pos).max() > 1e-2 * diag  # the load bends the beam
    err = np.abs(q - r.q).max() / diag
    assert err <= 1e-9, err
    s.close()


def test_mixed_path_with_gravity_matches_oracle(emu):
    mesh = _beam(0.5)
    r = _oracle(mesh, 0.5)
    s, st = _gpu(emu, mesh, 0.5, precision=1, tol=1e-6)
    assert st.status == 0 and st.rel_residual <= 1e-6
    err = np.abs(s.positions() - r.q).max() / _diag(mesh)
    assert err <= 1e-4, err
    s.close()


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-11, 1e-9), (1, 1e-6, 1e-4)])
def test_muscle_tendon_unit_with_gravity_matches_oracle(emu, precision, tol, bound):
    # two materials (tendon E = 1e8, muscle 6e5), a sideways load on top of the activation
    base = muscle_tendon_unit(4, 4, 14, h=0.01, radius_cells=1.9, frames=1, a_max=0.6)
    mesh = dataclasses.replace(base, f_ext=gravity_forces(base, g=(-20.0, 0.0, -9.81)))
    a = mesh.activations[0]
    r = _oracle(mesh, a, tol=1e-11 if precision == 0 else 1e-10)
    s, st = _gpu(emu, mesh, a, precision=precision, tol=tol)
    assert st.status == 0 and st.rel_residual <= tol
    err = np.abs(s.positions() - r.q).max() / _diag(mesh)
    assert err <= bound, (err, st.newton_iters, r.iterations)
    s.close()


def test_removing_the_forces_restores_the_unloaded_result(emu):
    mesh = _beam(0.4)
    plain = dataclasses.replace(mesh, f_ext=None)
    s0, _ = _gpu(emu, plain, 0.4, precision=1, tol=1e-6)
    q0 = s0.positions()
    s0.close()
    s, _ = _gpu(emu, mesh, 0.4, precision=1, tol=1e-6)
    q_loaded = s.positions()
    assert np.abs(q_loaded - q0).max() > 1e-3 * _diag(mesh)
    s.set_external_forces(None)
    s.reset()
    s.set_activation(np.full(mesh.n_tets, 0.4))
    st = s.solve()
    assert st.status == 0
    np.testing.assert_array_equal(s.positions(), q0)
    s.close()


def test_invalid_forces_are_rejected(emu):
    mesh = box_beam(1, 1, 2)
    s = emu.Solver(mesh, emu.Params())
    lib = s.lib
    import ctypes as C

    bad = np.zeros((mesh.n_verts + 1, 3))
    rc = lib.emu_set_external_forces(s.handle, bad.ctypes.data_as(C.POINTER(C.c_double)), mesh.n_verts + 1)
    assert rc == -1
    nan = np.zeros((mesh.n_verts, 3))
    nan[1, 2] = np.nan
    with pytest.raises(emu.EmuError) as e:
        s.set_external_forces(nan)
    assert e.value.code == -1
    s.close()
