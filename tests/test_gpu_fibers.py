"""GPU heat-equation fiber field (Sec. 3.6) against the oracle's.

emu_fiber_field solves the P1 Laplace equation on the device (FP64 CG to
1e-13) and normalises the per-tet gradients. Bounds: axial fibers between
the end faces of a box to 1e-10 (the exact answer), and 1e-8 per component
against the oracle's direct solve on cylinders whose field bends towards a
partial insertion (several CG blocks and a ragged tail).
"""
import dataclasses

import numpy as np
import pytest

from emu_inputs import box_beam, mtu_for_tet_count, muscle_tendon_unit
from oracle import EmuOracle, OracleParams
from oracle.fibers import fiber_field as oracle_fibers

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


def _ends(Q):
    L = Q[:, 2].max()
    origin = np.nonzero(Q[:, 2] == 0.0)[0]
    far = np.nonzero((np.abs(Q[:, 2] - L) < 1e-12) & (Q[:, 0] >= np.median(Q[:, 0])))[0]
    return origin, far


def test_end_faces_give_axial_fibers(emu):
    mesh = box_beam(3, 2, 7, h=0.01)
    Q = mesh.rest_pos
    L = Q[:, 2].max()
    origin = np.nonzero(Q[:, 2] == 0.0)[0]
    insertion = np.nonzero(np.abs(Q[:, 2] - L) < 1e-12)[0]
    u = emu.fiber_field(Q, mesh.tets, origin, insertion)
    np.testing.assert_allclose(u, np.broadcast_to([0.0, 0.0, 1.0], u.shape), atol=1e-10)


@pytest.mark.parametrize("kind", ["small", "large"])
def test_cylinder_fibers_match_the_oracle(emu, kind):
    mesh = (muscle_tendon_unit(6, 6, 20, h=0.01, radius_cells=2.6, frames=1) if kind == "small"
            else mtu_for_tet_count(40000))
    Q = mesh.rest_pos
    origin, far = _ends(Q)
    u_ref, _ = oracle_fibers(Q, mesh.tets, origin, far)
    u = emu.fiber_field(Q, mesh.tets, origin, far)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-12)
    assert np.abs(u - u_ref).max() <= 1e-8, np.abs(u - u_ref).max()


def test_solve_with_heat_equation_fibers_matches_the_oracle(emu):
    base = muscle_tendon_unit(4, 4, 14, h=0.01, radius_cells=1.9, frames=1, a_max=0.6)
    origin, far = _ends(base.rest_pos)
    mesh = dataclasses.replace(base, fiber_dir=emu.fiber_field(base.rest_pos, base.tets, origin, far))
    a = mesh.activations[0]
    r = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0)).solve(a, tol=1e-10)
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-6, precision=1))
    s.set_activation(a)
    st = s.solve()
    assert st.status == 0
    diag = float(np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0)))
    assert np.abs(s.positions() - r.q).max() / diag <= 1e-4
    s.close()


def test_invalid_inputs_are_rejected(emu):
    mesh = box_beam(1, 1, 2)
    Q = mesh.rest_pos
    with pytest.raises(emu.EmuError) as e:
        emu.fiber_field(Q, mesh.tets, [0, 1], [1, 5])   # a vertex in both sets
    assert e.value.code == -1
    with pytest.raises(emu.EmuError) as e:
        emu.fiber_field(Q, mesh.tets, [0], [Q.shape[0]])  # out of range
    assert e.value.code == -1
    flat = Q.copy()
    flat[:, 2] = 0.0                                      # every tet degenerate
    with pytest.raises(emu.EmuError) as e:
        emu.fiber_field(flat, mesh.tets, [0], [5])
    assert e.value.code == -1
