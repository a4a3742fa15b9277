"""Pins of the oracle's heat-equation fiber field (Sec. 3.6, "Modeling").

P1 elements reproduce linear fields exactly, so: with Dirichlet data taken
from a linear function on the whole boundary, the discrete harmonic field is
that function and every tet's fiber is its normalised gradient; with -1/+1
on the two end faces of a box (insulated sides) the field is linear along
the box and the fibers are axial. On a cylinder the field obeys the maximum
principle and the fibers are unit vectors running from origin to insertion.
"""
import numpy as np

from emu_inputs import box_beam, muscle_tendon_unit
from oracle.fibers import fiber_field, harmonic_field


def test_linear_boundary_data_give_the_linear_field_and_its_gradient():
    mesh = box_beam(3, 3, 4, h=0.01)
    Q = mesh.rest_pos
    lo, hi = Q.min(0), Q.max(0)
    bnd = np.nonzero(np.any((np.abs(Q - lo) < 1e-12) | (np.abs(Q - hi) < 1e-12), axis=1))[0]
    a = np.array([0.7, -1.3, 2.1])
    g = Q @ a + 0.25
    f, Gs = harmonic_field(Q, mesh.tets, bnd, g[bnd])
    np.testing.assert_allclose(f, g, atol=1e-12 * np.abs(g).max())
    grad = (Gs @ f).reshape(-1, 3)
    np.testing.assert_allclose(grad, np.broadcast_to(a, grad.shape), atol=1e-10 * np.linalg.norm(a))


def test_end_faces_give_axial_fibers():
    mesh = box_beam(2, 3, 5, h=0.01)
    Q = mesh.rest_pos
    L = Q[:, 2].max()
    origin = np.nonzero(Q[:, 2] == 0.0)[0]
    insertion = np.nonzero(np.abs(Q[:, 2] - L) < 1e-12)[0]
    u, f = fiber_field(Q, mesh.tets, origin, insertion)
    np.testing.assert_allclose(f, -1.0 + 2.0 * Q[:, 2] / L, atol=1e-12)
    np.testing.assert_allclose(u, np.broadcast_to([0.0, 0.0, 1.0], u.shape), atol=1e-12)


def test_cylinder_fibers_are_unit_and_run_from_origin_to_insertion():
    mesh = muscle_tendon_unit(6, 6, 20, h=0.01, radius_cells=2.6, frames=1)
    Q = mesh.rest_pos
    L = Q[:, 2].max()
    origin = np.nonzero(Q[:, 2] == 0.0)[0]
    # the insertion is a patch of the far end only: the field bends towards it
    far = np.nonzero((np.abs(Q[:, 2] - L) < 1e-12) & (Q[:, 0] >= np.median(Q[:, 0])))[0]
    u, f = fiber_field(Q, mesh.tets, origin, far)
    assert f.min() >= -1.0 - 1e-12 and f.max() <= 1.0 + 1e-12      # maximum principle
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-12)
    assert np.mean(u[:, 2]) > 0.8                                   # along the muscle, origin -> insertion
    # the field is not the trivial axial one: fibers near the far end lean towards the patch
    cen = Q[mesh.tets].mean(axis=1)
    near_end = cen[:, 2] > 0.9 * L
    assert np.mean(u[near_end, 0]) > 0.05
