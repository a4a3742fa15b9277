"""Pins of the bone-and-joint oracle (Sec. 3.3) against facts fixed by the
paper's constraints and by mathematics.

The reading of Sec. 3.3 that the oracle implements is stated in its module
header (one F per bone, bone rows as a penalty during Newton, joints as
least-squares affine fits, the slack schedule). Each test checks it against
something other than itself: finite differences of the energy, the plain
oracle when there are no bones, the exact constraints the final solve must
satisfy, and the kinematics a hinge allows.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from emu_inputs import arm_assembly, box_beam
from oracle import EmuOracle, OracleParams
from oracle.bones import BoneOracle, affine_fit_weights

PRM = OracleParams(alpha_rel=1.0, weight_mode=0)


@pytest.fixture(scope="module")
def arm():
    return arm_assembly(bone_w=2, bone_len=4, r0=2.0, frames=4)


@pytest.fixture(scope="module")
def arm_solved(arm):
    o = BoneOracle(arm, PRM)
    r = o.solve(arm.activations[2], tol=1e-10)
    return o, r


def _diag(mesh):
    return float(np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0)))


def test_arm_assembly_layout(arm):
    big = arm_assembly()
    assert 790_000 <= big.n_tets <= 810_000
    assert (big.bone_id == 0).sum() == (big.bone_id == 1).sum() == 50_112
    for mesh in (arm, arm_assembly(bone_w=3, bone_len=8, r0=3.0, frames=2)):
        T = mesh.tets
        v1, v2 = np.unique(T[mesh.bone_id == 0]), np.unique(T[mesh.bone_id == 1])
        vm = np.unique(T[mesh.bone_id < 0])
        assert np.intersect1d(v1, v2).size == 0             # a gap between the bones
        assert np.intersect1d(vm, v1).size > 0 and np.intersect1d(vm, v2).size > 0  # muscle fused to both
        n = mesh.n_verts
        A = sp.coo_matrix((np.ones(16 * T.shape[0]), (np.repeat(T, 4, axis=1).ravel(), np.tile(T, (1, 4)).ravel())),
                          shape=(n, n))
        assert connected_components(A)[0] == 1
        assert set(mesh.fixed_verts.tolist()) == set(v1.tolist())   # bone 1 pinned
        p0 = mesh.joints[0]["point"]
        assert mesh.rest_pos[v1, 2].max() < p0[2] < mesh.rest_pos[v2, 2].min()


def test_affine_fit_weights_reproduce_affine_fields():
    rng = np.random.default_rng(3)
    Q = rng.normal(size=(11, 3))
    A, t, p = rng.normal(size=(3, 3)), rng.normal(size=3), rng.normal(size=3)
    c = affine_fit_weights(Q, p)
    np.testing.assert_allclose(c @ (Q @ A.T + t), A @ p + t, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(c.sum(), 1.0, rtol=1e-13)


def test_without_bones_the_bone_oracle_is_the_plain_oracle():
    mesh = box_beam(2, 2, 4, activation=0.6)
    r0 = EmuOracle(mesh, PRM).solve(0.6, tol=1e-11)
    r1 = BoneOracle(mesh, PRM).solve(0.6, tol=1e-11)
    assert np.abs(r1.q - r0.q).max() <= 1e-10 * _diag(mesh)
    assert abs(r1.iterations - r0.iterations) <= 2


def test_reduced_gradient_matches_central_differences(arm):
    o = BoneOracle(arm, PRM)
    a = arm.activations[2]
    rng = np.random.default_rng(5)
    X = o.identity() + 0.01 * rng.normal(size=(o.nvar, 3, 3))

    def E(Y):
        return o.energy(Y, o.acap_solve(o.full_F(Y)), a)

    g = o.gradient(X, o.acap_solve(o.full_F(X)), a)
    for only_bone in (False, True):
        dX = rng.normal(size=X.shape)
        if only_bone:  # the free bone's F alone: sums over its tets
            keep = np.zeros(o.nvar, dtype=bool)
            keep[o.bone_slot[1]] = True
            dX[~keep] = 0.0
        h = 1e-6
        fd = (E(X + h * dX) - E(X - h * dX)) / (2 * h)
        assert abs(fd - np.sum(g * dX)) <= 1e-6 * abs(fd), (fd, np.sum(g * dX))


def test_joint_rows_hold_exactly_in_the_newton_phase(arm):
    o = BoneOracle(arm, PRM)
    rng = np.random.default_rng(6)
    for _ in range(2):
        X = o.identity() + 0.05 * rng.normal(size=(o.nvar, 3, 3))
        q = o.acap_solve(o.full_F(X))
        assert np.abs(o.joint_residual(q)).max() <= 1e-14 * _diag(arm)


def test_converged_state_is_stationary_by_finite_differences(arm, arm_solved):
    # independent of the gradient routine: E is flat at the result along
    # random directions, relative to its slope at the rest state. The
    # differences are taken term by term (delta_energy, pinned against plain
    # differences in the oracle's own tests): the bone's energy, V mu with
    # mu = 3.8e9, cancels to zero under rotation and a plain difference
    # would keep only its rounding
    o, r = arm_solved
    a = arm.activations[2]
    rng = np.random.default_rng(7)

    def slope(X, dX, h=1e-8):  # the bone's stiff third derivative wants a small h
        q = o.acap_solve(o.full_F(X))
        dq = o.acap_solve_d(o.full_d(dX))
        return (o.delta_energy(X, dX, q, dq, a, h) - o.delta_energy(X, dX, q, dq, a, -h)) / (2 * h)

    for _ in range(2):
        dX = rng.normal(size=r.F.shape)
        assert abs(slope(r.F, dX)) <= 1e-8 * abs(slope(o.identity(), dX))


def test_final_solve_makes_each_bone_follow_its_F(arm, arm_solved):
    o, r = arm_solved
    diag = _diag(arm)
    v1, v2 = o.bone_verts
    np.testing.assert_array_equal(r.q[v1], arm.rest_pos[v1])     # pinned bone at rest
    Fb = r.F[o.bone_slot[1]]
    aff = r.q[v2] - arm.rest_pos[v2] @ Fb.T
    assert np.abs(aff - aff.mean(0)).max() <= 1e-12 * diag    # q_v = F_b Q_v + t_b
    disp = np.abs(r.q - arm.rest_pos).max()
    assert disp > 1e-3 * diag
    # eps1 = -1e-4: the joint opens by a negligible amount ...
    assert np.abs(o.joint_residual(r.q.reshape(-1))).max() <= 1e-5 * disp
    # ... while without the joint the free bone is pulled far off the hinge
    free = BoneOracle(dataclasses.replace(arm, joints=None), PRM).solve(arm.activations[2], tol=1e-8)
    assert np.abs(o.joint_residual(free.q.reshape(-1))).max() >= 1e-2 * disp


def test_hinge_turns_the_free_bone_rigidly_about_its_axis(arm, arm_solved):
    o, r = arm_solved
    Fb = r.F[o.bone_slot[1]]
    U, S, Vt = np.linalg.svd(Fb)
    R = U @ Vt
    assert np.abs(S - 1.0).max() <= 1e-6        # E = 1e10: no visible stretch
    angle = np.arccos(np.clip(0.5 * (np.trace(R) - 1.0), -1.0, 1.0))
    axis = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    axis /= np.linalg.norm(axis)
    assert angle > 0.05                         # the muscle flexes the joint
    assert abs(axis @ np.asarray(arm.joints[0]["axis"])) >= 1.0 - 1e-8


def test_warm_started_frame_reaches_the_cold_solution(arm):
    # frames are solved from the previous frame's F (Sec. 4's sequences); the
    # stationary point must not depend on the start
    o = BoneOracle(arm, PRM)
    a1, a2 = arm.activations[1], arm.activations[2]
    r1 = o.solve(a1, tol=1e-10)
    warm = o.solve(a2, X0=r1.F, tol=1e-10)
    cold = o.solve(a2, tol=1e-10)
    assert np.abs(warm.q - cold.q).max() <= 1e-8 * _diag(arm)


def test_ball_joint_holds_its_point_and_lets_the_bone_turn(arm):
    ball = [dict(type="ball", bones=(0, 1), point=arm.joints[0]["point"])]
    mesh = dataclasses.replace(arm, joints=ball)
    o = BoneOracle(mesh, PRM)
    r = o.solve(mesh.activations[2], tol=1e-10)
    assert len(o.joint_points) == 1
    Fb = r.F[o.bone_slot[1]]
    v2 = o.bone_verts[1]
    t_b = (r.q[v2] - mesh.rest_pos[v2] @ Fb.T).mean(0)
    p0 = np.asarray(ball[0]["point"])
    disp = np.abs(r.q - mesh.rest_pos).max()
    # the free bone's affine map keeps the joint point (bone 1 is pinned at rest)
    assert np.linalg.norm(Fb @ p0 + t_b - p0) <= 1e-5 * disp
    U, S, Vt = np.linalg.svd(Fb)
    angle = np.arccos(np.clip(0.5 * (np.trace(U @ Vt) - 1.0), -1.0, 1.0))
    assert angle > 0.05


def test_reduced_capacitance_equals_its_gram_form_with_a_virtual_tet_per_bone(arm):
    # Eq. 12's capacitance Lambda - alpha B H^-1 B^T over the reduced
    # variables, assembled another way: every deformable tet as the Gram term
    # w Gamma^T N Gamma (N = I - alpha w H^-1), pinned-bone tets as
    # w Gamma^T Gamma, and a free bone as one tet of weight sum w, operator
    # the weighted mean of its tets' Gamma, plus their weighted variance
    o = BoneOracle(arm, PRM)
    a = arm.activations[2]
    rng = np.random.default_rng(1)
    X = o.identity() + 0.02 * rng.normal(size=(o.nvar, 3, 3))
    H = o.hessian_blocks(X, a)
    al = o.base.alpha
    Bt = o.B.T.reshape(o.nvar, 9, o.k)
    C_ref = o.Lhat - al * (o.B @ np.linalg.solve(H, Bt).reshape(9 * o.nvar, o.k))
    Gam = (o.base.G_f @ o.Phi).reshape(o.m, 9, o.k)
    w, slot, sb = o.w, o.slot, o.bone_slot[1]
    C = np.zeros((o.k, o.k))
    for i in range(o.m):
        if slot[i] < 0:
            C += w[i] * Gam[i].T @ Gam[i]
        elif slot[i] != sb:
            C += w[i] * Gam[i].T @ (np.eye(9) - al * w[i] * np.linalg.inv(H[slot[i]])) @ Gam[i]
    tb = np.nonzero(slot == sb)[0]
    wb = w[tb].sum()
    Gbar = np.einsum("i,ijk->jk", w[tb], Gam[tb]) / wb
    C += sum(w[i] * (Gam[i] - Gbar).T @ (Gam[i] - Gbar) for i in tb)
    C += wb * Gbar.T @ (np.eye(9) - al * wb * np.linalg.inv(H[sb])) @ Gbar
    assert np.abs(C - C_ref).max() <= 1e-12 * np.abs(C_ref).max()
