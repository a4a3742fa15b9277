"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself:
finite differences, closed forms, a second independent solver, symmetry or
a brute-force root. A dropped term, a wrong sign or index, or a transposed
operand anywhere in the oracle fails at least one of them.
"""
import dataclasses

import numpy as np
import pytest
import scipy.optimize as so

from emu_inputs import box_beam, muscle_tendon_unit
from oracle import (EmuOracle, OracleParams, psi, dpsi, d2psi, delta_psi, element_terms_s,
                    stretch_from_s, s_from_stretch, sym_basis, lame, rest_geometry, build_G,
                    INVERTED_ENERGY)
from oracle.vertex_space import envelope_solve, fem_solve

RNG = np.random.default_rng(20060882)


def _rand_F(n, scale=0.25):
    """Random rotation times random SPD stretch, det > 0."""
    A = RNG.normal(size=(n, 3, 3))
    Qr, _ = np.linalg.qr(A)
    Qr *= np.sign(np.linalg.det(Qr))[:, None, None]
    B = RNG.normal(size=(n, 3, 3)) * scale
    S = np.eye(3) + 0.5 * (B + np.swapaxes(B, 1, 2))
    return Qr @ S


def _mat(n):
    mu, lam = lame(np.full(n, 6e5), np.full(n, 0.45))
    ka = RNG.uniform(0.0, 1.0, size=n) * mu
    u = RNG.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return mu, lam, ka, u


# ---------------------------------------------------------------- p2: FD --
def test_first_piola_matches_central_differences():
    n = 16
    F = _rand_F(n)
    mu, lam, ka, u = _mat(n)
    P = dpsi(F, mu, lam, ka, u)
    h = 1e-6
    for r in range(3):
        for c in range(3):
            E = np.zeros((3, 3))
            E[r, c] = h
            fd = (psi(F + E, mu, lam, ka, u) - psi(F - E, mu, lam, ka, u)) / (2 * h)
            np.testing.assert_allclose(P[:, r, c], fd, rtol=1e-6, atol=1e-7 * mu[0])


def test_hessian_matches_central_differences():
    n = 16
    F = _rand_F(n)
    mu, lam, ka, u = _mat(n)
    H = d2psi(F, mu, lam, ka, u)
    h = 1e-6
    for k in range(9):
        E = np.zeros(9)
        E[k] = h
        E = E.reshape(3, 3)
        fd = (dpsi(F + E, mu, lam, ka, u) - dpsi(F - E, mu, lam, ka, u)).reshape(n, 9) / (2 * h)
        np.testing.assert_allclose(H[:, :, k], fd, rtol=1e-6, atol=1e-6 * mu[0])
    np.testing.assert_allclose(H, np.swapaxes(H, 1, 2), rtol=1e-12, atol=1e-9 * mu[0])


def test_rest_state_has_zero_elastic_stress_and_fiber_stress_2kauu():
    # Neo-Hookean: P(I) = 0. Fiber: d/dF (ka u^T F^T F u) = 2 ka F u u^T.
    n = 8
    mu, lam, ka, u = _mat(n)
    I = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    P = dpsi(I, mu, lam, ka, u)
    np.testing.assert_allclose(P, 2 * ka[:, None, None] * np.einsum("ni,nj->nij", u, u), atol=1e-9)
    np.testing.assert_allclose(psi(I, mu, lam, np.zeros(n), u), 0.0, atol=1e-12)


def test_inverted_element_gets_huge_energy():
    F = np.diag([1.0, 1.0, -1.0])[None]
    mu, lam, ka, u = _mat(1)
    assert psi(F, mu, lam, ka, u)[0] == INVERTED_ENERGY


def test_stretch_form_gradient_and_hessian_match_fd():
    n = 12
    mu, lam, ka, u = _mat(n)
    V = RNG.uniform(1e-7, 2e-7, size=n)
    B = RNG.normal(size=(n, 3, 3)) * 0.2
    S = np.eye(3) + 0.5 * (B + np.swapaxes(B, 1, 2))
    s = s_from_stretch(S)
    val, g, H = element_terms_s(s, mu, lam, ka, u, V)
    np.testing.assert_allclose(stretch_from_s(s), S, atol=1e-15)
    E = sym_basis()
    np.testing.assert_allclose(np.einsum("kij,lij->kl", E, E), np.eye(6), atol=1e-15)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fp, gp, _ = element_terms_s(s + e, mu, lam, ka, u, V)
        fm, gm, _ = element_terms_s(s - e, mu, lam, ka, u, V)
        np.testing.assert_allclose(g[:, k], (fp - fm) / (2 * h), rtol=1e-6, atol=1e-7 * np.max(V * mu))
        np.testing.assert_allclose(H[:, :, k], (gp - gm) / (2 * h), rtol=1e-6, atol=1e-6 * np.max(V * mu))


def test_delta_psi_matches_difference_and_derivative():
    n = 10
    F = _rand_F(n, 0.15)
    d = RNG.normal(size=(n, 3, 3)) * 0.05
    mu, lam, ka, u = _mat(n)
    for sigma in [1.0, 0.3]:
        ref = psi(F + sigma * d, mu, lam, ka, u) - psi(F, mu, lam, ka, u)
        np.testing.assert_allclose(delta_psi(F, d, sigma, mu, lam, ka, u), ref, rtol=1e-9, atol=1e-9)
    # tiny step: ratio tends to <P, d> (no cancellation loss)
    s = 1e-12
    lin = np.einsum("nij,nij->n", dpsi(F, mu, lam, ka, u), d)
    np.testing.assert_allclose(delta_psi(F, d, s, mu, lam, ka, u) / s, lin, rtol=1e-6)
    # inversion along the step is rejected
    bad = delta_psi(np.eye(3)[None], -2.0 * np.eye(3)[None], 1.0, mu[:1], lam[:1], ka[:1], u[:1])
    assert np.isinf(bad[0])


# ------------------------------------------------------- geometry / G ----
def test_G_reproduces_affine_fields_and_volumes():
    mesh = box_beam(2, 2, 3, h=0.01)
    Dm, Dinv, V = rest_geometry(mesh.rest_pos, mesh.tets)
    np.testing.assert_allclose(V.sum(), 2 * 2 * 3 * 1e-6, rtol=1e-12)
    G = build_G(mesh.n_verts, mesh.tets, Dinv)
    A = np.array([[1.1, 0.2, -0.1], [0.05, 0.9, 0.3], [0.0, -0.2, 1.2]])
    q = mesh.rest_pos @ A.T + np.array([0.3, -0.1, 0.2])
    F = (G @ q.ravel()).reshape(-1, 3, 3)
    np.testing.assert_allclose(F, np.broadcast_to(A, F.shape), atol=1e-12)
    # interior vertices: sum over incident tets of V_i grad N_v = 0
    o = EmuOracle(box_beam(3, 3, 3, h=0.01), OracleParams(weight_mode=0))
    GtV = o.G.T @ np.repeat(o.V, 9)
    Qv = o.Q
    interior = np.all((Qv > 1e-9) & (Qv < 0.03 - 1e-9), axis=1)
    assert interior.sum() == 8


# ------------------------------------------------------------ p1 rest ----
def test_rest_state_is_a_fixed_point_with_zero_iterations():
    mesh = box_beam(2, 2, 4)
    o = EmuOracle(mesh)
    r = o.solve(0.0)
    assert r.iterations == 0
    np.testing.assert_allclose(r.q, mesh.rest_pos, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r.F, np.broadcast_to(np.eye(3), r.F.shape), atol=0)
    assert abs(r.energy) < 1e-25


# ---------------------------------------------------- p2b global grad ----
def test_global_gradient_includes_cancelled_term_correctly():
    mesh = box_beam(1, 1, 2)
    o = EmuOracle(mesh, OracleParams(alpha_rel=2.0))
    a = np.full(o.m, 0.7)
    F = _rand_F(o.m, 0.1)
    q = o.acap_solve(F)
    g = o.gradient(F, q, a)
    h = 1e-7
    fd = np.zeros_like(g)
    for i in range(o.m):
        for r in range(3):
            for c in range(3):
                E = np.zeros_like(F)
                E[i, r, c] = h
                ep = o.energy(F + E, o.acap_solve(F + E), a)
                em = o.energy(F - E, o.acap_solve(F - E), a)
                fd[i, r, c] = (ep - em) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


# -------------------------------------------------- p3 Woodbury ----------
def test_woodbury_direction_equals_dense_lowrank_solve():
    mesh = box_beam(1, 1, 3)
    o = EmuOracle(mesh, OracleParams(k_modes=12))
    a = np.full(o.m, 0.5)
    F = _rand_F(o.m, 0.1)
    q = o.acap_solve(F)
    g = o.gradient(F, q, a).reshape(-1)
    H = o.hessian_blocks(F, a)
    d = o.woodbury_direction(H, g)
    Hd = np.zeros((9 * o.m, 9 * o.m))
    for i in range(o.m):
        Hd[9 * i:9 * i + 9, 9 * i:9 * i + 9] = H[i]
    Happrox = Hd - o.alpha * o.B.T @ np.diag(1.0 / o.Lam) @ o.B
    d_ref = -np.linalg.solve(Happrox, g)
    np.testing.assert_allclose(d, d_ref, rtol=1e-9, atol=1e-12 * np.abs(d_ref).max())
    assert float(g @ d) < 0.0
    assert np.all(np.linalg.eigvalsh(0.5 * (Happrox + Happrox.T)) > 0)


def test_full_rank_modes_give_the_exact_hessian_step():
    mesh = box_beam(1, 1, 2)
    o = EmuOracle(mesh, OracleParams(k_modes=10**6))
    assert o.k == o.free_dofs.size
    a = np.full(o.m, 0.5)
    F = _rand_F(o.m, 0.05)
    q = o.acap_solve(F)
    g = o.gradient(F, q, a).reshape(-1)
    H = o.hessian_blocks(F, a)
    d = o.woodbury_direction(H, g)
    # Eq. 8 with the exact dense ACAP term alpha (W - W G K^-1 G^T W)
    W = np.diag(o.w9)
    Gf = o.G_f.toarray()
    acap = o.alpha * (W - W @ Gf @ np.linalg.solve(o.K.toarray(), Gf.T @ W))
    Hd = np.zeros((9 * o.m, 9 * o.m))
    for i in range(o.m):
        Hd[9 * i:9 * i + 9, 9 * i:9 * i + 9] = H[i] - o.alpha * o.w[i] * np.eye(9)
    d_ref = -np.linalg.solve(Hd + acap, g)
    np.testing.assert_allclose(d, d_ref, rtol=1e-7, atol=1e-9 * np.abs(d_ref).max())


# --------------------------------- p4 vertex-space (envelope) Newton -----
@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (2, 2, 6)])
def test_emu_equals_vertex_space_newton_of_the_eliminated_energy(dims):
    mesh = box_beam(*dims, activation=0.5)
    o = EmuOracle(mesh, OracleParams(alpha_rel=1.0))
    r = o.solve(0.5, tol=1e-12)
    q_env = envelope_solve(o, 0.5, tol=1e-13)
    diag = np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0))
    assert np.abs(r.q - q_env).max() / diag < 1e-10
    assert np.abs(r.q - mesh.rest_pos).max() / diag > 1e-3  # it actually moved


# ------------------------------------------------- p5 alpha -> infinity ---
def test_alpha_to_infinity_approaches_fem_at_first_order():
    mesh = box_beam(1, 1, 3, activation=0.4)
    errs = []
    alphas = [1e2, 1e3, 1e4]
    q_fem = None
    for ar in alphas:
        o = EmuOracle(mesh, OracleParams(alpha_rel=ar, k_modes=10**6))
        if q_fem is None:
            q_fem = fem_solve(o, 0.4)
        r = o.solve(0.4, tol=1e-11)  # FP64 floor is near 1e-12 at alpha = 1e4 mu
        errs.append(np.abs(r.q - q_fem).max())
    slopes = np.diff(np.log(errs)) / np.diff(np.log(alphas))
    assert np.all(slopes < -0.9) and np.all(slopes > -1.1), (errs, slopes)


# --------------------------------------------------- p6 affine patch -----
def test_affine_patch_reproduces_uniform_deformation():
    mesh = box_beam(3, 3, 3, h=0.01, activation=0.3)
    Q = mesh.rest_pos
    L = 0.03
    bnd = np.nonzero(np.any((Q < 1e-12) | (Q > L - 1e-12), axis=1))[0].astype(np.int32)
    A = np.array([[1.05, 0.08, 0.0], [-0.03, 0.97, 0.05], [0.02, 0.0, 1.02]])
    b = np.array([0.001, -0.002, 0.003])
    mesh.fixed_verts = bnd
    mesh.fixed_pos = Q[bnd] @ A.T + b
    o = EmuOracle(mesh, OracleParams(weight_mode=0, alpha_rel=1.0))
    r = o.solve(0.3, tol=1e-13)
    np.testing.assert_allclose(r.q, Q @ A.T + b, atol=1e-13 * L)
    # every F_i solves V Psi'(F) + alpha V (F - A) = 0 (single-tet root)
    mu, lam = o.mu[0], o.lam[0]
    ka, u = o.kappa * 0.3, o.u[0]

    def res(x):
        F = x.reshape(1, 3, 3)
        return (dpsi(F, np.array([mu]), np.array([lam]), np.array([ka]), u[None])[0]
                + o.alpha * (F[0] - A)).ravel() / mu

    Fstar = so.fsolve(res, A.ravel(), xtol=1e-15).reshape(3, 3)
    np.testing.assert_allclose(r.F, np.broadcast_to(Fstar, r.F.shape), atol=1e-11)


# ------------------------------ p7 stress-free uniaxial fiber contraction --
def test_stress_free_fiber_contraction_is_reproduced_exactly():
    # Along u = e_z the activated material is stress free at
    # F* = diag(lt, lt, lf) with
    #   mu (lt^2 - 1) + lam ln J = 0,  mu (lf^2 - 1) + lam ln J + 2 ka lf^2 = 0.
    # Prescribing the boundary to F* Q makes F_i = F* and q = F* Q the
    # equilibrium: V Psi'(F*) = 0 and E_C = 0.
    mesh = box_beam(3, 3, 3, h=0.01, activation=0.5)
    o0 = EmuOracle(mesh)
    mu, lam, ka = o0.mu[0], o0.lam[0], o0.kappa * 0.5

    def eqs(x):
        lt, lf = x
        lnJ = np.log(lt * lt * lf)
        return [mu * (lt * lt - 1) + lam * lnJ, mu * (lf * lf - 1) + lam * lnJ + 2 * ka * lf * lf]

    lt, lf = so.fsolve(eqs, [1.1, 0.8], xtol=1e-15)
    assert lf < 1.0 < lt
    A = np.diag([lt, lt, lf])
    Q = mesh.rest_pos
    bnd = np.nonzero(np.any((Q < 1e-12) | (Q > 0.03 - 1e-12), axis=1))[0].astype(np.int32)
    mesh.fixed_verts = bnd
    mesh.fixed_pos = Q[bnd] @ A.T
    o = EmuOracle(mesh)
    r = o.solve(0.5, tol=1e-13)
    np.testing.assert_allclose(r.F, np.broadcast_to(A, r.F.shape), atol=1e-11)
    np.testing.assert_allclose(r.q, Q @ A.T, atol=1e-13)


# -------------------------------------------------- p9 symmetry ----------
def test_box_beam_solution_is_symmetric_under_x_y_swap():
    mesh = box_beam(2, 2, 6, activation=0.5)
    o = EmuOracle(mesh)
    r = o.solve(0.5, tol=1e-12)
    Q = mesh.rest_pos
    key = {tuple(np.round(p / 0.01).astype(int)): i for i, p in enumerate(Q)}
    perm = np.array([key[(int(round(p[1] / 0.01)), int(round(p[0] / 0.01)), int(round(p[2] / 0.01)))] for p in Q])
    q = r.q
    np.testing.assert_allclose(q[perm][:, [1, 0, 2]], q, atol=1e-12)


# ----------------------------------------- convergence / line search -----
def test_energy_decreases_monotonically_and_converges():
    mesh = muscle_tendon_unit(3, 3, 10, h=0.01, radius_cells=1.6, frames=1)
    o = EmuOracle(mesh, OracleParams(weight_mode=0))
    a = mesh.activations[0]
    F = np.broadcast_to(np.eye(3), (o.m, 3, 3)).copy()
    E_prev = o.energy(F, o.acap_solve(F), a)
    for it in range(15):
        r = o.solve(a, F0=F, max_newton=1, tol=0.0)
        E = o.energy(r.F, o.acap_solve(r.F), a)
        assert E <= E_prev + 1e-12 * abs(E_prev)
        E_prev, F = E, r.F
    r = o.solve(a, F0=F, tol=1e-8)
    assert r.rel_residual <= 1e-8


def _diag(mesh):
    return float(np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0)))


def test_converged_result_does_not_depend_on_the_mode_basis():
    # Eqs. 9-12 only shape the direction; the gradient is exact, so the
    # stationary point is the same for any number of modes
    mesh = box_beam(2, 2, 6, activation=0.5)
    qs = [EmuOracle(mesh, OracleParams(weight_mode=0, k_modes=k)).solve(0.5, tol=1e-11).q for k in (6, 24, 48)]
    for q in qs[1:]:
        assert np.abs(q - qs[0]).max() <= 1e-9 * _diag(mesh)


def test_converged_result_does_not_depend_on_the_line_search_start():
    # Algorithm 1's first trial step (10) or the Newton step (1): same point
    mesh = box_beam(2, 2, 6, activation=0.5)
    q1 = EmuOracle(mesh, OracleParams(weight_mode=0, ls_sigma0=1.0)).solve(0.5, tol=1e-11).q
    q10 = EmuOracle(mesh, OracleParams(weight_mode=0, ls_sigma0=10.0)).solve(0.5, tol=1e-11).q
    assert np.abs(q10 - q1).max() <= 1e-9 * _diag(mesh)


def test_rigid_motion_of_the_rest_state_moves_the_solution_with_it():
    # Eq. 2 uses edge differences and Psi, the fiber term and the ACAP term
    # are invariant under a rotation of the reference frame: rotating and
    # translating the rest mesh, its fibers and its pins rotates and
    # translates the converged positions
    mesh = box_beam(2, 2, 5, activation=0.6)
    A = RNG.normal(size=(3, 3))
    R0, _ = np.linalg.qr(A)
    R0 *= np.sign(np.linalg.det(R0))
    t0 = np.array([0.3, -0.2, 0.1])
    moved = dataclasses.replace(mesh, rest_pos=mesh.rest_pos @ R0.T + t0, fiber_dir=mesh.fiber_dir @ R0.T)
    q = EmuOracle(mesh, OracleParams(weight_mode=0)).solve(0.6, tol=1e-11).q
    qm = EmuOracle(moved, OracleParams(weight_mode=0)).solve(0.6, tol=1e-11).q
    assert np.abs(qm - (q @ R0.T + t0)).max() <= 1e-9 * _diag(mesh)


def test_scaling_the_mesh_or_the_moduli_leaves_the_shape_unchanged():
    # E(F) is a sum of V_i times per-volume densities, with w_i = V_i, and
    # alpha and kappa are multiples of the smallest shear modulus: scaling
    # every length by s scales every term by s^3, and scaling every Young's
    # modulus scales every term alike, so the stationary F is unchanged and
    # the positions scale with the mesh
    mesh = box_beam(2, 2, 5, activation=0.6)
    q = EmuOracle(mesh, OracleParams(weight_mode=0)).solve(0.6, tol=1e-11).q
    big = dataclasses.replace(mesh, rest_pos=2.0 * mesh.rest_pos)
    qb = EmuOracle(big, OracleParams(weight_mode=0)).solve(0.6, tol=1e-11).q
    assert np.abs(qb - 2.0 * q).max() <= 1e-9 * _diag(big)
    stiff = dataclasses.replace(mesh, youngs=37.0 * mesh.youngs)
    qs = EmuOracle(stiff, OracleParams(weight_mode=0)).solve(0.6, tol=1e-11).q
    assert np.abs(qs - q).max() <= 1e-9 * _diag(mesh)


def test_small_activations_act_linearly():
    # around the rest state the response is linear in a: doubling a small
    # activation doubles the displacement up to O(a^2)
    mesh = box_beam(2, 2, 5)
    o = EmuOracle(mesh, OracleParams(weight_mode=0))
    u1 = o.solve(1e-4, tol=1e-10).q - mesh.rest_pos
    u2 = o.solve(2e-4, tol=1e-10).q - mesh.rest_pos
    assert np.abs(u2 - 2.0 * u1).max() <= 1e-3 * np.abs(u1).max()
    assert np.abs(u1).max() > 0.0


# ------------------------------------------------------- p15: materials --
def test_lame_parameters_hand_computed():
    # mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu)(1 - 2 nu)), worked by hand
    mu, lam = lame(np.array([6e5, 1e10, 1e8]), np.array([0.45, 0.3, 0.0]))
    np.testing.assert_allclose(mu, [600000.0 / 2.9, 1e10 / 2.6, 5e7], rtol=1e-15)
    np.testing.assert_allclose(lam, [270000.0 / 0.145, 3e9 / 0.52, 0.0], rtol=1e-15, atol=0.0)
    np.testing.assert_allclose(mu[0], 206896.55172413793, rtol=1e-15)
    np.testing.assert_allclose(lam[0], 1862068.9655172413, rtol=1e-15)


@pytest.mark.parametrize("E,nu", [(6e5, 0.45), (1e10, 0.3), (1e8, 0.2)])
def test_small_strain_uniaxial_stress_recovers_youngs_modulus_and_poisson_ratio(E, nu):
    # The definitions of E and nu: under a small uniaxial stress the axial
    # stress over the axial strain is E, and the lateral strain over the
    # axial strain is -nu. The stress comes from the oracle's neo-Hookean
    # Piola stress with the oracle's Lame parameters (no fiber term), so a
    # wrong lame() or a wrong Psi' fails here.
    mu, lam = lame(E, nu)
    eps = 1e-7
    u = np.array([1.0, 0.0, 0.0])

    def lateral_stress(et):
        F = np.diag([1.0 + eps, 1.0 + et, 1.0 + et])
        return dpsi(F[None], np.array([mu]), np.array([lam]), np.zeros(1), u[None])[0][1, 1]

    et = so.brentq(lateral_stress, -eps, eps, xtol=1e-22, rtol=1e-15)
    F = np.diag([1.0 + eps, 1.0 + et, 1.0 + et])
    P = dpsi(F[None], np.array([mu]), np.array([lam]), np.zeros(1), u[None])[0]
    np.testing.assert_allclose(P[0, 0] / eps, E, rtol=1e-5)
    np.testing.assert_allclose(-et / eps, nu, rtol=1e-5)
