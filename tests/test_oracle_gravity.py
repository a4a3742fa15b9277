"""Pins of the oracle's external forces (Sec. 3.4, Eq. external-forces).

The oracle turns a constant per-vertex force f into the generalized force
nu on the deformation gradients and adds -<F, nu> to the energy. These tests
hold that against the definition of the work q*(F)^T f (computed with the
coupling solve, not with nu), against finite differences of the total
energy, against plain FEM with the same force as alpha grows (first order,
like p5), and against the direction and linearity of a small sag.
"""
import dataclasses

import numpy as np

from emu_inputs import box_beam, gravity_forces
from oracle import EmuOracle, OracleParams
from oracle.vertex_space import fem_solve

RNG = np.random.default_rng(34)


def _rand_F(n, scale=0.1):
    A = RNG.normal(size=(n, 3, 3))
    Qr, _ = np.linalg.qr(A)
    Qr *= np.sign(np.linalg.det(Qr))[:, None, None]
    B = RNG.normal(size=(n, 3, 3)) * scale
    return Qr @ (np.eye(3) + 0.5 * (B + np.swapaxes(B, 1, 2)))


def _loaded(mesh, g=(0.0, -300.0, -981.0), extra=True):
    f = gravity_forces(mesh, g=g)
    if extra:  # plus an arbitrary force field: nu must not rely on f being uniform
        f = f + RNG.normal(size=f.shape) * np.abs(f).max()
    return dataclasses.replace(mesh, f_ext=f)


def test_generalized_force_reproduces_the_work_of_the_force():
    mesh = _loaded(box_beam(2, 2, 4))
    o = EmuOracle(mesh, OracleParams(alpha_rel=3.0))
    f = mesh.f_ext.reshape(-1)
    for _ in range(3):
        F1, F2 = _rand_F(o.m), _rand_F(o.m)
        work = (o.acap_solve(F2) - o.acap_solve(F1)) @ f
        assert abs(np.sum((F2 - F1) * o.nu) - work) <= 1e-12 * abs(work) + 1e-18


def test_total_gradient_matches_central_differences_of_the_total_energy():
    mesh0 = box_beam(2, 2, 3, activation=0.4)
    mesh = _loaded(mesh0)
    o = EmuOracle(mesh, OracleParams(alpha_rel=2.0))
    o0 = EmuOracle(mesh0, OracleParams(alpha_rel=2.0))  # the same problem without the force
    f = mesh.f_ext.reshape(-1)
    a = np.full(o.m, 0.4)

    def total(F):  # Eq. 5 plus the work of f through q*(F), both from their definitions
        q = o0.acap_solve(F)
        return o0.energy(F, q, a) - q @ f

    F = _rand_F(o.m)
    g = o.gradient(F, o.acap_solve(F), a)
    for _ in range(4):
        D = RNG.normal(size=F.shape)
        h = 1e-6
        fd = (total(F + h * D) - total(F - h * D)) / (2 * h)
        assert abs(fd - np.sum(g * D)) <= 1e-6 * abs(fd) + 1e-9 * np.abs(g).max()
    # and the oracle's own energy differs from that total by a constant
    F2 = _rand_F(o.m)
    c1 = o.energy(F, o.acap_solve(F), a) - total(F)
    c2 = o.energy(F2, o.acap_solve(F2), a) - total(F2)
    assert abs(c1 - c2) <= 1e-10 * abs(total(F))


def test_alpha_to_infinity_with_the_force_approaches_fem_at_first_order():
    mesh = _loaded(box_beam(1, 1, 3, activation=0.4), g=(0.0, -2000.0, -4000.0), extra=False)
    errs = []
    alphas = [1e2, 1e3, 1e4]
    q_fem = None
    for ar in alphas:
        o = EmuOracle(mesh, OracleParams(alpha_rel=ar, k_modes=10**6))
        if q_fem is None:
            q_fem = fem_solve(o, 0.4)
        r = o.solve(0.4, tol=1e-11)
        errs.append(np.abs(r.q - q_fem).max())
    slopes = np.diff(np.log(errs)) / np.diff(np.log(alphas))
    assert np.all(slopes < -0.9) and np.all(slopes > -1.1), (errs, slopes)
    # the force matters at this size: FEM with and without it differ by far more
    o_nf = EmuOracle(dataclasses.replace(mesh, f_ext=None), OracleParams(alpha_rel=1e4, k_modes=10**6))
    assert np.abs(fem_solve(o_nf, 0.4) - q_fem).max() > 100 * errs[-1]


def test_a_small_load_sags_along_g_and_linearly():
    base = box_beam(2, 2, 6, activation=0.0)
    diag = np.linalg.norm(base.rest_pos.max(0) - base.rest_pos.min(0))
    g = np.array([0.0, -1.0, 0.0])
    disp = []
    for scale in (1.0, 2.0):
        mesh = dataclasses.replace(base, f_ext=gravity_forces(base, g=tuple(scale * g)))
        o = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0))
        r = o.solve(0.0, tol=1e-9)  # the normaliser |nu| is small: 1e-11 is below the energy's FP64 floor
        disp.append(r.q - base.rest_pos)
    u1, u2 = disp
    assert np.abs(u1).max() > 1e-6 * diag                     # it moved
    assert np.mean(u1 @ g) > 0 and np.mean(u2 @ g) > 0          # along g
    # a tip sag of 0.7 % of the beam: linear to a few parts in 1e3 (1.9e-3 measured)
    assert np.abs(u2 - 2.0 * u1).max() <= 5e-3 * np.abs(u2).max()
