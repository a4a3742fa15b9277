"""GPU parity of the F-form iteration (Sec. 3.2.1, Eqs. 10-12: one free F per
tet, 9 x 9 blocks) against the FP64 oracle, through the C ABI.

Element level: V Psi(F), V P(F) and the 9 x 9 block with the definiteness
fix, against the oracle's psi, dpsi and d2psi, the isotropic part projected
by the oracle's psd_project (a numerical eigen-decomposition) and the fiber
part taken as it stands. Relative bounds 1e-12 (energy, stress) and 1e-10
of the block's largest entry (Hessian: the analytic eigen-system against
LAPACK's).

Solves: converged positions within 1e-9 of the rest bounding-box diagonal
with both sides at a relative residual of 1e-11 (the bound of the other
FP64 parity tests), on box beams, the two-material muscle-tendon unit,
warm-started frames and a gravity load; the final F within 1e-8.
"""
import dataclasses

import numpy as np
import pytest

from emu_inputs import box_beam, gravity_forces, muscle_tendon_unit
from oracle import EmuOracle, OracleParams, d2psi, dpsi, lame, psd_project, psi, stretch_from_s

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


def _gpu(emu, mesh, a, tol=1e-11, **kw):
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=tol, form=emu.FORM_F, **kw))
    s.set_activation(a)
    st = s.solve()
    return s, st


def _oracle(mesh, a, tol=1e-11):
    o = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0))
    return o.solve(a, tol=tol)


def _random_F(rng, n, spread):
    A = rng.normal(size=(n, 3, 3))
    Qr, _ = np.linalg.qr(A)
    Qr *= np.sign(np.linalg.det(Qr))[:, None, None]
    B = rng.normal(size=(n, 3, 3))
    Bs = 0.5 * (B + np.swapaxes(B, 1, 2))
    w, Vv = np.linalg.eigh(Bs)
    sig = np.exp(spread * np.tanh(w))  # stretches in [e^-spread, e^spread]
    S = np.einsum("nij,nj,nkj->nik", Vv, sig, Vv)
    return Qr @ S


# ----------------------------------------------------------- element level --
@pytest.mark.parametrize("spread", [0.05, 0.5])
def test_fform_terms_match_oracle(emu, spread):
    import torch

    rng = np.random.default_rng(17)
    n = 301  # several blocks and a ragged tail
    F = _random_F(rng, n, spread)
    mu, lam = lame(np.full(n, 6e5), np.full(n, 0.45))
    ka = rng.uniform(0, 1, n) * mu
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    V = rng.uniform(1e-7, 2e-7, n)
    prm = np.zeros((n, 8))
    prm[:, 0], prm[:, 1], prm[:, 2], prm[:, 3], prm[:, 4:7] = V, mu, lam, ka, u
    val = V * psi(F, mu, lam, ka, u)
    P = V[:, None, None] * dpsi(F, mu, lam, ka, u)
    H_iso = V[:, None, None] * d2psi(F, mu, lam, np.zeros(n), u)
    H_fib = V[:, None, None] * (d2psi(F, mu, lam, ka, u) - d2psi(F, mu, lam, np.zeros(n), u))
    H_ref = psd_project(H_iso) + H_fib
    dev = torch.device("cuda:0")
    tF = torch.tensor(F.reshape(n, 9), device=dev)
    tp = torch.tensor(prm, device=dev)
    tpsi = torch.empty(n, dtype=torch.float64, device=dev)
    tg = torch.empty((n, 9), dtype=torch.float64, device=dev)
    th = torch.empty((n, 81), dtype=torch.float64, device=dev)
    emu.eval_fform_terms(tF.data_ptr(), tp.data_ptr(), n, tpsi.data_ptr(), tg.data_ptr(), th.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    scale = np.abs(V * mu).max()
    np.testing.assert_allclose(tpsi.cpu().numpy(), val, rtol=1e-12, atol=1e-12 * scale)
    np.testing.assert_allclose(tg.cpu().numpy(), P.reshape(n, 9), rtol=1e-12, atol=1e-12 * scale)
    Hg = th.cpu().numpy().reshape(n, 9, 9)
    hmax = np.abs(H_ref).max(axis=(1, 2))
    assert np.all(np.abs(Hg - H_ref).max(axis=(1, 2)) <= 1e-10 * hmax)
    # positive semi-definite, and the projection only acts where the
    # isotropic Hessian is indefinite
    assert np.all(np.linalg.eigvalsh(Hg) >= -1e-12 * hmax[:, None])
    indefinite = np.linalg.eigvalsh(0.5 * (H_iso + np.swapaxes(H_iso, 1, 2))).min(axis=1) < 0
    exact = ~indefinite
    full = V[:, None, None] * d2psi(F, mu, lam, ka, u)
    assert np.all(np.abs(Hg[exact] - full[exact]).max(axis=(1, 2)) <= 1e-10 * hmax[exact])
    if spread >= 0.5:
        assert indefinite.sum() > n // 4  # the large stretches exercise the clamp


# ------------------------------------------------------------- full solves --
@pytest.mark.parametrize("dims,act", [((2, 2, 6), 0.5), ((3, 5, 7), 0.8)])
def test_fform_box_beam_matches_oracle(emu, dims, act):
    mesh = box_beam(*dims, activation=act)
    r = _oracle(mesh, act)
    s, st = _gpu(emu, mesh, act)
    assert st.status == 0 and st.rel_residual <= 1e-11, (st.status, st.rel_residual)
    err = np.abs(s.positions() - r.q).max() / _diag(mesh)
    assert err <= 1e-9, (err, st.newton_iters, r.iterations)
    R, sv, F = s.element_state()
    np.testing.assert_allclose(F, r.F, atol=1e-8)
    np.testing.assert_allclose(np.einsum("nji,njk->nik", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    np.testing.assert_allclose(R @ stretch_from_s(sv), F, atol=1e-12)
    s.close()


def test_fform_muscle_tendon_unit_matches_oracle_and_rs_form(emu):
    mesh = muscle_tendon_unit(4, 4, 14, h=0.01, radius_cells=1.9, frames=1, a_max=0.6)
    a = mesh.activations[0]
    r = _oracle(mesh, a)
    s, st = _gpu(emu, mesh, a)
    assert st.status == 0 and st.rel_residual <= 1e-11, (st.status, st.rel_residual)
    err = np.abs(s.positions() - r.q).max() / _diag(mesh)
    assert err <= 1e-9, (err, st.newton_iters, r.iterations)
    rs = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-11))
    rs.set_activation(a)
    st_rs = rs.solve()
    assert st_rs.status == 0
    assert np.abs(s.positions() - rs.positions()).max() / _diag(mesh) <= 1e-9
    s.close()
    rs.close()


def test_fform_warm_started_frames_match_oracle(emu):
    mesh = muscle_tendon_unit(3, 3, 10, h=0.01, radius_cells=1.6, frames=3, a_max=0.8)
    o = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0))
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-11, form=emu.FORM_F))
    F = None
    for f in range(mesh.activations.shape[0]):
        a = mesh.activations[f]
        r = o.solve(a, F0=F, tol=1e-11)
        F = r.F
        s.set_activation(a)
        st = s.solve()
        assert st.status == 0
        err = np.abs(s.positions() - r.q).max() / _diag(mesh)
        assert err <= 1e-9, (f, err)
    s.close()


def test_fform_with_gravity_matches_oracle(emu):
    base = box_beam(2, 2, 6, activation=0.5)
    mesh = dataclasses.replace(base, f_ext=gravity_forces(base, g=(0.0, -40.0, -20.0)))
    r = _oracle(mesh, 0.5)
    s, st = _gpu(emu, mesh, 0.5)
    assert st.status == 0 and st.rel_residual <= 1e-11
    q = s.positions()
    assert np.abs(q - mesh.rest_pos).max() > 1e-2 * _diag(mesh)
    assert np.abs(q - r.q).max() / _diag(mesh) <= 1e-9
    s.close()


def test_fform_state_round_trip_and_resume(emu):
    # set (R, s) -> F = R S; an interrupted solve resumed from its state ends
    # where an uninterrupted one does (to rounding: F = R S is recomposed)
    mesh = box_beam(2, 2, 6, activation=0.5)
    p = emu.Params(tol_rel_residual=1e-11, form=emu.FORM_F)
    full = emu.Solver(mesh, p)
    full.set_activation(0.5)
    st_full = full.solve()
    part = emu.Solver(mesh, dataclasses.replace(p, max_newton=5))
    part.set_activation(0.5)
    st = part.solve(raise_on_error=False)
    assert st.newton_iters == 5
    R, sv, F = part.element_state()
    q = part.positions()
    resumed = emu.Solver(mesh, p)
    resumed.set_activation(0.5)
    resumed.set_element_state(R=R, s=sv, q=q)
    _, _, F2 = resumed.element_state()
    np.testing.assert_allclose(F2, F, atol=1e-13)
    st2 = resumed.solve()
    assert st2.status == 0 and st_full.status == 0
    np.testing.assert_allclose(resumed.positions(), full.positions(), atol=1e-10 * _diag(mesh))
    for x in (full, part, resumed):
        x.close()


def test_fform_rest_state_takes_zero_iterations(emu):
    mesh = box_beam(2, 2, 4)
    s, st = _gpu(emu, mesh, 0.0)
    assert st.newton_iters == 0
    np.testing.assert_allclose(s.positions(), mesh.rest_pos, atol=1e-13)
    s.close()


def test_fform_rejects_mixed_precision_and_bones(emu):
    mesh = box_beam(2, 2, 4)
    with pytest.raises(emu.EmuError) as e:
        emu.Solver(mesh, emu.Params(form=emu.FORM_F, precision=emu.PRECISION_MIXED))
    assert e.value.code == -10
    with pytest.raises(emu.EmuError) as e:
        emu.Solver(mesh, emu.Params(form=2))
    assert e.value.code == -1
    from emu_inputs import arm_assembly

    arm = arm_assembly(bone_w=2, bone_len=4, r0=2.0, frames=1)
    with pytest.raises(emu.EmuError) as e:
        emu.Solver(arm, emu.Params(form=emu.FORM_F))
    assert e.value.code == -10
