"""Pins of the oracle's 9 x 9 Hessian (Sec. 3.2.1) against the closed-form
eigen-system of an isotropic energy in the singular-value frame of F, the
form the GPU's F-form uses for its definiteness fix (reading r25).

For the neo-Hookean density of Sec. 3.1 with F = U diag(sig) V^T and
c = mu - lam ln J, the Hessian in vec(F) has
  * for each pair i < j the eigenvectors (u_i v_j^T +- u_j v_i^T) / sqrt2
    with eigenvalues mu +- c / (sig_i sig_j);
  * on span{u_i v_i^T} the 3 x 3 block lam / (sig_i sig_j)
    + [i = j] (mu + c / sig_i^2).
The fiber term of d2psi is 2 ka I (x) u u^T: eigenvalues 0 (six times) and
2 ka (three times). A dropped term, a wrong sign or a transposed index in
d2psi moves one of these eigenvalues or eigenvectors.
"""
import numpy as np
import pytest

from oracle import d2psi, lame, psd_project


def _random_F(rng, n, spread):
    A = rng.normal(size=(n, 3, 3))
    Q, _ = np.linalg.qr(A)
    Q *= np.sign(np.linalg.det(Q))[:, None, None]
    B = rng.normal(size=(n, 3, 3))
    w, Vv = np.linalg.eigh(0.5 * (B + np.swapaxes(B, 1, 2)))
    S = np.einsum("nij,nj,nkj->nik", Vv, np.exp(spread * np.tanh(w)), Vv)
    return Q @ S


@pytest.mark.parametrize("spread", [0.05, 0.6])
def test_isotropic_hessian_has_the_analytic_eigensystem(spread):
    rng = np.random.default_rng(23)
    n = 40
    F = _random_F(rng, n, spread)
    mu, lam = lame(np.full(n, 6e5), np.full(n, 0.45))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    H = d2psi(F, mu, lam, np.zeros(n), u)
    for e in range(n):
        Uu, sig, Vt = np.linalg.svd(F[e])
        Vm = Vt.T
        c = mu[e] - lam[e] * np.log(np.linalg.det(F[e]))
        scale = np.abs(H[e]).max()
        expect = []
        for i, j in ((0, 1), (0, 2), (1, 2)):
            for sgn in (1.0, -1.0):
                val = mu[e] + sgn * c / (sig[i] * sig[j])
                z = (np.outer(Uu[:, i], Vm[:, j]) + sgn * np.outer(Uu[:, j], Vm[:, i])).ravel() / np.sqrt(2.0)
                assert np.abs(H[e] @ z - val * z).max() <= 1e-10 * scale
                expect.append(val)
        A3 = lam[e] / np.outer(sig, sig) + np.diag(mu[e] + c / sig**2)
        D = np.stack([np.outer(Uu[:, i], Vm[:, i]).ravel() for i in range(3)], axis=1)  # 9 x 3
        np.testing.assert_allclose(D.T @ H[e] @ D, A3, rtol=1e-10, atol=1e-10 * scale)
        expect.extend(np.linalg.eigvalsh(A3))
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(0.5 * (H[e] + H[e].T))), np.sort(expect),
                                   rtol=1e-10, atol=1e-10 * scale)


def test_projection_clamps_exactly_the_negative_analytic_eigenvalues():
    rng = np.random.default_rng(29)
    n = 30
    F = _random_F(rng, n, 0.6)
    mu, lam = lame(np.full(n, 6e5), np.full(n, 0.45))
    u = np.tile([0.0, 0.0, 1.0], (n, 1))
    H = d2psi(F, mu, lam, np.zeros(n), u)
    Hp = psd_project(H)
    for e in range(n):
        ev = np.linalg.eigvalsh(0.5 * (H[e] + H[e].T))
        evp = np.linalg.eigvalsh(Hp[e])
        scale = np.abs(H[e]).max()
        np.testing.assert_allclose(np.sort(evp), np.sort(np.maximum(ev, 0.0)), atol=1e-10 * scale)


def test_fiber_term_is_two_ka_identity_kron_uu():
    rng = np.random.default_rng(31)
    n = 12
    F = _random_F(rng, n, 0.3)
    mu, lam = lame(np.full(n, 6e5), np.full(n, 0.45))
    ka = rng.uniform(0.1, 1.0, n) * mu
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Hf = d2psi(F, mu, lam, ka, u) - d2psi(F, mu, lam, np.zeros(n), u)
    for e in range(n):
        ref = 2.0 * ka[e] * np.kron(np.eye(3), np.outer(u[e], u[e]))
        np.testing.assert_allclose(Hf[e], ref, atol=1e-9 * ka[e])
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Hf[e])), [0] * 6 + [2 * ka[e]] * 3,
                                   atol=1e-9 * ka[e])
