"""Full size: the 401,920-tet muscle-tendon unit in the configuration the
benchmark times (mixed precision, a stream of its own, PyTorch's caching
allocator, warm-started ramp frames). The oracle's solver cannot run at
this size, so the oracle checks, in FP64 and with its own exact operator
G (Eq. 2), properties that hold at any size at the GPU's result (F = R S per
tet, q):

  * Eq. 4: q solves the coupling problem for F: the free-row residual
    G_f^T W (F - G q) is small against G_f^T W (F - I);
  * Eqs. 6-7: the oracle's gradient at (F, q), relative to its gradient at
    the unloaded state (F = I, q = Q = q*(I)), meets the solver's tolerance
    (up to the FP32 rounding of the mixed path's D_m^-1, V and w);
  * every rotation is orthonormal with det +1 and every stretch is SPD.
"""
import numpy as np
import pytest

from emu_inputs import muscle_tendon_unit
from oracle import EmuOracle, OracleParams, stretch_from_s

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


def test_muscle_tendon_unit_401920_tets_meets_eq4_and_the_tolerance(emu):
    import torch

    mesh = muscle_tendon_unit()  # 32 x 32 x 128, r = 12.9 h: 401,920 tets
    assert mesh.n_tets == 401920
    stream = torch.cuda.Stream()
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-6, precision=emu.PRECISION_MIXED),
                   stream=stream.cuda_stream, allocator=emu.TorchAllocator(torch.cuda.current_device()))
    for f in (1, 2, 3):
        s.set_activation(mesh.activations[f])
        st = s.solve()
        assert st.status == 0 and st.rel_residual <= 1e-6
    q = s.positions().ravel()
    R, sv, F = s.element_state()
    s.close()

    o = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0), modes="none", factor=False)
    a = mesh.activations[3]
    eye = np.broadcast_to(np.eye(3), F.shape)
    r = o.G_f.T @ (o.w9 * (F.reshape(-1) - o.G @ q))
    scale = o.G_f.T @ (o.w9 * (F - eye).reshape(-1))
    assert np.linalg.norm(r) <= 1e-7 * np.linalg.norm(scale)  # measured 1.8e-9
    g0 = np.linalg.norm(o.gradient(eye.copy(), mesh.rest_pos.ravel(), a))
    g = np.linalg.norm(o.gradient(F, q, a))
    assert g <= 2e-6 * g0, g / g0  # measured 9.5e-7 (the GPU reports 9.5e-7)
    np.testing.assert_allclose(np.einsum("nji,njk->nik", R, R), eye, atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    assert np.linalg.eigvalsh(stretch_from_s(sv)).min() > 0.0
