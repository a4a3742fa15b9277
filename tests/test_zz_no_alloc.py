"""Allocation-free coupling solve (emu_acap_solve_noalloc) against the solver.

Some callers cannot allocate device memory. For them the library offers
one entry point whose scratch lives in a fixed array inside the library. This
test checks it through the C ABI: after a converged FP64 solve, the positions
the solver reports are q*(F) for its final F (Eq. 4), so solving q*(F) from
that F with the allocation-free call must give the same positions. Two
calls in a row must agree: the shared array keeps the previous call's
contents, and a call must not depend on them.

This file is collected last on purpose (see its name).
"""
import numpy as np
import pytest

from emu_inputs import box_beam, muscle_tendon_unit

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


@pytest.mark.parametrize("mesh_fn", [lambda: box_beam(2, 2, 6, activation=0.5),
                                     lambda: muscle_tendon_unit(4, 4, 14, h=0.01, radius_cells=1.9, frames=1,
                                                                a_max=0.6)])
def test_noalloc_coupling_solve_matches_solver_positions(emu, mesh_fn):
    import torch

    mesh = mesh_fn()
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-10))
    s.set_activation(mesh.activations[0])
    s.solve()
    q_ref = s.positions()
    _, _, F = s.element_state()
    dev = torch.device("cuda:0")
    tF = torch.tensor(F.reshape(-1, 9), dtype=torch.float64, device=dev)
    diag = float(np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0)))
    outs = []
    for _ in range(2):
        tq = torch.full((mesh.n_verts, 3), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        rc = s.acap_solve_noalloc(tF.data_ptr(), tq.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == 0, rc
        q = tq.cpu().numpy()
        assert np.all(np.isfinite(q))
        err = np.abs(q - q_ref).max() / diag
        assert err <= 1e-9, err
        outs.append(q)
    np.testing.assert_array_equal(outs[0], outs[1])
    s.close()


def test_noalloc_coupling_solve_on_a_mixed_precision_handle(emu):
    # a mixed handle keeps an FP64 coupling operator built from its FP32
    # D_m^-1 and weights; the allocation-free call solves Eq. 4 with that
    # operator for the handle's final F, which must give the positions the
    # mixed solve reports (both coupling solves converged to 1e-10)
    import torch

    mesh = box_beam(4, 4, 16, activation=0.5)
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-6, pcg_tol=1e-10, precision=emu.PRECISION_MIXED))
    s.set_activation(0.5)
    st = s.solve()
    assert st.status == 0
    q_ref = s.positions()
    _, _, F = s.element_state()
    dev = torch.device("cuda:0")
    tF = torch.tensor(F.reshape(-1, 9), dtype=torch.float64, device=dev)
    diag = float(np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0)))
    outs = []
    for _ in range(2):
        tq = torch.full((mesh.n_verts, 3), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        rc = s.acap_solve_noalloc(tF.data_ptr(), tq.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == 0, (rc, s.lib.emu_last_error())
        q = tq.cpu().numpy()
        err = np.abs(q - q_ref).max() / diag
        assert err <= 1e-8, err
        outs.append(q)
    np.testing.assert_array_equal(outs[0], outs[1])
    s.close()


def test_noalloc_rejects_a_mesh_larger_than_its_fixed_scratch(emu):
    # 401,920 tets need 96 bytes per tet + 144 per vertex: more than the
    # fixed 32 MiB array, so the call must refuse before touching memory
    import torch

    mesh = muscle_tendon_unit(frames=1)
    s = emu.Solver(mesh, emu.Params(precision=emu.PRECISION_MIXED))
    dev = torch.device("cuda:0")
    tF = torch.zeros((mesh.n_tets, 9), dtype=torch.float64, device=dev)
    tq = torch.zeros((mesh.n_verts, 3), dtype=torch.float64, device=dev)
    rc = s.acap_solve_noalloc(tF.data_ptr(), tq.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == -1  # EMU_ERR_INVALID_ARG
    assert b"32 MiB" in s.lib.emu_last_error()
    assert torch.count_nonzero(tq).item() == 0
    s.close()
