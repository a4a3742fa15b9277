"""The set-up autotuner of the coupling solves (emu_params.autotune).

It times candidate launch settings on the mesh's own matrix and keeps the
fastest: the local polynomial's degree of the mixed path's pipelined CG
and the rows per block of the FP64 CG. Checked here: the choice is one of
the candidates, it is reused for a second handle of the same mesh (a batch
stays bit-identical to its meshes alone), and a tuned solve still meets the
parity bounds against the FP64 oracle (1e-4 of the diagonal for the mixed
path at 1e-6, 1e-9 for the FP64 path at 1e-11).
"""
import numpy as np
import pytest

from emu_inputs import box_beam, muscle_tendon_unit
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


def test_default_settings_are_reported_untuned(emu):
    mesh = muscle_tendon_unit(6, 6, 20, h=0.01, radius_cells=2.6, frames=1)
    s = emu.Solver(mesh, emu.Params(precision=emu.PRECISION_MIXED))
    t = s.tuning()
    assert not t["tuned"] and t["cg_local_degree"] == 4 and t["cg64_rows_per_block"] == 128
    s.close()


def test_mixed_autotune_picks_a_candidate_and_keeps_parity(emu):
    mesh = muscle_tendon_unit(6, 6, 20, h=0.01, radius_cells=2.6, frames=1, a_max=0.6)
    a = mesh.activations[0]
    p = emu.Params(precision=emu.PRECISION_MIXED, tol_rel_residual=1e-6, autotune=1)
    s = emu.Solver(mesh, p)
    t = s.tuning()
    assert t["tuned"] and t["cg_local_degree"] in (2, 3, 4, 6, 8), t
    s.set_activation(a)
    st = s.solve()
    assert st.status == 0 and st.rel_residual <= 1e-6
    r = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0)).solve(a, tol=1e-10)
    assert np.abs(s.positions() - r.q).max() / _diag(mesh) <= 1e-4
    # a second handle of the same mesh reuses the choice and the result
    s2 = emu.Solver(mesh, p)
    assert s2.tuning() == t
    s2.set_activation(a)
    s2.solve()
    np.testing.assert_array_equal(s2.positions(), s.positions())
    s.close()
    s2.close()


def test_fp64_autotune_picks_rows_per_block_and_keeps_parity(emu):
    mesh = box_beam(3, 5, 7, activation=0.8)
    p = emu.Params(tol_rel_residual=1e-11, autotune=1)
    s = emu.Solver(mesh, p)
    t = s.tuning()
    assert t["tuned"] and t["cg64_rows_per_block"] in (64, 128, 256), t
    s.set_activation(0.8)
    st = s.solve()
    assert st.status == 0 and st.rel_residual <= 1e-11
    r = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0)).solve(0.8, tol=1e-11)
    assert np.abs(s.positions() - r.q).max() / _diag(mesh) <= 1e-9
    s.close()


def test_autotune_flag_is_validated(emu):
    with pytest.raises(emu.EmuError) as e:
        emu.Solver(box_beam(1, 1, 2), emu.Params(autotune=2))
    assert e.value.code == -1
