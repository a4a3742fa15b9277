"""Batching (emu_batch_solve): independent meshes of uneven size solved
together, each on its own stream.

Every kernel of a solve is deterministic (fixed reduction orders, no
floating-point atomics) and a handle's work never reads another handle's
memory, so each mesh's result in the batch must be bit-identical to its
result solved alone; the FP64 path is also held to the oracle.
"""
import numpy as np
import pytest

from emu_inputs import batch_set, box_beam
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


def _solvers(emu, meshes, acts, params):
    import torch

    out = []
    for mesh, a in zip(meshes, acts):
        stream = torch.cuda.Stream()
        s = emu.Solver(mesh, params, stream=stream.cuda_stream)
        s.torch_stream = stream  # the stream must outlive the handle
        s.set_activation(a)
        out.append(s)
    return out


def test_batch_equals_each_mesh_alone_mixed(emu):
    # uneven sizes (log-uniform, as the 256-mesh batch), two frames each
    meshes = batch_set(count=7, seed=3, t_min=150.0, t_max=4000.0)
    acts = [np.full(m.tets.shape[0], float(m.activations[0][0])) for m in meshes]
    p = emu.Params(tol_rel_residual=1e-6, precision=emu.PRECISION_MIXED)
    alone = _solvers(emu, meshes, acts, p)
    ref_q, ref_it = [], []
    for s in alone:
        st = s.solve()
        ref_q.append(s.positions())
        ref_it.append(st.newton_iters)
    batch = _solvers(emu, meshes, acts, p)
    stats = emu.batch_solve(batch)
    for k, (s, st) in enumerate(zip(batch, stats)):
        assert st.status == 0 and st.rel_residual <= 1e-6
        assert st.newton_iters == ref_it[k]
        assert np.array_equal(s.positions(), ref_q[k]), k
    # a second frame from the resident (warm-started) states
    for s, a in zip(alone, acts):
        s.set_activation(0.5 * a)
        s.solve()
    for s, a in zip(batch, acts):
        s.set_activation(0.5 * a)
    emu.batch_solve(batch)
    for s_a, s_b in zip(alone, batch):
        assert np.array_equal(s_a.positions(), s_b.positions())


def test_batch_fp64_matches_oracle(emu):
    meshes = [box_beam(2, 2, 6, activation=0.5), box_beam(3, 3, 5, activation=0.8), box_beam(2, 3, 4, activation=0.3)]
    acts = [m.activations[0] for m in meshes]
    batch = _solvers(emu, meshes, acts, emu.Params(tol_rel_residual=1e-11))
    stats = emu.batch_solve(batch)
    for mesh, a, s, st in zip(meshes, acts, batch, stats):
        assert st.status == 0 and st.rel_residual <= 1e-11
        r = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0)).solve(a, tol=1e-11)
        err = np.abs(s.positions() - r.q).max() / _diag(mesh)
        assert err <= 1e-9, err


def test_batch_rejects_a_repeated_handle(emu):
    m = box_beam(2, 2, 3, activation=0.2)
    s = emu.Solver(m, emu.Params())
    s.set_activation(m.activations[0])
    with pytest.raises(emu.EmuError):
        emu.batch_solve([s, s])
