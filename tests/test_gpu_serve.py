"""Serving (emu_server_*): continuous batching under a device-memory budget.

A request's result must not depend on what else is in flight: every kernel
is deterministic and reads only its own handle's memory, so a request
solved alone, in a mix of concurrent requests, and through a plain Solver
must give bit-identical positions for every frame.
"""
import time

import numpy as np
import pytest

from emu_inputs import box_beam, mtu_for_tet_count

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


def _ramp(mesh, frames, a_max):
    a = mesh.activations[0] if len(mesh.activations) else np.ones(mesh.tets.shape[0])
    muscle = (np.asarray(a) > 0).astype(np.float64)
    return np.stack([muscle * a_max * (f + 1) / frames for f in range(frames)])


def _wait(srv, ids, timeout_s=300.0):
    left, t0, out = set(ids), time.time(), {}
    while left:
        for i in srv.poll():
            out[i] = srv.result(i)
            left.discard(i)
        assert time.time() - t0 < timeout_s, f"requests {sorted(left)} did not finish"
        time.sleep(0.002)
    return out


def _requests():
    # uneven sizes: muscle-tendon units of about 1k to 12k tets, 1 to 4 frames
    specs = [(1000, 0.05, 3, 0.7), (6000, 0.15, 2, 0.4), (2500, 0.1, 4, 0.9), (12000, 0.0, 1, 0.5),
             (1500, 0.2, 3, 0.3)]
    out = []
    for k, (t, tf, fr, am) in enumerate(specs):
        mesh = mtu_for_tet_count(t, tendon_frac=tf, seed=11 + k)
        out.append((mesh, _ramp(mesh, fr, am)))
    return out


def test_request_result_is_the_same_alone_in_the_mix_and_through_a_solver(emu):
    p = emu.Params(tol_rel_residual=1e-6, precision=emu.PRECISION_MIXED)
    reqs = _requests()
    probe_mesh, probe_acts = reqs[2]
    # 1. through a plain Solver, frame by frame
    s = emu.Solver(probe_mesh, p)
    ref = []
    for a in probe_acts:
        s.set_activation(a)
        s.solve()
        ref.append(s.positions())
    ref = np.stack(ref)
    s.close()
    srv = emu.Server(64 << 30, p)
    try:
        # 2. alone
        srv.submit(probe_mesh, probe_acts, 100)
        alone_q, alone_st = _wait(srv, [100])[100]
        assert alone_st.status == 0 and alone_st.frames_done == len(probe_acts)
        assert np.array_equal(alone_q, ref)
        # 3. in a mix submitted at once
        for k, (mesh, acts) in enumerate(reqs):
            srv.submit(mesh, acts, k)
        res = _wait(srv, list(range(len(reqs))))
        for k, (mesh, acts) in enumerate(reqs):
            q, st = res[k]
            assert st.status == 0 and st.frames_done == acts.shape[0], (k, st.status)
            assert st.rel_residual <= 1e-6
        assert np.array_equal(res[2][0], ref)
    finally:
        srv.close()


def test_admission_waits_for_memory_and_rejects_a_mesh_over_budget(emu):
    p = emu.Params(tol_rel_residual=1e-6, precision=emu.PRECISION_MIXED)
    mesh = mtu_for_tet_count(3000, tendon_frac=0.1, seed=5)
    need = emu.required_bytes(mesh, p)
    # room for one request at a time: the second waits for the first's memory
    srv = emu.Server(int(1.5 * need), p)
    try:
        acts = _ramp(mesh, 2, 0.6)
        srv.submit(mesh, acts, 1)
        srv.submit(mesh, acts, 2)
        res = _wait(srv, [1, 2])
        (q1, s1), (q2, s2) = res[1], res[2]
        assert s1.status == 0 and s2.status == 0
        assert np.array_equal(q1, q2)  # same mesh and activations, solved one after the other
        first, second = (s1, s2) if s1.queue_ms <= s2.queue_ms else (s2, s1)
        # the second was admitted only after the first finished
        assert second.queue_ms >= first.queue_ms + first.setup_ms + first.solve_ms - 1.0
        big = box_beam(8, 8, 40)
        with pytest.raises(emu.EmuError):
            srv.submit(big, np.full((1, big.tets.shape[0]), 0.5), 3)
    finally:
        srv.close()
