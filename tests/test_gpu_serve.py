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


def test_requests_arriving_mid_flight_overlap_and_each_matches_its_solo_run(emu):
    # continuous batching: requests submitted while others are being solved
    # (and while others are being set up) are admitted and run concurrently;
    # each result is bit-identical to the same request served alone, and the
    # whole mix takes clearly less than the requests one after another
    p = emu.Params(tol_rel_residual=1e-6, precision=emu.PRECISION_MIXED)
    reqs = _requests()
    srv = emu.Server(64 << 30, p)
    try:
        solo_q, solo_s = [], []
        for k, (mesh, acts) in enumerate(reqs):
            t0 = time.time()
            srv.submit(mesh, acts, 1000 + k)
            q, st = _wait(srv, [1000 + k])[1000 + k]
            solo_s.append(time.time() - t0)
            assert st.status == 0
            solo_q.append(q)
        t0 = time.time()
        srv.submit(reqs[3][0], reqs[3][1], 3)  # the largest first
        srv.submit(reqs[1][0], reqs[1][1], 1)
        time.sleep(0.05)  # the rest arrive while those two are in flight
        for k in (0, 2, 4):
            srv.submit(reqs[k][0], reqs[k][1], k)
        res = _wait(srv, list(range(len(reqs))))
        makespan = time.time() - t0
        for k in range(len(reqs)):
            q, st = res[k]
            assert st.status == 0 and st.frames_done == reqs[k][1].shape[0]
            assert np.array_equal(q, solo_q[k]), k
        assert makespan < 0.8 * sum(solo_s), (makespan, solo_s)
    finally:
        srv.close()


def test_a_request_with_bones_and_a_hinge_is_served_like_a_plain_solve(emu):
    from emu_inputs import arm_assembly

    arm = arm_assembly(bone_w=2, bone_len=4, r0=2.0, frames=4)
    p = emu.Params(tol_rel_residual=1e-6, precision=emu.PRECISION_MIXED)
    s = emu.Solver(arm, p)
    ref = []
    for f in (1, 2):
        s.set_activation(arm.activations[f])
        assert s.solve().status == 0
        ref.append(s.positions())
    s.close()
    srv = emu.Server(16 << 30, p)
    try:
        srv.submit(arm, arm.activations[1:3], 7)
        q, st = _wait(srv, [7])[7]
        assert st.status == 0 and st.frames_done == 2
        assert np.array_equal(q, np.stack(ref))
    finally:
        srv.close()
