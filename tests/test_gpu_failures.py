"""Failure detection and resume, on the GPU, in the forms that fault nothing.

* A bounded device wait that is made to run out (a grid barrier one block
  never reaches) returns EMU_ERR_TIMEOUT and leaves the context usable.
* Status paths: the Newton cap (EMU_ERR_NOT_CONVERGED, state kept), the CG
  cap (EMU_ERR_PCG), an allocator that fails (EMU_ERR_OOM, every successful
  allocation released), a served request that fails (the others' results
  unchanged).
* Resume: element state and positions saved after some frames and set on a
  fresh handle continue bit for bit like the uninterrupted run (FP64).
"""
import ctypes as C

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


def test_a_wait_that_runs_out_reports_timeout_and_the_context_stays_usable(emu):
    for wait_ns in (10_000_000, 200_000_000):  # 10 ms, 0.2 s
        assert emu.check_bounded_wait(wait_ns) == emu.binding.EMU_ERR_TIMEOUT
    mesh = box_beam(2, 2, 4, activation=0.4)
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-8))
    s.set_activation(0.4)
    assert s.solve().status == 0
    assert np.all(np.isfinite(s.positions()))
    s.close()


def test_newton_cap_reports_not_converged_and_keeps_a_usable_state(emu):
    mesh = box_beam(2, 2, 6, activation=0.5)
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-10, max_newton=1))
    s.set_activation(0.5)
    st = s.solve(raise_on_error=False)
    assert st.status == emu.binding.EMU_ERR_NOT_CONVERGED and st.newton_iters == 1
    R, sv, F = s.element_state()
    q = s.positions()
    assert np.all(np.isfinite(q)) and np.all(np.isfinite(F))
    np.testing.assert_allclose(np.einsum("nji,njk->nik", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    # the kept state is a valid warm start: a handle without the cap finishes from it
    t = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-10))
    t.set_element_state(R, sv, q)
    t.set_activation(0.5)
    assert t.solve().status == 0
    ref = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-10))
    ref.set_activation(0.5)
    ref.solve()
    diag = float(np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0)))
    assert np.abs(t.positions() - ref.positions()).max() <= 1e-9 * diag
    for x in (s, t, ref):
        x.close()


def test_cg_cap_reports_pcg_error(emu):
    mesh = box_beam(2, 2, 6, activation=0.5)
    s = emu.Solver(mesh, emu.Params(tol_rel_residual=1e-8, pcg_max=1))
    s.set_activation(0.5)
    st = s.solve(raise_on_error=False)
    assert st.status == emu.binding.EMU_ERR_PCG, st.status
    s.close()


def test_allocator_failure_reports_oom_and_releases_every_allocation(emu):
    import torch

    mesh = box_beam(2, 2, 4, activation=0.4)
    AF = emu.binding.emu_allocator._fields_[1][1]
    FF = emu.binding.emu_allocator._fields_[2][1]
    for fail_at in (1, 7, 30):
        live = {}
        calls = {"n": 0}

        def _alloc(ctx, size, stream):
            calls["n"] += 1
            if calls["n"] == fail_at:
                return None
            p = int(torch.cuda.caching_allocator_alloc(int(size), 0, stream))
            live[p] = size
            return p

        def _free(ctx, ptr, size, stream):
            assert int(ptr) in live
            del live[int(ptr)]
            torch.cuda.caching_allocator_delete(int(ptr))

        af, ff = AF(_alloc), FF(_free)

        class A:
            struct = emu.binding.emu_allocator(None, af, ff)

        with pytest.raises(emu.EmuError) as e:
            emu.Solver(mesh, emu.Params(), allocator=A())
        assert e.value.code == emu.binding.EMU_ERR_OOM
        assert calls["n"] >= fail_at and not live  # nothing leaked


def test_a_failing_served_request_leaves_the_others_unchanged(emu):
    good = [mtu_for_tet_count(1500, tendon_frac=0.1, seed=11), mtu_for_tet_count(2500, tendon_frac=0.15, seed=12)]
    bad = box_beam(2, 2, 3, activation=0.4)
    bad.rest_pos = bad.rest_pos.copy()
    bad.rest_pos[bad.tets[5][3]] = bad.rest_pos[bad.tets[5][0]]  # a degenerate tet: create fails
    acts = [np.stack([(m.material_id == 0) * a for a in (0.3, 0.6)]) for m in good]
    p = emu.Params(tol_rel_residual=1e-6, precision=emu.PRECISION_MIXED)
    solo = []
    for m, a in zip(good, acts):
        s = emu.Solver(m, p)
        q = []
        for f in range(a.shape[0]):
            s.set_activation(a[f])
            assert s.solve().status == 0
            q.append(s.positions())
        solo.append(np.stack(q))
        s.close()
    srv = emu.Server(8 << 30, p)
    srv.submit(good[0], acts[0], 1)
    srv.submit(bad, np.full((1, bad.n_tets), 0.4), 2)
    srv.submit(good[1], acts[1], 3)
    got = {}
    import time

    t0 = time.time()
    while len(got) < 3 and time.time() - t0 < 120:
        for i in srv.poll():
            got[i] = srv.result(i)
        time.sleep(0.001)
    srv.close()
    assert got[2][1].status == emu.binding.EMU_ERR_DEGENERATE_TET
    for k, rid in enumerate((1, 3)):
        assert got[rid][1].status == 0
        np.testing.assert_array_equal(got[rid][0], solo[k])


def test_resume_from_saved_state_is_bitwise_equal_to_the_uninterrupted_run(emu):
    mesh = box_beam(3, 3, 8, activation=np.linspace(0.0, 0.6, 5))
    p = emu.Params(tol_rel_residual=1e-9)
    full = emu.Solver(mesh, p)
    for f in (1, 2, 3, 4):
        full.set_activation(mesh.activations[f])
        assert full.solve().status == 0
    q_full = full.positions()
    first = emu.Solver(mesh, p)
    for f in (1, 2):
        first.set_activation(mesh.activations[f])
        first.solve()
    R, sv, _ = first.element_state()
    q2 = first.positions()
    first.close()
    resumed = emu.Solver(mesh, p)
    resumed.set_element_state(R, sv, q2)
    for f in (3, 4):
        resumed.set_activation(mesh.activations[f])
        assert resumed.solve().status == 0
    np.testing.assert_array_equal(resumed.positions(), q_full)
    full.close()
    resumed.close()
