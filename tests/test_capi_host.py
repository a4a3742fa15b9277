"""Host-only checks of the C ABI: the library builds, loads and exports every
entry point declared in include/emu.h; argument validation runs without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from emu_inputs import box_beam

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2006_08821_gb300 import build as b

    b.build()
    from paper_2006_08821_gb300 import binding

    return binding.load_library()


def _header_functions():
    text = open(os.path.join(ROOT, "include", "emu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(emu_[a-z_]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    from paper_2006_08821_gb300.binding import EXPORTED

    assert sorted(EXPORTED) == names


def test_default_params_and_status_strings(lib):
    from paper_2006_08821_gb300 import binding

    p = binding.default_params()
    assert p.k_modes == 48 and p.alpha_rel == 1.0 and p.weight_mode == 0
    assert p.ls_c == 1e-4 and p.ls_rho == 0.5  # Algorithm 1 constants
    assert lib.emu_status_string(0) == b"ok"
    assert lib.emu_status_string(-4) == b"not converged"


def _desc(mesh):
    from paper_2006_08821_gb300 import binding as B

    keep = [np.ascontiguousarray(x) for x in (mesh.rest_pos, mesh.tets.astype(np.int32), mesh.youngs,
                                                mesh.poisson, mesh.material_id.astype(np.uint8),
                                                mesh.fiber_dir, mesh.fixed_verts.astype(np.int32))]
    d = B.emu_mesh_desc()
    d.n_verts, d.n_tets = mesh.n_verts, mesh.n_tets
    d.rest_pos = keep[0].ctypes.data_as(C.POINTER(C.c_double))
    d.tets = keep[1].ctypes.data_as(C.POINTER(C.c_int32))
    d.n_materials = 1
    d.youngs = keep[2].ctypes.data_as(C.POINTER(C.c_double))
    d.poisson = keep[3].ctypes.data_as(C.POINTER(C.c_double))
    d.material_id = keep[4].ctypes.data_as(C.POINTER(C.c_uint8))
    d.fiber_dir = keep[5].ctypes.data_as(C.POINTER(C.c_double))
    d.n_fixed = len(keep[6])
    d.fixed_verts = keep[6].ctypes.data_as(C.POINTER(C.c_int32))
    return d, keep


@pytest.mark.parametrize("mutate,code", [
    ("bad_index", -1), ("no_pins", -1), ("bad_poisson", -1), ("bad_kmodes", -1), ("empty", -1),
    ("nan_rest", -1), ("bad_material", -1), ("bone", -1), ("joint", -1), ("neg_joints", -1),
    ("joint_without_bones", -1), ("bone_id_below_minus_one", -1),
])
def test_create_rejects_invalid_input_before_touching_the_device(lib, mutate, code):
    from paper_2006_08821_gb300 import binding as B

    mesh = box_beam(1, 1, 2)
    if mutate == "bad_index":
        mesh.tets = mesh.tets.copy()
        mesh.tets[0, 0] = mesh.n_verts + 5
    if mutate == "bad_poisson":
        mesh.poisson = np.array([0.5])
    if mutate == "nan_rest":
        mesh.rest_pos = mesh.rest_pos.copy()
        mesh.rest_pos[3, 1] = np.nan
    if mutate == "bad_material":
        mesh.material_id = mesh.material_id.copy()
        mesh.material_id[0] = 7
    d, keep = _desc(mesh)
    if mutate == "no_pins":
        d.n_fixed = 0
    if mutate == "empty":
        d.n_tets = 0
    if mutate in ("bone", "bone_id_below_minus_one"):
        # tet 0 touches the pinned face: a bone with part of its vertices pinned
        bid = np.full(mesh.n_tets, -1, dtype=np.int32)
        bid[0] = 0 if mutate == "bone" else -2
        keep.append(bid)
        d.bone_id = bid.ctypes.data_as(C.POINTER(C.c_int32))
    if mutate == "joint":  # joint arrays missing
        d.n_joints = 1
    if mutate == "joint_without_bones":
        jt = np.array([1], dtype=np.int32)
        jb = np.array([0, 1], dtype=np.int32)
        jp = np.zeros(3)
        ja = np.array([0.0, 1.0, 0.0])
        jh = np.array([0.01])
        keep += [jt, jb, jp, ja, jh]
        d.n_joints = 1
        d.joint_type = jt.ctypes.data_as(C.POINTER(C.c_int32))
        d.joint_bones = jb.ctypes.data_as(C.POINTER(C.c_int32))
        d.joint_point = jp.ctypes.data_as(C.POINTER(C.c_double))
        d.joint_axis = ja.ctypes.data_as(C.POINTER(C.c_double))
        d.joint_half_length = jh.ctypes.data_as(C.POINTER(C.c_double))
    if mutate == "neg_joints":
        d.n_joints = -1
    p = B.Params().to_c()
    if mutate == "bad_kmodes":
        p.k_modes = 50
    h = C.c_void_p()
    rc = lib.emu_create(C.byref(d), C.byref(p), None, None, C.byref(h))
    assert rc == code
    assert not h.value
    assert len(lib.emu_last_error()) > 0


def test_batch_solve_validates_its_arguments_without_a_device(lib):
    from paper_2006_08821_gb300 import binding as B

    assert lib.emu_batch_solve(None, 0, None) == B.EMU_OK  # empty batch: nothing to do
    assert lib.emu_batch_solve(None, 1, None) == B.EMU_ERR_INVALID_ARG
    hs = (C.c_void_p * 2)(None, None)
    assert lib.emu_batch_solve(hs, 2, None) == B.EMU_ERR_INVALID_ARG
    assert lib.emu_batch_solve(hs, -1, None) == B.EMU_ERR_INVALID_ARG


def test_server_calls_validate_their_arguments_without_a_device(lib):
    from paper_2006_08821_gb300 import binding as B

    n = C.c_int32()
    ids = (C.c_uint64 * 4)()
    assert lib.emu_server_poll(None, ids, 4, C.byref(n)) == B.EMU_ERR_INVALID_ARG
    assert lib.emu_server_result(None, 1, None, None) == B.EMU_ERR_INVALID_ARG
    assert lib.emu_server_submit(None, None, None, 1, 1) == B.EMU_ERR_INVALID_ARG
    assert lib.emu_server_create(1 << 30, None, None, None) == B.EMU_ERR_INVALID_ARG
    assert lib.emu_server_destroy(None) == B.EMU_OK
    assert lib.emu_required_bytes(None, None, None) == B.EMU_ERR_INVALID_ARG


def test_the_binding_fails_loudly_without_the_library(tmp_path):
    # there is no CPU fallback: a missing library is an error, not a detour
    from paper_2006_08821_gb300 import binding as B

    saved = B._lib
    B._lib = None
    try:
        with pytest.raises(RuntimeError):
            B.load_library(str(tmp_path / "missing.so"))
    finally:
        B._lib = saved
