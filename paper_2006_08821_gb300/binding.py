"""ctypes binding of the C ABI in ``include/emu.h`` (argument marshalling only).

Every computation runs in the CUDA library ``libemu_gb300.so``. This module
loads it, mirrors the structs of the header and wraps the entry points with
the same names. Loading fails loudly if the library is missing; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libemu_gb300.so")

EMU_OK = 0
EMU_ERR_INVALID_ARG = -1
EMU_ERR_DEGENERATE_TET = -2
EMU_ERR_OOM = -3
EMU_ERR_NOT_CONVERGED = -4
EMU_ERR_LINESEARCH = -5
EMU_ERR_PCG = -6
EMU_ERR_INVERTED = -7
EMU_ERR_TIMEOUT = -8
EMU_ERR_CUDA = -9
EMU_ERR_NOT_IMPLEMENTED = -10

PRECISION_FP64 = 0
PRECISION_MIXED = 1
FORM_RS = 0  # rotation-stretch chart (emu_form)
FORM_F = 1   # the F-form of Sec. 3.2.1

# Entry points declared in include/emu.h (checked by the export test).
EXPORTED = [
    "emu_default_params", "emu_status_string", "emu_last_error", "emu_create", "emu_destroy",
    "emu_set_activation", "emu_set_activation_device", "emu_solve_quasistatic", "emu_get_positions",
    "emu_get_element_state", "emu_set_element_state", "emu_reset", "emu_get_sizes",
    "emu_eval_stretch_terms", "emu_eval_polar", "emu_set_profiling", "emu_get_profile",
    "emu_acap_solve_noalloc", "emu_batch_solve", "emu_required_bytes", "emu_server_create",
    "emu_server_submit", "emu_server_poll", "emu_server_result", "emu_server_destroy", "emu_check_bounded_wait",
    "emu_eval_capacitance", "emu_set_external_forces", "emu_fiber_field", "emu_alpha_sweep",
    "emu_eval_fform_terms", "emu_get_tuning",
]

PHASES = ["rhs", "assemble", "pcg", "grad", "syrk", "small", "dir", "ls", "update"]


class EmuError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class emu_allocator(C.Structure):
    _fields_ = [
        ("ctx", C.c_void_p),
        ("alloc", C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)),
        ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)),
    ]


class emu_mesh_desc(C.Structure):
    _fields_ = [
        ("n_verts", C.c_int64),
        ("n_tets", C.c_int64),
        ("rest_pos", C.POINTER(C.c_double)),
        ("tets", C.POINTER(C.c_int32)),
        ("n_materials", C.c_int32),
        ("youngs", C.POINTER(C.c_double)),
        ("poisson", C.POINTER(C.c_double)),
        ("material_id", C.POINTER(C.c_uint8)),
        ("fiber_dir", C.POINTER(C.c_double)),
        ("n_fixed", C.c_int64),
        ("fixed_verts", C.POINTER(C.c_int32)),
        ("fixed_pos", C.POINTER(C.c_double)),
        ("bone_id", C.POINTER(C.c_int32)),
        ("n_joints", C.c_int32),
        ("joint_type", C.POINTER(C.c_int32)),
        ("joint_bones", C.POINTER(C.c_int32)),
        ("joint_point", C.POINTER(C.c_double)),
        ("joint_axis", C.POINTER(C.c_double)),
        ("joint_half_length", C.POINTER(C.c_double)),
    ]


class emu_params(C.Structure):
    _fields_ = [
        ("alpha_rel", C.c_double),
        ("weight_mode", C.c_int32),
        ("k_modes", C.c_int32),
        ("fiber_scale", C.c_double),
        ("tol_rel_residual", C.c_double),
        ("max_newton", C.c_int32),
        ("ls_sigma0", C.c_double),
        ("ls_c", C.c_double),
        ("ls_rho", C.c_double),
        ("ls_max_trials", C.c_int32),
        ("pcg_tol", C.c_double),
        ("pcg_max", C.c_int32),
        ("precision", C.c_int32),
        ("mode_iters", C.c_int32),
        ("seed", C.c_uint64),
        ("dq_tol", C.c_double),
        ("q_refresh", C.c_int32),
        ("eps_bone", C.c_double),
        ("eps_joint", C.c_double),
        ("cg_local_degree", C.c_int32),
        ("form", C.c_int32),
        ("autotune", C.c_int32),
    ]


class emu_solve_stats(C.Structure):
    _fields_ = [
        ("newton_iters", C.c_int32),
        ("ls_trials", C.c_int32),
        ("pcg_iters", C.c_int32),
        ("status", C.c_int32),
        ("rel_residual", C.c_double),
        ("energy_change", C.c_double),
        ("ms", C.c_double),
    ]


class emu_request_stats(C.Structure):
    _fields_ = [
        ("id", C.c_uint64),
        ("status", C.c_int32),
        ("frames_done", C.c_int32),
        ("newton_iters", C.c_int32),
        ("pcg_iters", C.c_int32),
        ("rel_residual", C.c_double),
        ("queue_ms", C.c_double),
        ("setup_ms", C.c_double),
        ("solve_ms", C.c_double),
        ("latency_ms", C.c_double),
        ("device_bytes", C.c_uint64),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2006_08821_gb300.build.build() "
                           "(needs nvcc); there is no CPU fallback")
    lib = C.CDLL(path)
    P = C.POINTER
    lib.emu_default_params.argtypes = [P(emu_params)]
    lib.emu_default_params.restype = None
    lib.emu_status_string.argtypes = [C.c_int]
    lib.emu_status_string.restype = C.c_char_p
    lib.emu_last_error.argtypes = []
    lib.emu_last_error.restype = C.c_char_p
    lib.emu_create.argtypes = [P(emu_mesh_desc), P(emu_params), P(emu_allocator), C.c_void_p, P(C.c_void_p)]
    lib.emu_destroy.argtypes = [C.c_void_p]
    lib.emu_set_activation.argtypes = [C.c_void_p, P(C.c_double), C.c_int64]
    lib.emu_set_external_forces.argtypes = [C.c_void_p, P(C.c_double), C.c_int64]
    lib.emu_alpha_sweep.argtypes = [P(emu_mesh_desc), P(emu_params), P(C.c_double), C.c_double, C.c_double,
                                    C.c_int32, C.c_double, P(C.c_double), P(C.c_int32), P(C.c_int32), C.c_void_p]
    lib.emu_fiber_field.argtypes = [C.c_int64, P(C.c_double), C.c_int64, P(C.c_int32), P(C.c_int32), C.c_int64,
                                    P(C.c_int32), C.c_int64, P(C.c_double), C.c_void_p]
    lib.emu_set_activation_device.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    lib.emu_solve_quasistatic.argtypes = [C.c_void_p, P(emu_solve_stats)]
    lib.emu_get_positions.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
    lib.emu_get_element_state.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double), P(C.c_double)]
    lib.emu_set_element_state.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double), P(C.c_double)]
    lib.emu_reset.argtypes = [C.c_void_p]
    lib.emu_get_sizes.argtypes = [C.c_void_p, P(C.c_int64), P(C.c_int64), P(C.c_int32)]
    lib.emu_eval_stretch_terms.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p]
    lib.emu_eval_polar.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.emu_set_profiling.argtypes = [C.c_void_p, C.c_int32]
    lib.emu_acap_solve_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.emu_get_profile.argtypes = [C.c_void_p, P(C.c_double), P(C.c_int32), C.c_int32, P(C.c_int64)]
    lib.emu_batch_solve.argtypes = [P(C.c_void_p), C.c_int32, P(emu_solve_stats)]
    lib.emu_required_bytes.argtypes = [P(emu_mesh_desc), P(emu_params), P(C.c_size_t)]
    lib.emu_server_create.argtypes = [C.c_size_t, P(emu_params), P(emu_allocator), P(C.c_void_p)]
    lib.emu_server_submit.argtypes = [C.c_void_p, P(emu_mesh_desc), P(C.c_double), C.c_int32, C.c_uint64]
    lib.emu_server_poll.argtypes = [C.c_void_p, P(C.c_uint64), C.c_int32, P(C.c_int32)]
    lib.emu_server_result.argtypes = [C.c_void_p, C.c_uint64, P(C.c_double), P(emu_request_stats)]
    lib.emu_server_destroy.argtypes = [C.c_void_p]
    lib.emu_check_bounded_wait.argtypes = [C.c_int64, C.c_void_p]
    lib.emu_eval_capacitance.argtypes = [C.c_int64, P(C.c_float), P(C.c_float), P(C.c_float), P(C.c_float),
                                         C.c_int32, P(C.c_double), P(C.c_double), C.c_void_p]
    for name in EXPORTED:
        if name not in ("emu_default_params", "emu_status_string", "emu_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(rc, lib=None):
    if rc != EMU_OK:
        lib = lib or load_library()
        raise EmuError(rc, f"{lib.emu_status_string(rc).decode()}: {lib.emu_last_error().decode()}")


def _dptr(a, dtype):
    """Host pointer of a C-contiguous numpy array of the given dtype (kept alive by the caller)."""
    return a.ctypes.data_as(C.POINTER(dtype))


@dataclasses.dataclass
class Params:
    """Mirror of emu_params with the library defaults."""
    alpha_rel: float = 1.0
    weight_mode: int = 0
    k_modes: int = 48
    fiber_scale: float = 1.0
    tol_rel_residual: float = 1e-6
    max_newton: int = 2000
    ls_sigma0: float = 4.0
    ls_c: float = 1e-4
    ls_rho: float = 0.5
    ls_max_trials: int = 40
    pcg_tol: float = 1e-8
    pcg_max: int = 5000
    precision: int = PRECISION_FP64
    mode_iters: int = 8
    seed: int = 12345
    dq_tol: float = 8e-2
    q_refresh: int = 32
    eps_bone: float = -1e-3
    eps_joint: float = -1e-4
    cg_local_degree: int = 4
    form: int = FORM_RS
    autotune: int = 0

    def to_c(self) -> emu_params:
        p = emu_params()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


def default_params() -> Params:
    lib = load_library()
    p = emu_params()
    lib.emu_default_params(C.byref(p))
    return Params(**{f.name: getattr(p, f.name) for f in dataclasses.fields(Params)})


class TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self, device=0):
        import torch

        self._torch = torch
        self.device = device
        AF = emu_allocator._fields_[1][1]
        FF = emu_allocator._fields_[2][1]

        def _alloc(ctx, size, stream):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(size), self.device, stream))
            except Exception:  # pragma: no cover - OOM path
                return None

        def _free(ctx, ptr, size, stream):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._af = AF(_alloc)
        self._ff = FF(_free)
        self.struct = emu_allocator(None, self._af, self._ff)


def mesh_desc(mesh):
    """emu_mesh_desc of a mesh (emu_inputs.MeshSpec-like) and the arrays it
    points into (keep them alive while the descriptor is used)."""
    Q = np.ascontiguousarray(mesh.rest_pos, dtype=np.float64)
    T = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    E = np.ascontiguousarray(mesh.youngs, dtype=np.float64)
    nu = np.ascontiguousarray(mesh.poisson, dtype=np.float64)
    mid = np.ascontiguousarray(mesh.material_id, dtype=np.uint8)
    fib = None if mesh.fiber_dir is None else np.ascontiguousarray(mesh.fiber_dir, dtype=np.float64)
    fx = np.ascontiguousarray(mesh.fixed_verts, dtype=np.int32)
    fp = None if getattr(mesh, "fixed_pos", None) is None else np.ascontiguousarray(mesh.fixed_pos, dtype=np.float64)
    d = emu_mesh_desc()
    d.n_verts = Q.shape[0]
    d.n_tets = T.shape[0]
    d.rest_pos = _dptr(Q, C.c_double)
    d.tets = _dptr(T, C.c_int32)
    d.n_materials = E.shape[0]
    d.youngs = _dptr(E, C.c_double)
    d.poisson = _dptr(nu, C.c_double)
    d.material_id = _dptr(mid, C.c_uint8)
    d.fiber_dir = _dptr(fib, C.c_double) if fib is not None else None
    d.n_fixed = fx.shape[0]
    d.fixed_verts = _dptr(fx, C.c_int32)
    d.fixed_pos = _dptr(fp, C.c_double) if fp is not None else None
    bid = getattr(mesh, "bone_id", None)
    bid = None if bid is None else np.ascontiguousarray(bid, dtype=np.int32)
    d.bone_id = _dptr(bid, C.c_int32) if bid is not None else None
    joints = getattr(mesh, "joints", None) or []
    jt = np.array([1 if j["type"] == "hinge" else 0 for j in joints], dtype=np.int32)
    jb = np.array([j["bones"] for j in joints], dtype=np.int32).reshape(-1, 2)
    jp = np.array([j["point"] for j in joints], dtype=np.float64).reshape(-1, 3)
    ja = np.array([j.get("axis", (0.0, 0.0, 0.0)) for j in joints], dtype=np.float64).reshape(-1, 3)
    jh = np.array([j.get("half_length", 0.0) for j in joints], dtype=np.float64)
    d.n_joints = len(joints)
    if joints:
        d.joint_type = _dptr(jt, C.c_int32)
        d.joint_bones = _dptr(jb, C.c_int32)
        d.joint_point = _dptr(jp, C.c_double)
        d.joint_axis = _dptr(ja, C.c_double)
        d.joint_half_length = _dptr(jh, C.c_double)
    return d, [Q, T, E, nu, mid, fib, fx, fp, bid, jt, jb, jp, ja, jh]


class Solver:
    """One mesh resident on the GPU (wraps emu_create ... emu_destroy)."""

    def __init__(self, mesh, params: Params | None = None, stream=None, allocator=None):
        self.lib = load_library()
        self.params = params or Params()
        d, self._keep = mesh_desc(mesh)
        self.n_verts = int(d.n_verts)
        self.n_tets = int(d.n_tets)
        self.stream = stream
        st = None if stream is None else C.c_void_p(int(stream))
        self._allocator = allocator
        ap = C.byref(allocator.struct) if allocator is not None else None
        h = C.c_void_p()
        cp = self.params.to_c()
        _check(self.lib.emu_create(C.byref(d), C.byref(cp), ap, st, C.byref(h)), self.lib)
        self.handle = h
        if getattr(mesh, "f_ext", None) is not None:  # constant per-vertex forces of the mesh
            self.set_external_forces(mesh.f_ext)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.emu_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_activation(self, a):
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (self.n_tets,)))
        _check(self.lib.emu_set_activation(self.handle, _dptr(a, C.c_double), a.shape[0]), self.lib)

    def set_external_forces(self, f):
        """Constant per-vertex forces (n_verts, 3), e.g. gravity; None removes them."""
        if f is None:
            _check(self.lib.emu_set_external_forces(self.handle, None, 0), self.lib)
            return
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        if f.shape != (self.n_verts, 3):
            raise ValueError("forces must have shape (n_verts, 3)")
        _check(self.lib.emu_set_external_forces(self.handle, _dptr(f, C.c_double), f.shape[0]), self.lib)

    def set_activation_device(self, a_dev_ptr: int):
        _check(self.lib.emu_set_activation_device(self.handle, C.c_void_p(a_dev_ptr), self.n_tets), self.lib)

    def solve(self, raise_on_error=True) -> emu_solve_stats:
        st = emu_solve_stats()
        rc = self.lib.emu_solve_quasistatic(self.handle, C.byref(st))
        if raise_on_error and rc not in (EMU_OK,):
            _check(rc, self.lib)
        st.status = rc
        return st

    def positions(self) -> np.ndarray:
        out = np.empty((self.n_verts, 3), dtype=np.float64)
        _check(self.lib.emu_get_positions(self.handle, out.ctypes.data_as(C.c_void_p), 0), self.lib)
        return out

    def positions_to_device(self, dev_ptr: int):
        _check(self.lib.emu_get_positions(self.handle, C.c_void_p(dev_ptr), 1), self.lib)

    def element_state(self):
        R = np.empty((self.n_tets, 3, 3))
        s = np.empty((self.n_tets, 6))
        F = np.empty((self.n_tets, 3, 3))
        _check(self.lib.emu_get_element_state(self.handle, _dptr(R, C.c_double), _dptr(s, C.c_double),
                                              _dptr(F, C.c_double)), self.lib)
        return R, s, F

    def set_element_state(self, R=None, s=None, q=None):
        arrs = [None if x is None else np.ascontiguousarray(x, dtype=np.float64) for x in (R, s, q)]
        ptrs = [None if x is None else _dptr(x, C.c_double) for x in arrs]
        _check(self.lib.emu_set_element_state(self.handle, *ptrs), self.lib)

    def reset(self):
        _check(self.lib.emu_reset(self.handle), self.lib)

    def tuning(self) -> dict:
        """emu_get_tuning: the coupling solves' launch settings in use."""
        d, r, t = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        _check(self.lib.emu_get_tuning(self.handle, C.byref(d), C.byref(r), C.byref(t)), self.lib)
        return {"cg_local_degree": int(d.value), "cg64_rows_per_block": int(r.value), "tuned": bool(t.value)}

    def acap_solve_noalloc(self, F_dev_ptr: int, q_dev_ptr: int, stream=None):
        """emu_acap_solve_noalloc: q = q*(F) with no device allocation (device pointers)."""
        st = C.c_void_p(int(stream)) if stream is not None else (
            C.c_void_p(int(self.stream)) if self.stream is not None else None)
        return self.lib.emu_acap_solve_noalloc(self.handle, C.c_void_p(int(F_dev_ptr)), C.c_void_p(int(q_dev_ptr)), st)

    def set_profiling(self, enable: bool):
        _check(self.lib.emu_set_profiling(self.handle, 1 if enable else 0), self.lib)

    def profile(self):
        """(dict phase -> (ms, launches), total launches) since profiling was enabled."""
        n = len(PHASES)
        ms = (C.c_double * n)()
        cnt = (C.c_int32 * n)()
        tot = C.c_int64()
        _check(self.lib.emu_get_profile(self.handle, ms, cnt, n, C.byref(tot)), self.lib)
        return {PHASES[k]: (ms[k], cnt[k]) for k in range(n)}, tot.value

    def sizes(self):
        n = C.c_int64()
        m = C.c_int64()
        k = C.c_int32()
        _check(self.lib.emu_get_sizes(self.handle, C.byref(n), C.byref(m), C.byref(k)), self.lib)
        return n.value, m.value, k.value


def batch_solve(solvers, raise_on_error=True):
    """emu_batch_solve over ``solvers`` (distinct Solver objects): one
    quasi-static solve each, interleaved on their streams. Returns the list
    of per-solver stats (``status`` set on each)."""
    solvers = list(solvers)
    lib = load_library()
    n = len(solvers)
    hs = (C.c_void_p * max(n, 1))(*[s.handle for s in solvers])
    st = (emu_solve_stats * max(n, 1))()
    rc = lib.emu_batch_solve(hs, n, st)
    if raise_on_error and rc != EMU_OK:
        _check(rc, lib)
    return [st[i] for i in range(n)]


def required_bytes(mesh, params: Params | None = None) -> int:
    """emu_required_bytes: device memory bound of a mesh (needs a GPU)."""
    lib = load_library()
    d, keep = mesh_desc(mesh)
    cp = (params or Params()).to_c()
    out = C.c_size_t()
    _check(lib.emu_required_bytes(C.byref(d), C.byref(cp), C.byref(out)), lib)
    return int(out.value)


class Server:
    """emu_server_*: persistent request loop with a device-memory budget."""

    def __init__(self, budget_bytes: int, params: Params | None = None):
        self.lib = load_library()
        self.params = params or Params()
        cp = self.params.to_c()
        h = C.c_void_p()
        _check(self.lib.emu_server_create(C.c_size_t(int(budget_bytes)), C.byref(cp), None, C.byref(h)), self.lib)
        self.handle = h
        self._shape = {}

    def submit(self, mesh, activations, request_id: int):
        """activations: (frames, n_tets) float64 (a 1-D array is one frame)."""
        d, keep = mesh_desc(mesh)
        a = np.ascontiguousarray(np.atleast_2d(np.asarray(activations, dtype=np.float64)))
        if a.shape[1] != d.n_tets:
            raise ValueError("activations must have n_tets columns")
        _check(self.lib.emu_server_submit(self.handle, C.byref(d), _dptr(a, C.c_double), a.shape[0],
                                          C.c_uint64(int(request_id))), self.lib)
        self._shape[int(request_id)] = (a.shape[0], int(d.n_verts))

    def poll(self, cap: int = 256):
        ids = (C.c_uint64 * cap)()
        n = C.c_int32()
        _check(self.lib.emu_server_poll(self.handle, ids, cap, C.byref(n)), self.lib)
        return [int(ids[k]) for k in range(n.value)]

    def result(self, request_id: int):
        """(positions (frames, n_verts, 3), emu_request_stats) of a finished request."""
        frames, n = self._shape.pop(int(request_id))
        pos = np.empty((frames, n, 3), dtype=np.float64)
        st = emu_request_stats()
        _check(self.lib.emu_server_result(self.handle, C.c_uint64(int(request_id)), _dptr(pos, C.c_double),
                                          C.byref(st)), self.lib)
        return pos, st

    def close(self):
        if getattr(self, "handle", None):
            self.lib.emu_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eval_stretch_terms(s_dev, params_dev, n, mixed, psi_dev, grad_dev, hess_dev, stream=0):
    """emu_eval_stretch_terms on device pointers (ints)."""
    lib = load_library()
    cv = lambda x: None if x is None else C.c_void_p(int(x))  # noqa: E731
    _check(lib.emu_eval_stretch_terms(cv(s_dev), cv(params_dev), n, mixed, cv(psi_dev), cv(grad_dev),
                                      cv(hess_dev), cv(stream)), lib)


def eval_fform_terms(F_dev, params_dev, n, psi_dev, grad_dev, hess_dev, stream=0):
    """emu_eval_fform_terms on device pointers (ints)."""
    lib = load_library()
    cv = lambda x: None if x is None else C.c_void_p(int(x))  # noqa: E731
    _check(lib.emu_eval_fform_terms(cv(F_dev), cv(params_dev), n, cv(psi_dev), cv(grad_dev), cv(hess_dev),
                                    cv(stream)), lib)


def check_bounded_wait(wait_ns: int, stream=0) -> int:
    """emu_check_bounded_wait: status of a grid-barrier wait that must run out
    (EMU_ERR_TIMEOUT is the expected result)."""
    lib = load_library()
    return lib.emu_check_bounded_wait(int(wait_ns), C.c_void_p(int(stream)) if stream else None)


def alpha_sweep(mesh, activation, params: Params | None = None, alpha0=1.0, factor=10.0, max_steps=6, jump=3.0,
                stream=0):
    """emu_alpha_sweep: (chosen alpha_rel, the alpha_rel values tried, their
    Newton counts, -1 where a solve did not converge)."""
    lib = load_library()
    d, keep = mesh_desc(mesh)
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(activation, dtype=np.float64), (mesh.n_tets,)))
    cp = (params or Params()).to_c()
    out = C.c_double(0.0)
    iters = np.full(max_steps, -1, dtype=np.int32)
    n = C.c_int32(0)
    _check(lib.emu_alpha_sweep(C.byref(d), C.byref(cp), _dptr(a, C.c_double), alpha0, factor, max_steps, jump,
                               C.byref(out), _dptr(iters, C.c_int32), C.byref(n),
                               C.c_void_p(int(stream)) if stream else None), lib)
    k = int(n.value)
    return float(out.value), [alpha0 * factor ** i for i in range(k)], [int(x) for x in iters[:k]]


def fiber_field(rest_pos, tets, origin, insertion, stream=0):
    """emu_fiber_field: unit fiber directions (n_tets, 3) from the heat
    equation with -1 on ``origin`` and +1 on ``insertion`` vertices."""
    lib = load_library()
    Q = np.ascontiguousarray(rest_pos, dtype=np.float64)
    T = np.ascontiguousarray(tets, dtype=np.int32)
    o = np.ascontiguousarray(origin, dtype=np.int32)
    ins = np.ascontiguousarray(insertion, dtype=np.int32)
    out = np.zeros((T.shape[0], 3))
    _check(lib.emu_fiber_field(Q.shape[0], _dptr(Q, C.c_double), T.shape[0], _dptr(T, C.c_int32), _dptr(o, C.c_int32),
                               o.size, _dptr(ins, C.c_int32), ins.size, _dptr(out, C.c_double),
                               C.c_void_p(int(stream)) if stream else None), lib)
    return out


def eval_capacitance(U, gamma, y, w, kernel=0, stream=0):
    """emu_eval_capacitance: (C 48 x 48, By 48) from component-major float32
    host arrays U (54, m), gamma (48, m), y (9, m), w (m,)."""
    lib = load_library()
    U = np.ascontiguousarray(U, dtype=np.float32)
    gamma = np.ascontiguousarray(gamma, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    m = w.shape[0]
    if U.shape != (54, m) or gamma.shape != (48, m) or y.shape != (9, m):
        raise ValueError("U (54, m), gamma (48, m), y (9, m), w (m,) expected")
    Cm = np.zeros((48, 48))
    By = np.zeros(48)
    _check(lib.emu_eval_capacitance(m, _dptr(U, C.c_float), _dptr(gamma, C.c_float), _dptr(y, C.c_float),
                                    _dptr(w, C.c_float), int(kernel), _dptr(Cm, C.c_double), _dptr(By, C.c_double),
                                    C.c_void_p(int(stream)) if stream else None), lib)
    return Cm, By


def eval_polar(F_dev, n, R_dev, s_dev, stream=0):
    lib = load_library()
    _check(lib.emu_eval_polar(C.c_void_p(int(F_dev)), n, C.c_void_p(int(R_dev)), C.c_void_p(int(s_dev)),
                              C.c_void_p(int(stream))), lib)
