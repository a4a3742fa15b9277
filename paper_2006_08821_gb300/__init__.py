"""GB300-native quasi-static solver of EMU (arXiv 2006.08821).

The compute path is the CUDA library ``libemu_gb300.so`` (sm_103a) behind the
C ABI of ``include/emu.h``; ``binding`` mirrors that ABI with ctypes. PyTorch
is only used to provide device memory and streams.
"""
from .binding import (  # noqa: F401
    EXPORTED,
    LIB_PATH,
    EmuError,
    Params,
    Server,
    Solver,
    alpha_sweep,
    batch_solve,
    check_bounded_wait,
    mesh_desc,
    required_bytes,
    TorchAllocator,
    default_params,
    eval_capacitance,
    fiber_field,
    eval_polar,
    eval_stretch_terms,
    eval_fform_terms,
    load_library,
    PRECISION_FP64,
    PRECISION_MIXED,
    FORM_RS,
    FORM_F,
)
