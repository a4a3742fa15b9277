"""FP64 CPU oracle (test infrastructure only; see emu_oracle's header)."""
from .emu_oracle import (  # noqa: F401
    EmuOracle, OracleParams, OracleResult, lame, rest_geometry, build_G, psi, dpsi, d2psi,
    psd_project, delta_psi, sym_basis, stretch_from_s, s_from_stretch, element_terms_s,
    INVERTED_ENERGY,
)
from .bones import BoneOracle, affine_fit_weights  # noqa: F401,E402
