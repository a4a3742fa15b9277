"""Host logic of the bench line's roofline figures (no GPU)."""
import math

import bench


def _prof():
    # phase -> (ms, launches) over 10 Newton iterations of a 400k-tet mesh
    return {"rhs": (0.1, 1), "assemble": (0.2, 10), "pcg": (3.4, 11), "grad": (0.8, 22), "syrk": (1.2, 10),
            "small": (0.3, 20), "dir": (0.5, 10), "ls": (0.6, 10), "update": (0.16, 20)}


def test_dominant_phase_with_little_dram_traffic_is_latency_bound():
    m, n, nnz = 400000, 75000, 1000000
    roof = bench.dominant_roofline(_prof(), True, m, n, nnz, 300.0, 6800.0, "measured",
                                   {"pcg": (20e6, "profiles/x.md")})
    assert roof["kernel"] == "pcg" and roof["bound"] == "latency"
    per_launch = bench.algorithmic_bytes("pcg", True, m, n, nnz, 300.0) / 11
    assert math.isclose(roof["bytes_per_launch"], per_launch)
    assert math.isclose(roof["frac"], per_launch / (3.4e-3 / 11) / 1e9 / 6800.0)
    assert math.isclose(roof["dram_frac"], 20e6 / (3.4e-3 / 11) / 1e9 / 6800.0)
    # without a DRAM figure a system well inside L2 is latency-bound by size ...
    roof = bench.dominant_roofline(_prof(), True, m, n, nnz, 300.0, 6800.0, "measured", {})
    assert roof["bound"] == "latency" and roof["traffic"] is None and "by size" in roof["note"]
    # ... and one too large for L2 is labelled by its algorithmic bytes
    roof = bench.dominant_roofline(_prof(), True, 40 * m, 40 * n, 40 * nnz, 300.0, 6800.0, "measured", {})
    assert roof["bound"] == "hbm" and roof["traffic"] is None


def test_per_tet_fractions_and_whole_iteration():
    m, n, nnz = 400000, 75000, 1000000
    pt = bench.per_tet_fractions(_prof(), True, m, n, nnz, 6800.0)
    assert set(pt) == {"grad", "syrk", "dir", "ls", "update"}
    b = bench.algorithmic_bytes("update", True, m, n, nnz, 0.0)
    # the update phase holds two launches per iteration, one of them per tet
    assert math.isclose(pt["update"]["us_per_launch"], 16.0)
    assert math.isclose(pt["update"]["frac"], round(b / 16e-6 / 1e9 / 6800.0, 3))
    w = bench.whole_iteration(_prof(), True, m, n, nnz, 300.0, 10, 6800.0, 5e8)
    assert math.isclose(w["scope_ceiling_tet_iters_s"], 6800e9 / (560 + 140 * 30.0))
    assert math.isclose(w["frac_of_scope_ceiling"], 5e8 / w["scope_ceiling_tet_iters_s"])
    assert math.isclose(w["us_per_iter"], 1e3 * sum(v[0] for v in _prof().values()) / 10)


def test_fform_byte_accounting():
    # the F-form (FP64) keeps F (72 B) as its state instead of R and s
    # (120 B) and a 45-entry factor instead of the 54-entry chart factor
    m, n, nnz = 1000, 300, 4000
    for phase, dstate, dfac in [("grad", 48, 9 * 8), ("dir", 0, 9 * 8), ("syrk", 0, 9 * 8), ("ls", 48, 0),
                                ("update", 96, 0), ("rhs", 48, 0)]:
        rs = bench.algorithmic_bytes(phase, False, m, n, nnz, 0.0)
        ff = bench.algorithmic_bytes(phase, False, m, n, nnz, 0.0, fform=True)
        assert math.isclose(rs - ff, (dstate + dfac) * m), phase
    # the coupling solve does not depend on the form
    assert bench.algorithmic_bytes("pcg", False, m, n, nnz, 10.0) == bench.algorithmic_bytes(
        "pcg", False, m, n, nnz, 10.0, fform=True)
