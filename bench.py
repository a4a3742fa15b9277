"""Benchmark of the GB300 quasi-static solve (tet-iterations per second).

Workload (default): the muscle-tendon unit, a 32x32x128 Kuhn-split cube grid
masked to a cylinder (401,920 tets, 74,929 vertices). The outer 10% of its
length is tendon (E = 1e8 Pa), the rest muscle (E = 6e5 Pa). Fibers follow
the axis with a seeded 5-degree Gaussian tilt, and a 60-frame activation ramp
goes from 0 to 1. Each frame is solved from the previous frame's state to a
relative residual of 1e-6. A step is one frame. Warm-up frames come first,
then K timed frames; the L2 cache is flushed between frames, outside the
timed intervals.

Reported:
  value      tet-iterations/s = sum(n_tets * newton_iters) / sum(frame device time)
  e2e        the same metric through the public API with host buffers: each
             frame's activation upload, solve and position download inside
             the host-clocked interval.
  roofline   the kernel with the most device time: algorithmic bytes per
             launch over its average CUDA-event duration, against the
             measured HBM copy peak; labelled latency-bound (with its DRAM
             fraction beside it) when ncu shows its operands stay in L2.
  per_tet_kernels_hbm, whole_iteration
             each per-tet kernel's fraction of the HBM peak, and one Newton
             iteration's algorithmic bytes over its device time.
  error_vs_oracle
             positions of the benchmarked configuration on the CPU
             baseline's sample against the oracle's (re-converged to 1e-10).
  cpu_baseline / --impl reference: the FP64 CPU oracle on a bounded sample of
             the same workload.

Multi-GPU: one process per GPU (torchrun), each solving an independent
replica of the workload ("replicas only": the method has no exchange step);
max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from emu_inputs import arm_assembly, batch_set, box_beam, mtu_for_tet_count, muscle_tendon_unit, request_stream  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129e6  # GB300 L2

# DRAM bytes (read + write) per launch of a phase's kernel from one ncu
# capture of the unchanged kernel (summaries under profiles/); None once the
# kernel has changed since.
NCU_TRAFFIC = {
    "pcg": (18.21e6, "profiles/pcg32p_kernel_mtu401920.md"),
    "grad": (124.19e6, "profiles/k_grad_m_mtu401920.md"),
    "dir": (230.63e6, "profiles/k_dir_m_mtu401920.md"),
    "ls": (82.91e6, "profiles/k_ls_m_mtu401920.md"),
    "syrk": (183.30e6, "profiles/k_syrk05_mtu401920.md"),
}


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        for key in ("hbm_gbs", "hbm_GBs", "hbm"):
            if key in pk:
                v = pk[key]
                if isinstance(v, dict):
                    v = v.get("value", v.get("gbs"))
                return float(v), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def make_workload(name):
    if name == "mtu":
        mesh = muscle_tendon_unit()  # 32x32x128, r = 12.9h, 60 frames
        desc = (f"muscle-tendon unit: 32x32x128 Kuhn grid masked to a cylinder, {mesh.n_tets} tets, "
                f"{mesh.n_verts} verts, 10% tendon E=1e8, muscle E=6e5, nu=0.45, fibers +-5deg, "
                f"60-frame activation ramp 0->1, warm starts, rel residual 1e-6")
        return mesh, desc
    if name == "box":
        mesh = box_beam(4, 4, 16, activation=np.linspace(0.0, 0.5, 6))
        return mesh, "box beam 4x4x16 (1,536 tets), activation ramp to 0.5, rel residual 1e-6"
    if name == "mtu_small":
        mesh = muscle_tendon_unit(8, 8, 32, h=0.01, radius_cells=12.9 / 4, frames=60)
        return mesh, f"muscle-tendon unit 8x8x32 ({mesh.n_tets} tets), 60-frame ramp, rel residual 1e-6"
    if name == "arm":
        # the arm-like assembly at the largest size the method converges on
        # within the Newton cap (the 799,152-tet default does not, in the
        # oracle either; see the design notes)
        mesh = arm_assembly(bone_w=6, bone_len=24, r0=10.0, frames=120)
        desc = (f"arm-like assembly: two box bones (E=1e10, 6x6x24 cells each, bone 1 pinned), hinge joint, "
                f"fusiform muscle and tendon bars, {mesh.n_tets} tets, {mesh.n_verts} verts, "
                f"120-frame activation sin^2 ramp, warm starts, rel residual 1e-6, final solve with affine bones")
        return mesh, desc
    raise ValueError(name)


def algorithmic_bytes(phase, mixed, m, n, nnz, cg_iters, fform=False):
    """Minimum bytes one launch of a phase must move (each array read or
    written once; vertex arrays once per vertex), for the roofline.

    Per-tet phases count per-tet records of the mixed (FP32) or FP64 layout;
    the ACAP solve counts, per CG iteration, the CSR matrix (value + column
    index), D^-1, the 16 coarse-basis values and six 3-vectors read and
    written once, times the CG iterations of the launch. The F-form (FP64)
    keeps F (9 values) as its state and a 45-entry factor per tet."""
    f = 4 if mixed else 8
    rec = 16 + 9 * f + 6 * f + 3 * f          # tet, D^-1, V c w mu lam ka, u
    state = (16 + 6 * 4) if mixed else (72 if fform else 72 + 48)
    fac = 45 if fform else 54
    vert = 24 * n / m                          # q gathered, each vertex once
    per_tet = {
        "grad": rec + state + vert + 9 * f + 9 * f + 9 * f + fac * f,   # + E0 (mixed), write g, y, Uw
        "dir": 48 * f + fac * f + 9 * f + 9 * f + 9 * f + f + 9 * f + 96,  # gam, Uw, y, g, D^-1, w -> d, corner terms
        "ls": rec + state + 9 * f + 2 * vert + (9 * 4 if mixed else 0),
        "update": 2 * state + 9 * f,
        "syrk": fac * f + 48 * f + 9 * f + f,
        "rhs": 16 + 9 * f + state + f + 96,
    }
    if phase in per_tet:
        return per_tet[phase] * m
    if phase == "pcg":
        per_iter = nnz * (f + 4) + n * (4 + f + 16 * f + 6 * 2 * 3 * f)
        return per_iter * cg_iters
    return None


# per-tet kernels launched per launch of a profiled phase (the update phase
# also launches the per-vertex position update, the mixed gradient phase the
# per-vertex split of the displacement)
PER_TET_KERNELS = {"grad": 0.5, "syrk": 1.0, "dir": 1.0, "ls": 1.0, "update": 0.5}
PER_TET_KERNELS_FP64 = {"grad": 1.0, "syrk": 1.0, "dir": 1.0, "ls": 1.0, "update": 0.5}


def per_tet_kernels(mixed):
    return PER_TET_KERNELS if mixed else PER_TET_KERNELS_FP64


def per_tet_fractions(prof, mixed, m, n, nnz, peak, traffic_table=None, fform=False):
    """Each per-tet kernel's algorithmic bytes per launch over its average
    CUDA-event duration, against the HBM peak; with the kernel's ncu DRAM
    bytes per launch beside it where a capture of the unchanged kernel exists."""
    out = {}
    for name, per in per_tet_kernels(mixed).items():
        ms, nl = prof.get(name, (0.0, 0))
        if nl <= 0 or ms <= 0:
            continue
        launches = nl * per
        b = algorithmic_bytes(name, mixed, m, n, nnz, 0.0, fform)
        us = 1e3 * ms / launches
        gbs = b / (us * 1e-6) / 1e9
        out[name] = {"bytes_per_launch": b, "us_per_launch": round(us, 2), "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / peak, 3)}
        tr = (traffic_table or {}).get(name)
        if tr:
            out[name]["ncu_dram_bytes"] = tr[0]
            out[name]["ncu_dram_frac"] = round(tr[0] / (us * 1e-6) / 1e9 / peak, 3)
    return out


def dominant_roofline(prof, mixed, m, n, nnz, cg_total, peak, peak_kind, traffic_table, fform=False):
    """Roofline entry of the phase with the most device time. The coupling
    solve's system (CSR, vectors, coarse rows) is L2-resident on the
    benchmark meshes: when its measured DRAM traffic is far below the
    algorithmic bytes it is reported as latency-bound, with both fractions."""
    name, (ms_tot, nl) = max(prof.items(), key=lambda kv: kv[1][0])
    total = algorithmic_bytes(name, mixed, m, n, nnz, cg_total, fform)
    if total is None or nl <= 0 or ms_tot <= 0:
        return None
    per_launch = total / nl if name == "pcg" else total
    avg_s = ms_tot / nl / 1e3
    achieved = per_launch / avg_s / 1e9
    tr = traffic_table.get(name)
    traffic = tr[0] if tr else None
    bound = "hbm"
    if traffic is not None and traffic < 0.25 * per_launch:
        bound = "latency"
    # without a capture of this workload: the coupling solve's system (CSR,
    # D^-1, coarse rows, six 3-vectors) well inside the 129 MB L2 is
    # latency-bound by construction (grid barriers and L2 round trips)
    f = 4 if mixed else 8
    system_bytes = nnz * (f + 4) + n * (f + 16 * f + 6 * 3 * f)
    l2_resident = name == "pcg" and traffic is None and system_bytes < 0.5 * L2_BYTES
    if l2_resident:
        bound = "latency"
    roof = {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_source": tr[1] if tr else None,
            "peak_source": peak_kind, "bytes_per_launch": per_launch, "avg_launch_ms": 1e3 * avg_s,
            "share_of_device_time": ms_tot / max(1e-9, sum(v[0] for v in prof.values()))}
    if traffic is not None:
        roof["dram_gbs"] = traffic / avg_s / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / peak
    if bound == "latency":
        roof["note"] = ("L2-resident: DRAM traffic per launch is far below the algorithmic bytes, so frac "
                        "measures how fast the solve streams its operands from L2; the limit is grid-barrier "
                        "and L2 latency")
        if l2_resident:
            roof["note"] = (f"L2-resident by size (system {system_bytes / 1e6:.1f} MB against the 129 MB L2; no "
                            "ncu capture of this workload): frac measures how fast the solve streams its operands "
                            "from L2; the limit is grid-barrier and L2 latency")
    return roof


def whole_iteration(prof, mixed, m, n, nnz, cg_total, iters, peak, value, fform=False):
    """One Newton iteration against the HBM roofline: the algorithmic bytes
    of every per-tet kernel and of the coupling solve over the device time
    per iteration, and the measured tet-iters/s against the scope's ceiling
    peak / (560 + 140 N_cg) bytes per tet-iteration."""
    if iters <= 0:
        return None
    b = 0.0
    for name, per in per_tet_kernels(mixed).items():
        ms, nl = prof.get(name, (0.0, 0))
        b += algorithmic_bytes(name, mixed, m, n, nnz, 0.0, fform) * nl * per
    b += algorithmic_bytes("pcg", mixed, m, n, nnz, cg_total)
    b /= iters
    t = sum(v[0] for v in prof.values()) / 1e3 / iters
    ncg = cg_total / iters
    ceiling = peak * 1e9 / (560.0 + 140.0 * ncg)
    return {"bytes_per_iter": b, "us_per_iter": 1e6 * t, "achieved_gbs": b / t / 1e9, "frac": b / t / 1e9 / peak,
            "scope_ceiling_tet_iters_s": ceiling, "frac_of_scope_ceiling": value / ceiling}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def solver_nnz(mesh):
    """Non-zeros of the scalar ACAP Laplacian (free-free couplings plus the
    pinned identity rows), counted from the tet connectivity."""
    T = np.asarray(mesh.tets, dtype=np.int64)
    fixed = np.zeros(mesh.n_verts, dtype=bool)
    fixed[np.asarray(mesh.fixed_verts)] = True
    a = T[:, :, None].repeat(4, 2).reshape(-1)
    b = T[:, None, :].repeat(4, 1).reshape(-1)
    keep = ~fixed[a] & ~fixed[b]
    pairs = np.unique(a[keep] * mesh.n_verts + b[keep])
    return int(pairs.size + fixed.sum())


def threads_used(cpu_s, wall_s):
    """Threads a host computation kept busy on average: process CPU time (all
    threads) over wall time, at least 1."""
    return max(1, int(round(cpu_s / wall_s))) if wall_s > 0 else 1


def oracle_sample(workload_name):
    """The CPU sample of a workload: (mesh, description, oracle, solve) with
    solve(oracle, activation, previous F or None, tol, max_newton)."""
    from oracle import EmuOracle, OracleParams

    prm = OracleParams(alpha_rel=1.0, weight_mode=0)
    if workload_name == "arm":
        from oracle.bones import BoneOracle

        mesh = arm_assembly(bone_w=3, bone_len=8, r0=3.0, frames=120)
        sample = f"arm-like assembly 3x3x8-cell bones ({mesh.n_tets} tets, same construction), warm-started frames"
        return mesh, sample, BoneOracle(mesh, prm), \
            lambda o, a, F, tol, mx: o.solve(a, X0=F, tol=tol, max_newton=mx)
    if workload_name in ("mtu", "mtu_small", "serve"):
        mesh = muscle_tendon_unit(8, 8, 32, h=0.01, radius_cells=12.9 / 4, frames=60)
        sample = f"muscle-tendon unit 8x8x32 grid ({mesh.n_tets} tets, same construction), warm-started ramp frames"
    else:
        mesh = box_beam(4, 4, 16, activation=np.linspace(0.0, 0.5, 12))
        sample = "box beam 4x4x16, ramp frames"
    return mesh, sample, EmuOracle(mesh, prm), lambda o, a, F, tol, mx: o.solve(a, F0=F, tol=tol, max_newton=mx)


def cpu_baseline(workload_name, budget_s=15.0, ref_tol=1e-10):
    """FP64 oracle on a bounded sample of the workload (tet-iters/s).

    Returns the baseline entry and, for the parity figure of the line, the
    sample mesh, the frames it solved and the oracle's positions of the last
    of them re-converged (untimed) to ``ref_tol`` from its own state."""
    mesh, sample, o, solve = oracle_sample(workload_name)
    F = None
    t0, c0 = time.perf_counter(), time.process_time()
    tets_iters = 0
    frames = 0
    for f in range(1, mesh.activations.shape[0]):
        r = solve(o, mesh.activations[f], F, 1e-6, 5000)
        F = r.F
        tets_iters += mesh.n_tets * r.iterations
        frames += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = threads_used(time.process_time() - c0, dt)
    ref = None
    # a stiff assembly's FP64 floor can lie above ref_tol (weak activations)
    for tol in (ref_tol, 10 * ref_tol, 100 * ref_tol, 1000 * ref_tol):
        try:
            ref = solve(o, mesh.activations[frames], F, tol, 20000)
            ref_tol = tol
            break
        except RuntimeError:
            continue
    if ref is None:
        return cb_entry(tets_iters, dt, cores, sample, frames), None
    cb = cb_entry(tets_iters, dt, cores, sample, frames)
    return cb, {"mesh": mesh, "frames": frames, "q_ref": ref.q, "ref_tol": ref_tol, "sample": sample}


def cb_entry(tets_iters, dt, cores, sample, frames):
    return {"value": tets_iters / dt, "unit": "tet-iters/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample}; frames 1..{frames} ({tets_iters} tet-iters, {dt:.1f} s; "
                      f"{os.cpu_count()} host cores, {cores} busy on average)"}


def error_vs_oracle(emu, params, ref):
    """Positions of the GPU path (the bench's parameters) on the baseline's
    sample, frames 1..k warm-started as the oracle solved them, against the
    oracle's frame k: max over vertices of |q_gpu - q_oracle| over the rest
    bounding-box diagonal (the parity metric of the tests)."""
    mesh = ref["mesh"]
    s = emu.Solver(mesh, params)
    st = None
    for f in range(1, ref["frames"] + 1):
        s.set_activation(mesh.activations[f])
        st = s.solve(raise_on_error=False)
    q = s.positions()
    s.close()
    diag = float(np.linalg.norm(mesh.rest_pos.max(0) - mesh.rest_pos.min(0)))
    disp = float(np.abs(ref["q_ref"] - mesh.rest_pos).max())
    err = float(np.abs(q - ref["q_ref"]).max())
    return {"max_pos_err_rel_diag": err / diag, "max_pos_err_rel_disp": err / disp if disp > 0 else None,
            "bound_rel_diag": 1e-4 if params.precision == emu.PRECISION_MIXED else 1e-9,
            "gpu_rel_residual": float(st.rel_residual), "gpu_status": int(st.status),
            "oracle_tol": ref["ref_tol"], "frame": ref["frames"],
            "sample": f"{ref['sample']}; frame {ref['frames']} after warm-started frames 1..{ref['frames']}"}


def batch_desc(meshes, tol):
    return (f"batch of {len(meshes)} box beams, log-uniform 1k-60k tets "
            f"(sum {sum(mm.n_tets for mm in meshes)} tets), activation U[0,1], from rest, rel residual {tol:g}, "
            "one emu_batch_solve per step, one stream per mesh")


def serve_desc(args, n_requests):
    return (f"serving: first {n_requests} requests of a Poisson stream at {args.rate:g}/s, "
            "muscle-tendon units log-uniform 1k-200k tets, 1-30 frames, tendon U[0,0.2], "
            f"budget {args.budget_gb:g} GB, rel residual {args.tol:g}")


def run_reference(args, rank, world):
    """The oracle (FP64 CPU) as the reference arm: a step is one warm-started
    frame of a bounded sample of the workload (the same construction at
    6,080 tets for the muscle-tendon unit); W untimed frames, then K timed."""
    if rank != 0:
        return
    if args.workload == "batch":
        return run_reference_batch(args)
    mesh, sample, o, solve = oracle_sample(args.workload)
    if args.workload == "serve":
        desc = serve_desc(args, args.requests)
    else:
        _, desc = make_workload(args.workload)
    nf = mesh.activations.shape[0]
    F = None
    f = 1
    for _ in range(args.warmup):
        r = solve(o, mesh.activations[f], F, args.tol, 5000)
        F, f = r.F, f % (nf - 1) + 1
    t0, c0 = time.perf_counter(), time.process_time()
    tet_iters = 0
    for _ in range(args.steps):
        r = solve(o, mesh.activations[f], F, args.tol, 5000)
        F, f = r.F, f % (nf - 1) + 1
        tet_iters += mesh.n_tets * r.iterations
    dt = time.perf_counter() - t0
    value = tet_iters / dt
    cb = {"value": value, "unit": "tet-iters/s", "cores": threads_used(time.process_time() - c0, dt), "kind": "oracle",
          "sample": f"{sample}; {args.steps} timed frames after {args.warmup} warm-up frames "
                    f"({tet_iters} tet-iters, {dt:.1f} s)"}
    line = {"impl": "reference", "metric": "tet-iters/s", "value": value, "unit": "tet-iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "tet-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_batch(args):
    """Reference arm of the batch: a step is one mesh of the same 256-mesh set
    (in order, from rest), on the host cores."""
    from oracle import EmuOracle, OracleParams

    meshes = batch_set(count=args.meshes, seed=3)
    order = iter(range(len(meshes)))
    done, tet_iters, dt, cpu = 0, 0, 0.0, 0.0
    for phase, count in (("warmup", args.warmup), ("timed", args.steps)):
        for _ in range(count):
            k = next(order)
            mesh = meshes[k]
            t0, c0 = time.perf_counter(), time.process_time()
            r = EmuOracle(mesh, OracleParams(alpha_rel=1.0, weight_mode=0)).solve(
                mesh.activations[0], tol=args.tol, max_newton=5000)
            if phase == "timed":
                dt += time.perf_counter() - t0
                cpu += time.process_time() - c0
                tet_iters += mesh.n_tets * r.iterations
                done += 1
    value = tet_iters / dt if dt > 0 else 0.0
    cb = {"value": value, "unit": "tet-iters/s", "cores": threads_used(cpu, dt), "kind": "oracle",
          "sample": f"meshes {args.warmup}..{args.warmup + done - 1} of the batch set, from rest "
                    f"({tet_iters} tet-iters, {dt:.1f} s; setup and solve timed)"}
    line = {"impl": "reference", "metric": "tet-iters/s", "value": value, "unit": "tet-iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": batch_desc(meshes, args.tol)}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "tet-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_over_ranks(dist, maxes, sums, device="cuda"):
    """Whole-job totals of a replica run: the maximum over ranks of each entry
    of ``maxes`` (times) and the sum over ranks of each entry of ``sums``
    (units of work). Without a process group the local values come back."""
    if not dist:
        return [float(x) for x in maxes], [float(x) for x in sums]
    import torch

    t = torch.tensor([float(x) for x in maxes], device=device, dtype=torch.float64)
    u = torch.tensor([float(x) for x in sums], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.tolist(), u.tolist()


def make_params(emu, args, mixed):
    """Solver parameters of a bench leg: tolerance, precision and, with
    ``--ls-sigma0`` / ``--cg-degree``, the first line-search trial step and
    the local preconditioner degree of the dq solves (else the library's)."""
    p = emu.Params(tol_rel_residual=args.tol, precision=emu.PRECISION_MIXED if mixed else emu.PRECISION_FP64)
    if args.ls_sigma0 is not None:
        p.ls_sigma0 = args.ls_sigma0
    if args.cg_degree is not None:
        p.cg_local_degree = args.cg_degree
    if getattr(args, "form", "rs") == "f":
        p.form = emu.FORM_F
    if getattr(args, "autotune", False):
        p.autotune = 1
    return p


def _finish_line(line, rank, dist):
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batch(args, emu, torch, rank, world, dist):
    """Independent box beams of log-uniform size (1k-60k tets, activation
    U[0, 1]), all solved together by emu_batch_solve, each mesh on its own
    stream. A step resets every mesh to rest and solves the batch once; the
    host clock spans the whole batch (synchronized on both sides)."""
    meshes = batch_set(count=args.meshes, seed=3)
    mixed = args.precision == "mixed"
    params = make_params(emu, args, mixed)
    t_setup = time.perf_counter()
    streams, solvers = [], []
    for mesh in meshes:
        st = torch.cuda.Stream()
        s = emu.Solver(mesh, params, stream=st.cuda_stream)
        s.set_activation(mesh.activations[0])
        streams.append(st)
        solvers.append(s)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    m_each = np.array([mm.n_tets for mm in meshes], dtype=np.float64)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")

    def step():
        for s in solvers:
            s.reset()
        for s, mesh in zip(solvers, meshes):
            s.set_activation(mesh.activations[0])
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = emu.batch_solve(solvers, raise_on_error=False)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, stats

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    times, tet_iters, iters, resid, failed = [], 0.0, [], [], []
    for _ in range(args.steps):
        dt, stats = step()
        times.append(dt)
        its = np.array([st.newton_iters for st in stats], dtype=np.float64)
        tet_iters += float((m_each * its).sum())
        iters.append(int(its.sum()))
        ok = [st for st in stats if st.status == 0]
        resid.append(max(st.rel_residual for st in ok) if ok else float("nan"))
        failed.append([{"mesh": k, "tets": int(m_each[k]), "activation": float(meshes[k].activations[0][0]),
                        "status": int(st.status), "newton_iters": int(st.newton_iters),
                        "rel_residual": float(st.rel_residual)} for k, st in enumerate(stats) if st.status != 0])
    clk = clocks.stop()
    (total,), (tet_iters_job,) = reduce_over_ranks(dist, [float(np.sum(times))], [tet_iters])
    value = tet_iters_job / total
    line = {
        "metric": "tet-iters/s", "value": value, "unit": "tet-iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": batch_desc(meshes, args.tol),
                   "precision": args.precision, "l2": "inputs larger than L2; flushed between steps",
                   "tets": int(m_each.sum()), "meshes": len(meshes), "ls_sigma0": params.ls_sigma0, "cg_local_degree": params.cg_local_degree},
        "newton_iters_per_step": iters, "max_rel_residual_converged": float(np.max(resid)),
        "not_converged": failed[-1], "setup_s": setup_s,
        "roofline": None, "cpu_baseline": None,
        "e2e": {"value": value, "unit": "tet-iters/s", "h2d_bytes_per_step": int(8 * m_each.sum()), "d2h_bytes_per_step": 0},
        "clocks": clk,
    }
    for s in solvers:
        s.close()
    _finish_line(line, rank, dist)


def run_serve(args, emu, torch, rank, world, dist):
    """Poisson stream of quasi-static requests (muscle-tendon units of 1k to
    200k tets, 1-30 frames each, tendon fraction U[0, 0.2]) submitted at their
    arrival times to one emu_server with a device-memory budget; reports the
    sustained tet-iters/s over the makespan and p50/p99 request latency."""
    reqs = request_stream(rate_hz=args.rate, seed=4, max_requests=args.requests)
    built = []
    for r in reqs:
        mesh = mtu_for_tet_count(r["tets"], tendon_frac=r["tendon_frac"], seed=r["seed"])
        muscle = (mesh.material_id == 0).astype(np.float64)
        fr = r["frames"]
        acts = np.stack([muscle * r["a_max"] * (f + 1) / fr for f in range(fr)])
        built.append((r, mesh, acts))
    mixed = args.precision == "mixed"
    params = make_params(emu, args, mixed)
    srv = emu.Server(int(args.budget_gb * (1 << 30)), params)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    pending = list(built)
    results = {}
    done_at = {}
    while len(results) < len(built):
        now = time.perf_counter() - t0
        while pending and pending[0][0]["arrival_s"] - reqs[0]["arrival_s"] <= now:
            r, mesh, acts = pending.pop(0)
            srv.submit(mesh, acts, r["id"])
        for i in srv.poll():
            results[i] = srv.result(i)
            done_at[i] = time.perf_counter() - t0
        time.sleep(0.0005)
    makespan = max(done_at.values())
    clk = clocks.stop()
    srv.close()
    tet_iters = 0.0
    lat, bad = [], 0
    by_id = {r["id"]: (r, mesh) for r, mesh, _ in built}
    for i, (q, st) in results.items():
        r, mesh = by_id[i]
        tet_iters += float(mesh.n_tets) * st.newton_iters
        lat.append(st.latency_ms)
        bad += int(st.status != 0)
    (makespan,), (tet_iters_job,) = reduce_over_ranks(dist, [makespan], [tet_iters])
    value = tet_iters_job / makespan
    line = {
        "metric": "tet-iters/s", "value": value, "unit": "tet-iters/s", "n_gpus": world, "steps": len(built),
        "warmup": 0, "ms_per_step": 1e3 * makespan / len(built), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": serve_desc(args, len(built)),
                   "precision": args.precision, "requests": len(built), "ls_sigma0": params.ls_sigma0,
                   "tets_mean": float(np.mean([mm.n_tets for _, mm, _ in built]))},
        "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
        "failed_requests": bad, "makespan_s": makespan,
        "roofline": None, "cpu_baseline": None,
        "e2e": {"value": value, "unit": "tet-iters/s",
                "h2d_bytes_per_step": int(np.mean([8 * a.size for _, _, a in built])),
                "d2h_bytes_per_step": int(np.mean([24 * mm.n_verts * a.shape[0] for _, mm, a in built]))},
        "clocks": clk,
    }
    _finish_line(line, rank, dist)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mtu", choices=["mtu", "box", "mtu_small", "arm", "batch", "serve"])
    ap.add_argument("--meshes", type=int, default=256, help="batch: number of meshes")
    ap.add_argument("--requests", type=int, default=24, help="serve: requests taken from the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate (1/s)")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: device-memory budget")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--autotune", action="store_true",
                    help="let the library time and pick the coupling solves' launch settings at set-up")
    ap.add_argument("--form", default="rs", choices=["rs", "f"],
                    help="Newton variables: rotation-stretch chart (rs) or the F-form of Sec. 3.2.1 (f, FP64 only)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--ls-sigma0", type=float, default=None,
                    help="first line-search trial step (default: the library's, 4)")
    ap.add_argument("--cg-degree", type=int, default=None,
                    help="degree of the block-local polynomial in the dq solves' preconditioner (default: the library's, 4)")
    args = ap.parse_args()
    if args.form == "f" and args.precision != "fp64":
        ap.error("--form f runs in FP64: add --precision fp64")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    cb, cb_ref = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, cb_ref = cpu_baseline(args.workload)  # before any GPU work (no fork after CUDA init)

    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2006_08821_gb300 import build as b

    b.build()
    import paper_2006_08821_gb300 as emu

    if args.workload == "batch":
        return run_batch(args, emu, torch, rank, world, dist)
    if args.workload == "serve":
        return run_serve(args, emu, torch, rank, world, dist)
    mesh, desc = make_workload(args.workload)
    frames = mesh.activations.shape[0]
    n_prof = 2  # profiled frames after the timed ones (per-phase CUDA events)
    if args.warmup + args.steps + n_prof > frames - 1:
        raise SystemExit(f"workload has {frames} frames; warmup + steps must be <= {frames - 1 - n_prof}")
    mixed = args.precision == "mixed"
    stream = torch.cuda.Stream()
    params = make_params(emu, args, mixed)
    t_setup = time.perf_counter()
    solver = emu.Solver(mesh, params, stream=stream.cuda_stream, allocator=emu.TorchAllocator(local))
    setup_s = time.perf_counter() - t_setup
    tuning = solver.tuning()
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    m, n = mesh.n_tets, mesh.n_verts

    # warm-up frames 1..W (frame 0 is the unloaded state)
    for f in range(1, 1 + args.warmup):
        solver.set_activation(mesh.activations[f])
        solver.solve()
    solver.set_profiling(False)  # profiling off; zeroes the launch counter
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    frame_ms, e2e_s, iters, resid, cg = [], [], [], [], []
    act_pinned = torch.empty(m, dtype=torch.float64).pin_memory()
    for f in range(1 + args.warmup, 1 + args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        act_pinned.numpy()[:] = mesh.activations[f]
        t0 = time.perf_counter()
        solver.set_activation(act_pinned.numpy())
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = solver.solve()
        e1.record(stream)
        q = solver.positions()
        t1 = time.perf_counter()
        e1.synchronize()
        frame_ms.append(e0.elapsed_time(e1))
        e2e_s.append(t1 - t0)
        iters.append(st.newton_iters)
        resid.append(st.rel_residual)
        cg.append(st.pcg_iters)
    torch.cuda.synchronize()
    clk = clocks.stop()
    _, launches = solver.profile()  # kernels the library launched in the timed frames
    # per-phase device times: the library's CUDA events on the solver's
    # stream, on the next frames (profiling replaces the per-iteration CUDA
    # graph by direct launches, so it stays out of the timed frames)
    solver.set_profiling(True)
    prof_its = 0
    prof_cg = 0
    for f in range(1 + args.warmup + args.steps, 1 + args.warmup + args.steps + n_prof):
        solver.set_activation(mesh.activations[f])
        st = solver.solve()
        prof_its += st.newton_iters
        prof_cg += st.pcg_iters
    torch.cuda.synchronize()
    prof, _ = solver.profile()
    (total_ms, total_e2e), (tet_iters,) = reduce_over_ranks(
        dist, [float(np.sum(frame_ms)), float(np.sum(e2e_s))], [float(m * np.sum(iters))])
    value = tet_iters / (total_ms / 1e3)
    e2e_value = tet_iters / total_e2e

    # roofline (device times from the library's per-phase CUDA events on the
    # solver's stream, profiled frames)
    peak, peak_kind = hbm_peak()
    nnz = solver_nnz(mesh)
    cg_per_iter = prof_cg / max(prof_its, 1)
    dev_ms = sum(v[0] for v in prof.values())
    fform = args.form == "f"
    per_tet = per_tet_fractions(prof, mixed, m, n, nnz, peak,
                                NCU_TRAFFIC if (mixed and args.workload == "mtu") else {}, fform)
    roof = dominant_roofline(prof, mixed, m, n, nnz, float(prof_cg), peak, peak_kind,
                             NCU_TRAFFIC if (mixed and args.workload == "mtu") else {}, fform)
    whole = whole_iteration(prof, mixed, m, n, nnz, float(prof_cg), prof_its, peak, value, fform)
    err = None
    if cb_ref is not None:
        err = error_vs_oracle(emu, params, cb_ref)
    line = {
        "metric": "tet-iters/s", "value": value, "unit": "tet-iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": desc, "precision": args.precision, "l2": f"flushed ({args.flush_mb} MB write) between steps",
                   "tets": m, "verts": n, "ls_sigma0": params.ls_sigma0, "cg_local_degree": params.cg_local_degree,
                   "form": args.form, "tuning": tuning},
        "ms_per_converged_frame_p50": float(np.median(frame_ms)),
        "frame_ms_p99": float(np.percentile(frame_ms, 99)),
        "newton_iters_per_frame": [int(x) for x in iters],
        "cg_iters_per_frame": [int(x) for x in cg],
        "max_rel_residual": float(np.max(resid)),
        "setup_s": setup_s,
        "phase_us_per_newton_iter": {k: round(1e3 * v[0] / max(prof_its, 1), 1) for k, v in prof.items()},
        "phase_launches": {k: v[1] for k, v in prof.items()},
        "phase_source": f"{n_prof} profiled frames after the timed ones ({prof_its} Newton iterations)",
        "roofline": roof,
        "per_tet_kernels_hbm": per_tet,
        "whole_iteration": whole,
        "cg_iters_per_newton_iter": round(cg_per_iter, 2),
        "error_vs_oracle": err,
        "cpu_baseline": cb,
        "e2e": {"value": e2e_value, "unit": "tet-iters/s", "h2d_bytes_per_step": 8 * m, "d2h_bytes_per_step": 24 * n},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
