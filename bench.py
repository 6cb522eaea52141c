#!/usr/bin/env python
"""Benchmark of the tangent-point hot path on one GB300 (or N replicas).

One step = one pass of the whole hot path on the 20,000-face torus
(R=1, r=0.3, 200 x 50 grid, N(0, 0.005^2) noise), starting from the same
seeded positions every step:
  face geometry -> constrained preconditioned descent step (direct FP32
  pair terms for E, dE, A = B + B0 and L^{2-s} inside flexible GMRES,
  cotan CG solves, FP64 Schur complement, Armijo line search, corrective
  projection) -> Barnes-Hut (theta = 0.5) energy and differential.

Metric: pair interactions per second (every evaluated (target, source face)
or (target, BVH node) term of the step), plus steps/s and step latency.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "torus_20k"
METRIC = "pair interactions/s"
UNIT = "pairs/s"
# algorithmic FP32 flops per pair interaction (FMA = 2, MUFU not counted);
# operator applies: kernel evaluation + 2 per accumulator, KC columns per launch
FLOPS_PER_PAIR = {"energy_direct": 20, "diff_direct": 57, "bh_energy": 20, "bh_diff": 51}
# static-obstacle pair (surface face, obstacle face) with its gradient: d (3), |d|^2 (5),
# |d|^-6 (2), times a (1), sum (1), |d|^-8 a (1), 3 gradient FMAs (6)
OBSTACLE_FLOPS_PER_PAIR = 19
APPLY_FLOPS = {"apply_A": lambda kc: 26 + 2 * (2 + 4 * kc), "apply_B": lambda kc: 9 + 2 * (1 + 3 * kc),
               "apply_B0": lambda kc: 26 + 2 * (1 + kc), "apply_L": lambda kc: 9 + 2 * (1 + kc)}


def flops_per_pair(name, stat):
    if name in FLOPS_PER_PAIR:
        return FLOPS_PER_PAIR[name]
    if name in APPLY_FLOPS:
        kc = stat.get("columns", 0.0) / max(1, stat["launches"]) or 3.0
        return APPLY_FLOPS[name](kc)
    return None
KERNEL_SOURCE = {"energy_direct": "pairs.cu", "diff_direct": "pairs.cu", "apply_A": "pairs.cu",
                 "apply_B": "pairs.cu", "apply_B0": "pairs.cu", "apply_L": "pairs.cu",
                 "bh_energy": "bvh.cu", "bh_diff": "bvh.cu", "bh_apply": "pairs.cu", "cg": "cg.cu",
                 "bvh_build": "bvh.cu",
                 "chol_factor": "chol.cu", "chol_solve": "chol.cu", "obstacle_direct": "obstacle.cu",
                 "bh_obstacle": "obstacle.cu"}
FP32_LANES_PER_SM = 128


def step_params(tp):
    """The timed step: FP32 pair terms, flexible GMRES to 1e-5 on the exact
    operator, the preconditioner's Poisson solves to 1e-4 (inside flexible
    GMRES they are preconditioner applications: their accuracy moves the
    iteration count, not the converged direction; 27 iterations on torus_20k
    at 1e-4 as at 1e-6), and an Armijo line search whose first trial moves no
    vertex by more than a quarter of the mean face size (tau0_disp = 0.25)."""
    return tp.params(theta=0.0, precision=tp.TP_PREC_FP32, krylov_tol=1e-5, krylov_max=60,
                     gmres_restart=30, cg_tol=1e-4, cg_max=20000, proj_iters=1, tau0_disp=0.25)


def bh_params(tp):
    return tp.params(theta=0.5, precision=tp.TP_PREC_FP32, leaf_size=8)


# ---------------------------------------------------------------------------
# CPU side: the oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------

def sample_desc(scale, procs=1):
    per = "per process, " if procs > 1 else ""
    return (f"oracle (numpy FP64) on {WORKLOAD}, {procs} process(es) with 1 thread each; {per}energy rows of "
            f"{32 * scale} target faces, dE at {3 * scale} vertices, A.u and L.u at {3 * scale} vertices each; "
            "pairs = rows evaluated x (nf - 1)")


def oracle_timed_loop(scale, seed, warm, reps, start_at):
    """Reference arm, one process: `warm` untimed samples, then from the
    wall-clock time start_at `reps` timed ones; returns (pairs, start, end)."""
    for _ in range(warm):
        oracle_sample_pairs_per_s(scale, seed)
    time.sleep(max(0.0, start_at - time.time()))
    pairs, w0, w1 = 0.0, None, None
    for k in range(reps):
        r = oracle_sample_pairs_per_s(scale, seed + 1000 * (k + 1))
        pairs += r[2]
        w0 = r[3] if w0 is None else w0
        w1 = r[4]
    return pairs, w0, w1


def oracle_sample_pairs_per_s(scale, seed=4242, start_at=None):
    """Run in a subprocess with single-threaded BLAS; returns (pairs/s,
    seconds, pairs, start, end) with start/end on the wall clock (time.time);
    with start_at the work waits until that wall-clock time, so that
    concurrent processes compute over the same window."""
    import numpy as np
    from oracle import tp_oracle as O
    from synth import vertex_vectors, workload
    V, F = workload(WORKLOAD)
    nf = len(F)
    rng = np.random.default_rng(seed)
    targets = rng.choice(nf, 32 * scale, replace=False)
    nvs = 3 * scale
    verts = rng.choice(len(V), 3 * nvs, replace=False)
    u = vertex_vectors(len(V), 3, 202)
    if start_at is not None:
        time.sleep(max(0.0, start_at - time.time()))
    w0 = time.time()
    t0 = time.perf_counter()
    O.energy_rows(V, F, 6.0, targets)
    O.differential_at_vertices(V, F, verts[:nvs])
    O.apply_operator_at_vertices(V, F, u, "A", verts[nvs:2 * nvs])
    O.apply_operator_at_vertices(V, F, u, "L", verts[2 * nvs:])
    dt = time.perf_counter() - t0
    w1 = time.time()

    def inc_rows(vs):
        return len(np.unique(np.concatenate([np.nonzero(np.any(F == v, axis=1))[0] for v in vs])))
    rows = len(targets) + inc_rows(verts[:nvs]) + inc_rows(verts[nvs:2 * nvs]) + inc_rows(verts[2 * nvs:])
    pairs = float(rows) * (nf - 1)
    return pairs / dt, dt, pairs, w0, w1


def _oracle_procs(scale, procs):
    """procs concurrent single-threaded oracle processes (different seeded
    samples of the same workload); returns (summed pairs / wall seconds,
    wall seconds)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    # every process loads its inputs first and starts computing at the same
    # wall-clock time; the window is from that time to the last process's end
    start_at = time.time() + 4.0 + 0.25 * procs
    cmds = []
    for i in range(procs):
        code = ("import json,sys; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.oracle_sample_pairs_per_s(%d, %d, %r)))"
                % (ROOT, scale, 4242 + i, start_at if procs > 1 else None))
        cmds.append([sys.executable, "-c", code])
    ps = [subprocess.Popen(c, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for c in cmds]
    pairs, w0, w1 = 0.0, [], []
    for pr in ps:
        out, err = pr.communicate(timeout=900)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        r = json.loads(out.strip().splitlines()[-1])
        pairs += r[2]
        w0.append(r[3])
        w1.append(r[4])
    wall = max(w1) - min(w0)
    return pairs / wall, wall


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_cpu_sample(scale=48, all_scale=6):
    """The oracle on the host cores: one single-threaded process, and one
    single-threaded process per core at once (the all-cores figure is the
    reported value)."""
    v1, dt1 = _oracle_procs(scale, 1)
    n = host_cores()
    vn, dtn = _oracle_procs(all_scale, n)
    return {"value": vn, "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample_desc(all_scale, n),
            "seconds": round(dtn, 2),
            "single_thread": {"value": v1, "cores": 1, "sample": sample_desc(scale), "seconds": round(dt1, 2)}}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def profile_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary of this kernel, or
    None when the summary is missing or the kernel's source changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2107_01664_gb300", "csrc", KERNEL_SOURCE.get(kernel, ""))
    if not os.path.exists(src) or "source_sha256" not in vals or "dram_bytes_per_launch" not in vals:
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != vals["source_sha256"]:
        return None
    return float(vals["dram_bytes_per_launch"])


# ---------------------------------------------------------------------------
# large single mesh: Barnes-Hut on the 1,310,720-face icosphere
# ---------------------------------------------------------------------------

def fp32_peak_tflops(dev):
    import torch
    peaks, _ = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz"


def kernel_roofline(name, stat, flops_per_unit, workload, dev, bytes_per_unit=None):
    """Roofline of one kernel class from its profile statistics: FP32
    TFLOP/s against the FP32 peak (ALU-bound pair kernels) or GB/s against
    the measured HBM copy bandwidth (bytes_per_unit given); DRAM bytes per
    launch from the committed ncu summary of this kernel and workload."""
    n = max(1, stat["launches"])
    ms = stat["ms"] / n
    units = stat["units"] / n
    peaks, src = measured_peaks()
    tr = profile_traffic(name, workload)
    out = {"ms_per_launch": ms, "units_per_launch": units, "per_s": units / (ms / 1e3) if ms > 0 else None,
           "launches": stat["launches"], "traffic": tr}
    if ms <= 0:
        return out
    if bytes_per_unit is None:
        peak, basis = fp32_peak_tflops(dev)
        ach = flops_per_unit * units / (ms / 1e3) / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "peak_basis": basis})
    else:
        peak = float(peaks.get("hbm_gbs", 6800.0))
        ach = bytes_per_unit * units / (ms / 1e3) / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "peak_basis": f"hbm_gbs ({src})"})
    if tr is not None:
        out["dram_gbs"] = tr / (ms / 1e3) / 1e9
    return out


def large_mesh(tp, dev, reps=3):
    """The 1,310,720-face icosphere with spherical-harmonic bumps: Barnes-Hut
    (theta = 0.5, leaf 8) E, dE and A v (3 columns) in FP32 with their
    rooflines; their errors against stored FP64 direct sums of the oracle
    (energy rows at 20,000 seeded target faces, dE and A u at 64 seeded
    vertices; tests/golden/make_l8_samples.py); the FP32 direct rows of the
    same 20,000 targets; the Poisson solve of the preconditioner (9 columns,
    cg_tol 1e-6) with its HBM throughput; one direct all-pairs energy."""
    import numpy as np
    import torch
    from synth import vertex_vectors, workload
    t_start = time.perf_counter()
    V, F = workload("icosphere_l8")
    smp = json.load(open(os.path.join(ROOT, "tests", "golden", "icosphere_l8_samples.json")))
    mesh = tp.Mesh(torch.tensor(V, dtype=torch.float64, device=dev),
                   torch.tensor(F, dtype=torch.int32, device=dev), device=dev.index or 0)
    pb = bh_params(tp)
    dE = torch.empty((len(V), 3), dtype=torch.float64, device=dev)
    v3 = torch.tensor(vertex_vectors(len(V), 3, 507), dtype=torch.float64, device=dev)
    tp.tp_energy(mesh, pb)
    tp.tp_differential(mesh, pb, like=dE)
    tp.fractional_apply(mesh, "A", v3, pb)
    torch.cuda.synchronize()
    tp.tp_profile_read(mesh)
    tp.tp_profile_enable(mesh, True)
    for _ in range(reps):
        tp.tp_mesh_set_positions(mesh, torch.tensor(V, dtype=torch.float64, device=dev))  # rebuilds the BVH
        E_bh = tp.tp_energy(mesh, pb)
        g_bh, _ = tp.tp_differential(mesh, pb, like=dE)
        Au_bh = tp.fractional_apply(mesh, "A", v3, pb)
    torch.cuda.synchronize()
    prof = tp.tp_profile_read(mesh)
    out = {"workload": "icosphere_l8", "nf": int(len(F)), "nv": int(len(V)), "theta": pb.theta,
           "leaf_size": pb.leaf_size, "dtype": "f32"}
    for k, fl in (("bh_energy", FLOPS_PER_PAIR["bh_energy"]), ("bh_diff", FLOPS_PER_PAIR["bh_diff"]),
                  ("bh_apply", APPLY_FLOPS["apply_A"](3)), ("bvh_build", None)):
        if k in prof and prof[k]["launches"]:
            out[k] = kernel_roofline(k, prof[k], fl or 0.0, "icosphere_l8", dev) if fl else \
                {"ms_per_launch": prof[k]["ms"] / prof[k]["launches"]}
    bh_ms = sum(prof[k]["ms"] / prof[k]["launches"] for k in ("bh_energy", "bh_diff", "bh_apply") if k in prof)
    bh_units = sum(prof[k]["units"] / prof[k]["launches"] for k in ("bh_energy", "bh_diff", "bh_apply") if k in prof)
    out["bh_E_dE_Av"] = {"ms": bh_ms, "interactions": bh_units,
                         "interactions_per_s": bh_units / (bh_ms / 1e3) if bh_ms > 0 else None}
    # accuracy against the stored FP64 direct sums
    rel = lambda a, b: float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))
    mx = lambda a, b: float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())
    tg = torch.tensor(np.array(smp["targets"], dtype=np.int32), device=dev)
    rows_ref = np.array(smp["rows"])
    rows_bh = tp.tp_energy_rows(mesh, tg, pb).cpu().numpy()
    tp.tp_profile_read(mesh)
    rows_d = tp.tp_energy_rows(mesh, tg, tp.params()).cpu().numpy()
    pd = tp.tp_profile_read(mesh)
    vi = np.array(smp["vertices"])
    g_h = g_bh.cpu().numpy()[vi]
    a_h = Au_bh.cpu().numpy()[vi]
    out["accuracy_vs_fp64_direct"] = {
        "reference": "oracle FP64 direct sums (stored): energy rows at 20,000 targets, dE and A u at 64 vertices",
        "bh_theta_0.5": {"rows": rel(rows_bh, rows_ref), "rows_max": mx(rows_bh, rows_ref),
                         "dE": rel(g_h, smp["dE"]), "Au": rel(a_h, smp["Au"])},
        "fp32_direct": {"rows": rel(rows_d, rows_ref), "rows_max": mx(rows_d, rows_ref)},
        "E_bh": E_bh}
    if "energy_direct" in pd and pd["energy_direct"]["launches"]:
        out["direct_rows_20k"] = kernel_roofline("energy_direct", pd["energy_direct"],
                                                 FLOPS_PER_PAIR["energy_direct"], "icosphere_l8", dev)
    # Poisson solve of the preconditioner on 655,362 vertices
    info = tp.cotan_factor_info(mesh)
    b = torch.tensor(vertex_vectors(len(V), 9, 508), dtype=torch.float64, device=dev)
    tp.cotan_solve(mesh, b, tp.params(cg_tol=1e-6))
    torch.cuda.synchronize()
    tp.tp_profile_read(mesh)
    z, iters = tp.cotan_solve(mesh, b, tp.params(cg_tol=1e-6))
    torch.cuda.synchronize()
    pp = tp.tp_profile_read(mesh)
    key = "chol_solve" if ("chol_solve" in pp and pp["chol_solve"]["launches"]) else "cg"
    poisson = {"solver": "sparse Cholesky + FP64 refinement" if key == "chol_solve" else "Jacobi CG (FP64)",
               "factor_available": bool(info["available"]), "columns": 9, "cg_tol": 1e-6, "iterations": iters}
    if key in pp and pp[key]["ms"] > 0:
        d = pp[key]
        poisson.update({"ms": d["ms"], "bytes": d["units"],
                        "achieved_gbs": d["units"] / (d["ms"] / 1e3) / 1e9,
                        "hbm_peak_gbs": float(measured_peaks()[0].get("hbm_gbs", 6800.0))})
        poisson["frac"] = poisson["achieved_gbs"] / poisson["hbm_peak_gbs"]
    out["poisson_solve"] = poisson
    # one direct all-pairs energy (FP32)
    tp.tp_profile_read(mesh)
    tp.tp_energy(mesh, tp.params())
    torch.cuda.synchronize()
    pe = tp.tp_profile_read(mesh)
    if "energy_direct" in pe:
        out["energy_direct_all_pairs"] = kernel_roofline("energy_direct", pe["energy_direct"],
                                                         FLOPS_PER_PAIR["energy_direct"], "icosphere_l8", dev)
    tp.tp_profile_enable(mesh, False)
    mesh.close()
    out["bh_step_linked_tori"] = bh_step(tp, dev)
    out["section_s"] = round(time.perf_counter() - t_start, 1)
    return out


def obstacle_scene(tp, dev, reps=5, steps=2):
    """Static-obstacle term (§7.3.2) on torus_20k around the 20,480-face ball
    in its hole: device time of the direct FP32 energy + differential (all
    20,000 x 20,480 pairs), of the Barnes-Hut one (theta = 0.5, leaf 8), and
    of constrained steps whose energy includes the obstacle term."""
    import numpy as np
    import torch
    from synth import obstacle, workload
    V, F = workload(WORKLOAD)
    VO, FO = obstacle("ball_in_torus_hole")
    f0 = torch.tensor(V, dtype=torch.float64, device=dev)
    mesh = tp.Mesh(f0, torch.tensor(F, dtype=torch.int32, device=dev), device=dev.index or 0)
    tp.tp_obstacle_set(mesh, torch.tensor(VO, dtype=torch.float64, device=dev),
                       torch.tensor(FO, dtype=torch.int32, device=dev), 1.0)
    dE = torch.empty((len(V), 3), dtype=torch.float64, device=dev)
    pd, pb = tp.params(), bh_params(tp)
    tp.tp_obstacle_energy(mesh, pd, like=dE)
    tp.tp_obstacle_energy(mesh, pb, like=dE)
    torch.cuda.synchronize()
    tp.tp_profile_read(mesh)
    tp.tp_profile_enable(mesh, True)
    E = Eb = None
    for _ in range(reps):
        E, _ = tp.tp_obstacle_energy(mesh, pd, like=dE)
        Eb, _ = tp.tp_obstacle_energy(mesh, pb, like=dE)
    torch.cuda.synchronize()
    prof = tp.tp_profile_read(mesh)
    tp.tp_profile_enable(mesh, False)
    out = {"workload": "torus_20k+ball_in_torus_hole", "nf": int(len(F)), "nf_obstacle": int(len(FO)),
           "E_direct": E, "E_bh": Eb}
    for k in ("obstacle_direct", "bh_obstacle"):
        if k in prof and prof[k]["launches"]:
            d = prof[k]
            n = d["launches"]
            out[k] = {"ms_per_launch": d["ms"] / n, "units_per_launch": d["units"] / n,
                      "per_s": d["units"] / (d["ms"] / 1e3) if d["ms"] > 0 else None}
    if "obstacle_direct" in out and prof["obstacle_direct"]["ms"] > 0:
        d = prof["obstacle_direct"]
        peaks, _ = measured_peaks()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        tfl = OBSTACLE_FLOPS_PER_PAIR * d["units"] / (d["ms"] / 1e3) / 1e12
        out["obstacle_direct"]["tflops"] = tfl
        out["obstacle_direct"]["frac_of_fp32_peak"] = tfl / peak
    # constrained steps on E + E_O (direct pairs, the benchmark's step settings)
    A0 = float(np.sum(0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)))
    Vol0 = float(np.sum(V[F[:, 0]] * np.cross(V[F[:, 1]], V[F[:, 2]])) / 6.0)
    cons = tp.tp_constraints(flags=tp.TP_CONSTRAINT_AREA | tp.TP_CONSTRAINT_VOLUME, A0=A0, V0=Vol0)
    ps = step_params(tp)
    tp.precond_step(mesh, cons, ps)
    tp.tp_mesh_set_positions(mesh, f0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps_ = []
    e0.record()
    for _ in range(steps):
        tp.tp_mesh_set_positions(mesh, f0)
        reps_.append(tp.precond_step(mesh, cons, ps))
    e1.record()
    torch.cuda.synchronize()
    mesh.close()
    out["step"] = {"ms_per_step": e0.elapsed_time(e1) / steps,
                   "E_before": reps_[0]["E_before"], "E_after": reps_[0]["E_after"],
                   "tau": reps_[0]["tau"], "status": [r["status"] for r in reps_]}
    return out


def pinned_steps(tp, dev, steps=2):
    """Vertex pins as fast positional constraints (§7.1.2, §7.2): constrained
    steps on torus_20k with 8 pinned vertices (the benchmark's step settings),
    and the Krylov iterations to krylov_tol on the smooth torus (no noise)
    with the barycenter constraint and with the pins."""
    import numpy as np
    import torch
    from synth import torus, workload
    pins = np.arange(0, 10000, 1250, dtype=np.int32)

    def cons_of(V, F):
        A0 = float(np.sum(0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)))
        Vol0 = float(np.sum(V[F[:, 0]] * np.cross(V[F[:, 1]], V[F[:, 2]])) / 6.0)
        return tp.tp_constraints(flags=tp.TP_CONSTRAINT_AREA | tp.TP_CONSTRAINT_VOLUME, A0=A0, V0=Vol0)

    V, F = workload(WORKLOAD)
    cons = cons_of(V, F)
    ps = step_params(tp)
    f0 = torch.tensor(V, dtype=torch.float64, device=dev)
    mesh = tp.Mesh(f0, torch.tensor(F, dtype=torch.int32, device=dev), device=dev.index or 0)
    tp.tp_pins_set(mesh, pins)
    tp.precond_step(mesh, cons, ps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = []
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        tp.tp_mesh_set_positions(mesh, f0)
        reps.append(tp.precond_step(mesh, cons, ps))
    e1.record()
    torch.cuda.synchronize()
    f = tp.tp_mesh_get_positions(mesh)
    mesh.close()
    out = {"workload": "torus_20k", "pins": int(len(pins)), "ms_per_step": e0.elapsed_time(e1) / steps,
           "krylov_iters_per_step": sum(r["krylov_iters"] for r in reps) / steps,
           "pins_moved": bool(np.any(f[pins] != V[pins])), "status": [r["status"] for r in reps]}
    # Krylov iterations to tolerance on the smooth torus
    Vs, Fs = torus(200, 50, 1.0, 0.3)
    cs = cons_of(Vs, Fs)
    pt = tp.params(krylov_tol=1e-5, krylov_max=400, cg_tol=1e-6)
    its = {}
    for name, pv in (("barycenter", None), ("pins", pins)):
        m2 = tp.Mesh(torch.tensor(Vs, dtype=torch.float64, device=dev),
                     torch.tensor(Fs, dtype=torch.int32, device=dev), device=dev.index or 0)
        if pv is not None:
            tp.tp_pins_set(m2, pv)
        r = tp.precond_step(m2, cs, pt)
        its[name] = {"krylov_iters": r["krylov_iters"], "status": r["status"]}
        m2.close()
    out["smooth_torus_krylov"] = its
    return out


def willmore_steps(tp, dev, steps=2, weight=100.0):
    """Willmore term (§7.3.5) on torus_20k: device time of E_W + dE_W, and
    constrained steps minimising E + w E_W with the H^2 term in the operator
    (w = 100 makes w E_W about a sixth of E on this mesh)."""
    import numpy as np
    import torch
    from synth import workload
    V, F = workload(WORKLOAD)
    A0 = float(np.sum(0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)))
    Vol0 = float(np.sum(V[F[:, 0]] * np.cross(V[F[:, 1]], V[F[:, 2]])) / 6.0)
    cons = tp.tp_constraints(flags=tp.TP_CONSTRAINT_AREA | tp.TP_CONSTRAINT_VOLUME, A0=A0, V0=Vol0)
    f0 = torch.tensor(V, dtype=torch.float64, device=dev)
    mesh = tp.Mesh(f0, torch.tensor(F, dtype=torch.int32, device=dev), device=dev.index or 0)
    dE = torch.empty((len(V), 3), dtype=torch.float64, device=dev)
    EW, _ = tp.tp_willmore_energy(mesh, like=dE)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        tp.tp_willmore_energy(mesh, like=dE)
    e1.record()
    torch.cuda.synchronize()
    ew_ms = e0.elapsed_time(e1) / 10
    tp.tp_willmore_set(mesh, weight)
    ps = step_params(tp)
    tp.precond_step(mesh, cons, ps)
    reps = []
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        tp.tp_mesh_set_positions(mesh, f0)
        reps.append(tp.precond_step(mesh, cons, ps))
    e1.record()
    torch.cuda.synchronize()
    mesh.close()
    return {"workload": "torus_20k", "weight": weight, "E_W": EW, "E_W_and_dE_W_ms": ew_ms,
            "ms_per_step": e0.elapsed_time(e1) / steps,
            "krylov_iters_per_step": sum(r["krylov_iters"] for r in reps) / steps,
            "E_before": reps[0]["E_before"], "E_after": reps[0]["E_after"], "status": [r["status"] for r in reps]}


def tensor_core_apply(tp, dev, reps=5):
    """The 9-column A apply on torus_20k with its accumulation on tcgen05
    tensor cores (tensor_cores = 1: split TF32 products, FP32 accumulators in
    tensor memory, compensated read-back every 128 sources) beside the
    CUDA-core kernel (the step's default): kernel time per launch, the
    algorithmic FP32 rate (102 flop per pair, as apply_A), and the relative
    difference of the two results."""
    import numpy as np
    import torch
    from synth import vertex_vectors, workload
    V, F = workload(WORKLOAD)
    out = {"workload": WORKLOAD, "columns": 9}
    with tp.Mesh(torch.tensor(V, dtype=torch.float64, device=dev),
                 torch.tensor(F, dtype=torch.int32, device=dev), device=dev.index or 0) as m:
        u = torch.tensor(vertex_vectors(len(V), 9, 11), dtype=torch.float64, device=dev)
        ys = {}
        for name, tc in (("cuda_cores", 0), ("tensor_cores", 1)):
            pp = tp.params(tensor_cores=tc)
            ys[name] = tp.fractional_apply(m, "A", u, pp).cpu().numpy()
            torch.cuda.synchronize()
            tp.tp_profile_read(m)
            tp.tp_profile_enable(m, True)
            for _ in range(reps):
                tp.fractional_apply(m, "A", u, pp)
            torch.cuda.synchronize()
            d = tp.tp_profile_read(m)["apply_A"]
            tp.tp_profile_enable(m, False)
            ms = d["ms"] / d["launches"]
            pairs = d["units"] / d["launches"]
            out[name] = {"ms_per_launch": ms,
                         "tflops": APPLY_FLOPS["apply_A"](9) * pairs / (ms / 1e3) / 1e12}
        a, b = ys["tensor_cores"], ys["cuda_cores"]
        out["rel_difference"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return out


def accuracy(tp, dev):
    """Errors on torus_20k against the FP64 oracle, from stored oracle values
    (tests/golden: the energy, and dE and A u (u = 3 seeded N(0,1) columns)
    at 64 sampled vertices): the FP32 direct path and Barnes-Hut at
    theta = 0.25 and 0.5 (relative 2-norm errors over the sampled rows)."""
    import numpy as np
    import torch
    from synth import vertex_vectors, workload
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "full_size.json")))[WORKLOAD]
    smp = json.load(open(os.path.join(ROOT, "tests", "golden", "torus20k_samples.json")))
    V, F = workload(WORKLOAD)
    idx = np.array(smp["vertices"])
    dE_ref, Au_ref = np.array(smp["dE"]), np.array(smp["Au"])
    u = torch.tensor(vertex_vectors(len(V), 3, 202), dtype=torch.float64, device=dev)
    mesh = tp.Mesh(torch.tensor(V, dtype=torch.float64, device=dev), torch.tensor(F, dtype=torch.int32, device=dev),
                   device=dev.index or 0)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out = {"workload": WORKLOAD, "reference": "FP64 oracle (stored: energy, dE and A u at 64 vertices)"}
    for name, p in (("fp32_direct", tp.params()), ("bh_theta_0.25", tp.params(theta=0.25)),
                    ("bh_theta_0.5", tp.params(theta=0.5))):
        E = tp.tp_energy(mesh, p)
        dE, _ = tp.tp_differential(mesh, p)
        Au = tp.fractional_apply(mesh, "A", u, p).cpu().numpy()
        out[name] = {"E": abs(E - gold["energy"]) / abs(gold["energy"]), "dE": rel(dE[idx], dE_ref),
                     "Au": rel(Au[idx], Au_ref)}
    mesh.close()
    return out


def bh_step(tp, dev, steps=2):
    """Constrained steps with every pair sum on the tree (theta = 0.5: energy,
    differential, and the A and L^{2-s} applies of the Krylov loop) on the
    two linked 25,000-face tori; device time per step."""
    import numpy as np
    import torch
    from synth import workload
    V, F = workload("linked_tori_50k")
    A0 = float(np.sum(0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)))
    Vol0 = float(np.sum(V[F[:, 0]] * np.cross(V[F[:, 1]], V[F[:, 2]])) / 6.0)
    cons = tp.tp_constraints(flags=tp.TP_CONSTRAINT_AREA | tp.TP_CONSTRAINT_VOLUME, A0=A0, V0=Vol0)
    p = tp.params(theta=0.5, krylov_tol=1e-5, krylov_max=60, cg_tol=1e-6)
    f0 = torch.tensor(V, dtype=torch.float64, device=dev)
    mesh = tp.Mesh(f0, torch.tensor(F, dtype=torch.int32, device=dev), device=dev.index or 0)
    tp.precond_step(mesh, cons, p)                        # warm-up (tree, factor, graphs)
    tp.tp_mesh_set_positions(mesh, f0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = []
    e0.record()
    for _ in range(steps):
        reps.append(tp.precond_step(mesh, cons, p))
    e1.record()
    torch.cuda.synchronize()
    mesh.close()
    ms = e0.elapsed_time(e1) / steps
    return {"workload": "linked_tori_50k", "nf": int(len(F)), "theta": 0.5, "ms_per_step": ms,
            "interactions_per_step": sum(r["pair_interactions"] for r in reps) / steps,
            "krylov_iters_per_step": sum(r["krylov_iters"] for r in reps) / steps,
            "E": [r["E_after"] for r in reps], "status": [r["status"] for r in reps]}


def long_run(args):
    """Long Barnes-Hut run on the two linked 25,000-face tori: args.long_run
    constrained steps (area + volume) with every pair sum on the tree
    (theta = 0.5); the tree is refit each step and rebuilt every 20 steps.
    Reports the energy trace, device time per step, the tree's share and the
    plateau: the first step after which no 10-step window lowers the energy
    by 0.1% or more."""
    import numpy as np
    import torch
    import paper_2107_01664_gb300 as tp
    from synth import workload
    dev = torch.device("cuda", 0)
    V, F = workload("linked_tori_50k")
    A0 = float(np.sum(0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)))
    Vol0 = float(np.sum(V[F[:, 0]] * np.cross(V[F[:, 1]], V[F[:, 2]])) / 6.0)
    cons = tp.tp_constraints(flags=tp.TP_CONSTRAINT_AREA | tp.TP_CONSTRAINT_VOLUME, A0=A0, V0=Vol0)
    mesh = tp.Mesh(torch.tensor(V, dtype=torch.float64, device=dev),
                   torch.tensor(F, dtype=torch.int32, device=dev), device=0)
    base = dict(theta=0.5, krylov_tol=1e-5, krylov_max=60, cg_tol=1e-6)
    E_exact0 = tp.tp_energy(mesh, tp.params())
    tp.tp_profile_read(mesh)
    tp.tp_profile_enable(mesh, True)
    E, ms, status = [], [], []
    wall0 = time.perf_counter()
    for k in range(args.long_run):
        p = tp.params(bvh_refit=0 if k % 20 == 0 else 1, **base)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rep = tp.precond_step(mesh, cons, p)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        E.append(rep["E_after"])
        status.append(rep["status"])
    wall = time.perf_counter() - wall0
    # plateau: the first step after which no 10-step window lowers E by 0.1%
    drops = [k for k in range(10, len(E)) if (E[k - 10] - E[k]) >= 1e-3 * abs(E[k])]
    plateau = (drops[-1] + 1) if drops else 0
    if plateau >= len(E):
        plateau = None
    prof = tp.tp_profile_read(mesh)
    tp.tp_profile_enable(mesh, False)
    E_exact = tp.tp_energy(mesh, tp.params())
    f = tp.tp_mesh_get_positions(mesh)
    mesh.close()
    A1 = float(np.sum(0.5 * np.linalg.norm(np.cross(f[F[:, 1]] - f[F[:, 0]], f[F[:, 2]] - f[F[:, 0]]), axis=1)))
    total_ms = sum(ms)
    out = {"mode": "long_run", "workload": "linked_tori_50k", "steps": args.long_run, "theta": 0.5,
           "tree": "refit each step, rebuilt every 20", "ms_per_step_mean": total_ms / len(ms),
           "device_s_total": total_ms / 1e3, "wall_s": wall,
           "plateau_step": plateau, "time_to_plateau_s": (sum(ms[:plateau + 1]) / 1e3) if plateau is not None else None,
           "E_exact_start": E_exact0, "E_exact_end": E_exact, "E_bh_trace_every_10": E[::10],
           "area_rel_drift_end": abs(A1 - A0) / A0, "krylov_converged_steps": sum(1 for s_ in status if s_ == 0),
           "bvh_build_share": (prof["bvh_build"]["ms"] / total_ms) if "bvh_build" in prof else None,
           "kernel_ms": {k: round(v["ms"], 1) for k, v in prof.items()}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def aggregate_ranks(dev_ms, units, device, world):
    """Whole-job aggregate over the ranks of the process group: the maximum
    device time and the summed work (replicas: no data-path collective)."""
    if world <= 1:
        return dev_ms, units
    import torch
    import torch.distributed as dist
    tmax = torch.tensor([dev_ms], dtype=torch.float64, device=device)
    tsum = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax.item()), float(tsum.item())


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2107_01664_gb300 as tp
    from synth import workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    V, F = workload(WORKLOAD)
    f0 = torch.tensor(V, dtype=torch.float64, device=dev)
    faces = torch.tensor(F, dtype=torch.int32, device=dev)
    mesh = tp.Mesh(f0, faces, device=local)
    A0 = float(np.sum(0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)))
    Vol0 = float(np.sum(V[F[:, 0]] * np.cross(V[F[:, 1]], V[F[:, 2]])) / 6.0)
    cons = tp.tp_constraints(flags=tp.TP_CONSTRAINT_AREA | tp.TP_CONSTRAINT_VOLUME, A0=A0, V0=Vol0)
    ps, pb = step_params(tp), bh_params(tp)
    dE_buf = torch.empty((len(V), 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def one_step(f_in, like=None):
        tp.tp_mesh_set_positions(mesh, f_in)
        rep = tp.precond_step(mesh, cons, ps)
        Eb = tp.tp_energy(mesh, pb)
        dEb, _ = tp.tp_differential(mesh, pb, like=like if like is not None else dE_buf)
        return rep, Eb, dEb

    for _ in range(args.warmup):
        one_step(f0)
    torch.cuda.synchronize()
    tp.tp_profile_read(mesh)                      # discard warm-up statistics
    tp.tp_profile_enable(mesh, True)

    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    reps = []
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = tp.tp_launch_count()
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_steps")     # lets a profiler select the timed launches
    for k in range(args.steps):
        flush.zero_()                              # L2 flushed between timed steps
        ev[k][0].record(stream)
        rep, Eb, dEb = one_step(f0)
        ev[k][1].record(stream)
        reps.append(rep)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - wall0
    launches = tp.tp_launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    if world > 1:
        dist.barrier()
    prof = tp.tp_profile_read(mesh)
    tp.tp_profile_enable(mesh, False)

    pair_kernels = [k for k in prof if k in FLOPS_PER_PAIR or k in APPLY_FLOPS]
    pairs_total = sum(prof[k]["units"] for k in pair_kernels)
    dev_ms = float(sum(step_ms))
    dev_ms_all, pairs_all = aggregate_ranks(dev_ms, pairs_total, dev, world)
    value = pairs_all / (dev_ms_all / 1e3)
    # the energies of rejected Armijo trials are pair work too; the figure
    # without them counts only the accepted trial of each step
    nf = len(F)
    rejected = sum(max(0, r["ls_trials"] - 1) for r in reps) * float(nf) * (nf - 1)
    pairs_acc_all = aggregate_ranks(dev_ms, pairs_total - rejected, dev, world)[1]

    # e2e through the C ABI with host buffers: pinned positions in, positions + dE out
    f_host = torch.tensor(V, dtype=torch.float64).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_pairs = 0.0
    for _ in range(e2e_steps):
        tp.tp_mesh_set_positions(mesh, f_host)
        rep = tp.precond_step(mesh, cons, ps)
        tp.tp_energy(mesh, pb)
        tp.tp_differential(mesh, pb, like=None)      # dE to host
        tp.tp_mesh_get_positions(mesh, None)          # positions to host
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    pairs_per_step = pairs_total / args.steps
    e2e = {"value": pairs_per_step / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(len(V) * 3 * 8),
           "d2h_bytes_per_step": int(2 * len(V) * 3 * 8 + 8 * 3)}

    # roofline of the dominant kernel
    dom = max(prof, key=lambda k: prof[k]["ms"]) if prof else None
    peaks, src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    roof = None
    if dom is not None:
        d = prof[dom]
        per_launch_ms = d["ms"] / max(1, d["launches"])
        if flops_per_pair(dom, d) is not None:
            clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
            peak = sms * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
            achieved = flops_per_pair(dom, d) * d["units"] / (d["ms"] / 1e3) / 1e12
            roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {clock_mhz:.0f} MHz"}
        else:
            peak = float(peaks.get("hbm_gbs", 6800.0))
            achieved = d["units"] / (d["ms"] / 1e3) / 1e9
            roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_basis": f"hbm_gbs ({src})"}
        tr = profile_traffic(dom, WORKLOAD)
        roof["traffic"] = tr
        roof["launch_ms"] = per_launch_ms
        roof["launches"] = d["launches"]

    lat = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded torus, no dataset)",
        "config": {"workload": WORKLOAD, "nv": int(len(V)), "nf": int(len(F)),
                   "step": "set positions + precond_step(area+volume; direct FP32 pairs, FP64 solver) + BH theta=0.5 E+dE",
                   "solver_dtype": "f64 (CG, FGMRES, Schur)", "krylov_tol": ps.krylov_tol, "cg_tol": ps.cg_tol,
                   "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{world}"},
        "steps_per_s": 1e3 * args.steps / dev_ms_all,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "pairs_per_step": pairs_per_step,
        "value_without_rejected_trials": pairs_acc_all / (dev_ms_all / 1e3),
        "rejected_trial_pairs_per_step": rejected / args.steps,
        "ls_trials_per_step": sum(r["ls_trials"] for r in reps) / len(reps),
        "krylov_iters_per_step": sum(r["krylov_iters"] for r in reps) / len(reps),
        # steps whose FGMRES met krylov_tol within krylov_max (status 0); status 4 = the
        # fixed iteration budget ran out first (the step is still taken)
        "krylov_converged_steps": sum(1 for r in reps if r["status"] == 0),
        "cg_iters_per_step": sum(r["cg_iters"] for r in reps) / len(reps),
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "units": v["units"],
                        "tflops": (flops_per_pair(k, v) * v["units"] / (v["ms"] / 1e3) / 1e12
                                   if flops_per_pair(k, v) and v["ms"] > 0 else None)}
                    for k, v in prof.items()},
        "wall_s": wall, "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "clocks": clk,
    }
    if not args.no_large:
        line["large_mesh"] = large_mesh(tp, dev)
        line["accuracy"] = accuracy(tp, dev)
        line["tensor_core_apply"] = tensor_core_apply(tp, dev)
        line["serving"] = serving(tp, dev, n=args.serve_n, slots=args.serve_slots)
        line["obstacle"] = obstacle_scene(tp, dev)
        line["pins"] = pinned_steps(tp, dev)
        line["willmore"] = willmore_steps(tp, dev)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = run_cpu_sample()
    mesh.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands on the host cores
# ---------------------------------------------------------------------------

def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # one single-threaded oracle process per host core: W untimed samples
    # each, then K timed samples each from a common start time
    n = host_cores()
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    start_at = time.time() + 6.0 + 0.6 * args.warmup
    ps = []
    for i in range(n):
        code = ("import json,sys; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.oracle_timed_loop(1, %d, %d, %d, %r)))"
                % (ROOT, 4242 + i, args.warmup, args.steps, start_at))
        ps.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                   stderr=subprocess.PIPE, text=True))
    pairs, w0, w1 = 0.0, [], []
    for pr in ps:
        out, err = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        r = json.loads(out.strip().splitlines()[-1])
        pairs += r[0]
        w0.append(r[1])
        w1.append(r[2])
    secs = max(w1) - min(w0)
    value = pairs / secs
    cpu = {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
           "sample": sample_desc(1, n) + f"; {args.steps} timed samples per process"}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded torus, no dataset)",
        "config": {"workload": WORKLOAD, "step": "bounded oracle sample (see cpu_baseline.sample)"},
        "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# serving: continuous batching of descent steps
# ---------------------------------------------------------------------------

def serve_arm(args):
    """Serving alone (the same section the default run reports)."""
    import torch
    import paper_2107_01664_gb300 as tp
    torch.cuda.set_device(0)
    print(json.dumps({"serving": serving(tp, torch.device("cuda", 0), n=args.serve_n, f_max=args.serve_fmax,
                                         slots=args.serve_slots)}))


SERVE_BH_ABOVE = 30000


def serving(tp, dev, n=512, f_min=2000, f_max=200000, slots=4, fp64_n=16, fp64_fmax=8000, pilot=64):
    """Serving as the benchmark's fourth configuration: n one-step requests
    (perturbed icospheres and tori, sigma = 0.01, faces log-uniform in
    [f_min, f_max], seed 404) arriving as a Poisson process at 0.7x the
    capacity measured closed-loop on `pilot` requests spread evenly over the
    stream (every n/pilot-th request, so the size mix is the stream's); FP32 pair
    terms with FP64 solves, Barnes-Hut (theta = 0.5) above SERVE_BH_ABOVE
    faces, admission by HBM footprint, smallest-first within a 1 s fairness
    window. The plain FP64 direct path serves a seeded sub-stream (the first
    fp64_n requests of the stream with at most fp64_fmax faces) with the same
    arrivals as the FP32 path; the full stream in FP64 would take hours (FP64
    pair terms run at 1/64 of the FP32 rate). The line search of a served step
    starts where no vertex moves by more than a quarter of a face size
    (tau0_disp = 0.25)."""
    import numpy as np
    from paper_2107_01664_gb300 import serve
    t_start = time.perf_counter()
    p32 = tp.params(precision=tp.TP_PREC_FP32, krylov_tol=1e-5, krylov_max=30, cg_tol=1e-4, tau0_disp=0.25)
    p64 = tp.params(precision=tp.TP_PREC_FP64, krylov_tol=1e-5, krylov_max=30, cg_tol=1e-4, tau0_disp=0.25)
    reqs = serve.make_requests(n, f_min, f_max, rate=1.0, seed=404)

    def at_rate(rs, rate, seed):
        rng = np.random.default_rng(seed)
        t = np.cumsum(rng.exponential(1.0 / rate, len(rs)))
        return [serve.Request(arrival=float(t[i]), rid=r.rid, V=r.V, F=r.F) for i, r in enumerate(rs)]

    def run(rs, p, bh_above):
        srv = serve.Server(slots=slots, step_params=p, bh_above=bh_above, keep_positions=True)
        res = srv.run(rs)
        summ = serve.summarize(res, srv.wall)
        summ.update({"max_concurrency": srv.max_concurrency, "peak_admitted_bytes": srv.peak_used,
                     "budget_bytes": srv.budget})
        return summ, res

    stride = max(1, n // pilot)
    closed = [serve.Request(arrival=0.0, rid=r.rid, V=r.V, F=r.F) for r in reqs[::stride][:pilot]]
    cap, _ = run(closed, p32, SERVE_BH_ABOVE)
    rate = 0.7 * cap["steps_per_s"]
    main_stream = at_rate(reqs, rate, 405)
    summ, res = run(main_stream, p32, SERVE_BH_ABOVE)
    nfs = np.array([len(r.F) for r in reqs])
    lat = {r.rid: r.latency for r in res if r.status == "ok"}
    svc = {r.rid: r.end - r.start for r in res if r.status == "ok"}
    classes = {}
    for name, lo, hi in (("2k-8k", 0, 8000), ("8k-30k", 8000, 30000), ("30k-200k", 30000, 10 ** 9)):
        ids = [i for i in range(len(reqs)) if lo < nfs[i] <= hi and i in lat]
        if ids:
            ls = np.array([lat[i] for i in ids]) * 1e3
            sv = np.array([svc[i] for i in ids]) * 1e3
            classes[name] = {"requests": len(ids), "p50_ms": float(np.percentile(ls, 50)),
                             "p99_ms": float(np.percentile(ls, 99)),
                             "service_p50_ms": float(np.percentile(sv, 50))}
    out = {"metric": "served steps/s", "requests": n, "faces": [f_min, f_max], "slots": slots,
           "bh_above_faces": SERVE_BH_ABOVE, "pilot_closed_loop_steps_per_s": cap["steps_per_s"],
           "arrival_rate_per_s": rate, "fp32_pairs": summ, "latency_by_size": classes,
           "krylov_converged": int(sum(1 for r in res if r.status == "ok" and r.report.get("status") == 0))}
    # the FP64 direct path on the seeded sub-stream
    sub = [r for r in main_stream if len(r.F) <= fp64_fmax][:fp64_n]
    t0 = sub[0].arrival if sub else 0.0
    sub = [serve.Request(arrival=r.arrival - t0, rid=r.rid, V=r.V, F=r.F) for r in sub]
    s32, r32 = run(sub, p32, None)
    s64, r64 = run(sub, p64, None)
    # per request: E at the start of the step (the quantity the 1e-5 FP32
    # tolerance is stated for), the step length, and the step per unit
    # length (f_new - f) / tau of both paths
    dE0, dtau, dstep = [], [], []
    byid = {r.rid: r for r in sub}
    for a, b in zip(r32, r64):
        if a.status != "ok" or b.status != "ok":
            continue
        f0 = byid[a.rid].V
        dE0.append(abs(a.report["E_before"] - b.report["E_before"]) / abs(b.report["E_before"]))
        dtau.append(abs(a.report["tau"] - b.report["tau"]) / b.report["tau"])
        xa, xb = (a.positions - f0) / a.report["tau"], (b.positions - f0) / b.report["tau"]
        dstep.append(float(np.linalg.norm(xa - xb) / max(np.linalg.norm(xb), 1e-300)))
    out["fp64_comparison"] = {"sub_stream": f"first {len(sub)} requests with at most {fp64_fmax} faces, same arrivals",
                              "fp32_pairs": s32, "fp64_direct": s64,
                              "max_rel_E_difference": max(dE0) if dE0 else None,
                              "max_rel_tau_difference": max(dtau) if dtau else None,
                              "max_rel_step_per_tau_difference": max(dstep) if dstep else None}
    out["section_s"] = round(time.perf_counter() - t_start, 1)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the extra sections (1.31M-face mesh, serving, obstacle, pins, Willmore, accuracy)")
    ap.add_argument("--large", action="store_true", help="run only the 1.31M-face section instead")
    ap.add_argument("--serve", action="store_true", help="run the serving benchmark instead")
    ap.add_argument("--long-run", type=int, default=0, help="run N Barnes-Hut steps on the linked tori instead")
    ap.add_argument("--obstacle", action="store_true",
                    help="run only the static-obstacle scene (torus_20k around a ball) instead")
    ap.add_argument("--pins", action="store_true",
                    help="run only the vertex-pin steps (torus_20k with 8 pins) instead")
    ap.add_argument("--accuracy", action="store_true",
                    help="report only the errors on torus_20k against stored oracle values instead")
    ap.add_argument("--willmore", action="store_true",
                    help="run only the Willmore steps (torus_20k, weight 100) instead")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="run only the tensor-core A apply beside the CUDA-core one (torus_20k) instead")
    ap.add_argument("--serve-n", type=int, default=512)
    ap.add_argument("--serve-fmax", type=int, default=200000)
    ap.add_argument("--serve-slots", type=int, default=4)
    args = ap.parse_args()
    if args.serve:
        serve_arm(args)
        return
    if args.long_run:
        long_run(args)
        return
    if args.obstacle:
        import torch
        import paper_2107_01664_gb300 as tp
        torch.cuda.set_device(0)
        print(json.dumps({"obstacle": obstacle_scene(tp, torch.device("cuda", 0))}))
        return
    if args.pins:
        import torch
        import paper_2107_01664_gb300 as tp
        torch.cuda.set_device(0)
        print(json.dumps({"pins": pinned_steps(tp, torch.device("cuda", 0))}))
        return
    if args.large:
        import torch
        import paper_2107_01664_gb300 as tp
        torch.cuda.set_device(0)
        print(json.dumps({"large_mesh": large_mesh(tp, torch.device("cuda", 0))}))
        return
    if args.accuracy:
        import torch
        import paper_2107_01664_gb300 as tp
        torch.cuda.set_device(0)
        print(json.dumps({"accuracy": accuracy(tp, torch.device("cuda", 0))}))
        return
    if args.willmore:
        import torch
        import paper_2107_01664_gb300 as tp
        torch.cuda.set_device(0)
        print(json.dumps({"willmore": willmore_steps(tp, torch.device("cuda", 0))}))
        return
    if args.tensor_cores:
        import torch
        import paper_2107_01664_gb300 as tp
        torch.cuda.set_device(0)
        print(json.dumps({"tensor_core_apply": tensor_core_apply(tp, torch.device("cuda", 0))}))
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
