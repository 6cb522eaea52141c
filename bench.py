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
                 "bh_energy": "bvh.cu", "bh_diff": "bvh.cu", "cg": "cg.cu", "bvh_build": "bvh.cu",
                 "chol_factor": "chol.cu", "chol_solve": "chol.cu", "obstacle_direct": "obstacle.cu",
                 "bh_obstacle": "obstacle.cu"}
FP32_LANES_PER_SM = 128


def step_params(tp):
    return tp.params(theta=0.0, precision=tp.TP_PREC_FP32, krylov_tol=1e-5, krylov_max=60,
                     gmres_restart=30, cg_tol=1e-6, cg_max=20000, proj_iters=1)


def bh_params(tp):
    return tp.params(theta=0.5, precision=tp.TP_PREC_FP32, leaf_size=8)


# ---------------------------------------------------------------------------
# CPU side: the oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------

def sample_desc(scale):
    return (f"oracle (numpy FP64, 1 thread) on {WORKLOAD}: energy rows of {32 * scale} target faces, "
            f"dE at {3 * scale} vertices, A.u and L.u at {3 * scale} vertices each; "
            "pairs = rows evaluated x (nf - 1)")


def oracle_sample_pairs_per_s(scale):
    """Run in a subprocess with single-threaded BLAS; returns (pairs/s, seconds, pairs)."""
    import numpy as np
    from oracle import tp_oracle as O
    from synth import vertex_vectors, workload
    V, F = workload(WORKLOAD)
    nf = len(F)
    rng = np.random.default_rng(4242)
    targets = rng.choice(nf, 32 * scale, replace=False)
    nvs = 3 * scale
    verts = rng.choice(len(V), 3 * nvs, replace=False)
    u = vertex_vectors(len(V), 3, 202)
    t0 = time.perf_counter()
    O.energy_rows(V, F, 6.0, targets)
    O.differential_at_vertices(V, F, verts[:nvs])
    O.apply_operator_at_vertices(V, F, u, "A", verts[nvs:2 * nvs])
    O.apply_operator_at_vertices(V, F, u, "L", verts[2 * nvs:])
    dt = time.perf_counter() - t0

    def inc_rows(vs):
        return len(np.unique(np.concatenate([np.nonzero(np.any(F == v, axis=1))[0] for v in vs])))
    rows = len(targets) + inc_rows(verts[:nvs]) + inc_rows(verts[nvs:2 * nvs]) + inc_rows(verts[2 * nvs:])
    pairs = float(rows) * (nf - 1)
    return pairs / dt, dt, pairs


def run_cpu_sample(scale=48):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample_pairs_per_s(%d)))" % (ROOT, scale))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    v, dt, pairs = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample_desc(scale),
            "seconds": round(dt, 2)}


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

def large_bh(tp, dev, reps=3):
    """Device time of the Barnes-Hut (theta = 0.5, leaf 8) energy and
    differential on icosphere level 8 with spherical-harmonic bumps, and of one
    direct all-pairs energy for comparison (interactions per second)."""
    import torch
    from synth import workload
    V, F = workload("icosphere_l8")
    mesh = tp.Mesh(torch.tensor(V, dtype=torch.float64, device=dev),
                   torch.tensor(F, dtype=torch.int32, device=dev), device=dev.index or 0)
    pb = bh_params(tp)
    dE = torch.empty((len(V), 3), dtype=torch.float64, device=dev)
    tp.tp_energy(mesh, pb)
    tp.tp_differential(mesh, pb, like=dE)
    torch.cuda.synchronize()
    tp.tp_profile_read(mesh)
    tp.tp_profile_enable(mesh, True)
    for _ in range(reps):
        tp.tp_mesh_set_positions(mesh, torch.tensor(V, dtype=torch.float64, device=dev))  # rebuilds the BVH
        tp.tp_energy(mesh, pb)
        tp.tp_differential(mesh, pb, like=dE)
    tp.tp_energy(mesh, tp.params())                       # one direct pass
    # Barnes-Hut operator applies: A and L^{2-s} on 3 columns
    v3 = torch.randn((len(V), 3), dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(7))
    for op in ("A", "L"):
        tp.fractional_apply(mesh, op, v3, pb)
    torch.cuda.synchronize()
    prof = tp.tp_profile_read(mesh)
    tp.tp_profile_enable(mesh, False)
    mesh.close()
    out = {"workload": "icosphere_l8", "nf": int(len(F)), "theta": pb.theta, "leaf_size": pb.leaf_size}
    for k in ("bh_energy", "bh_diff", "bh_apply", "bvh_build", "energy_direct"):
        if k in prof and prof[k]["launches"]:
            d = prof[k]
            n = d["launches"]
            out[k] = {"ms_per_launch": d["ms"] / n, "units_per_launch": d["units"] / n,
                      "per_s": d["units"] / (d["ms"] / 1e3) if d["ms"] > 0 else None}
    out["bh_step_linked_tori"] = bh_step(tp, dev)
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
        line["large_mesh_bh"] = large_bh(tp, dev)
        line["obstacle"] = obstacle_scene(tp, dev)
        line["pins"] = pinned_steps(tp, dev)
        line["willmore"] = willmore_steps(tp, dev)
        line["accuracy"] = accuracy(tp, dev)
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
    for _ in range(args.warmup):       # untimed
        run_cpu_sample(scale=4)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        r = run_cpu_sample(scale=4)
        vals.append(r["value"])
        secs += r["seconds"]
    value = sum(vals) / len(vals)
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample_desc(4)}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded torus, no dataset)",
        "config": {"workload": WORKLOAD, "step": "bounded oracle sample (see cpu_baseline.sample)"},
        "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# serving: continuous batching of descent steps (separate report)
# ---------------------------------------------------------------------------

SERVE_DESC = ("Poisson arrivals of one-step requests on perturbed icospheres and tori (sigma=0.01), "
              "face counts log-uniform in [f_min, f_max]; slots = concurrent host threads on their own "
              "CUDA streams; admission by tp_mesh_footprint_bytes against an HBM budget")


def serve_arm(args):
    """Serving (continuous batching of one-step requests).

    1. fp32_pairs: the FP32-pair / FP64-solve path on a stream of
       args.serve_n meshes of 2k-serve_fmax faces. A closed-loop run (all
       requests present at t = 0) measures the capacity; the reported run
       replays the stream with Poisson arrivals at 0.8x that capacity.
    2. same_stream: a smaller stream (2k-8k faces) served once on the FP32
       path and once on the plain FP64 direct path, same arrivals, same
       meshes; steps/s, p50/p99 latency of both and the largest relative
       difference between the two paths' new positions (per request:
       |f32 - f64| / |f64 - f_start|). The full FP64 stream of 2k-200k
       faces would take hours (FP64 pair terms run at 1/64 of FP32)."""
    import numpy as np
    import paper_2107_01664_gb300 as tp
    from paper_2107_01664_gb300 import serve
    out = {"metric": "served steps/s", "unit": "steps/s", "mode": "serve", "description": SERVE_DESC}

    def run(reqs, prec, rate):
        p = tp.params(precision=prec, krylov_tol=1e-5, krylov_max=30, cg_tol=1e-6)
        stream = [serve.Request(arrival=(0.0 if rate is None else r.arrival), rid=r.rid, V=r.V, F=r.F, A0=r.A0,
                                V0=r.V0) for r in reqs]
        srv = serve.Server(slots=args.serve_slots, step_params=p)
        res = srv.run(stream)
        summ = serve.summarize(res, srv.wall)
        summ.update({"n_requests": len(reqs), "rate_per_s": rate, "slots": args.serve_slots,
                     "max_concurrency": srv.max_concurrency, "peak_admitted_bytes": srv.peak_used,
                     "budget_bytes": srv.budget, "krylov_max": p.krylov_max})
        return summ, res

    def at_rate(reqs, rate, seed):
        rng = np.random.default_rng(seed)
        t = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
        return [serve.Request(arrival=float(t[i]), rid=r.rid, V=r.V, F=r.F, A0=r.A0, V0=r.V0)
                for i, r in enumerate(reqs)]

    reqs = serve.make_requests(args.serve_n, 2000, args.serve_fmax, rate=1.0, seed=404)
    cap, _ = run(reqs, tp.TP_PREC_FP32, None)
    rate = 0.8 * cap["steps_per_s"]
    summ, _ = run(at_rate(reqs, rate, 405), tp.TP_PREC_FP32, rate)
    summ.update({"f_range": [2000, args.serve_fmax], "closed_loop_capacity_steps_per_s": cap["steps_per_s"]})
    out["fp32_pairs"] = summ

    small = serve.make_requests(max(4, args.serve_n // 4), 2000, 8000, rate=1.0, seed=406)
    cap64, _ = run(small, tp.TP_PREC_FP64, None)
    rate_s = 0.8 * cap64["steps_per_s"]
    stream = at_rate(small, rate_s, 407)
    s32, r32 = run(stream, tp.TP_PREC_FP32, rate_s)
    s64, r64 = run(stream, tp.TP_PREC_FP64, rate_s)
    # accuracy of the FP32 path against the FP64 one, per request: E at the
    # start of the step (the quantity the 1e-5 tolerance is stated for), the
    # Armijo step length, and the step itself where both took the same step
    # length (a different tau is a discrete line-search decision, not an
    # arithmetic error)
    dE0, same_tau, dstep = [], 0, []
    for a, b, q in zip(r32, r64, small):
        if a.status != "ok" or b.status != "ok":
            continue
        dE0.append(abs(a.report["E_before"] - b.report["E_before"]) / abs(b.report["E_before"]))
        if a.report["tau"] == b.report["tau"]:
            same_tau += 1
            dstep.append(float(np.linalg.norm(a.positions - b.positions) /
                               max(np.linalg.norm(b.positions - q.V), 1e-300)))
    out["same_stream"] = {"f_range": [2000, 8000], "rate_per_s": rate_s,
                          "fp64_closed_loop_capacity_steps_per_s": cap64["steps_per_s"],
                          "fp32_pairs": s32, "fp64_direct": s64,
                          "max_rel_E_difference_fp32_vs_fp64": max(dE0) if dE0 else None,
                          "requests_with_same_tau": same_tau,
                          "max_rel_step_difference_same_tau": max(dstep) if dstep else None}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-large", action="store_true", help="skip the 1.31M-face Barnes-Hut section")
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
    ap.add_argument("--serve-n", type=int, default=64)
    ap.add_argument("--serve-fmax", type=int, default=50000)
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
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
