"""Serving loop: continuous batching of constrained descent steps.

Requests (one precond_step on a mesh of its own) arrive over time; each is
admitted as soon as a slot is free and its device footprint
(tp_mesh_footprint_bytes) fits in the remaining HBM budget. Every slot is a
host thread with its own CUDA stream; the library releases the GIL during
its calls, so the slots' kernels overlap on the GPU. Mesh state stays on the
device for the life of the request. Latency = completion time - arrival
time; the report gives steps/s and p50/p99 latency.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import (Mesh, TpError, params, precond_step, tp_constraints, tp_mesh_footprint_bytes,
               tp_mesh_get_positions)


@dataclass(order=True)
class Request:
    arrival: float                               # seconds after the start of the run
    rid: int = field(compare=False)
    V: np.ndarray = field(compare=False, repr=False)
    F: np.ndarray = field(compare=False, repr=False)
    A0: float = field(compare=False, default=0.0)
    V0: float = field(compare=False, default=0.0)


@dataclass
class Result:
    rid: int
    nf: int
    arrival: float
    start: float
    end: float
    positions: np.ndarray
    report: dict
    status: str = "ok"

    @property
    def latency(self) -> float:
        return self.end - self.arrival


class Server:
    """Slots x streams over one GPU, admission by HBM footprint."""

    def __init__(self, slots: int = 4, hbm_budget: int | None = None, step_params=None, device: int = 0,
                 keep_positions: bool = True):
        import torch
        self.torch = torch
        self.device = device
        self.slots = slots
        self.params = step_params or params()
        if hbm_budget is None:
            free, _total = torch.cuda.mem_get_info(device)
            hbm_budget = int(0.8 * free)
        self.budget = hbm_budget
        self.peak_used = 0
        self.keep_positions = keep_positions
        self._lock = threading.Condition()
        self._used = 0
        self._pending: list[Request] = []      # arrived, waiting for admission (FIFO by arrival)
        self._results: list[Result] = []
        self._done = False
        self.max_concurrency = 0
        self._running = 0

    def footprint(self, r: Request) -> int:
        return int(tp_mesh_footprint_bytes(len(r.V), len(r.F), self.params))

    def _admit(self) -> Request | None:
        # oldest request whose footprint fits; requests larger than the whole
        # budget are admitted alone
        for i, r in enumerate(self._pending):
            fp = self.footprint(r)
            if self._used + fp <= self.budget or (self._used == 0 and fp > self.budget):
                self._pending.pop(i)
                self._used += fp
                self.peak_used = max(self.peak_used, self._used)
                return r
        return None

    def _worker(self, t0: float):
        import contextlib
        torch = self.torch
        gpu = torch.cuda.is_available()
        if gpu:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(self.device)
        ctx = (lambda: torch.cuda.stream(stream)) if gpu else contextlib.nullcontext
        while True:
            with self._lock:
                while True:
                    r = self._admit()
                    if r is not None or (self._done and not self._pending):
                        break
                    self._lock.wait(0.01)
                if r is None:
                    return
                self._running += 1
                self.max_concurrency = max(self.max_concurrency, self._running)
            start = time.perf_counter() - t0
            status, rep, pos = "ok", {}, None
            with ctx():
                try:
                    with Mesh(r.V, r.F, device=self.device) as mesh:
                        c = tp_constraints(flags=3, A0=r.A0, V0=r.V0)
                        rep = precond_step(mesh, c, self.params)
                        pos = tp_mesh_get_positions(mesh) if self.keep_positions else None
                except (TpError, ImportError, OSError) as e:
                    status = f"error: {e}"
            end = time.perf_counter() - t0
            with self._lock:
                self._used -= self.footprint(r)
                self._running -= 1
                self._results.append(Result(r.rid, len(r.F), r.arrival, start, end, pos, rep, status))
                self._lock.notify_all()

    def run(self, requests: list[Request]) -> list[Result]:
        """Serve the requests at their arrival times; returns results by rid."""
        arrivals = sorted(requests)
        t0 = time.perf_counter()
        workers = [threading.Thread(target=self._worker, args=(t0,), daemon=True) for _ in range(self.slots)]
        for w in workers:
            w.start()
        for r in arrivals:
            delay = r.arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            with self._lock:
                self._pending.append(r)
                self._lock.notify_all()
        with self._lock:
            self._done = True
            self._lock.notify_all()
        for w in workers:
            w.join()
        self.wall = time.perf_counter() - t0
        return sorted(self._results, key=lambda x: x.rid)


def summarize(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results if r.status == "ok"])
    ok = len(lat)
    return {
        "requests": len(results), "completed": ok,
        "steps_per_s": ok / wall if wall > 0 else 0.0,
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3) if ok else None,
                       "p99": float(np.percentile(lat, 99) * 1e3) if ok else None,
                       "mean": float(lat.mean() * 1e3) if ok else None},
        "wall_s": wall,
        "pair_interactions": float(sum(r.report.get("pair_interactions", 0.0) for r in results)),
    }


def make_requests(n: int, f_min: int, f_max: int, rate: float, seed: int) -> list[Request]:
    """n requests with Poisson arrivals at `rate` per second; each a perturbed
    icosphere or torus whose face count is drawn log-uniformly in
    [f_min, f_max] (icospheres take the nearest subdivision level). Uses the
    seeded mesh generators of the benchmark inputs."""
    from synth import gaussian_noise, icosphere, torus
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        target = float(np.exp(rng.uniform(np.log(f_min), np.log(f_max))))
        if rng.random() < 0.5:
            lvl = int(np.clip(round(np.log(target / 20.0) / np.log(4.0)), 1, 8))
            V, F = icosphere(lvl)
        else:
            nm = max(8, int(round(np.sqrt(target / 2.0 * 4.0))))
            nn = max(4, int(round(target / 2.0 / nm)))
            V, F = torus(nm, nn, 1.0, 0.3)
        V = gaussian_noise(V, 0.01, int(rng.integers(1 << 30)))
        Fi = np.asarray(F)
        fi, fj, fk = V[Fi[:, 0]], V[Fi[:, 1]], V[Fi[:, 2]]
        A0 = float(0.5 * np.linalg.norm(np.cross(fj - fi, fk - fi), axis=1).sum())
        V0 = float(np.sum(fi * np.cross(fj, fk)) / 6.0)
        out.append(Request(arrival=t, rid=i, V=V, F=F, A0=A0, V0=V0))
    return out
