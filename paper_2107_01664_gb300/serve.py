"""Serving loop: continuous batching of constrained descent steps.

Requests (one precond_step on a mesh of its own) arrive over time; each is
admitted as soon as a slot is free and its device footprint
(tp_mesh_footprint_bytes) fits in the remaining HBM budget. Every slot is a
host thread with its own CUDA stream; the library releases the GIL during
its calls, so the slots' kernels overlap on the GPU. Mesh state stays on the
device for the life of the request. Latency = completion time - arrival
time; the report gives steps/s and p50/p99 latency.

Admission order: among the waiting requests that fit, the smallest mesh goes
first, except that a request that has waited longer than the fairness window
goes before any younger one (oldest first), so that large meshes are not
starved and small ones do not queue behind them. Meshes above `bh_above`
faces take the Barnes-Hut pair sums (theta = 0.5) for every pair term of the
step; the constraint targets A0 and V0 are the mesh's own total area and
volume (tp_mesh_area_volume) unless the request gives them.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import (Mesh, TpError, params, precond_step, tp_constraints, tp_mesh_area_volume,
               tp_mesh_footprint_bytes, tp_mesh_get_positions)


@dataclass(order=True)
class Request:
    arrival: float                               # seconds after the start of the run
    rid: int = field(compare=False)
    V: np.ndarray = field(compare=False, repr=False)
    F: np.ndarray = field(compare=False, repr=False)
    A0: float | None = field(compare=False, default=None)   # None: the mesh's own area
    V0: float | None = field(compare=False, default=None)   # None: the mesh's own volume


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
                 keep_positions: bool = True, bh_above: int | None = None, bh_theta: float = 0.5,
                 fair_s: float | None = 1.0):
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
        self.bh_above = bh_above
        self.bh_theta = bh_theta
        self.fair_s = fair_s
        self._t0 = None
        self._lock = threading.Condition()
        self._used = 0
        self._pending: list[Request] = []      # arrived, waiting for admission (FIFO by arrival)
        self._results: list[Result] = []
        self._done = False
        self.max_concurrency = 0
        self._running = 0

    def params_for(self, r: Request):
        """The step parameters of a request: Barnes-Hut above bh_above faces."""
        if self.bh_above is not None and len(r.F) > self.bh_above and self.params.precision == 0:
            import copy
            p = copy.copy(self.params)
            p.theta = self.bh_theta
            return p
        return self.params

    def footprint(self, r: Request) -> int:
        return int(tp_mesh_footprint_bytes(len(r.V), len(r.F), self.params_for(r)))

    def _order(self) -> list[int]:
        """Indices of the pending requests in admission order: those older
        than the fairness window first (oldest first), then the rest by
        footprint (smallest first, ties by arrival)."""
        now = (time.perf_counter() - self._t0) if self._t0 is not None else None
        def key(i):
            r = self._pending[i]
            old = self.fair_s is None or now is None or now - r.arrival > self.fair_s
            return (0, r.arrival, 0) if old else (1, self.footprint(r), r.arrival)
        return sorted(range(len(self._pending)), key=key)

    def _admit(self) -> Request | None:
        # first request in admission order whose footprint fits; requests
        # larger than the whole budget are admitted alone
        for i in self._order():
            r = self._pending[i]
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
                        A0, V0 = r.A0, r.V0
                        if A0 is None or V0 is None:
                            a, v = tp_mesh_area_volume(mesh)
                            A0 = a if A0 is None else A0
                            V0 = v if V0 is None else V0
                        c = tp_constraints(flags=3, A0=A0, V0=V0)
                        rep = precond_step(mesh, c, self.params_for(r))
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
        self._t0 = t0
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
    out = {
        "requests": len(results), "completed": ok,
        "steps_per_s": ok / wall if wall > 0 else 0.0,
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3) if ok else None,
                       "p99": float(np.percentile(lat, 99) * 1e3) if ok else None,
                       "mean": float(lat.mean() * 1e3) if ok else None},
        "wall_s": wall,
        "pair_interactions": float(sum(r.report.get("pair_interactions", 0.0) for r in results)),
    }
    if ok and out["latency_ms"]["p50"]:
        out["p99_over_p50"] = out["latency_ms"]["p99"] / out["latency_ms"]["p50"]
    return out


_BASE_MESHES: dict = {}


def _base_mesh(kind: str, a: int, b: int = 0):
    """Unperturbed icosphere of level a or torus of a x b (cached: requests
    share base meshes and differ by their noise)."""
    from synth import icosphere, torus
    key = (kind, a, b)
    if key not in _BASE_MESHES:
        _BASE_MESHES[key] = icosphere(a) if kind == "ico" else torus(a, b, 1.0, 0.3)
    return _BASE_MESHES[key]


def make_requests(n: int, f_min: int, f_max: int, rate: float, seed: int) -> list[Request]:
    """n requests with Poisson arrivals at `rate` per second; each a perturbed
    icosphere or torus (50/50) whose face count is drawn log-uniformly in
    [f_min, f_max] (icospheres take the nearest subdivision level inside
    that range), with
    seeded N(0, 0.01^2) noise per vertex coordinate. The constraint targets
    are left to the server (the mesh's own area and volume)."""
    from synth import gaussian_noise
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        target = float(np.exp(rng.uniform(np.log(f_min), np.log(f_max))))
        if rng.random() < 0.5:
            # the nearest level whose 20 * 4^l faces lie in [f_min, f_max]
            # (the nearest level overall when none does)
            lo = int(np.ceil(np.log(f_min / 20.0) / np.log(4.0) - 1e-9))
            hi = int(np.floor(np.log(f_max / 20.0) / np.log(4.0) + 1e-9))
            lvl = int(round(np.log(target / 20.0) / np.log(4.0)))
            lvl = int(np.clip(lvl, lo, hi)) if lo <= hi else lvl
            V, F = _base_mesh("ico", int(np.clip(lvl, 1, 8)))
        else:
            nm = max(8, int(round(np.sqrt(target / 2.0 * 4.0))))
            nn = max(4, int(round(target / 2.0 / nm)))
            V, F = _base_mesh("torus", nm, nn)
        V = gaussian_noise(V, 0.01, int(rng.integers(1 << 30)))
        out.append(Request(arrival=t, rid=i, V=V, F=F))
    return out
