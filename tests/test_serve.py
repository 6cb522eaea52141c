"""Serving loop: admission by HBM footprint, overlap of requests, results
independent of the mix (GPU), and host-side failure handling (CPU: requests
that fail are reported and the loop keeps serving)."""
import numpy as np
import pytest

from paper_2107_01664_gb300 import serve


def test_failing_requests_do_not_stop_the_loop():
    # host-side fault: a request with an invalid face index fails at mesh
    # creation (no GPU work is started for it); the others are still served.
    # Without a GPU every request fails the same way, which exercises the
    # same path; with a GPU only the bad one fails.
    import torch
    reqs = serve.make_requests(6, 300, 800, rate=1000.0, seed=3)
    bad = reqs[2]
    bad.F = bad.F.copy()
    bad.F[0, 0] = len(bad.V) + 5
    srv = serve.Server(slots=2, hbm_budget=1 << 40)
    res = srv.run(reqs)
    assert [r.rid for r in res] == list(range(6))
    assert res[2].status.startswith("error")
    if torch.cuda.is_available():
        assert all(r.status == "ok" for r in res if r.rid != 2)
    assert srv._used == 0                      # every admission was released


def _bare_server(budget, fair_s=None, t0=None):
    srv = serve.Server.__new__(serve.Server)
    srv.params = None
    srv.budget = budget
    srv._used = 0
    srv.peak_used = 0
    srv.fair_s = fair_s
    srv._t0 = t0
    srv.bh_above = None
    return srv


def test_admission_respects_the_budget_without_gpu_work():
    # fair_s = None: first come, first served among the requests that fit
    srv = _bare_server(100)
    srv.params = None
    srv.budget = 100
    srv._used = 0
    srv.peak_used = 0
    sizes = {0: 60, 1: 50, 2: 30, 3: 200}
    srv.footprint = lambda r: sizes[r.rid]
    srv._pending = [serve.Request(arrival=float(i), rid=i, V=np.zeros((3, 3)), F=np.zeros((1, 3))) for i in range(4)]
    first = srv._admit()
    assert first.rid == 0 and srv._used == 60
    second = srv._admit()                      # 50 does not fit (60+50 > 100); 30 does
    assert second.rid == 2 and srv._used == 90
    assert srv._admit() is None
    srv._used = 0
    assert srv._admit().rid == 1
    srv._used = 0
    srv._pending = [r for r in srv._pending if r.rid == 3]
    assert srv._admit().rid == 3               # larger than the budget: admitted alone


def test_admission_smallest_first_within_the_fairness_window():
    import time
    # requests that arrived less than fair_s ago go smallest first; one that
    # waited longer goes before all of them
    now = time.perf_counter()
    srv = _bare_server(1000, fair_s=5.0, t0=now - 10.0)      # "now" is 10 s into the run
    sizes = {0: 300, 1: 100, 2: 200, 3: 50}
    arrivals = {0: 9.0, 1: 9.5, 2: 2.0, 3: 9.8}                # rid 2 has waited 8 s
    srv.footprint = lambda r: sizes[r.rid]
    srv._pending = [serve.Request(arrival=arrivals[i], rid=i, V=np.zeros((3, 3)), F=np.zeros((1, 3)))
                    for i in range(4)]
    order = [srv._admit().rid for _ in range(4)]
    assert order == [2, 3, 1, 0]


def test_bh_above_switches_large_meshes_to_barnes_hut():
    import paper_2107_01664_gb300 as tp
    srv = _bare_server(1 << 40)
    srv.params = tp.params()
    srv.bh_above, srv.bh_theta = 1000, 0.5
    small = serve.Request(arrival=0.0, rid=0, V=np.zeros((3, 3)), F=np.zeros((800, 3)))
    large = serve.Request(arrival=0.0, rid=1, V=np.zeros((3, 3)), F=np.zeros((5000, 3)))
    assert srv.params_for(small).theta == 0.0
    assert srv.params_for(large).theta == 0.5 and srv.params.theta == 0.0


@pytest.mark.gpu
def test_results_are_the_same_alone_and_in_the_mix(lib):
    import paper_2107_01664_gb300 as tp
    p = tp.params(cg_tol=1e-6, krylov_max=40)
    reqs = serve.make_requests(8, 500, 3000, rate=200.0, seed=11)
    fps = [tp.tp_mesh_footprint_bytes(len(r.V), len(r.F), p) for r in reqs]
    budget = 3 * max(fps)
    mix = serve.Server(slots=4, hbm_budget=budget, step_params=p)
    res_mix = mix.run(reqs)
    assert all(r.status == "ok" for r in res_mix)
    assert mix.peak_used <= budget
    assert mix.max_concurrency >= 2
    alone = serve.Server(slots=1, hbm_budget=budget, step_params=p)
    res_alone = alone.run([serve.Request(arrival=0.0, rid=r.rid, V=r.V, F=r.F) for r in reqs])
    for a, b in zip(res_mix, res_alone):
        d = np.linalg.norm(a.positions - b.positions) / np.linalg.norm(b.positions)
        assert d <= 1e-12, (a.rid, d)
        assert a.report["E_after"] == pytest.approx(b.report["E_after"], rel=1e-12)
    s = serve.summarize(res_mix, mix.wall)
    assert s["completed"] == 8 and s["latency_ms"]["p99"] >= s["latency_ms"]["p50"]


def test_request_sizes_stay_in_the_configured_range():
    # icospheres take a subdivision level whose 20 * 4^l faces lie in
    # [f_min, f_max]; tori round the drawn face count; arrivals increase
    f_min, f_max = 2000, 200000
    reqs = serve.make_requests(40, f_min, f_max, rate=10.0, seed=5)
    t = [r.arrival for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    kinds = set()
    for r in reqs:
        nf = len(r.F)
        is_ico = len(r.V) == nf // 2 + 2 and nf % 20 == 0 and (nf // 20) & (nf // 20 - 1) == 0
        kinds.add(is_ico)
        if is_ico:
            assert f_min <= nf <= f_max, nf
        else:
            assert 0.9 * f_min <= nf <= 1.1 * f_max, nf
        assert r.F.min() >= 0 and r.F.max() < len(r.V)
    assert kinds == {True, False}
