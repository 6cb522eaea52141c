"""GPU parity of the Barnes-Hut path (§4) against the FP64 oracle, through
the C ABI: theta = 0 equals the direct sum; at theta in {0.25, 0.5} the GPU
energy, energy rows and both differential modes equal the oracle's
Barnes-Hut evaluation over the same tree (FP32 pair terms: 1e-5); the
approximation error against the direct sum is reported and falls with
theta. The Barnes-Hut operator applies (A, B, B0, L^{2-s}, 3 and 9
columns) equal the oracle's over the same tree to 1e-5 and keep constants
in the nullspace; a constrained step runs on them. Full sizes: the
20,000-face torus and a 64-target sample of the 1,310,720-face icosphere."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import small_mesh, workload

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    """max |a - b| over max |b|: a few wrong entries that a 2-norm hides show here"""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda:0", dtype=dtype)


@pytest.fixture(scope="module")
def meshes(lib):
    import torch
    out = {}
    for name in ["ico3", "torus30x11", "ico1"]:
        V, F = small_mesh(name, seed=31)
        out[name] = (V, F, lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)))
    yield out
    for v in out.values():
        v[2].close()


@pytest.mark.parametrize("name", ["ico3", "torus30x11", "ico1"])
@pytest.mark.parametrize("leaf", [8, 3])
def test_theta_zero_equals_direct(lib, meshes, name, leaf):
    V, F, m = meshes[name]
    E_bh = lib.tp_energy(m, lib.params(theta=1e-9, leaf_size=leaf))
    assert rel(E_bh, O.energy(V, F)) <= TOL32
    g, _ = lib.tp_differential(m, lib.params(theta=1e-9, leaf_size=leaf))
    assert rel(g, O.differential(V, F)) <= TOL32


@pytest.mark.parametrize("name", ["ico3", "torus30x11"])
@pytest.mark.parametrize("theta", [0.25, 0.5])
def test_bh_energy_matches_oracle_bh(lib, meshes, name, theta):
    V, F, m = meshes[name]
    p = lib.params(theta=theta)
    E = lib.tp_energy(m, p)
    E_ref = O.bh_energy(V, F, theta)
    assert rel(E, E_ref) <= TOL32
    tg = np.array([0, 17, len(F) // 2, len(F) - 1], dtype=np.int32)
    rows = lib.tp_energy_rows(m, tg, p)
    ref_rows, _ = O.bh_energy_rows(V, F, theta, 8, 6.0, tg)
    assert rel(rows, ref_rows) <= TOL32


@pytest.mark.parametrize("name", ["ico3", "torus30x11"])
@pytest.mark.parametrize("theta", [0.25, 0.5])
@pytest.mark.parametrize("mode", ["full", "literal"])
def test_bh_differential_matches_oracle_bh(lib, meshes, name, theta, mode):
    V, F, m = meshes[name]
    p = lib.params(theta=theta, bh_diff_mode=lib.TP_BH_DIFF_FULL if mode == "full" else lib.TP_BH_DIFF_LITERAL)
    g, E = lib.tp_differential(m, p)
    assert rel(g, O.bh_differential(V, F, theta, mode=mode)) <= TOL32
    assert rel(E, O.bh_energy(V, F, theta)) <= TOL32


def test_bh_error_falls_with_theta(lib, meshes):
    V, F, m = meshes["ico3"]
    E = O.energy(V, F)
    g_ref = O.differential(V, F)
    errE, errG = [], []
    for th in (0.25, 0.5, 1.0):
        p = lib.params(theta=th)
        errE.append(abs(lib.tp_energy(m, p) - E) / E)
        errG.append(rel(lib.tp_differential(m, p)[0], g_ref))
    print("BH relative error vs theta (0.25, 0.5, 1.0): E", errE, "dE", errG)
    assert errE[0] < errE[1] < errE[2]
    assert errG[0] < errG[1] < errG[2]


def test_bh_rows_with_device_targets_and_repeat(lib, meshes):
    V, F, m = meshes["torus30x11"]
    p = lib.params(theta=0.5)
    tg = np.arange(0, len(F), 7, dtype=np.int32)
    r1 = lib.tp_energy_rows(m, dev(tg), p).cpu().numpy()
    r2 = lib.tp_energy_rows(m, tg, p)
    assert np.array_equal(r1, r2)
    ref, _ = O.bh_energy_rows(V, F, 0.5, 8, 6.0, tg)
    assert rel(r1, ref) <= TOL32


@pytest.mark.parametrize("op", ["A", "B", "B0", "L"])
@pytest.mark.parametrize("name", ["ico3", "torus30x11"])
@pytest.mark.parametrize("k", [3, 9])
def test_bh_apply_matches_oracle_bh(lib, meshes, op, name, k):
    from synth import vertex_vectors
    V, F, m = meshes[name]
    v = vertex_vectors(len(V), k, 13)
    ref = O.bh_apply_operator(V, F, v, op, 0.5)
    got = lib.fractional_apply(m, op, v, lib.params(theta=0.5))
    assert rel(got, ref) <= TOL32


@pytest.mark.parametrize("op", ["A", "L"])
def test_bh_apply_tiny_theta_is_direct_and_keeps_constants(lib, meshes, op):
    from synth import vertex_vectors
    V, F, m = meshes["ico3"]
    v = vertex_vectors(len(V), 3, 14)
    got = lib.fractional_apply(m, op, v, lib.params(theta=1e-9))
    assert rel(got, O.apply_operator(V, F, v, op)) <= TOL32
    scale = np.abs(lib.fractional_apply(m, op, v, lib.params(theta=0.7))).max()
    one = lib.fractional_apply(m, op, np.ones((len(V), 1)), lib.params(theta=0.7))
    assert np.abs(one).max() <= 1e-5 * scale


def test_bh_apply_leaf_size_and_error_trend(lib, meshes):
    from synth import vertex_vectors
    V, F, m = meshes["torus30x11"]
    v = vertex_vectors(len(V), 3, 15)
    exact = O.apply_operator(V, F, v, "A")
    errs = []
    for th in (0.25, 0.5, 1.0):
        got = lib.fractional_apply(m, "A", v, lib.params(theta=th, leaf_size=4))
        assert rel(got, O.bh_apply_operator(V, F, v, "A", th, leaf=4)) <= TOL32
        errs.append(rel(got, exact))
    assert errs[0] < errs[1] < errs[2]


def test_precond_step_on_bh_applies(lib):
    # theta > 0: energy, differential and every operator apply of the step
    # use the tree; the step descends and meets the constraints
    import torch
    V, F = workload("icosphere_l3")
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        c = lib.tp_constraints(flags=3, A0=A0, V0=V0)
        rep_bh = lib.precond_step(m, c, lib.params(theta=0.5, krylov_max=300, proj_iters=3))
        f_bh = m.get_positions()
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        rep = lib.precond_step(m, c, lib.params(krylov_max=300, proj_iters=3))
    assert rep_bh["status"] == 0 and rep_bh["slope"] < 0 and rep_bh["E_after"] < rep_bh["E_before"]
    assert abs(O.total_area(f_bh, F) - A0) < 1e-7 * A0
    assert 0 < rep_bh["pair_interactions"] < rep["pair_interactions"]


def test_torus20k_bh_apply(lib):
    # full size: constants in the nullspace, approximation error of the
    # 9-column A apply against the direct apply at theta = 0.5
    import torch
    from synth import vertex_vectors
    V, F = workload("torus_20k")
    v = vertex_vectors(len(V), 9, 16)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        d = lib.fractional_apply(m, "A", v, lib.params())
        b = lib.fractional_apply(m, "A", v, lib.params(theta=0.5))
        one = lib.fractional_apply(m, "A", np.ones((len(V), 1)), lib.params(theta=0.5))
    assert rel(b, d) < 2e-3
    assert np.abs(one).max() <= 1e-5 * np.abs(b).max()


def test_torus20k_bh(lib):
    import torch
    V, F = workload("torus_20k")
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        p = lib.params(theta=0.5)
        E = lib.tp_energy(m, p)
        g, _ = lib.tp_differential(m, p)
    assert rel(E, O.bh_energy(V, F, 0.5)) <= TOL32
    idx = np.random.default_rng(5).choice(len(V), 32, replace=False)
    ref = O.bh_differential(V, F, 0.5, mode="full")
    assert rel(g[idx], ref[idx]) <= TOL32 and maxrel(g[idx], ref[idx]) <= 4 * TOL32


def test_icosphere_l8_bh_sample(lib):
    import torch
    V, F = workload("icosphere_l8")
    tg = np.random.default_rng(505).choice(len(F), 64, replace=False).astype(np.int32)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        rows = lib.tp_energy_rows(m, tg, lib.params(theta=0.5))
        rows_direct = lib.tp_energy_rows(m, tg, lib.params())
    tree = O.bvh_build(V, F, 8)
    Tr, L = O.bh_interactions(V, F, 0.5, 8, tg, tree)
    ref_bh, _ = O.bh_energy_rows(V, F, 0.5, 8, 6.0, tg)
    ref_direct = O.energy_rows(V, F, 6.0, tg)
    assert rel(rows, ref_bh) <= TOL32 and maxrel(rows, ref_bh) <= 4 * TOL32
    assert rel(rows_direct, ref_direct) <= TOL32 and maxrel(rows_direct, ref_direct) <= 4 * TOL32
    print("icosphere_l8 sample: BH(0.5) vs direct FP64 rows, relative error", rel(rows, ref_direct))


def test_bvh_refit_matches_oracle_refit(lib):
    # build on V, move to W: with bvh_refit the tree keeps V's face order
    # (oracle: bh_energy over that order at W); without, it is rebuilt
    import torch
    from synth import vertex_vectors
    V, F = small_mesh("torus30x11", seed=41)
    W = V + 0.004 * vertex_vectors(len(V), 3, 42)
    order_V = O.bvh_build(V, F, 8)["order"]
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        p_refit = lib.params(theta=0.5, bvh_refit=1)
        E_V = lib.tp_energy(m, p_refit)                 # first build (Morton order of V)
        assert rel(E_V, O.bh_energy(V, F, 0.5)) <= TOL32
        m.set_positions(dev(W, torch.float64))
        E_refit = lib.tp_energy(m, p_refit)
        assert rel(E_refit, O.bh_energy(W, F, 0.5, order=order_V)) <= TOL32
        g, _ = lib.tp_differential(m, p_refit)
        m.set_positions(dev(W, torch.float64))
        E_build = lib.tp_energy(m, lib.params(theta=0.5))
        assert rel(E_build, O.bh_energy(W, F, 0.5)) <= TOL32
    assert np.all(np.isfinite(g))


def _l8_samples():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "icosphere_l8_samples.json")
    return json.load(open(path))


@pytest.fixture(scope="module")
def icosphere_l8(lib):
    import torch
    V, F = workload("icosphere_l8")
    m = lib.Mesh(dev(V, torch.float64), dev(F, torch.int32))
    yield V, F, m
    m.close()


def test_icosphere_l8_direct_rows_20k_targets(lib, icosphere_l8):
    # full size (1,310,720 faces): FP32 direct rows of 20,000 seeded targets
    # against the oracle's stored FP64 direct rows (tests/golden/make_l8_samples.py);
    # the Barnes-Hut rows at theta = 0.5 against the same rows (approximation
    # error, reported; bounded loosely so that a broken traversal fails: on
    # this smooth bumpy sphere the oracle's own Barnes-Hut rows are 8-9% off
    # the direct sums at theta = 0.5 and 2-3% at theta = 0.25, levels 4-6)
    V, F, m = icosphere_l8
    smp = _l8_samples()
    tg = np.array(smp["targets"], dtype=np.int32)
    ref = np.array(smp["rows"])
    rows = lib.tp_energy_rows(m, dev(tg), lib.params()).cpu().numpy()
    assert rel(rows, ref) <= TOL32 and maxrel(rows, ref) <= 4 * TOL32
    rows_bh = lib.tp_energy_rows(m, dev(tg), lib.params(theta=0.5)).cpu().numpy()
    err = rel(rows_bh, ref)
    print("icosphere_l8, 20,000 targets: BH(0.5) rows vs FP64 direct, relative error", err)
    assert err < 0.15


def test_icosphere_l8_bh_differential_and_apply_sampled(lib, icosphere_l8):
    import torch
    from synth import vertex_vectors
    V, F, m = icosphere_l8
    smp = _l8_samples()
    vi = np.array(smp["vertices"])
    p = lib.params(theta=0.5)
    like = torch.empty((len(V), 3), dtype=torch.float64, device="cuda:0")
    g, _ = lib.tp_differential(m, p, like=like)
    u = dev(vertex_vectors(len(V), 3, 507), torch.float64)
    y = lib.fractional_apply(m, "A", u, p)
    eg = rel(g.cpu().numpy()[vi], smp["dE"])
    ey = rel(y.cpu().numpy()[vi], smp["Au"])
    print("icosphere_l8, 64 vertices: BH(0.5) vs FP64 direct: dE", eg, "A u", ey)
    assert eg < 0.3 and ey < 0.3


def test_icosphere_l8_poisson_solve_residual(lib, icosphere_l8):
    # the Poisson solve of the preconditioner at full size (655,362
    # vertices): the residual of the oracle's cotan matrix, and zero mean
    from synth import vertex_vectors
    V, F, m = icosphere_l8
    b = vertex_vectors(len(V), 3, 508)
    z, it = lib.cotan_solve(m, b, lib.params(cg_tol=1e-6))
    C = O.cotan_laplacian(V, F)
    bp = O.project_mean_zero(b)
    assert np.linalg.norm(C @ z - bp) <= 1.01e-6 * np.linalg.norm(bp)
    assert np.abs(z.mean(axis=0)).max() <= 1e-9 * np.abs(z).max()
