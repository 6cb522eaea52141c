"""GPU parity of the static-obstacle term (§7.3.2) against the FP64 oracle,
through the C ABI: direct sums in FP32 and FP64 (several tiles, ragged
tails, near pairs, a generic exponent), Barnes-Hut over the obstacle's BVH
(same admissible sets, counted interactions), the frame refresh after the
surface moves, the constrained step with an obstacle, and the full-size
scene (torus_20k around a 20,480-face ball) in the benchmark's launch
configuration."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import icosphere, obstacle, small_mesh, workload

pytestmark = pytest.mark.gpu

TOL32, TOL64 = 1e-5, 1e-10


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


def scene(name):
    """(surface V, F, obstacle VO, FO) of small parity scenes."""
    if name == "ico3_in_ball":          # 1280 targets, 1280 sources: 10 x 10 tiles
        V, F = small_mesh("ico3", seed=4)
        VO, FO = icosphere(3, 1.6)
        return 0.8 * V, F, VO + np.array([0.05, -0.1, 0.02]), FO
    if name == "torus_around_octa":     # 182 targets (ragged), 8 sources (one partial tile)
        V, F = small_mesh("torus13x7", seed=5)
        VO, FO = small_mesh("octa")
        return V, F, 0.4 * VO, FO
    if name == "tetra_near_ico2":       # 4 targets, 320 sources, surface close to the obstacle
        V, F = small_mesh("tetra")
        VO, FO = icosphere(2, 1.0)
        return 0.05 * V + np.array([0.0, 0.0, 0.9]), F, VO, FO
    if name == "ico2_beside_torus":     # obstacle outside the surface, ragged both ways
        V, F = small_mesh("ico2", seed=6)
        VO, FO = small_mesh("torus13x7", seed=9)
        return 0.3 * V + np.array([1.0, 0.0, 0.0]), F, VO, FO
    raise KeyError(name)


SCENES = ["ico3_in_ball", "torus_around_octa", "tetra_near_ico2", "ico2_beside_torus"]


def _mesh_with_obstacle(lib, V, F, VO, FO, w=1.0):
    import torch
    m = lib.Mesh(dev(V, torch.float64), dev(F, torch.int32))
    lib.tp_obstacle_set(m, dev(VO, torch.float64), dev(FO, torch.int32), w)
    return m


@pytest.mark.parametrize("name", SCENES)
@pytest.mark.parametrize("prec", [0, 1])
def test_direct_energy_and_differential(lib, name, prec):
    V, F, VO, FO = scene(name)
    w = 0.75
    with _mesh_with_obstacle(lib, V, F, VO, FO, w) as m:
        E, g = lib.tp_obstacle_energy(m, lib.params(precision=prec))
        E_only, none = lib.tp_obstacle_energy(m, lib.params(precision=prec), grad=False)
    tol = TOL32 if prec == 0 else TOL64
    E_ref = O.obstacle_energy(V, F, VO, FO, 6.0, w)
    g_ref = O.obstacle_differential(V, F, VO, FO, 6.0, w)
    assert none is None
    assert rel(E, E_ref) <= tol and rel(E_only, E_ref) <= tol
    assert rel(g, g_ref) <= tol
    assert np.abs(g - g_ref).max() <= 10 * tol * np.abs(g_ref).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [4.5, 3.0])
def test_direct_generic_exponent(lib, prec, p):
    V, F, VO, FO = scene("ico3_in_ball")
    with _mesh_with_obstacle(lib, V, F, VO, FO) as m:
        E, g = lib.tp_obstacle_energy(m, lib.params(precision=prec, p=p))
    tol = TOL32 if prec == 0 else TOL64
    assert rel(E, O.obstacle_energy(V, F, VO, FO, p)) <= tol
    assert rel(g, O.obstacle_differential(V, F, VO, FO, p)) <= tol


def test_frame_follows_the_surface(lib):
    # after the surface moves (new reference frame) the obstacle, which did
    # not move, is re-expressed in the new frame
    import torch
    V, F, VO, FO = scene("ico3_in_ball")
    with _mesh_with_obstacle(lib, V, F, VO, FO) as m:
        V2 = 0.9 * V + np.array([0.2, 0.1, -0.15])
        m.set_positions(dev(V2, torch.float64))
        E, g = lib.tp_obstacle_energy(m, lib.params())
        assert rel(E, O.obstacle_energy(V2, F, VO, FO)) <= TOL32
        assert rel(g, O.obstacle_differential(V2, F, VO, FO)) <= TOL32
        # replacing the obstacle and removing it
        lib.tp_obstacle_set(m, dev(2.0 * VO, torch.float64), dev(FO, torch.int32), 2.0)
        E2, _ = lib.tp_obstacle_energy(m, lib.params(), grad=False)
        assert rel(E2, O.obstacle_energy(V2, F, 2.0 * VO, FO, 6.0, 2.0)) <= TOL32
        lib.tp_obstacle_set(m, None)
        with pytest.raises(lib.TpError):
            lib.tp_obstacle_energy(m, lib.params())


def test_invalid_obstacles_are_rejected(lib):
    import torch
    V, F, VO, FO = scene("torus_around_octa")
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        bad = FO.copy()
        bad[0, 0] = len(VO)
        with pytest.raises(lib.TpError):
            lib.tp_obstacle_set(m, VO, bad, 1.0)
        with pytest.raises(lib.TpError):
            lib.tp_obstacle_set(m, VO, FO, -1.0)
        flat = VO.copy()
        flat[:, 1:] = 0.0                  # every vertex on the x axis: zero-area faces
        with pytest.raises(lib.TpError):
            lib.tp_obstacle_set(m, flat, FO, 1.0)
        # the mesh still works without an obstacle
        assert rel(lib.tp_energy(m, lib.params(precision=1)), O.energy(V, F)) <= TOL64


def _bh_count(lib, m):
    st = lib.tp_profile_read(m)
    return st.get("bh_obstacle", {}).get("units", 0.0)


@pytest.mark.parametrize("theta,leaf,err", [(0.5, 8, 5e-3), (0.3, 4, 2e-3), (1.0, 1, 0.1)])
def test_barnes_hut_matches_oracle(lib, theta, leaf, err):
    V, F, VO, FO = scene("ico3_in_ball")
    w = 1.25
    with _mesh_with_obstacle(lib, V, F, VO, FO, w) as m:
        lib.tp_profile_read(m)
        E, g = lib.tp_obstacle_energy(m, lib.params(theta=theta, leaf_size=leaf))
        n = _bh_count(lib, m)
    E_ref, g_ref, n_ref = O.bh_obstacle_energy(V, F, VO, FO, theta, leaf, 6.0, w)
    assert n == n_ref
    assert rel(E, E_ref) <= TOL32
    assert rel(g, g_ref) <= TOL32
    # and it approximates the direct sum (oracle: 1.5e-3, 5e-4, 7.2e-2)
    assert rel(E, O.obstacle_energy(V, F, VO, FO, 6.0, w)) < err


def test_barnes_hut_tiny_theta_is_the_direct_sum(lib):
    V, F, VO, FO = scene("ico2_beside_torus")
    with _mesh_with_obstacle(lib, V, F, VO, FO) as m:
        E, g = lib.tp_obstacle_energy(m, lib.params(theta=1e-4))
    assert rel(E, O.obstacle_energy(V, F, VO, FO)) <= TOL32
    assert rel(g, O.obstacle_differential(V, F, VO, FO)) <= TOL32


def test_precond_step_with_obstacle_matches_oracle(lib):
    import torch
    V, F = small_mesh("ico2", seed=3)
    V = 0.4 * V
    VO, FO = icosphere(2, 1.0)
    VO = VO + np.array([0.3, 0.0, 0.0])
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    tau = 0.05
    ref = O.precond_step(V, F, A0, V0, fixed_tau=tau, obstacle=(VO, FO, 0.5))
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        lib.tp_obstacle_set(m, VO, FO, 0.5)
        c = lib.tp_constraints(flags=lib.TP_CONSTRAINT_AREA | lib.TP_CONSTRAINT_VOLUME, A0=A0, V0=V0)
        p = lib.params(precision=1, krylov_tol=1e-11, cg_tol=1e-12, fixed_tau=1, tau0=tau)
        rep = lib.precond_step(m, c, p)
        f_new = m.get_positions()
    assert rep["status"] == 0 and rep["slope"] < 0
    assert rel(rep["E_before"], ref["E0"]) < 1e-10
    assert rel(f_new - V, ref["f_new"] - V) < 1e-7
    assert rel(rep["E_after"], ref["E1"]) < 1e-8


def test_armijo_steps_with_obstacle_descend(lib):
    # FP32 path, line search on E + E_O, direct then Barnes-Hut for both
    # terms. The weight keeps E_O comparable to E: at weight 1 this scene's
    # first direction is 55 times the sphere's radius and the oracle's step
    # blows the sphere apart too (Armijo accepts the far-away minimum).
    import torch
    V, F = small_mesh("ico3", seed=2)
    V = 0.5 * V
    VO, FO = icosphere(3, 1.0)
    VO = VO + np.array([0.35, 0.0, 0.0])
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        lib.tp_obstacle_set(m, VO, FO, 0.01)
        c = lib.tp_constraints(flags=3, A0=A0, V0=V0)
        for theta in (0.0, 0.5):
            p = lib.params(theta=theta, krylov_max=300, proj_iters=2)
            for _ in range(2):
                rep = lib.precond_step(m, c, p)
                assert rep["slope"] < 0 and rep["E_after"] < rep["E_before"]
        f = m.get_positions()
    E_tot = O.energy(f, F) + O.obstacle_energy(f, F, VO, FO, 6.0, 0.01)
    assert E_tot < O.energy(V, F) + O.obstacle_energy(V, F, VO, FO, 6.0, 0.01)


# ---------------------------------------------------------------------------
# full size: torus_20k around the 20,480-face ball, benchmark configuration
# ---------------------------------------------------------------------------

def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size.json")
    return json.load(open(path))[name]


def test_torus20k_ball_obstacle_full(lib):
    import torch
    V, F = workload("torus_20k")
    VO, FO = obstacle("ball_in_torus_hole")
    with _mesh_with_obstacle(lib, V, F, VO, FO) as m:
        E, g = lib.tp_obstacle_energy(m, lib.params())
        Eb, gb = lib.tp_obstacle_energy(m, lib.params(theta=0.5))
    assert rel(E, _golden("torus_20k+ball_in_torus_hole")["obstacle_energy"]) <= TOL32
    # sampled vertices: the obstacle term of a face depends on that face
    # alone, so the faces incident to the sampled vertices give their rows
    idx = np.random.default_rng(31).choice(len(V), 64, replace=False)
    inc = np.nonzero(np.isin(F, idx).any(axis=1))[0]
    ref = O.obstacle_differential(V, F[inc], VO, FO)[idx]
    assert rel(g[idx], ref) <= TOL32 and maxrel(g[idx], ref) <= 4 * TOL32
    # Barnes-Hut at the benchmark's theta: the oracle's Barnes-Hut over the
    # same tree (its error against the direct sum is about 4% here)
    Eb_ref, gb_ref, _ = O.bh_obstacle_energy(V, F, VO, FO, 0.5, 8)
    assert rel(Eb, Eb_ref) <= TOL32
    assert rel(gb, gb_ref) <= TOL32 and maxrel(gb, gb_ref) <= 4 * TOL32


def test_free_barycenter_step_matches_oracle(lib):
    # barycenter motion (§7.1.1) with an obstacle: the FP64 step equals the
    # oracle's; the surface is translated away from the nearer wall; pins
    # and a free barycenter are rejected together
    import torch
    V, F = icosphere(2, 0.2)
    V = V + np.array([0.4, 0.0, 0.0])
    VO, FO = icosphere(3, 1.0)
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    ref = O.precond_step(V, F, A0, V0, fixed_tau=0.02, obstacle=(VO, FO, 1e-3), free_barycenter=True)
    flags = lib.TP_CONSTRAINT_AREA | lib.TP_CONSTRAINT_VOLUME | lib.TP_CONSTRAINT_FREE_BARYCENTER
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        lib.tp_obstacle_set(m, VO, FO, 1e-3)
        c = lib.tp_constraints(flags=flags, A0=A0, V0=V0)
        p = lib.params(precision=1, krylov_tol=1e-11, cg_tol=1e-12, fixed_tau=1, tau0=0.02, krylov_max=400)
        rep = lib.precond_step(m, c, p)
        f_new = m.get_positions()
        assert rep["status"] == 0 and rep["slope"] < 0
        # FP32 Armijo steps keep moving the sphere towards the centre
        for _ in range(2):
            rep = lib.precond_step(m, c, lib.params(krylov_max=300, proj_iters=2))
            assert rep["E_after"] < rep["E_before"]
        f2 = m.get_positions()
        lib.tp_pins_set(m, np.array([0], dtype=np.int32))
        with pytest.raises(lib.TpError):
            lib.precond_step(m, c, lib.params())
    assert rel(f_new - V, ref["f_new"] - V) < 1e-7
    assert f_new.mean(axis=0)[0] < V.mean(axis=0)[0]
    assert f2.mean(axis=0)[0] < f_new.mean(axis=0)[0]
