"""Pins of the Barnes-Hut part of the oracle (§4): theta = 0 is the exact
sum, the error falls with theta like O(theta^2), the 'full' differential is
the exact gradient of the frozen-list Barnes-Hut energy (central
differences), and the tree is a valid partition."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import small_mesh

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("mesh,leaf", [("ico3", 8), ("torus20x9", 4), ("ico2", 1)])
def test_theta_zero_is_exact(mesh, leaf):
    V, F = small_mesh(mesh, seed=2)
    assert O.bh_energy(V, F, 0.0, leaf) == pytest.approx(O.energy(V, F), rel=1e-13)


def test_tree_partitions_faces_and_nodes_aggregate():
    V, F = small_mesh("torus20x9", seed=1)
    T = O.bvh_build(V, F, 8)
    assert sorted(T["order"]) == list(range(len(F)))
    a = O.face_geometry(V, F)[2]
    assert T["a"][0] == pytest.approx(a.sum(), rel=1e-13)
    # escape index = first node after the subtree; leaves cover the faces once
    leaves = np.nonzero(T["leaf"])[0]
    assert T["count"][leaves].sum() == len(F)
    assert all(T["skip"][i] == i + 1 for i in leaves)
    assert T["skip"][0] == len(T["first"])
    # the radius bounds every vertex of the node
    vx = V[F] - T["c"]
    for nid in range(len(T["first"])):
        Tf = T["order"][T["first"][nid]:T["first"][nid] + T["count"][nid]]
        d = np.linalg.norm(vx[Tf].reshape(-1, 3) - T["X"][nid], axis=1)
        assert d.max() <= T["r"][nid] * (1 + 1e-12)


def test_error_falls_like_theta_squared():
    V, F = small_mesh("ico3", seed=2)
    E = O.energy(V, F)
    err = {th: abs(O.bh_energy(V, F, th) - E) / E for th in (0.25, 0.5, 1.0)}
    assert err[0.25] < err[0.5] < err[1.0]
    assert err[0.5] / err[0.25] > 2.5          # roughly quadratic in theta


def test_full_differential_is_gradient_of_frozen_energy():
    V, F = small_mesh("ico2", seed=3)
    T, L = O.bh_interactions(V, F, 0.5)
    g = O.bh_differential(V, F, 0.5, mode="full")
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        dv = rng.standard_normal(V.shape)
        fd = (O.bh_energy_frozen(V + h * dv, F, T, L) - O.bh_energy_frozen(V - h * dv, F, T, L)) / (2 * h)
        assert np.sum(g * dv) == pytest.approx(fd, rel=1e-6)
    assert O.bh_energy_frozen(V, F, T, L) == pytest.approx(O.bh_energy(V, F, 0.5), rel=1e-13)


def test_full_differential_at_theta_zero_is_exact():
    V, F = small_mesh("ico2", seed=4)
    g = O.bh_differential(V, F, 0.0, mode="full")
    ref = O.differential(V, F)
    assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)


def test_literal_differential_keeps_only_target_side():
    # literal = full minus the source-side terms; at theta = 0 it is the
    # derivative of sum_S sum_T K(S,T) a_S a_T through S's own data only
    V, F = small_mesh("ico1", seed=4)
    gl = O.bh_differential(V, F, 0.0, mode="literal")
    gX, gN, ga = O.face_adjoints(V, F)
    ref = O.differential(V, F)
    assert np.linalg.norm(gl - ref) > 0.1 * np.linalg.norm(ref)
