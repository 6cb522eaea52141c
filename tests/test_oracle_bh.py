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


# ---------------------------------------------------------------------------
# Barnes-Hut operator applies (the kernel-matrix products of §5.1.1-5.1.3
# over the admissible sets of §4.1, node-average projector of §5.1.4)
# ---------------------------------------------------------------------------

OPS = ["A", "B", "B0", "L"]


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("mesh,leaf", [("ico3", 8), ("torus20x9", 4)])
def test_bh_apply_theta_zero_is_the_direct_apply(op, mesh, leaf):
    from synth import vertex_vectors
    V, F = small_mesh(mesh, seed=3)
    v = vertex_vectors(len(V), 3, 5)
    ref = O.apply_operator(V, F, v, op)
    got = O.bh_apply_operator(V, F, v, op, 0.0, leaf)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("op", OPS)
def test_bh_apply_keeps_constants_in_the_nullspace(op):
    # r = H~ a uses the same approximation as H~ W, so O 1 = 0 at any theta
    from synth import vertex_vectors
    V, F = small_mesh("ico3", seed=4)
    scale = np.abs(O.bh_apply_operator(V, F, vertex_vectors(len(V), 1, 6), op, 0.7)).max()
    one = O.bh_apply_operator(V, F, np.ones((len(V), 1)), op, 0.7)
    assert np.abs(one).max() <= 1e-11 * scale


@pytest.mark.parametrize("op", OPS)
def test_bh_apply_error_falls_with_theta(op):
    from synth import vertex_vectors
    V, F = small_mesh("ico3", seed=5)
    v = vertex_vectors(len(V), 3, 7)
    ref = O.apply_operator(V, F, v, op)
    errs = [np.linalg.norm(O.bh_apply_operator(V, F, v, op, th) - ref) / np.linalg.norm(ref)
            for th in (0.25, 0.5, 1.0)]
    assert errs[0] < errs[1] < errs[2]
    assert errs[1] < 5e-3


def test_bh_apply_translation_and_scaling():
    # the tree is built in the frame of the bounding-box centre from codes
    # quantised to the bounding box: translation and uniform scaling keep the
    # tree and the admissible sets, so the applies transform like the exact
    # ones (A(lambda f) = lambda^(2 - 2s) A(f), L(lambda f) = lambda^(2s - 2) L(f))
    from synth import vertex_vectors
    V, F = small_mesh("torus20x9", seed=6)
    v = vertex_vectors(len(V), 2, 8)
    s = O.sobolev_s(6.0)
    for op, expo in (("A", 2.0 - 2.0 * s), ("L", 2.0 * s - 2.0)):
        y = O.bh_apply_operator(V, F, v, op, 0.6)
        yt = O.bh_apply_operator(V + np.array([0.3, -1.7, 2.2]), F, v, op, 0.6)
        ys = O.bh_apply_operator(2.5 * V, F, v, op, 0.6)
        assert np.linalg.norm(yt - y) <= 1e-9 * np.linalg.norm(y)
        assert np.linalg.norm(ys - 2.5 ** expo * y) <= 1e-9 * np.linalg.norm(y)


def _two_patches(D, seed, planar):
    """Two disjoint small patches: a planar 2x2 grid near the origin (the
    targets) and an irregular 8-face source patch (one leaf) centred near
    (D, 0, 0), curved or planar and tilted."""
    rng = np.random.default_rng(seed)
    g = np.array([[x, y, 0.0] for y in range(3) for x in range(3)], float) * 0.1
    quads = [(0, 1, 4, 3), (1, 2, 5, 4), (3, 4, 7, 6), (4, 5, 8, 7)]
    Fa = []
    for a_, b_, c_, d_ in quads:
        Fa += [(a_, b_, c_), (a_, c_, d_)]
    h = g.copy()
    h[:, :2] += 0.02 * rng.standard_normal((9, 2))          # irregular areas
    h[:, 2] = 0.3 * h[:, 0] + 0.2 * h[:, 1]                  # tilted plane
    if not planar:
        h[:, 2] += 2.0 * (h[:, 0] - 0.1) ** 2
    h = h + np.array([D, 0.0, 0.0])
    V = np.concatenate([g, h])
    F = np.array(Fa + [(i + 9, j + 9, k + 9) for i, j, k in Fa], dtype=np.int64)
    return V, F


@pytest.mark.parametrize("kind,planar", [("plain", False), ("low", True)])
def test_bh_far_field_is_second_order(kind, planar):
    # W = a on the source patch, 0 on the targets: the target rows of z are
    # -(H W), a pure far-field sum over the source node. X_I is the
    # area-weighted barycenter, so the first-order (dipole) term of the
    # Taylor expansion cancels and the relative error falls like (r_I / D)^2:
    # doubling D divides it by about four (a plain centroid would leave a
    # first-order error, ratio ~2). For the low-order kernel the source
    # patch is planar, where the node-average projector is the faces' own.
    errs = []
    for D in (1.0, 2.0, 4.0):
        V, F = _two_patches(D, 9, planar)
        X, N, a = O.face_geometry(V, F)
        T, L = O.bh_interactions(V, F, 0.9, leaf=8)
        assert set(range(8)) <= set(L["far_s"].tolist())     # the source leaf is a far node
        assert not np.any(L["near_s"] < 8) or np.all(L["near_t"][L["near_s"] < 8] < 8)
        Pbar = O.bvh_average_projectors(V, F, T)
        W = np.where(np.arange(len(F)) >= 8, a, 0.0)[:, None]
        z_bh = O.bh_kernel_apply(T, L, T["Xr"], N, a, W, kind, 10.0 / 3.0, Pbar)[:8, 0]
        z_ex = O.kernel_apply(T["Xr"], N, a, W, kind, 10.0 / 3.0)[:8, 0]
        errs.append(np.abs(z_bh - z_ex).max() / np.abs(z_ex).max())
    assert errs[0] < 0.1
    assert 3.0 < errs[0] / errs[1] < 5.5 and 3.0 < errs[1] / errs[2] < 5.5


def test_bh_low_order_uses_the_average_projector():
    # a curved source node: |P_I d|^2 with the average projector differs from
    # the average of |P_T d|^2, so the low-order far term keeps an error that
    # does not vanish with D, while the plain kernel's does
    e_low, e_plain = [], []
    for D in (2.0, 4.0):
        V, F = _two_patches(D, 9, planar=False)
        X, N, a = O.face_geometry(V, F)
        T, L = O.bh_interactions(V, F, 0.9, leaf=8)
        Pbar = O.bvh_average_projectors(V, F, T)
        W = np.where(np.arange(len(F)) >= 8, a, 0.0)[:, None]
        for kind, out in (("low", e_low), ("plain", e_plain)):
            z_bh = O.bh_kernel_apply(T, L, T["Xr"], N, a, W, kind, 10.0 / 3.0, Pbar)[:8, 0]
            z_ex = O.kernel_apply(T["Xr"], N, a, W, kind, 10.0 / 3.0)[:8, 0]
            out.append(np.abs(z_bh - z_ex).max() / np.abs(z_ex).max())
    assert e_plain[0] / e_plain[1] > 3.0
    assert e_low[0] / e_low[1] < 2.0
    # the node projector is the area average of the faces' projectors and
    # is no projector itself (its square differs from it)
    V, F = _two_patches(4.0, 9, planar=False)
    T, _ = O.bh_interactions(V, F, 0.9, leaf=8)
    P = O.bvh_average_projectors(V, F, T)
    leaf = [i for i in range(len(T["first"])) if T["leaf"][i] and T["first"][i] == 8][0]
    assert np.trace(P[leaf]) == pytest.approx(1.0, rel=1e-12)
    assert np.linalg.norm(P[leaf] @ P[leaf] - P[leaf]) > 1e-4


def test_bh_far_field_pin_catches_a_plain_centroid():
    # plant a mistake in the oracle's tree (node X_I = plain centroid of the
    # face barycenters): the second-order pin above must no longer hold
    errs = []
    for D in (1.0, 2.0, 4.0):
        V, F = _two_patches(D, 9, planar=False)
        X, N, a = O.face_geometry(V, F)
        T, L = O.bh_interactions(V, F, 0.9, leaf=8)
        bad = dict(T)
        bad["X"] = T["X"].copy()
        for nid in range(len(T["first"])):
            Tf = T["order"][T["first"][nid]:T["first"][nid] + T["count"][nid]]
            bad["X"][nid] = T["Xr"][Tf].mean(axis=0)
        Pbar = O.bvh_average_projectors(V, F, T)
        W = np.where(np.arange(len(F)) >= 8, a, 0.0)[:, None]
        z_bh = O.bh_kernel_apply(bad, L, T["Xr"], N, a, W, "plain", 10.0 / 3.0, Pbar)[:8, 0]
        z_ex = O.kernel_apply(T["Xr"], N, a, W, "plain", 10.0 / 3.0)[:8, 0]
        errs.append(np.abs(z_bh - z_ex).max() / np.abs(z_ex).max())
    assert not (3.0 < errs[0] / errs[1] < 5.5 and 3.0 < errs[1] / errs[2] < 5.5)


# ---------------------------------------------------------------------------
# refit: a tree keeps the face order of other positions (only node data move)
# ---------------------------------------------------------------------------

def test_refit_tree_is_valid_for_any_order():
    # any face order gives a partition: theta = 0 stays exact, node data are
    # those of the new positions, radii bound the vertices
    V, F = small_mesh("torus20x9", seed=11)
    order = np.random.default_rng(3).permutation(len(F))
    T = O.bvh_build(V, F, 8, order=order)
    assert list(T["order"]) == list(order)
    assert O.bh_energy(V, F, 0.0, 8, order=order) == pytest.approx(O.energy(V, F), rel=1e-13)
    a = O.face_geometry(V, F)[2]
    assert T["a"][0] == pytest.approx(a.sum(), rel=1e-13)
    vx = V[F] - T["c"]
    for nid in range(len(T["first"])):
        Tf = T["order"][T["first"][nid]:T["first"][nid] + T["count"][nid]]
        assert np.linalg.norm(vx[Tf].reshape(-1, 3) - T["X"][nid], axis=1).max() <= T["r"][nid] * (1 + 1e-12)


def test_refit_with_the_own_order_is_the_build_and_drifts_gently():
    V, F = small_mesh("ico3", seed=12)
    own = O.bvh_build(V, F, 8)["order"]
    assert O.bh_energy(V, F, 0.5, order=own) == pytest.approx(O.bh_energy(V, F, 0.5), rel=1e-14)
    # a small motion: the refit (old order) approximates the new energy as
    # well as a rebuild does (the tree quality drifts only with large motion)
    from synth import vertex_vectors
    for eps in (0.001, 0.01):
        W = V + eps * vertex_vectors(len(V), 3, 13)
        ex = O.energy(W, F)
        e_refit = abs(O.bh_energy(W, F, 0.5, order=own) - ex) / ex
        e_build = abs(O.bh_energy(W, F, 0.5) - ex) / ex
        assert e_refit <= 1.2 * e_build + 1e-3
