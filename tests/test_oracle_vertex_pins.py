"""Pins of the vertex-pin part of the oracle (§7.1.2, §7.2).

The Poisson solve with pin rows appended returns y exactly when the
right-hand side is C y for a y that vanishes at the pins, and equals the
elimination of the pinned rows and columns; the pinned descent direction
is zero at the pins, tangent to the area and volume constraints, a descent
direction, the same by the dense saddle solve and by the Schur complement
with the pin rows kept in the matrix, and without area/volume rows it is
-A_FF^{-1} g_F; a pinned step keeps the pinned vertices where they are and
projects onto the constraints."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import tp_oracle as O
from synth import icosphere, small_mesh

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def two_spheres():
    V1, F1 = small_mesh("ico2", seed=4)
    V2, F2 = small_mesh("ico1", seed=5)
    V = np.concatenate([V1, 0.5 * V2 + np.array([3.0, 0.0, 0.0])])
    F = np.concatenate([F1, F2 + len(V1)])
    return V, F, [5, len(V1) + 3]


@pytest.mark.parametrize("case", ["ico2", "torus13x7", "two_spheres"])
def test_pinned_poisson_solve_reproduces_and_eliminates(case):
    if case == "two_spheres":
        V, F, pins = two_spheres()
    else:
        V, F = small_mesh(case, seed=2)
        pins = [0, 7, 40]
    C = O.cotan_laplacian(V, F)
    rng = np.random.default_rng(3)
    y = rng.standard_normal((len(V), 3))
    y[pins] = 0.0
    z = O.pinned_poisson_solve(C, C @ y, pins)
    assert np.abs(z - y).max() < 1e-10 * np.abs(y).max()
    # elimination of the pinned rows and columns, any right-hand side
    b = rng.standard_normal((len(V), 2))
    z = O.pinned_poisson_solve(C, b, pins)
    free = np.setdiff1d(np.arange(len(V)), pins)
    lu = spla.splu(C[free][:, free].tocsc())
    for c in range(2):
        assert np.allclose(z[free, c], lu.solve(b[free, c]), rtol=1e-10, atol=1e-12)
    assert np.all(z[pins] == 0.0) or np.abs(z[pins]).max() < 1e-13


def test_pinned_direction_properties():
    V, F = small_mesh("ico2", seed=6)
    pins = [3, 50, 121]
    x, g = O.descent_direction(V, F, pins=pins)
    assert np.abs(x[pins]).max() < 1e-11 * np.abs(x).max()
    gA, gV = O.area_gradient(V, F), O.volume_gradient(V, F)
    assert abs(np.sum(gA * x)) < 1e-10 * np.linalg.norm(gA) * np.linalg.norm(x)
    assert abs(np.sum(gV * x)) < 1e-10 * np.linalg.norm(gV) * np.linalg.norm(x)
    assert np.sum(g * x) < 0
    xs, Z, S = O.schur_direction(V, F, pins=pins)
    assert np.abs(x - xs).max() < 1e-9 * np.abs(x).max()
    # the barycenter is free to move once pins are used
    assert np.linalg.norm(x.mean(axis=0)) > 1e-6 * np.abs(x).max()


def test_pinned_direction_without_area_volume_is_the_restricted_solve():
    V, F = small_mesh("torus13x7", seed=1)
    pins = [0, 50]
    x, g = O.descent_direction(V, F, use_area=False, use_volume=False, pins=pins)
    A = O.operator_matrix(V, F, "A")
    free = np.setdiff1d(np.arange(len(V)), pins)
    xf = -np.linalg.solve(A[np.ix_(free, free)], g[free])
    assert np.allclose(x[free], xf, rtol=1e-9, atol=1e-12 * np.abs(xf).max())


def test_pinned_step_keeps_pins_and_projects():
    V, F = small_mesh("ico2", seed=9)
    pins = [1, 60, 140]
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    r = O.precond_step(V, F, A0, V0, proj_iters=3, pins=pins)
    assert np.abs(r["f_new"][pins] - V[pins]).max() < 1e-13
    assert abs(O.total_area(r["f_new"], F) - A0) < 1e-8 * A0
    assert abs(O.total_volume(r["f_new"], F) - V0) < 1e-8 * abs(V0)
    assert r["E1"] < r["E0"]


def test_pinned_preconditioner_is_symmetric_and_zero_at_pins():
    V, F = small_mesh("ico2", seed=2)
    pins = [0, 100]
    rng = np.random.default_rng(8)
    u, v = rng.standard_normal((len(V), 1)), rng.standard_normal((len(V), 1))
    u[pins] = 0.0
    v[pins] = 0.0
    Pu = O.precond_apply(V, F, u, pins=pins)
    Pv = O.precond_apply(V, F, v, pins=pins)
    assert np.abs(Pu[pins]).max() < 1e-12 * np.abs(Pu).max()
    assert float(np.sum(v * Pu)) == pytest.approx(float(np.sum(u * Pv)), rel=1e-9)
    assert float(np.sum(u * Pu)) > 0
