"""Mutation checks of the newer parts of the oracle: plant a plausible slip
in the oracle (on the CPU, by monkeypatching) and check that one of its
pins fails. Obstacles (§7.3.2): an unweighted sum over the obstacle faces,
and a flipped gradient. Willmore (§7.3.5): cotan weights without their 1/2.
Vertex pins (§7.2): zeroing the pinned rows of an unpinned solve instead of
appending the pin rows. Components (§7.1.1): one mean for the whole mesh."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import icosphere, small_mesh

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def sphere_closed_form(r, R, p):
    return 2.0 * np.pi * R / (r * (p - 2.0)) * (abs(R - r) ** (2.0 - p) - (R + r) ** (2.0 - p))


def test_unweighted_obstacle_sum_fails_the_sphere_closed_form(monkeypatch):
    V, F = icosphere(4, 1.0)
    x = np.array([[0.18, 0.24, 0.0]])
    assert O.obstacle_potential(x, V, F)[0] == pytest.approx(sphere_closed_form(0.3, 1.0, 6.0), rel=1e-2)
    orig = O.face_geometry

    def unweighted(f, faces):
        X, N, a = orig(f, faces)
        return X, N, np.ones_like(a)          # the slip: a_O(S) left out
    monkeypatch.setattr(O, "face_geometry", unweighted)
    assert O.obstacle_potential(x, V, F)[0] != pytest.approx(sphere_closed_form(0.3, 1.0, 6.0), rel=1e-1)


def test_flipped_obstacle_gradient_fails_central_differences(monkeypatch):
    V, F = small_mesh("ico2", seed=3)
    V = 0.35 * V
    VO, FO = icosphere(2, 1.0)
    orig = O.obstacle_potential

    def flipped(x, fO, facesO, p=6.0, grad=False):
        if not grad:
            return orig(x, fO, facesO, p)
        phi, g = orig(x, fO, facesO, p, grad=True)
        return phi, -g                         # the slip: d = x - f_O(S)
    monkeypatch.setattr(O, "obstacle_potential", flipped)
    g = O.obstacle_differential(V, F, VO, FO)
    dv = np.random.default_rng(1).standard_normal(V.shape)
    h = 1e-6
    fd = (O.obstacle_energy(V + h * dv, F, VO, FO) - O.obstacle_energy(V - h * dv, F, VO, FO)) / (2 * h)
    assert abs(np.sum(g * dv) - fd) > 1e-3 * abs(fd)


def test_cotan_weights_without_half_fail_the_sphere_value(monkeypatch):
    V, F = icosphere(4)
    assert O.willmore_energy(V, F) == pytest.approx(16 * np.pi, rel=5e-3)
    orig = O.cotan_laplacian
    monkeypatch.setattr(O, "cotan_laplacian", lambda f, faces: 2.0 * orig(f, faces))   # cot, not cot/2
    assert O.willmore_energy(V, F) != pytest.approx(16 * np.pi, rel=0.5)


def test_zeroed_rows_instead_of_pin_rows_fail_the_reproduction(monkeypatch):
    V, F = small_mesh("ico2", seed=2)
    pins = [0, 7, 40]
    C = O.cotan_laplacian(V, F)
    y = np.random.default_rng(3).standard_normal((len(V), 2))
    y[pins] = 0.0

    def zeroed(C, b, pins):
        z = O.poisson_solve(C, b)              # the slip: an unpinned solve ...
        z[np.asarray(pins)] = 0.0              # ... with the pinned rows set to 0
        return z
    monkeypatch.setattr(O, "pinned_poisson_solve", zeroed)
    z = O.pinned_poisson_solve(C, C @ y, pins)
    assert np.abs(z - y).max() > 1e-3 * np.abs(y).max()


def test_whole_mesh_mean_fails_the_per_component_solve(monkeypatch):
    A = small_mesh("ico2", seed=3)
    B = small_mesh("torus13x7", seed=4)
    V = np.concatenate([A[0], 0.6 * B[0] + np.array([2.2, 0.0, 0.0])])
    F = np.concatenate([A[1], B[1] + len(A[0])])
    na = len(A[0])
    b = np.random.default_rng(2).standard_normal((len(V), 1))
    orig = O.project_mean_zero
    monkeypatch.setattr(O, "project_mean_zero", lambda b, comp=None: orig(b))   # the slip: one mean
    comp = O.mesh_components(len(V), F)
    z = O.poisson_solve(O.cotan_laplacian(V, F), b, comp)
    za = orig(O.poisson_solve(O.cotan_laplacian(*A), b[:na]))
    assert np.abs(z[:na] - za).max() > 1e-6 * np.abs(za).max()
