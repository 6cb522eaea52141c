"""Pins of the within-face term of the preconditioner's L^{2-s} (oracle).

The term is a face-weighted P1 stiffness matrix: constants are in its
nullspace, it is symmetric positive semidefinite, it equals w times the
cotan matrix when every face has the same area, and on a planar mesh its
quadratic form of a linear function u = c.x is sum_S w_S a_S |c|^2. With
it, the preconditioned operator's condition number stays small on a rough
torus (without it, it is in the hundreds and grows with refinement)."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import gaussian_noise, small_mesh, torus

SIG = 2.0 - O.sobolev_s(6.0)


def flat_grid(n, jitter=0.0, seed=0):
    xs = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(n * n)], axis=1)
    if jitter:
        rng = np.random.default_rng(seed)
        inner = (X.ravel() > 0) & (X.ravel() < 1) & (Y.ravel() > 0) & (Y.ravel() < 1)
        V[inner, :2] += jitter / n * rng.uniform(-1, 1, (inner.sum(), 2))
    F = []
    for i in range(n - 1):
        for j in range(n - 1):
            a, b, c, d = i * n + j, (i + 1) * n + j, (i + 1) * n + j + 1, i * n + j + 1
            F += [[a, b, c], [a, c, d]]
    return V, np.array(F)


def test_nullspace_symmetry_psd():
    V, F = small_mesh("torus13x7", seed=3)
    G = O.self_term_stiffness(V, F, SIG, 8.0).toarray()
    assert np.abs(G @ np.ones(len(V))).max() < 1e-12 * np.abs(G).max()
    assert np.abs(G - G.T).max() < 1e-14 * np.abs(G).max()
    assert np.linalg.eigvalsh(G).min() > -1e-12 * np.abs(G).max()


def test_equal_areas_give_a_multiple_of_the_cotan_matrix():
    V, F = flat_grid(7)
    a = O.face_geometry(V, F)[2]
    assert np.ptp(a) < 1e-15
    G = O.self_term_stiffness(V, F, SIG, 3.0).toarray()
    C = O.cotan_laplacian(V, F).toarray()
    assert np.allclose(G, 3.0 * a[0] ** (1.0 - SIG) * C, rtol=1e-12, atol=1e-14)


def test_linear_function_on_a_planar_mesh():
    V, F = flat_grid(9, jitter=0.3, seed=4)
    c = np.array([0.7, -1.3, 0.0])
    u = V @ c
    kappa = 2.5
    G = O.self_term_stiffness(V, F, SIG, kappa)
    a = O.face_geometry(V, F)[2]
    expect = np.sum(kappa * a ** (1.0 - SIG) * a) * (c @ c)
    assert float(u @ (G @ u)) == pytest.approx(expect, rel=1e-12)


def test_preconditioned_condition_number():
    V, F = torus(40, 14, 1.0, 0.3)
    V = gaussian_noise(V, 0.005, 2)
    A = O.operator_matrix(V, F, "A")
    conds = {}
    for kappa in (0.0, 8.0):
        P = O.precond_apply(V, F, np.eye(len(V)), self_weight=kappa)
        ev = np.sort(np.linalg.eigvals(P @ A).real)[1:]
        conds[kappa] = ev.max() / ev.min()
    assert conds[0.0] > 200
    assert conds[8.0] < 10


def test_preconditioner_with_the_term_is_symmetric_positive():
    V, F = small_mesh("ico2", seed=5)
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal((len(V), 1)), rng.standard_normal((len(V), 1))
    u -= u.mean()
    v -= v.mean()
    Pu, Pv = O.precond_apply(V, F, u), O.precond_apply(V, F, v)
    assert float(np.sum(v * Pu)) == pytest.approx(float(np.sum(u * Pv)), rel=1e-10)
    assert float(np.sum(u * Pu)) > 0
