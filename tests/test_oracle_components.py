"""Pins of the multi-component handling of the oracle (§7.1.1: for several
components, one barycenter per component): on two disjoint meshes the
Poisson solve equals the per-component solves, the dense saddle direction
keeps each component's barycenter, and it equals the Schur-complement
direction computed in the subspace of zero mean per component."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import small_mesh

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def two_meshes():
    A = small_mesh("ico2", seed=3)
    B = small_mesh("torus13x7", seed=4)
    V = np.concatenate([A[0], 0.6 * B[0] + np.array([2.2, 0.0, 0.0])])
    F = np.concatenate([A[1], B[1] + len(A[0])])
    return V, F, len(A[0]), A, B


def test_components_and_per_component_poisson():
    V, F, na, A, B = two_meshes()
    comp = O.mesh_components(len(V), F)
    assert len(np.unique(comp)) == 2 and np.all(comp[:na] == comp[0]) and np.all(comp[na:] != comp[0])
    b = np.random.default_rng(2).standard_normal((len(V), 2))
    z = O.poisson_solve(O.cotan_laplacian(V, F), b, comp)
    za = O.poisson_solve(O.cotan_laplacian(*A), b[:na])
    zb = O.poisson_solve(O.cotan_laplacian(0.6 * B[0], B[1]), b[na:])
    assert np.allclose(z[:na], za, rtol=1e-10, atol=1e-12)
    assert np.allclose(z[na:], zb, rtol=1e-10, atol=1e-12)


def test_direction_keeps_each_barycenter_and_matches_schur():
    V, F, na, _, _ = two_meshes()
    x, g = O.descent_direction(V, F)
    scale = np.abs(x).max()
    assert np.abs(x[:na].sum(axis=0)).max() < 1e-10 * scale * na
    assert np.abs(x[na:].sum(axis=0)).max() < 1e-10 * scale * (len(V) - na)
    xs, _, _ = O.schur_direction(V, F)
    assert np.abs(x - xs).max() < 1e-8 * scale
    assert np.sum(g * x) < 0
