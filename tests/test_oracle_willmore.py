"""Pins of the Willmore part of the oracle (§7.3.5).

E_W = f^T C M^{-1} C f of an icosphere converges at second order to the
smooth value int 4 H^2 dA = 16 pi of the round sphere (H = 1/R); E_W is
invariant under dilations and rigid motions; its differential matches
central differences; the H^2 term C M^{-1} C is symmetric positive
semidefinite with the constants in its nullspace; a step with the Willmore
term descends and is the plain step at weight 0."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import icosphere, small_mesh

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_sphere_converges_to_16_pi():
    err = [abs(O.willmore_energy(*icosphere(l)) / (16 * np.pi) - 1) for l in (3, 4, 5)]
    assert err[2] < 5e-4
    assert 3.5 < err[0] / err[1] < 4.5 and 3.5 < err[1] / err[2] < 4.5


def test_scale_and_rigid_motion_invariance():
    V, F = small_mesh("torus13x7", seed=2)
    E = O.willmore_energy(V, F)
    assert O.willmore_energy(3.7 * V, F) == pytest.approx(E, rel=1e-12)
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((3, 3)))
    assert O.willmore_energy(V @ Q.T + np.array([1.0, -2.0, 0.5]), F) == pytest.approx(E, rel=1e-12)


@pytest.mark.parametrize("name", ["ico2", "torus13x7"])
def test_differential_matches_central_differences(name):
    V, F = small_mesh(name, seed=3)
    g = O.willmore_differential(V, F)
    h = 1e-6
    rng = np.random.default_rng(5)
    for v in rng.choice(len(V), 5, replace=False):
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            fd = (O.willmore_energy(Vp, F) - O.willmore_energy(Vm, F)) / (2 * h)
            assert g[v, c] == pytest.approx(fd, rel=1e-6, abs=1e-8 * np.abs(g).max())


def test_metric_term():
    V, F = small_mesh("ico1", seed=2)
    W = O.willmore_metric(V, F)
    assert np.abs(W - W.T).max() < 1e-12 * np.abs(W).max()
    assert np.abs(W @ np.ones(len(V))).max() < 1e-10 * np.abs(W).max()
    assert np.linalg.eigvalsh(0.5 * (W + W.T)).min() > -1e-10 * np.abs(W).max()


def test_step_with_willmore():
    V, F = small_mesh("ico2", seed=4)
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    r = O.precond_step(V, F, A0, V0, fixed_tau=0.05, willmore=0.3)
    assert r["slope"] < 0
    r0 = O.precond_step(V, F, A0, V0, fixed_tau=0.05, willmore=0.0)
    rp = O.precond_step(V, F, A0, V0, fixed_tau=0.05)
    assert np.allclose(r0["f_new"], rp["f_new"], rtol=0, atol=1e-14)
    assert np.abs(r["x"] - rp["x"]).max() > 1e-6
    # with the Willmore energy and metric, the step lowers E + w E_W
    r = O.precond_step(V, F, A0, V0, willmore=0.3)
    assert r["E1"] < r["E0"]
