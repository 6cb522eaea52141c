"""Pins of the static-obstacle part of the oracle (§7.3.2).

The potential of a finely meshed sphere converges (second order in the edge
length) to the closed form of the sphere integral
    int_{|y|=R} |y - x|^{-p} dA = 2 pi R / (r (p-2)) [|R-r|^{2-p} - (R+r)^{2-p}],
r = |x| (4 pi R^{2-p} at r = 0); its gradient to the radial derivative of that
closed form. The differential is checked against central differences of the
energy, the energy against its scaling law lambda^{4-p} under a common
dilation, rigid motions, and the far-field limit A_surface A_obstacle D^{-p}.
The Barnes-Hut variant is the exact sum at theta = 0 and its error shrinks
with theta."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import icosphere, small_mesh

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def sphere_closed_form(r, R, p):
    if r == 0.0:
        return 4.0 * np.pi * R ** (2.0 - p)
    return 2.0 * np.pi * R / (r * (p - 2.0)) * (abs(R - r) ** (2.0 - p) - (R + r) ** (2.0 - p))


def scene(seed=3, level=2):
    """Small surface (noisy icosphere, radius 0.35) inside a unit-sphere
    obstacle shifted off-centre."""
    V, F = small_mesh("ico2", seed=seed)
    VO, FO = icosphere(level, 1.0)
    return 0.35 * V, F, VO + np.array([0.1, -0.05, 0.02]), FO


@pytest.mark.parametrize("p", [6.0, 4.5])
@pytest.mark.parametrize("r", [0.0, 0.3, 0.6, 1.8])
def test_sphere_potential_converges_to_closed_form(p, r):
    x = np.array([[0.6 * r, 0.8 * r, 0.0]])
    cf = sphere_closed_form(r, 1.0, p)
    err = []
    for lvl in (4, 5):
        V, F = icosphere(lvl, 1.0)
        err.append(abs(O.obstacle_potential(x, V, F, p)[0] / cf - 1.0))
    assert err[1] < 3e-3
    assert 3.0 < err[0] / err[1] < 5.0      # second-order convergence


@pytest.mark.parametrize("r", [0.3, 0.6, 1.8])
def test_sphere_gradient_is_radial_derivative_of_closed_form(r):
    p, R = 6.0, 1.0
    V, F = icosphere(5, R)
    u = np.array([0.6, 0.8, 0.0])
    _, g = O.obstacle_potential(r * u[None, :], V, F, p, grad=True)
    h = 1e-5
    dphi = (sphere_closed_form(r + h, R, p) - sphere_closed_form(r - h, R, p)) / (2 * h)
    gr = float(g[0] @ u)
    assert gr == pytest.approx(dphi, rel=5e-3)
    assert np.linalg.norm(g[0] - gr * u) < 1e-2 * abs(gr)


@pytest.mark.parametrize("p", [6.0, 4.5])
def test_differential_matches_central_differences(p):
    V, F, VO, FO = scene()
    w = 0.7
    g = O.obstacle_differential(V, F, VO, FO, p, w)
    rng = np.random.default_rng(4)
    h = 1e-6
    for v in rng.choice(len(V), 6, replace=False):
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            fd = (O.obstacle_energy(Vp, F, VO, FO, p, w) - O.obstacle_energy(Vm, F, VO, FO, p, w)) / (2 * h)
            assert g[v, c] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(g).max())


def test_scaling_rigid_motion_and_weight():
    V, F, VO, FO = scene()
    p = 6.0
    E = O.obstacle_energy(V, F, VO, FO, p)
    lam = 1.7
    assert O.obstacle_energy(lam * V, F, lam * VO, FO, p) == pytest.approx(lam ** (4.0 - p) * E, rel=1e-12)
    Q, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((3, 3)))
    t = np.array([3.0, -1.0, 2.0])
    assert O.obstacle_energy(V @ Q.T + t, F, VO @ Q.T + t, FO, p) == pytest.approx(E, rel=1e-12)
    assert O.obstacle_energy(V, F, VO, FO, p, 2.5) == pytest.approx(2.5 * E, rel=1e-14)
    # moving only the surface changes it
    assert abs(O.obstacle_energy(V + 0.05, F, VO, FO, p) - E) > 1e-3 * E


def test_far_field_limit():
    V, F = icosphere(2, 0.1)
    VO, FO = icosphere(2, 0.1)
    D = 20.0
    A = O.total_area(V, F)
    AO = O.total_area(VO, FO)
    for p in (6.0, 4.5):
        E = O.obstacle_energy(V, F, VO + np.array([D, 0.0, 0.0]), FO, p)
        assert E == pytest.approx(A * AO * D ** (-p), rel=1e-2)


def test_descends_away_from_the_obstacle():
    # the negative differential pushes a small sphere sitting off-centre in a
    # spherical obstacle back towards the centre (away from the nearer wall)
    V, F = icosphere(2, 0.2)
    VO, FO = icosphere(3, 1.0)
    off = np.array([0.4, 0.0, 0.0])
    g = O.obstacle_differential(V + off, F, VO, FO)
    assert g.sum(axis=0)[0] > 0 and abs(g.sum(axis=0)[1]) < 1e-6 * g.sum(axis=0)[0]


def test_bh_theta_zero_is_exact_and_error_shrinks():
    V, F, VO, FO = scene(level=3)
    X = O.face_geometry(V, F)[0]
    exact, gx = O.obstacle_potential(X, VO, FO, grad=True)
    phi0, g0, n0 = O.bh_obstacle_potential(X, VO, FO, 0.0, leaf=8, grad=True)
    assert np.allclose(phi0, exact, rtol=1e-13)
    assert np.allclose(g0, gx, rtol=1e-12, atol=1e-12 * np.abs(gx).max())
    assert n0 == len(X) * len(FO)
    errs = []
    for th in (0.8, 0.4, 0.2):
        phi, _, n = O.bh_obstacle_potential(X, VO, FO, th, leaf=4)
        errs.append(np.abs(phi / exact - 1).max())
        assert n < len(X) * len(FO)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 3e-3


def test_bh_energy_and_differential_are_consistent():
    # with the lists fixed the differential is exact for the approximation:
    # central differences of the Barnes-Hut energy (small steps keep the
    # interaction lists) match it
    V, F, VO, FO = scene(seed=6)
    E, g, _ = O.bh_obstacle_energy(V, F, VO, FO, 0.5, leaf=4)
    h = 1e-7
    for v in (0, 7, 31):
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[v, c] += h
            Vm[v, c] -= h
            fd = (O.bh_obstacle_energy(Vp, F, VO, FO, 0.5, leaf=4)[0]
                  - O.bh_obstacle_energy(Vm, F, VO, FO, 0.5, leaf=4)[0]) / (2 * h)
            assert g[v, c] == pytest.approx(fd, rel=1e-5, abs=1e-8 * np.abs(g).max())
    assert E == pytest.approx(O.obstacle_energy(V, F, VO, FO), rel=1e-2)


def test_step_with_obstacle_descends_and_zero_weight_is_plain_step():
    V, F = small_mesh("ico1", seed=2)
    V = 0.4 * V
    VO, FO = icosphere(2, 1.0)
    VO = VO + np.array([0.25, 0.0, 0.0])
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    r = O.precond_step(V, F, A0, V0, fixed_tau=0.1, obstacle=(VO, FO, 1.0))
    assert r["slope"] < 0
    r0 = O.precond_step(V, F, A0, V0, fixed_tau=0.1, obstacle=(VO, FO, 0.0))
    rp = O.precond_step(V, F, A0, V0, fixed_tau=0.1)
    assert np.allclose(r0["f_new"], rp["f_new"], rtol=0, atol=1e-14)
    # the obstacle term changes the direction
    assert np.abs(r["x"] - rp["x"]).max() > 1e-6


def test_free_barycenter_moves_the_surface_away_from_the_obstacle():
    # with the barycenter free (§7.1.1), a small sphere off-centre in a
    # spherical obstacle is translated towards the centre; the area and
    # volume still hold, and without the option the barycenter stays
    V, F = icosphere(2, 0.2)
    V = V + np.array([0.4, 0.0, 0.0])
    VO, FO = icosphere(3, 1.0)
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    ob = (VO, FO, 1e-3)
    r = O.precond_step(V, F, A0, V0, proj_iters=2, obstacle=ob, free_barycenter=True)
    r0 = O.precond_step(V, F, A0, V0, proj_iters=2, obstacle=ob)
    assert r["f_new"].mean(axis=0)[0] < V.mean(axis=0)[0] - 1e-6
    assert abs(r0["f_new"].mean(axis=0)[0] - V.mean(axis=0)[0]) < 1e-12
    assert abs(O.total_area(r["f_new"], F) - A0) < 1e-6 * A0
    assert r["E1"] < r["E0"]
    # the translation is the area-weighted mean of -dE, the same for all vertices
    t = O.barycenter_motion(V, F, np.ones_like(V))
    assert np.allclose(t, -1.0)
