"""GPU parity of the Willmore term (§7.3.5) against the FP64 oracle, through
the C ABI: E_W and dE_W on closed meshes of one and two components, the
icosphere's approach to 16 pi, the constrained step with the Willmore
energy and its H^2 operator term against the oracle's dense saddle solve
(FP64), FP32 Armijo steps that descend, invalid weights rejected, and the
benchmark torus."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import icosphere, small_mesh, workload

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda:0", dtype=dtype)


def two_meshes():
    A = small_mesh("ico2", seed=3)
    B = small_mesh("torus13x7", seed=4)
    V = np.concatenate([A[0], 0.6 * B[0] + np.array([2.2, 0.0, 0.0])])
    F = np.concatenate([A[1], B[1] + len(A[0])]).astype(np.int32)
    return V, F


def mesh(name):
    if name == "two":
        return two_meshes()
    return small_mesh(name, seed=6)


@pytest.mark.parametrize("name", ["tetra", "ico3", "torus13x7", "two"])
def test_energy_and_differential(lib, name):
    import torch
    V, F = mesh(name)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        E, g = lib.tp_willmore_energy(m)
        E2, g2 = lib.tp_willmore_energy(m, like=dev(V, torch.float64))
    gref = O.willmore_differential(V, F)
    assert rel(E, O.willmore_energy(V, F)) < 1e-12
    # (the regular tetrahedron is a critical point: its differential is 0)
    assert np.abs(g - gref).max() <= 1e-11 * max(np.abs(gref).max(), E)
    assert E2 == E and np.array_equal(g2.cpu().numpy(), g)


def test_sphere_value(lib):
    import torch
    V, F = icosphere(5)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        E, _ = lib.tp_willmore_energy(m)
    assert abs(E / (16 * np.pi) - 1) < 5e-4


def test_step_with_willmore_matches_exact_saddle_solution(lib):
    import torch
    V, F = small_mesh("ico2", seed=4)
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    w = 0.3
    ref = O.precond_step(V, F, A0, V0, fixed_tau=0.05, willmore=w)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        lib.tp_willmore_set(m, w)
        c = lib.tp_constraints(flags=3, A0=A0, V0=V0)
        p = lib.params(precision=1, krylov_tol=1e-11, cg_tol=1e-12, fixed_tau=1, tau0=0.05, krylov_max=400)
        rep = lib.precond_step(m, c, p)
        f_new = m.get_positions()
    assert rep["status"] == 0 and rep["slope"] < 0
    assert rel(rep["E_before"], ref["E0"]) < 1e-10
    assert rel(f_new - V, ref["f_new"] - V) < 1e-7
    assert rel(rep["E_after"], ref["E1"]) < 1e-8


def test_fp32_steps_with_willmore_descend(lib):
    import torch
    V, F = small_mesh("ico3", seed=8)
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    w = 0.1
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        lib.tp_willmore_set(m, w)
        c = lib.tp_constraints(flags=3, A0=A0, V0=V0)
        for theta in (0.0, 0.5):
            for _ in range(2):
                rep = lib.precond_step(m, c, lib.params(theta=theta, krylov_max=300))
                assert rep["slope"] < 0 and rep["E_after"] < rep["E_before"]
        f = m.get_positions()
        with pytest.raises(lib.TpError):
            lib.tp_willmore_set(m, -1.0)
        lib.tp_willmore_set(m, 0.0)
        E_plain = lib.precond_step(m, c, lib.params(krylov_max=300))["E_before"]
    assert E_plain == pytest.approx(O.energy(f, F), rel=1e-5)
    assert O.energy(f, F) + w * O.willmore_energy(f, F) < O.energy(V, F) + w * O.willmore_energy(V, F)


def test_torus20k_willmore(lib):
    # full size: E_W and dE_W against the oracle (sparse, fast at any size),
    # and a constrained step with the Willmore term
    import torch
    V, F = workload("torus_20k")
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        E, g = lib.tp_willmore_energy(m)
        lib.tp_willmore_set(m, 1.0)
        c = lib.tp_constraints(flags=3, A0=A0, V0=V0)
        rep = lib.precond_step(m, c, lib.params(krylov_tol=1e-5, krylov_max=60, cg_tol=1e-6))
    assert rel(E, O.willmore_energy(V, F)) < 1e-12
    assert rel(g, O.willmore_differential(V, F)) < 1e-11
    assert rep["slope"] < 0 and rep["E_after"] < rep["E_before"]
