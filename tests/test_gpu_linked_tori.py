"""Differentiation on the 50,000-face linked tori (two R=1, r=0.25 tori,
the second rotated 90 degrees about x and moved by (1,0,0)): the energy
behind TangentPointEnergy (autograd) with the library's differential as its
backward, checked by central differences with h = 1e-6 along 64 seeded unit
directions of the FP64 GPU energy, against the stored oracle energy, and
against the oracle gradient at sampled vertices."""
import json
import os

import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import workload

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    """max |a - b| over max |b|: a few wrong entries that a 2-norm hides show here"""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def tori(lib):
    import torch
    V, F = workload("linked_tori_50k")
    f = torch.tensor(V, dtype=torch.float64, device="cuda")
    m = lib.Mesh(f, torch.tensor(F, dtype=torch.int32, device="cuda"))
    yield V, F, f, m
    m.close()


def test_energy_matches_stored_oracle(lib, tori):
    V, F, f, m = tori
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "full_size.json")))["linked_tori_50k"]
    assert rel(lib.tp_energy(m, lib.params()), gold["energy"]) <= 1e-5
    assert rel(lib.tp_energy(m, lib.params(precision=1)), gold["energy"]) <= 1e-10


def test_autograd_backward_matches_central_differences(lib, tori):
    import torch
    V, F, f, m = tori
    x = f.clone().requires_grad_(True)
    E = lib.TangentPointEnergy.apply(x, m, lib.params())
    E.backward()
    g = x.grad.detach().cpu().numpy()
    p64 = lib.params(precision=1)
    rng = np.random.default_rng(303)
    h = 1e-6
    dd, fd = [], []
    for _ in range(64):
        dv = rng.standard_normal(V.shape)
        dv /= np.linalg.norm(dv)
        lib.tp_mesh_set_positions(m, V + h * dv)
        ep = lib.tp_energy(m, p64)
        lib.tp_mesh_set_positions(m, V - h * dv)
        em = lib.tp_energy(m, p64)
        fd.append((ep - em) / (2 * h))
        dd.append(float(np.sum(g * dv)))
    lib.tp_mesh_set_positions(m, V)
    fd, dd = np.array(fd), np.array(dd)
    # FP32-path gradient vs FP64 central differences, relative to the gradient norm
    assert np.abs(dd - fd).max() <= 1e-5 * np.linalg.norm(g)
    assert rel(dd, fd) <= 1e-5


def test_gradient_matches_oracle_at_sampled_vertices(lib, tori):
    V, F, f, m = tori
    g, _ = lib.tp_differential(m, lib.params())
    idx = np.random.default_rng(3).choice(len(V), 24, replace=False)
    ref = O.differential_at_vertices(V, F, idx)
    assert rel(g[idx], ref) <= 1e-5 and maxrel(g[idx], ref) <= 4e-5


def test_constrained_step_converges_with_one_barycenter_per_torus(lib):
    # one barycenter per component: the Krylov space (per-component mean-zero
    # preconditioner outputs) contains the solution, so FGMRES converges on
    # the two tori; each torus keeps its barycenter
    import torch
    V, F = workload("linked_tori_50k")
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    comp = O.mesh_components(len(V), F)
    with lib.Mesh(torch.tensor(V, dtype=torch.float64, device="cuda"),
                  torch.tensor(F, dtype=torch.int32, device="cuda")) as m:
        c = lib.tp_constraints(flags=3, A0=A0, V0=V0)
        rep = lib.precond_step(m, c, lib.params(theta=0.5, krylov_tol=1e-5, krylov_max=60, cg_tol=1e-6))
        f = m.get_positions()
    assert rep["status"] == 0 and rep["slope"] < 0 and rep["E_after"] < rep["E_before"]
    for lab in np.unique(comp):
        sel = comp == lab
        assert np.abs(f[sel].mean(axis=0) - V[sel].mean(axis=0)).max() < 1e-6
