"""Parity of the benchmarked constrained step: FP32 pair terms (E, dE, A and
L^{2-s} in the Krylov loop), the preconditioner's Cholesky Poisson solves at
cg_tol = 1e-4 and flexible GMRES at krylov_tol = 1e-5 -- exactly the
parameters bench.py times (bench.step_params) -- against the FP64 oracle.

What the step promises (§3.3, Eq. 14; §5.3, Eq. 17-18). The direction x
solves the saddle problem [A dPhi^T; dPhi 0][x; lambda] = [-dE; 0] (with the
barycenter rows of §7.1.1) through three Krylov solves A z_k = b_k (b_1 = dE,
b_2, b_3 = the area and volume gradients) in the Schur complement form
x = -(z_1 - Z (dPhi Z)^-1 dPhi z_1). Each solve stops at
|b_k - A~ z_k| <= tol |b_k| with the FP32 operator A~, so

    min_lambda |A x + dE + J^T lambda|
        <= tol (|dE| + sum_k |lambda_k| |J_k|) + eps_A |A x| + eps_g |dE|,

where J holds the area, volume and barycenter rows, eps_A bounds the relative
error of the FP32 operator and eps_g that of the FP32 differential against the
FP64 definitions (both 1e-5, the tolerance the other parity tests enforce on
them). The tests measure the left side with the oracle's exact operator and
differential and check it against the right side (x from the GPU step at a
fixed step length without projection, so f_new = f + tau x exactly). On the
642-vertex icosphere they also bound the direction error: on the constrained
subspace |x - x*| <= (residual) / lambda_min(A), lambda_min the smallest
non-zero eigenvalue of A (computed densely by the oracle), so
|x - x*| / |x*| <= (the bound above) / (lambda_min |x*|).
"""
import numpy as np
import pytest

import bench
from oracle import tp_oracle as O
from synth import workload

pytestmark = pytest.mark.gpu

EPS_A = EPS_G = 1e-5


def dev(x, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda:0", dtype=dtype)


def _bench_step_direction(lib, V, F, tau):
    """x of the benchmark's step (its parameters, at a fixed step length,
    no corrective projection) and the report."""
    import torch
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    p = bench.step_params(lib)
    # exactly tau: no line search, no displacement bound on the step, no projection
    p.fixed_tau, p.tau0, p.tau0_disp, p.proj_iters = 1, tau, 0.0, 0
    c = lib.tp_constraints(flags=lib.TP_CONSTRAINT_AREA | lib.TP_CONSTRAINT_VOLUME, A0=A0, V0=V0)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        rep = lib.precond_step(m, c, p)
        f_new = m.get_positions()
    return (f_new - V) / tau, rep, p


def _rows(V, F, idx=None):
    """Constraint rows [area, volume, barycenter x, y, z] as [5, nv, 3]
    (restricted to the vertices idx)."""
    nv = len(V)
    J = np.concatenate([O._constraint_rows(V, F, True, True), O._barycenter_rows(nv)], axis=0)
    J = J.reshape(5, nv, 3)
    return J if idx is None else J[:, idx, :]


def _residual_and_bound(Ax, g, J, tol):
    """min over lambda of |A x + g + J^T lambda| and the bound of the module
    docstring, on the rows given (full or sampled)."""
    r = (Ax + g).reshape(-1)
    Jm = J.reshape(J.shape[0], -1)
    lam, *_ = np.linalg.lstsq(Jm.T, -r, rcond=None)
    res = float(np.linalg.norm(r + Jm.T @ lam))
    gn = float(np.linalg.norm(g))
    bound = tol * (gn + sum(abs(lam[k]) * np.linalg.norm(Jm[k]) for k in range(2))) \
        + EPS_A * float(np.linalg.norm(Ax)) + EPS_G * gn
    return res, bound, lam


def test_bench_step_solves_the_saddle_problem_icosphere_l3(lib):
    V, F = workload("icosphere_l3")
    tau = 0.5
    x, rep, p = _bench_step_direction(lib, V, F, tau)
    assert rep["status"] == 0, rep
    g = O.differential(V, F)
    Ax = O.apply_operator(V, F, x, "A")
    J = _rows(V, F)
    res, bound, lam = _residual_and_bound(Ax, g, J, p.krylov_tol)
    assert res <= bound, (res, bound)
    # area and volume rows: dPhi x = 0 up to FP64 rounding of the Schur solve
    for k in range(2):
        assert abs(float(np.sum(J[k] * x))) <= 1e-9 * np.linalg.norm(J[k]) * np.linalg.norm(x)
    # barycenter: x has zero mean
    assert np.abs(x.mean(axis=0)).max() <= 1e-10 * np.abs(x).max()
    # the direction against the exact dense saddle solve
    x_star, _ = O.descent_direction(V, F)
    A = O.operator_matrix(V, F, "A")
    lam_min = np.linalg.eigvalsh(A)[1]          # the constants span the nullspace
    err = np.linalg.norm(x - x_star) / np.linalg.norm(x_star)
    assert err <= bound / (lam_min * np.linalg.norm(x_star)), err
    # energies: E(f) at the FP32 tolerance, E(f + tau x) consistent with the oracle
    assert abs(rep["E_before"] - O.energy(V, F)) <= 1e-5 * O.energy(V, F)
    E_new = O.energy(V + tau * x, F)
    assert abs(rep["E_after"] - E_new) <= 1e-5 * E_new
    assert rep["E_after"] < rep["E_before"] and rep["slope"] < 0


def test_bench_step_saddle_residual_torus20k_sampled(lib):
    # full size, the benchmark's mesh and launch configuration: the residual
    # of Eq. 14 at sampled vertices with the oracle's operator rows
    V, F = workload("torus_20k")
    tau = 1e-6
    x, rep, p = _bench_step_direction(lib, V, F, tau)
    assert rep["status"] == 0, rep
    idx = np.random.default_rng(2024).choice(len(V), 48, replace=False)
    g = O.differential_at_vertices(V, F, idx)
    Ax = O.apply_operator_at_vertices(V, F, x, "A", idx)
    J = _rows(V, F, idx)
    res, bound, _ = _residual_and_bound(Ax, g, J, p.krylov_tol)
    # sampled rows: the bound is a statement about full norms; on a uniform
    # sample of rows both sides scale alike, a factor 3 covers the sampling
    assert res <= 3.0 * bound, (res, bound)
    Jf = _rows(V, F)
    for k in range(2):
        assert abs(float(np.sum(Jf[k] * x))) <= 1e-9 * np.linalg.norm(Jf[k]) * np.linalg.norm(x)
    assert np.abs(x.mean(axis=0)).max() <= 1e-9 * np.abs(x).max()
