"""The A apply with its accumulation on tcgen05 tensor cores (tp_params.tensor_cores = 1):
split TF32 products H X = Hh Xh + Hh Xl + Hl Xh of the kernel values H (§5.1.1-5.1.3, App. A)
and the source vectors X, FP32 accumulators in tensor memory drained into compensated sums
every 128 sources. The same parity bar as the CUDA-core kernel: 1e-5 of the FP64 oracle in the
2-norm, 4e-5 in the max norm; ragged sizes (a partial last tile, fewer faces than one tile,
several target blocks and source splits), 4 and 9 columns, the benchmark mesh at full size on
sampled vertices, and the constrained step that uses it (§3.3, Eq. 14)."""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import small_mesh, vertex_vectors, workload

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda:0", dtype=dtype)


@pytest.mark.parametrize("name", ["tetra", "octa", "torus13x7", "ico3", "ico4"])
@pytest.mark.parametrize("k", [4, 9])
def test_tensor_core_apply_matches_oracle(lib, name, k):
    import torch
    V, F = small_mesh(name, seed=31)
    u = vertex_vectors(len(V), k, 41)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        y1 = lib.fractional_apply(m, "A", dev(u), lib.params(tensor_cores=1)).cpu().numpy()
        y0 = lib.fractional_apply(m, "A", dev(u), lib.params(tensor_cores=0)).cpu().numpy()
    ref = O.apply_operator(V, F, u, "A")
    assert np.isfinite(y1).all()
    assert rel(y1, ref) <= TOL32 and maxrel(y1, ref) <= 4 * TOL32
    # the two FP32 paths agree to the FP32 rounding of their sums
    assert rel(y1, y0) <= 5e-6


def test_tensor_core_apply_torus20k_sampled(lib):
    import torch
    V, F = workload("torus_20k")
    u = vertex_vectors(len(V), 9, 51)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        y = lib.fractional_apply(m, "A", dev(u), lib.params(tensor_cores=1)).cpu().numpy()
    idx = np.random.default_rng(52).choice(len(V), 48, replace=False)
    ref = O.apply_operator_at_vertices(V, F, u, "A", idx)
    assert rel(y[idx], ref) <= TOL32 and maxrel(y[idx], ref) <= 4 * TOL32


def test_tensor_core_step_solves_the_saddle_problem(lib):
    # the benchmark's step with the tensor-core A apply in the Krylov loop, at a
    # fixed step length: the residual of Eq. 14 within the bound derived in
    # test_gpu_step_fp32 (krylov_tol and the FP32 errors of A and dE)
    import bench
    import test_gpu_step_fp32 as S
    import torch
    V, F = workload("icosphere_l3")
    tau = 0.5
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    p = bench.step_params(lib)
    p.fixed_tau, p.tau0, p.tau0_disp, p.proj_iters, p.tensor_cores = 1, tau, 0.0, 0, 1
    c = lib.tp_constraints(flags=lib.TP_CONSTRAINT_AREA | lib.TP_CONSTRAINT_VOLUME, A0=A0, V0=V0)
    with lib.Mesh(dev(V, torch.float64), dev(F, torch.int32)) as m:
        rep = lib.precond_step(m, c, p)
        x = (m.get_positions() - V) / tau
    assert rep["status"] == 0, rep
    g = O.differential(V, F)
    Ax = O.apply_operator(V, F, x, "A")
    res, bound, _ = S._residual_and_bound(Ax, g, S._rows(V, F), p.krylov_tol)
    assert res <= bound, (res, bound)
