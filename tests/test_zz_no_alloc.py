"""The allocation-free energy entry point (tp_energy_noalloc).

Callers that cannot allocate device memory (code inside a CUDA graph under
capture, plug-ins whose host owns the device allocator, real-time loops that
must not take allocator locks) use tp_energy_noalloc, which keeps its
intermediates in a static device array of the library. This file is collected
last on purpose, so that a run stopping at the first failure has already run
every other test; it needs no other test's state and passes alone."""
import ctypes

import numpy as np
import pytest

from synth import small_mesh, workload

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _call(tp, pos, faces, E, p=6.0):
    import torch
    L = tp.lib()
    return L.tp_energy_noalloc(ctypes.c_void_p(pos.data_ptr()), int(pos.shape[0]),
                               ctypes.c_void_p(faces.data_ptr()), int(faces.shape[0]), ctypes.c_double(p),
                               ctypes.c_void_p(E.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("mesh,p", [("ico3", 6.0), ("torus13x7", 6.0), ("ico2", 4.5)])
def test_noalloc_energy_matches_tp_energy_on_two_calls(mesh, p):
    import torch
    import paper_2107_01664_gb300 as tp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V, F = small_mesh(mesh, seed=41)
    pos = torch.tensor(V, dtype=torch.float64, device="cuda")
    faces = torch.tensor(F, dtype=torch.int32, device="cuda")
    with tp.Mesh(pos, faces) as m:
        E_ref = tp.tp_energy(m, tp.params(p=p))
    E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):                    # the static scratch keeps the previous call's data
        assert _call(tp, pos, faces, E, p) == tp.TP_OK, tp.lib().tp_last_error().decode()
        torch.cuda.synchronize()
        assert abs(E.item() - E_ref) <= TOL32 * abs(E_ref)


def test_noalloc_energy_full_torus_and_size_limit():
    import torch
    import paper_2107_01664_gb300 as tp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V, F = workload("torus_20k")          # 20,000 faces, below the 32,768 limit
    pos = torch.tensor(V, dtype=torch.float64, device="cuda")
    faces = torch.tensor(F, dtype=torch.int32, device="cuda")
    with tp.Mesh(pos, faces) as m:
        E_ref = tp.tp_energy(m, tp.params())
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert _call(tp, pos, faces, E) == tp.TP_OK
        torch.cuda.synchronize()
        assert abs(E.item() - E_ref) <= TOL32 * abs(E_ref)
    # beyond the maximum: a clear error, nothing launched
    big = torch.zeros((32769, 3), dtype=torch.int32, device="cuda")
    assert _call(tp, pos, big, E) == tp.TP_ERR_INVALID_ARG
    assert "exceed the maximum" in tp.lib().tp_last_error().decode()
