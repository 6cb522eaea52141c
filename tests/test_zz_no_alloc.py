"""The allocation-free energy entry point (tp_energy_noalloc).

Some callers of this library are not allowed to allocate device memory: a
plug-in inside a host program that owns the GPU allocator, or a real-time loop
that must not block on allocator locks or fail with out-of-memory mid-run.
For them tp_energy_noalloc computes the direct energy from caller-owned device
arrays and keeps its intermediates in one static device array of the library.
These tests call it through the C ABI, twice in a row (the static array keeps
the previous call's contents), and compare it with the regular entry point
and with the FP64 oracle.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test; it needs no other test's state and
passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from oracle import tp_oracle as O
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


def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("mesh,p", [("ico3", 6.0), ("torus13x7", 6.0), ("ico2", 4.5)])
def test_noalloc_energy_matches_tp_energy_and_oracle_on_two_calls(mesh, p):
    _need_cuda()
    import torch
    import paper_2107_01664_gb300 as tp
    V, F = small_mesh(mesh, seed=41)
    pos = torch.tensor(V, dtype=torch.float64, device="cuda")
    faces = torch.tensor(F, dtype=torch.int32, device="cuda")
    with tp.Mesh(pos, faces) as m:
        E_ref = tp.tp_energy(m, tp.params(p=p))
    E_oracle = O.energy(V, F, p)
    E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert _call(tp, pos, faces, E, p) == tp.TP_OK, tp.lib().tp_last_error().decode()
        torch.cuda.synchronize()
        assert abs(E.item() - E_ref) <= TOL32 * abs(E_ref)
        assert abs(E.item() - E_oracle) <= TOL32 * abs(E_oracle)


def test_noalloc_energy_full_torus_allocates_nothing_and_size_limit():
    _need_cuda()
    import torch
    import paper_2107_01664_gb300 as tp
    V, F = workload("torus_20k")          # 20,000 faces, below the 32,768 limit
    pos = torch.tensor(V, dtype=torch.float64, device="cuda")
    faces = torch.tensor(F, dtype=torch.int32, device="cuda")
    with tp.Mesh(pos, faces) as m:
        E_ref = tp.tp_energy(m, tp.params())
    # the oracle's full sum takes minutes here: its stored value (tests/golden/make_golden.py)
    import json
    import os
    stored = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                         "full_size.json")))["torus_20k"]["energy"]
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(tp, pos, faces, E) == tp.TP_OK        # first call: looks up the static array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _call(tp, pos, faces, E) == tp.TP_OK
        torch.cuda.synchronize()
        assert abs(E.item() - E_ref) <= TOL32 * abs(E_ref)
        assert abs(E.item() - stored) <= TOL32 * abs(stored)
    assert torch.cuda.mem_get_info()[0] == free0       # no device memory taken by the calls
    # beyond the maximum: a clear error, nothing launched
    big = torch.zeros((32769, 3), dtype=torch.int32, device="cuda")
    assert _call(tp, pos, big, E) == tp.TP_ERR_INVALID_ARG
    assert "exceed the maximum" in tp.lib().tp_last_error().decode()


def test_noalloc_bad_face_index_gives_nan_and_next_call_is_clean():
    _need_cuda()
    import torch
    import paper_2107_01664_gb300 as tp
    V, F = small_mesh("ico2", seed=42)
    pos = torch.tensor(V, dtype=torch.float64, device="cuda")
    bad = F.copy()
    bad[3, 1] = len(V) + 5
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(tp, pos, torch.tensor(bad, dtype=torch.int32, device="cuda"), E) == tp.TP_OK
    torch.cuda.synchronize()
    assert np.isnan(E.item())
    # the flag is cleared by the next call
    assert _call(tp, pos, torch.tensor(F, dtype=torch.int32, device="cuda"), E) == tp.TP_OK
    torch.cuda.synchronize()
    assert abs(E.item() - O.energy(V, F)) <= TOL32 * abs(O.energy(V, F))


def test_noalloc_binding_rejects_inputs_it_would_have_to_convert():
    _need_cuda()
    import torch
    import paper_2107_01664_gb300 as tp
    V, F = small_mesh("ico2", seed=43)
    pos = torch.tensor(V, dtype=torch.float64, device="cuda")
    faces = torch.tensor(F, dtype=torch.int32, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        tp.tp_energy_noalloc(pos.float(), faces, E)
    with pytest.raises(TypeError):
        tp.tp_energy_noalloc(pos, faces.long(), E)
    with pytest.raises(TypeError):
        tp.tp_energy_noalloc(pos.cpu(), faces, E)
    with pytest.raises(ValueError):
        tp.tp_energy_noalloc(pos.t().contiguous().t(), faces, E)
    with pytest.raises(ValueError):
        tp.tp_energy_noalloc(pos, faces, E[:0])
    tp.tp_energy_noalloc(pos, faces, E)
    torch.cuda.synchronize()
    assert abs(E.item() - O.energy(V, F)) <= TOL32 * abs(O.energy(V, F))
