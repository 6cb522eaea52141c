"""Library contexts (tp_create / tp_destroy) and the caller-set allocator of
a context's device memory, through the C ABI: meshes created in a context
compute bitwise the same results as meshes of the default context, their
memory is accounted and returned, PyTorch's caching allocator can serve it,
an allocator that refuses is reported as TP_ERR_OOM, and a context with live
meshes is not destroyed."""
import ctypes

import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import small_mesh, vertex_vectors

pytestmark = pytest.mark.gpu


def _mesh_results(lib, m, V, F):
    p = lib.params()
    E = lib.tp_energy(m, p)
    g, _ = lib.tp_differential(m, p)
    y = lib.fractional_apply(m, "A", vertex_vectors(len(V), 9, 3), p)
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    rep = lib.precond_step(m, lib.tp_constraints(flags=3, A0=A0, V0=V0), lib.params(krylov_max=60))
    return E, g, y, rep["E_after"], m.get_positions()


def test_context_default_allocator_matches_default_context(lib):
    V, F = small_mesh("ico3", seed=61)
    with lib.Mesh(V, F) as m0:
        ref = _mesh_results(lib, m0, V, F)
    with lib.Context(0) as ctx:
        with lib.Mesh(V, F, ctx=ctx) as m:
            used, peak = ctx.memory()
            assert 0 < used <= peak
            got = _mesh_results(lib, m, V, F)
            assert ctx.memory()[0] >= used          # workspaces were added
            # a context with a live mesh is not destroyed
            assert lib.lib().tp_destroy(ctx.handle) == lib.TP_ERR_INVALID_ARG
        assert ctx.memory()[0] == 0                 # everything returned
    for a, b in zip(ref, got):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_context_torch_allocator_shares_the_pool(lib):
    import torch
    V, F = small_mesh("torus13x7", seed=62)
    with lib.Mesh(V, F) as m0:
        ref = _mesh_results(lib, m0, V, F)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    with lib.Context(0, allocator="torch") as ctx:
        with lib.Mesh(V, F, ctx=ctx) as m:
            got = _mesh_results(lib, m, V, F)
            torch.cuda.synchronize()
            used = ctx.memory()[0]
            assert used > 0
            assert torch.cuda.memory_allocated() - before >= used
        assert ctx.memory()[0] == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    for a, b in zip(ref, got):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_context_allocator_refusal_is_reported(lib):
    # host-side fault injection: an allocator that refuses every request
    V, F = small_mesh("ico2", seed=63)
    calls = []

    @lib._ALLOC_FN
    def refuse(nbytes, device, user):
        calls.append(nbytes)
        return None

    @lib._FREE_FN
    def never(ptr, nbytes, device, user):
        raise AssertionError("nothing was allocated")

    with lib.Context(0) as ctx:
        a = lib.tp_allocator(refuse, never, None)
        lib._check(lib.lib().tp_ctx_set_allocator(ctx.handle, ctypes.byref(a)))
        with pytest.raises(lib.TpError) as e:
            lib.Mesh(V, F, ctx=ctx)
        assert e.value.code == lib.TP_ERR_OOM
        assert calls
        assert ctx.memory()[0] == 0
        # back to cudaMalloc: the same context now serves the mesh
        lib.tp_ctx_set_allocator(ctx, None)
        with lib.Mesh(V, F, ctx=ctx) as m:
            assert abs(lib.tp_energy(m, lib.params()) - O.energy(V, F)) <= 1e-5 * O.energy(V, F)


def test_context_argument_errors(lib):
    with pytest.raises(lib.TpError):
        lib.Context(4096)
    with lib.Context(0) as ctx:
        half = lib.tp_allocator()
        half.alloc = lib._ALLOC_FN(lambda n, d, u: None)
        with pytest.raises(lib.TpError):
            lib._check(lib.lib().tp_ctx_set_allocator(ctx.handle, ctypes.byref(half)))
    assert lib.lib().tp_destroy(None) == lib.TP_OK
