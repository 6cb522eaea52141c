"""Python binding of libtpsurf, the GB300 tangent-point surface-flow library.

A thin ctypes layer over the C ABI of include/tp.h: the functions have the
same names and do argument marshalling only. Every step of the computation
runs in the library's CUDA kernels; there is no CPU or PyTorch fallback, and
importing this package fails loudly when the compiled library is missing.

Arrays may be numpy arrays or CPU tensors (host memory) or CUDA tensors
(device memory of the mesh's GPU). Results come back in the same kind of
memory as the input; CUDA work is queued on torch's current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "TP_OK", "TP_OP_A", "TP_OP_B", "TP_OP_B0", "TP_OP_L", "TP_PREC_FP32", "TP_PREC_FP64",
    "TP_CONSTRAINT_AREA", "TP_CONSTRAINT_VOLUME", "TP_CONSTRAINT_FREE_BARYCENTER", "TP_BH_DIFF_FULL", "TP_BH_DIFF_LITERAL",
    "TpError", "tp_params", "tp_constraints", "tp_step_report", "params", "Mesh",
    "tp_mesh_create", "tp_mesh_set_positions", "tp_mesh_get_positions", "tp_mesh_destroy",
    "tp_mesh_footprint_bytes", "tp_energy", "tp_energy_rows", "tp_differential",
    "fractional_apply", "cotan_solve", "precond_apply", "precond_step", "TangentPointEnergy",
    "lib_path", "lib", "tp_kernel_stat", "tp_profile_enable", "tp_profile_read", "tp_launch_count",
    "tp_energy_noalloc", "tp_chol_info", "cotan_factor_info", "TP_POISSON_CHOLESKY", "TP_POISSON_CG",
    "tp_obstacle_set", "tp_obstacle_energy", "tp_pins_set", "TP_MAX_PINS", "tp_willmore_set",
    "tp_willmore_energy", "tp_selftest_wait", "Context", "tp_allocator", "tp_create", "tp_destroy",
    "tp_ctx_set_allocator", "tp_ctx_memory", "tp_mesh_create_ctx", "tp_mesh_area_volume",
]

TP_OK, TP_ERR_INVALID_ARG, TP_ERR_DEGENERATE, TP_ERR_OOM = 0, 1, 2, 3
TP_ERR_NOT_CONVERGED, TP_ERR_TIMEOUT, TP_ERR_CUDA = 4, 5, 6
TP_PTR_HOST, TP_PTR_DEVICE = 0, 1
TP_PREC_FP32, TP_PREC_FP64 = 0, 1
TP_OP_A, TP_OP_B, TP_OP_B0, TP_OP_L = 0, 1, 2, 3
TP_BH_DIFF_FULL, TP_BH_DIFF_LITERAL = 0, 1
TP_CONSTRAINT_AREA, TP_CONSTRAINT_VOLUME, TP_CONSTRAINT_FREE_BARYCENTER = 1, 2, 4
TP_POISSON_CHOLESKY, TP_POISSON_CG = 0, 1
TP_MAX_PINS = 64
_OPS = {"A": TP_OP_A, "B": TP_OP_B, "B0": TP_OP_B0, "L": TP_OP_L}


class TpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tp status {code}: {msg}")
        self.code = code


class tp_params(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_double), ("theta", ctypes.c_double), ("leaf_size", ctypes.c_int),
        ("precision", ctypes.c_int), ("bh_diff_mode", ctypes.c_int),
        ("krylov_tol", ctypes.c_double), ("krylov_max", ctypes.c_int), ("gmres_restart", ctypes.c_int),
        ("cg_tol", ctypes.c_double), ("cg_max", ctypes.c_int), ("armijo_c", ctypes.c_double),
        ("armijo_shrink", ctypes.c_double), ("tau0", ctypes.c_double), ("ls_max", ctypes.c_int),
        ("fixed_tau", ctypes.c_int), ("proj_iters", ctypes.c_int), ("poisson_solver", ctypes.c_int),
        ("bvh_refit", ctypes.c_int), ("prec_self_weight", ctypes.c_double), ("tau0_disp", ctypes.c_double),
        ("tensor_cores", ctypes.c_int),
    ]


class tp_constraints(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_int), ("A0", ctypes.c_double), ("V0", ctypes.c_double)]


class tp_step_report(ctypes.Structure):
    _fields_ = [
        ("E_before", ctypes.c_double), ("E_after", ctypes.c_double), ("tau", ctypes.c_double),
        ("slope", ctypes.c_double), ("phi_before", ctypes.c_double * 2),
        ("phi_after", ctypes.c_double * 2), ("krylov_iters", ctypes.c_int),
        ("cg_iters", ctypes.c_int), ("ls_trials", ctypes.c_int), ("status", ctypes.c_int),
        ("pair_interactions", ctypes.c_double),
    ]


class tp_chol_info(ctypes.Structure):
    _fields_ = [("available", ctypes.c_int), ("components", ctypes.c_int), ("unknowns", ctypes.c_int),
                ("supernodes", ctypes.c_int), ("levels", ctypes.c_int), ("max_front", ctypes.c_int),
                ("factor_floats", ctypes.c_double), ("update_floats", ctypes.c_double)]


class tp_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("units", ctypes.c_double), ("columns", ctypes.c_double)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)


class tp_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded libtpsurf (ctypes.CDLL); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libtpsurf.so is not built ({path}); run "
                          "python -c 'import __graft_entry__ as g; g.build()'")
    L = ctypes.CDLL(path)
    c_int, c_double, vp, c_size = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "tp_params_default": (None, [P(tp_params)]),
        "tp_mesh_create": (c_int, [c_int, c_int, c_int, vp, vp, c_int, vp, P(vp)]),
        "tp_mesh_create_ctx": (c_int, [vp, c_int, c_int, vp, vp, c_int, vp, P(vp)]),
        "tp_create": (c_int, [c_int, P(vp)]),
        "tp_destroy": (c_int, [vp]),
        "tp_ctx_set_allocator": (c_int, [vp, P(tp_allocator)]),
        "tp_ctx_memory": (c_int, [vp, P(c_size), P(c_size)]),
        "tp_mesh_set_positions": (c_int, [vp, vp, c_int, vp]),
        "tp_mesh_get_positions": (c_int, [vp, vp, c_int, vp]),
        "tp_mesh_destroy": (c_int, [vp]),
        "tp_mesh_area_volume": (c_int, [vp, P(c_double), P(c_double), vp]),
        "tp_mesh_footprint_bytes": (c_size, [c_int, c_int, P(tp_params)]),
        "tp_energy": (c_int, [vp, P(tp_params), P(c_double), vp]),
        "tp_energy_rows": (c_int, [vp, P(tp_params), vp, c_int, vp, c_int, vp]),
        "tp_differential": (c_int, [vp, P(tp_params), vp, c_int, P(c_double), vp]),
        "fractional_apply": (c_int, [vp, P(tp_params), c_int, vp, c_int, vp, c_int, vp]),
        "cotan_solve": (c_int, [vp, P(tp_params), vp, c_int, vp, c_int, vp, P(c_int)]),
        "cotan_factor_info": (c_int, [vp, P(tp_chol_info)]),
        "precond_apply": (c_int, [vp, P(tp_params), vp, c_int, vp, c_int, vp]),
        "precond_step": (c_int, [vp, P(tp_params), P(tp_constraints), P(tp_step_report), vp]),
        "tp_last_error": (ctypes.c_char_p, []),
        "tp_profile_enable": (c_int, [vp, c_int]),
        "tp_profile_read": (c_int, [vp, P(tp_kernel_stat), c_int, P(c_int)]),
        "tp_launch_count": (ctypes.c_ulonglong, []),
        "tp_energy_noalloc": (c_int, [vp, c_int, vp, c_int, c_double, vp, vp]),
        "tp_obstacle_set": (c_int, [vp, c_int, c_int, vp, vp, c_double, c_int, vp]),
        "tp_pins_set": (c_int, [vp, c_int, vp, c_int, vp]),
        "tp_willmore_set": (c_int, [vp, c_double]),
        "tp_selftest_wait": (c_int, [c_int, P(c_int)]),
        "tp_willmore_energy": (c_int, [vp, P(c_double), vp, c_int, vp]),
        "tp_obstacle_energy": (c_int, [vp, P(tp_params), P(c_double), vp, c_int, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code):
    if code != TP_OK:
        raise TpError(code, lib().tp_last_error().decode())


def params(**overrides) -> tp_params:
    """tp_params with the library defaults and the given fields replaced."""
    p = tp_params()
    lib().tp_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(f"tp_params has no field {k}")
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _stream_ptr(x=None):
    if x is None or not _is_cuda(x):
        try:
            torch = _torch()
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(_torch().cuda.current_stream(x.device).cuda_stream)


def _as_buffer(x, dtype):
    """(pointer, kind, keepalive) of a contiguous array of the given numpy dtype."""
    if _is_cuda(x):
        torch = _torch()
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        t = x.to(tdt).contiguous()
        return ctypes.c_void_p(t.data_ptr()), TP_PTR_DEVICE, t
    if hasattr(x, "numpy"):
        x = x.detach().cpu().numpy()
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), TP_PTR_HOST, a


def _empty_like_kind(ref, shape, dtype=np.float64):
    if _is_cuda(ref):
        torch = _torch()
        t = torch.empty(shape, dtype=torch.float64, device=ref.device)
        return t, ctypes.c_void_p(t.data_ptr()), TP_PTR_DEVICE
    a = np.empty(shape, dtype=dtype)
    return a, ctypes.c_void_p(a.ctypes.data), TP_PTR_HOST


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------

class Context:
    """Owns a tp_ctx: a device and the allocator of its meshes' device memory.

    allocator=None keeps cudaMalloc / cudaFree. allocator="torch" takes the
    memory from PyTorch's caching allocator on that device, so the library's
    workspaces share one pool with the caller's tensors."""

    def __init__(self, device: int = 0, allocator=None):
        self.device = device
        self.handle = tp_create(device)
        self._cb = None
        if allocator == "torch":
            self.set_torch_allocator()
        elif allocator is not None:
            raise ValueError("allocator must be None or 'torch'")

    def set_torch_allocator(self):
        torch = _torch()

        def _alloc(nbytes, device, user):
            try:
                with torch.cuda.device(device):
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), device,
                                                                  torch.cuda.current_stream(device)))
            except Exception:
                return None

        def _free(ptr, nbytes, device, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        cb = (_ALLOC_FN(_alloc), _FREE_FN(_free))
        a = tp_allocator(cb[0], cb[1], None)
        _check(lib().tp_ctx_set_allocator(self.handle, ctypes.byref(a)))
        self._cb = cb          # the callbacks must outlive the context

    def memory(self):
        """(bytes in use, peak bytes) of the context's meshes."""
        return tp_ctx_memory(self)

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().tp_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tp_create(device: int = 0):
    h = ctypes.c_void_p()
    _check(lib().tp_create(int(device), ctypes.byref(h)))
    return h


def tp_destroy(ctx: Context):
    ctx.close()


def tp_ctx_set_allocator(ctx: Context, allocator=None):
    """allocator: None (cudaMalloc) or 'torch' (PyTorch's caching allocator)."""
    if allocator == "torch":
        ctx.set_torch_allocator()
    elif allocator is None:
        _check(lib().tp_ctx_set_allocator(ctx.handle, None))
        ctx._cb = None
    else:
        raise ValueError("allocator must be None or 'torch'")


def tp_ctx_memory(ctx: Context):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().tp_ctx_memory(ctx.handle, ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


class Mesh:
    """Owns a tp_mesh handle (positions, face tables, BVH, Laplacian on the GPU),
    in the device's default context or in the given Context."""

    def __init__(self, positions, faces, device: int = 0, ctx: Context | None = None):
        if ctx is not None:
            self.handle = tp_mesh_create_ctx(ctx, positions, faces)
            device = ctx.device
        else:
            self.handle = tp_mesh_create(positions, faces, device)
        self.ctx = ctx          # keeps the context alive while the mesh is
        self.nv = int(np.shape(positions)[0])
        self.nf = int(np.shape(faces)[0])
        self.device = device

    def set_positions(self, positions):
        tp_mesh_set_positions(self, positions)

    def get_positions(self, like=None):
        return tp_mesh_get_positions(self, like)

    def close(self):
        if getattr(self, "handle", None):
            lib().tp_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tp_mesh_create(positions, faces, device: int = 0):
    pp, pk, keep_p = _as_buffer(positions, np.float64)
    fp, fk, keep_f = _as_buffer(faces, np.int32)
    if pk != fk:
        raise ValueError("positions and faces must both be host or both be device arrays")
    h = ctypes.c_void_p()
    nv, nf = int(np.shape(positions)[0]), int(np.shape(faces)[0])
    _check(lib().tp_mesh_create(device, nv, nf, pp, fp, pk, _stream_ptr(positions), ctypes.byref(h)))
    return h


def tp_mesh_create_ctx(ctx: Context, positions, faces):
    pp, pk, keep_p = _as_buffer(positions, np.float64)
    fp, fk, keep_f = _as_buffer(faces, np.int32)
    if pk != fk:
        raise ValueError("positions and faces must both be host or both be device arrays")
    h = ctypes.c_void_p()
    nv, nf = int(np.shape(positions)[0]), int(np.shape(faces)[0])
    _check(lib().tp_mesh_create_ctx(ctx.handle, nv, nf, pp, fp, pk, _stream_ptr(positions), ctypes.byref(h)))
    return h


def tp_mesh_set_positions(mesh: Mesh, positions):
    pp, pk, keep = _as_buffer(positions, np.float64)
    _check(lib().tp_mesh_set_positions(mesh.handle, pp, pk, _stream_ptr(positions)))


def tp_mesh_get_positions(mesh: Mesh, like=None):
    out, ptr, kind = _empty_like_kind(like, (mesh.nv, 3))
    _check(lib().tp_mesh_get_positions(mesh.handle, ptr, kind, _stream_ptr(like)))
    return out


def tp_mesh_area_volume(mesh: Mesh):
    """(total area, enclosed signed volume) of the mesh's current positions (§7.1.3, §7.1.4)."""
    A, V = ctypes.c_double(), ctypes.c_double()
    _check(lib().tp_mesh_area_volume(mesh.handle, ctypes.byref(A), ctypes.byref(V), _stream_ptr()))
    return A.value, V.value


def tp_mesh_destroy(mesh: Mesh):
    mesh.close()


def tp_mesh_footprint_bytes(nv: int, nf: int, p: tp_params | None = None) -> int:
    p = p or params()
    return int(lib().tp_mesh_footprint_bytes(nv, nf, ctypes.byref(p)))


def tp_energy(mesh: Mesh, p: tp_params | None = None) -> float:
    p = p or params()
    E = ctypes.c_double()
    _check(lib().tp_energy(mesh.handle, ctypes.byref(p), ctypes.byref(E), _stream_ptr()))
    return E.value


def tp_energy_rows(mesh: Mesh, targets, p: tp_params | None = None):
    p = p or params()
    tp_, tk, keep = _as_buffer(targets, np.int32)
    n = int(np.shape(targets)[0])
    out, ptr, kind = _empty_like_kind(targets, (n,))
    _check(lib().tp_energy_rows(mesh.handle, ctypes.byref(p), tp_, n, ptr, kind, _stream_ptr(targets)))
    return out


def tp_differential(mesh: Mesh, p: tp_params | None = None, like=None):
    """(dE [nv,3], E); dE in the memory kind of `like` (host by default)."""
    p = p or params()
    out, ptr, kind = _empty_like_kind(like, (mesh.nv, 3))
    E = ctypes.c_double()
    _check(lib().tp_differential(mesh.handle, ctypes.byref(p), ptr, kind, ctypes.byref(E), _stream_ptr(like)))
    return out, E.value


def fractional_apply(mesh: Mesh, op, v, p: tp_params | None = None):
    p = p or params()
    op = _OPS.get(op, op)
    vp, vk, keep = _as_buffer(v, np.float64)
    k = 1 if len(np.shape(v)) == 1 else int(np.shape(v)[1])
    out, ptr, kind = _empty_like_kind(v, tuple(np.shape(v)))
    _check(lib().fractional_apply(mesh.handle, ctypes.byref(p), int(op), vp, k, ptr, vk, _stream_ptr(v)))
    return out


def cotan_solve(mesh: Mesh, b, p: tp_params | None = None):
    p = p or params()
    bp, bk, keep = _as_buffer(b, np.float64)
    k = 1 if len(np.shape(b)) == 1 else int(np.shape(b)[1])
    out, ptr, kind = _empty_like_kind(b, tuple(np.shape(b)))
    it = ctypes.c_int()
    _check(lib().cotan_solve(mesh.handle, ctypes.byref(p), bp, k, ptr, bk, _stream_ptr(b), ctypes.byref(it)))
    return out, it.value


def cotan_factor_info(mesh: Mesh) -> dict:
    """Structure of the sparse Cholesky factor of the mesh's cotan Laplacian."""
    info = tp_chol_info()
    _check(lib().cotan_factor_info(mesh.handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in tp_chol_info._fields_}


def precond_apply(mesh: Mesh, b, p: tp_params | None = None):
    p = p or params()
    bp, bk, keep = _as_buffer(b, np.float64)
    k = 1 if len(np.shape(b)) == 1 else int(np.shape(b)[1])
    out, ptr, kind = _empty_like_kind(b, tuple(np.shape(b)))
    _check(lib().precond_apply(mesh.handle, ctypes.byref(p), bp, k, ptr, bk, _stream_ptr(b)))
    return out


def precond_step(mesh: Mesh, constraints: tp_constraints, p: tp_params | None = None) -> dict:
    p = p or params()
    rep = tp_step_report()
    _check(lib().precond_step(mesh.handle, ctypes.byref(p), ctypes.byref(constraints), ctypes.byref(rep),
                              _stream_ptr()))
    return {
        "E_before": rep.E_before, "E_after": rep.E_after, "tau": rep.tau, "slope": rep.slope,
        "phi_before": list(rep.phi_before), "phi_after": list(rep.phi_after),
        "krylov_iters": rep.krylov_iters, "cg_iters": rep.cg_iters, "ls_trials": rep.ls_trials,
        "status": rep.status, "pair_interactions": rep.pair_interactions,
    }


def tp_selftest_wait(device: int = 0):
    """(status, timed_out) of the bounded-wait self-test (no exception: a
    TP_ERR_TIMEOUT status is the expected outcome)."""
    t = ctypes.c_int()
    code = lib().tp_selftest_wait(int(device), ctypes.byref(t))
    return code, t.value


def tp_willmore_set(mesh: Mesh, weight: float):
    """Weight of the Willmore term and its H^2 metric term in precond_step (§7.3.5)."""
    _check(lib().tp_willmore_set(mesh.handle, float(weight)))


def tp_willmore_energy(mesh: Mesh, like=None):
    """(E_W, dE_W [nv,3]) of the current positions; dE_W in the memory kind of `like`."""
    out, ptr, kind = _empty_like_kind(like, (mesh.nv, 3))
    E = ctypes.c_double()
    _check(lib().tp_willmore_energy(mesh.handle, ctypes.byref(E), ptr, kind, _stream_ptr(like)))
    return E.value, out


def tp_pins_set(mesh: Mesh, vertices=None):
    """Pin the given vertices (§7.1.2, §7.2); None or an empty list removes the pins."""
    if vertices is None or len(vertices) == 0:
        _check(lib().tp_pins_set(mesh.handle, 0, None, TP_PTR_HOST, _stream_ptr()))
        return
    vp, vk, keep = _as_buffer(vertices, np.int32)
    _check(lib().tp_pins_set(mesh.handle, int(np.shape(vertices)[0]), vp, vk, _stream_ptr(vertices)))


def tp_obstacle_set(mesh: Mesh, positions=None, faces=None, weight: float = 1.0):
    """Attach a static obstacle mesh (§7.3.2) to `mesh`; positions=None removes it."""
    if positions is None:
        _check(lib().tp_obstacle_set(mesh.handle, 0, 0, None, None, 0.0, TP_PTR_HOST, _stream_ptr()))
        return
    pp, pk, keep_p = _as_buffer(positions, np.float64)
    fp, fk, keep_f = _as_buffer(faces, np.int32)
    if pk != fk:
        raise ValueError("positions and faces must both be host or both be device arrays")
    nv, nf = int(np.shape(positions)[0]), int(np.shape(faces)[0])
    _check(lib().tp_obstacle_set(mesh.handle, nv, nf, pp, fp, float(weight), pk, _stream_ptr(positions)))


def tp_obstacle_energy(mesh: Mesh, p: tp_params | None = None, like=None, grad: bool = True):
    """(E_O, dE_O [nv,3] or None) of the obstacle set on `mesh`; dE_O in the
    memory kind of `like` (host by default)."""
    p = p or params()
    E = ctypes.c_double()
    if not grad:
        _check(lib().tp_obstacle_energy(mesh.handle, ctypes.byref(p), ctypes.byref(E), None, TP_PTR_HOST,
                                        _stream_ptr(like)))
        return E.value, None
    out, ptr, kind = _empty_like_kind(like, (mesh.nv, 3))
    _check(lib().tp_obstacle_energy(mesh.handle, ctypes.byref(p), ctypes.byref(E), ptr, kind, _stream_ptr(like)))
    return E.value, out


def tp_profile_enable(mesh: Mesh, on: bool = True):
    _check(lib().tp_profile_enable(mesh.handle, 1 if on else 0))


def tp_profile_read(mesh: Mesh) -> dict:
    """{kernel: {launches, ms, units}} accumulated since the last read (then reset)."""
    buf = (tp_kernel_stat * 32)()
    n = ctypes.c_int()
    _check(lib().tp_profile_read(mesh.handle, buf, 32, ctypes.byref(n)))
    return {buf[i].name.decode(): {"launches": buf[i].launches, "ms": buf[i].ms, "units": buf[i].units,
                                   "columns": buf[i].columns}
            for i in range(n.value)}


def tp_launch_count() -> int:
    return int(lib().tp_launch_count())


def tp_energy_noalloc(positions, faces, E_out, p: float = 6.0) -> None:
    """Direct energy into the CUDA tensor E_out (float64, at least 1 element)
    with no device allocation, for callers that may not allocate (see
    include/tp.h). positions [nv,3] float64 and faces [nf,3] int32 must be
    contiguous CUDA tensors on the current device (at most 32768 faces).
    Inputs of another dtype, layout or device are rejected, not converted:
    converting would allocate. A face index outside 0..nv-1 makes E_out NaN."""
    torch = _torch()
    cur = torch.cuda.current_device()
    for name, t, dt in (("positions", positions, torch.float64), ("faces", faces, torch.int32),
                        ("E_out", E_out, torch.float64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"tp_energy_noalloc: {name} must be a CUDA tensor")
        if t.dtype != dt:
            raise TypeError(f"tp_energy_noalloc: {name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"tp_energy_noalloc: {name} must be contiguous")
        if t.device.index != cur:
            raise ValueError(f"tp_energy_noalloc: {name} is on cuda:{t.device.index}, "
                             f"the current device is cuda:{cur}")
    if positions.dim() != 2 or positions.shape[1] != 3:
        raise ValueError("tp_energy_noalloc: positions must have shape [nv, 3]")
    if faces.dim() != 2 or faces.shape[1] != 3:
        raise ValueError("tp_energy_noalloc: faces must have shape [nf, 3]")
    if E_out.numel() < 1:
        raise ValueError("tp_energy_noalloc: E_out needs at least one element")
    _check(lib().tp_energy_noalloc(ctypes.c_void_p(positions.data_ptr()), int(positions.shape[0]),
                                   ctypes.c_void_p(faces.data_ptr()), int(faces.shape[0]), float(p),
                                   ctypes.c_void_p(E_out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))


# ---------------------------------------------------------------------------
# autograd: E with the hand-written dE as its backward
# ---------------------------------------------------------------------------

def _make_autograd():
    torch = _torch()

    class _TangentPointEnergy(torch.autograd.Function):
        """E(f) of Eq. 10 (or its Barnes-Hut approximation); its backward is
        the library's differential kernel. f is a float64 CUDA tensor [nv,3]."""

        @staticmethod
        def forward(ctx, positions, mesh, p):
            f = positions.detach().contiguous()
            tp_mesh_set_positions(mesh, f)
            ctx.save_for_backward(f)
            ctx.mesh, ctx.p = mesh, p
            return positions.new_tensor(tp_energy(mesh, p))

        @staticmethod
        def backward(ctx, grad_out):
            (f,) = ctx.saved_tensors
            tp_mesh_set_positions(ctx.mesh, f)
            dE, _ = tp_differential(ctx.mesh, ctx.p, like=f)
            return grad_out * dE, None, None

    return _TangentPointEnergy


class _Lazy:
    _fn = None

    def apply(self, positions, mesh, p=None):
        if _Lazy._fn is None:
            _Lazy._fn = _make_autograd()
        return _Lazy._fn.apply(positions, mesh, p or params())


TangentPointEnergy = _Lazy()
