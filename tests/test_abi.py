"""The C-ABI library builds, loads and exports every symbol of include/tp.h
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted({n for n in names if n not in ("defined",)})


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ["tp_energy", "tp_differential", "fractional_apply", "precond_step", "precond_apply",
              "cotan_solve", "tp_mesh_create", "tp_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import os as _os
    from paper_2107_01664_gb300 import build as b
    path = b.build()
    # RTLD_NOW resolves every symbol at load time: an undefined one fails here
    lib = ctypes.CDLL(path, mode=_os.RTLD_NOW | _os.RTLD_LOCAL)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_default_and_host_logic():
    import paper_2107_01664_gb300 as tp
    p = tp.params()
    assert p.p == 6.0 and p.theta == 0.0 and p.leaf_size == 8 and p.precision == tp.TP_PREC_FP32
    assert p.prec_self_weight == 24.0 and p.bvh_refit == 0 and p.tau0_disp == 0.0 and p.tensor_cores == 0   # last fields: layouts agree
    q = tp.params(theta=0.5, leaf_size=4)
    assert q.theta == 0.5 and q.leaf_size == 4
    with pytest.raises(AttributeError):
        tp.params(nonexistent=1)
    # footprint is a pure host computation and grows with the mesh
    small = tp.tp_mesh_footprint_bytes(642, 1280)
    big = tp.tp_mesh_footprint_bytes(655362, 1310720)
    assert 0 < small < big


def test_errors_without_device_are_reported_not_crashing():
    import numpy as np
    import paper_2107_01664_gb300 as tp
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the no-device error path")
    V = np.zeros((4, 3))
    F = np.array([[0, 1, 2]], dtype=np.int32)
    with pytest.raises(tp.TpError):
        tp.Mesh(V, F, device=0)


def test_context_without_device_is_an_error_not_a_crash():
    import paper_2107_01664_gb300 as tp
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the no-device error path")
    with pytest.raises(tp.TpError) as e:
        tp.Context(0)
    assert e.value.code == tp.TP_ERR_INVALID_ARG
    assert tp.lib().tp_destroy(None) == tp.TP_OK
