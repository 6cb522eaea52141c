"""Failure detection on the GPU without a fault: a kernel waits, with the
bounded wait of the sparse Cholesky sweep, for a device word that nothing
sets; the wait gives up after about a second, the library reports
TP_ERR_TIMEOUT, and the context keeps working."""
import time

import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import small_mesh

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_stays_usable(lib):
    import torch
    t0 = time.perf_counter()
    code, timed_out = lib.tp_selftest_wait(0)
    dt = time.perf_counter() - t0
    assert code == lib.TP_ERR_TIMEOUT and timed_out == 1
    assert 0.2 < dt < 30.0
    V, F = small_mesh("ico2", seed=1)
    with lib.Mesh(torch.tensor(V, device="cuda:0"), torch.tensor(F, dtype=torch.int32, device="cuda:0")) as m:
        E = lib.tp_energy(m, lib.params(precision=1))
    assert abs(E - O.energy(V, F)) <= 1e-10 * abs(O.energy(V, F))
