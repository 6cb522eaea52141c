"""Write icosphere_l8_samples.json: oracle (FP64 direct) values on the
1,310,720-face icosphere with spherical-harmonic bumps, for the full-size
parity test and the accuracy report of the benchmark's large-mesh section:

- the energy rows of Eq. 10 at 20,000 seeded target faces,
- the differential at 64 seeded vertices,
- A u at 64 seeded vertices for a seeded u with 3 columns.

Calls only the FP64 oracle and the seeded input generators; the rows are
computed in a process pool (the oracle's arithmetic is unchanged, only the
batches are smaller so that each worker stays within a few GB).

    python tests/golden/make_l8_samples.py [workers]
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tp_oracle as O  # noqa: E402
from synth import vertex_vectors, workload  # noqa: E402

N_TARGETS, N_VERTS = 20000, 64
_mesh = {}


def _init():
    O.CHUNK = 16
    _mesh["VF"] = workload("icosphere_l8")


def _rows(batch):
    V, F = _mesh["VF"]
    return O.energy_rows(V, F, 6.0, np.asarray(batch))


def _dE(batch):
    V, F = _mesh["VF"]
    return O.differential_at_vertices(V, F, np.asarray(batch))


def _Au(batch):
    V, F = _mesh["VF"]
    u = vertex_vectors(len(V), 3, 507)
    return O.apply_operator_at_vertices(V, F, u, "A", np.asarray(batch))


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    V, F = workload("icosphere_l8")
    targets = np.random.default_rng(505).choice(len(F), N_TARGETS, replace=False)
    verts = np.random.default_rng(506).choice(len(V), N_VERTS, replace=False)
    t = time.time()
    with mp.get_context("spawn").Pool(workers, initializer=_init) as pool:
        rows = np.concatenate(pool.map(_rows, [targets[i:i + 16] for i in range(0, N_TARGETS, 16)]))
        dE = np.concatenate(pool.map(_dE, [verts[i:i + 2] for i in range(0, N_VERTS, 2)]))
        Au = np.concatenate(pool.map(_Au, [verts[i:i + 2] for i in range(0, N_VERTS, 2)]))
    out = {"workload": "icosphere_l8", "p": 6.0, "reference": "FP64 direct sums of the oracle",
           "targets": [int(x) for x in targets], "rows": [float(x) for x in rows],
           "vertices": [int(x) for x in verts], "dE": dE.tolist(),
           "u": "vertex_vectors(nv, 3, seed 507)", "Au": Au.tolist(),
           "oracle_seconds": round(time.time() - t, 1), "workers": workers}
    with open(os.path.join(HERE, "icosphere_l8_samples.json"), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))
    print("icosphere_l8 samples:", out["oracle_seconds"], "s on", workers, "workers")


if __name__ == "__main__":
    main()
