"""Write torus20k_samples.json: oracle values of the 20,000-face torus at
sampled vertices (the differential, and A u for a seeded u with 3 columns),
for the accuracy report of the benchmark. Calls only the FP64 oracle and the
seeded input generators.

    python tests/golden/make_samples.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tp_oracle as O  # noqa: E402
from synth import vertex_vectors, workload  # noqa: E402


def main():
    V, F = workload("torus_20k")
    t = time.time()
    verts = np.random.default_rng(808).choice(len(V), 64, replace=False)
    u = vertex_vectors(len(V), 3, 202)
    out = {"workload": "torus_20k", "p": 6.0, "u": "vertex_vectors(nv, 3, seed 202)",
           "vertices": [int(v) for v in verts],
           "dE": O.differential_at_vertices(V, F, verts).tolist(),
           "Au": O.apply_operator_at_vertices(V, F, u, "A", verts).tolist(),
           "oracle_seconds": None}
    out["oracle_seconds"] = round(time.time() - t, 1)
    with open(os.path.join(HERE, "torus20k_samples.json"), "w") as fh:
        json.dump(out, fh)
    print("samples", out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
