"""Write full_size.json: oracle values at the full workload sizes whose
direct evaluation takes minutes on a CPU (so the GPU tests compare against
stored values): the energy of Eq. 10 of the named workloads and the
static-obstacle energy of §7.3.2 of torus_20k around its ball obstacle. Calls only the FP64 oracle and the seeded input generators.

    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tp_oracle as O  # noqa: E402
from synth import obstacle, workload  # noqa: E402


def main():
    out = {}
    for name in ("torus_20k", "linked_tori_50k"):
        V, F = workload(name)
        t = time.time()
        E = O.energy(V, F)
        out[name] = {"nv": int(len(V)), "nf": int(len(F)), "p": 6.0, "energy": E,
                     "area": O.total_area(V, F), "volume": O.total_volume(V, F),
                     "oracle_seconds": round(time.time() - t, 1)}
        print(name, out[name], flush=True)
    # static obstacle (§7.3.2): torus_20k around the ball in its hole
    V, F = workload("torus_20k")
    VO, FO = obstacle("ball_in_torus_hole")
    t = time.time()
    E = O.obstacle_energy(V, F, VO, FO, 6.0, 1.0)
    out["torus_20k+ball_in_torus_hole"] = {"nf": int(len(F)), "nf_obstacle": int(len(FO)), "p": 6.0,
                                           "weight": 1.0, "obstacle_energy": E,
                                           "oracle_seconds": round(time.time() - t, 1)}
    print("torus_20k+ball_in_torus_hole", out["torus_20k+ball_in_torus_hole"], flush=True)
    with open(os.path.join(HERE, "full_size.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
