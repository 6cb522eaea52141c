"""Host helpers of the library (csrc/host_util.h), compiled with g++ into a
small driver: connected components of triangle meshes (against scipy's
graph components, labels in the order of the smallest vertex) and the dense
inverse of the pins' small system (against numpy, and a singular matrix
detected). No GPU."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import small_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_01664_gb300", "csrc")


@pytest.fixture(scope="module")
def driver():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="host_util_")
    exe = os.path.join(d, "drv")
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "host_util_driver.cpp"),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def call(driver, text):
    r = subprocess.run([driver], input=text, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    return r.stdout.split()


def mesh_union(parts, shuffle_seed=None):
    Vs, Fs, off = [], [], 0
    for V, F in parts:
        Vs.append(V)
        Fs.append(np.asarray(F) + off)
        off += len(V)
    V, F = np.concatenate(Vs), np.concatenate(Fs)
    if shuffle_seed is not None:
        perm = np.random.default_rng(shuffle_seed).permutation(len(V))
        inv = np.empty_like(perm)
        inv[perm] = np.arange(len(V))
        V, F = V[perm], inv[F]
    return V, F


@pytest.mark.parametrize("case", ["one", "three", "shuffled", "isolated"])
def test_components(driver, case):
    parts = [small_mesh("ico2", seed=1)]
    if case != "one":
        parts += [small_mesh("torus13x7", seed=2), small_mesh("octa")]
    V, F = mesh_union(parts, 5 if case == "shuffled" else None)
    nv = len(V) + (2 if case == "isolated" else 0)     # two vertices in no face
    out = call(driver, "components %d %d %s" % (nv, len(F), " ".join(map(str, F.ravel()))))
    nc, comp = int(out[0]), np.array(list(map(int, out[1:])))
    ref = O.mesh_components(nv, F)
    assert nc == len(np.unique(ref))
    # same partition, labels numbered by first appearance
    first = {}
    for v, c in enumerate(ref):
        first.setdefault(c, len(first))
    assert np.array_equal(comp, np.array([first[c] for c in ref]))


def test_invert_matches_numpy_and_detects_singular(driver):
    rng = np.random.default_rng(3)
    for n in (1, 5, 13):
        a = rng.standard_normal((n, n)) + n * np.eye(n)
        out = call(driver, "invert %d %s" % (n, " ".join("%.17g" % x for x in a.ravel())))
        assert out[0] == "ok"
        inv = np.array(list(map(float, out[1:]))).reshape(n, n)
        assert np.allclose(inv, np.linalg.inv(a), rtol=1e-12, atol=1e-14)
    # a saddle matrix like the pins' one: [-W E; E^T 0] with W SPD
    W = rng.standard_normal((4, 4))
    W = W @ W.T + np.eye(4)
    E = np.array([[1.0], [1.0], [1.0], [1.0]])
    M = np.block([[-W, E], [E.T, np.zeros((1, 1))]])
    out = call(driver, "invert 5 %s" % " ".join("%.17g" % x for x in M.ravel()))
    inv = np.array(list(map(float, out[1:]))).reshape(5, 5)
    assert np.allclose(inv @ M, np.eye(5), atol=1e-12)
    assert call(driver, "invert 2 1 2 2 4") == ["singular"]    # rank 1
