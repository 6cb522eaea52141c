"""Host analysis of the sparse Cholesky factor of the cotan Laplacian (§5.2
pre-factorisation): the nested-dissection order, supernodal tree and index
maps of paper_2107_01664_gb300/csrc/chol_symbolic.h, exercised on the CPU by
an FP64 multifrontal factorisation through those maps (tests/
chol_symbolic_driver.cpp) and compared with the oracle's exact sparse
solve. No GPU."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import small_mesh, vertex_vectors, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_01664_gb300", "csrc")


@pytest.fixture(scope="module")
def driver():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="chol_drv_")
    exe = os.path.join(d, "drv")
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "chol_symbolic_driver.cpp"),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def run(driver, C, b, leaf):
    C = C.tocsr()
    C.sort_indices()
    nv, k = b.shape
    with tempfile.TemporaryDirectory() as d:
        fin, fout = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
        with open(fin, "wb") as f:
            np.array([nv, C.nnz, k, leaf], dtype=np.int32).tofile(f)
            C.indptr.astype(np.int32).tofile(f)
            C.indices.astype(np.int32).tofile(f)
            C.data.astype(np.float64).tofile(f)
            np.ascontiguousarray(b, dtype=np.float64).tofile(f)
        r = subprocess.run([driver, fin, fout], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        raw = open(fout, "rb").read()
    hdr = np.frombuffer(raw[:20], dtype=np.int32)
    z = np.frombuffer(raw[20:], dtype=np.float64).reshape(nv, k)
    return dict(n=int(hdr[0]), ncomp=int(hdr[1]), nnode=int(hdr[2]), levels=int(hdr[3]), max_front=int(hdr[4])), z


def union(meshes):
    Vs, Fs, off = [], [], 0
    for V, F in meshes:
        Vs.append(V)
        Fs.append(F + off)
        off += len(V)
    return np.concatenate(Vs), np.concatenate(Fs)


def comp_project(x, comp):
    x = x.copy()
    for c in np.unique(comp):
        x[comp == c] -= x[comp == c].mean(axis=0)
    return x


@pytest.mark.parametrize("name,leaf", [("tetra", 64), ("octa", 2), ("torus13x7", 8), ("ico3", 64), ("ico3", 5)])
def test_factor_solve_matches_exact_solve(driver, name, leaf):
    V, F = small_mesh(name, seed=21)
    C = O.cotan_laplacian(V, F)
    b = O.project_mean_zero(vertex_vectors(len(V), 3, 4))
    info, z = run(driver, C, b, leaf)
    assert info["ncomp"] == 1 and info["n"] == len(V) - 1
    ref = O.poisson_solve(C, b)
    assert np.linalg.norm(O.project_mean_zero(z) - ref) <= 1e-10 * np.linalg.norm(ref)
    # the pinned vertex is the first one, as in the oracle: z itself solves C z = b
    assert np.all(z[0] == 0.0)
    assert np.linalg.norm(C @ z - b) <= 1e-10 * np.linalg.norm(b)


def test_two_components_pin_one_vertex_each(driver):
    A = small_mesh("ico2", seed=3)
    B = small_mesh("torus13x7", seed=4)
    B = (B[0] + np.array([5.0, 0.0, 0.0]), B[1])
    V, F = union([A, B])
    comp = np.r_[np.zeros(len(A[0]), int), np.ones(len(B[0]), int)]
    C = O.cotan_laplacian(V, F)
    b = comp_project(vertex_vectors(len(V), 2, 7), comp)
    info, z = run(driver, C, b, 16)
    assert info["ncomp"] == 2 and info["n"] == len(V) - 2
    assert z[0].tolist() == [0.0, 0.0] and z[len(A[0])].tolist() == [0.0, 0.0]
    # each component against the oracle's solve of that component alone
    for (Vc, Fc), sl in ((A, slice(0, len(A[0]))), (B, slice(len(A[0]), len(V)))):
        ref = O.poisson_solve(O.cotan_laplacian(Vc, Fc), b[sl])
        got = O.project_mean_zero(z[sl])
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_benchmark_torus_tree_shape(driver):
    # the 20,000-face torus: the tree the device factorisation runs on
    V, F = workload("torus_20k")
    C = O.cotan_laplacian(V, F)
    b = O.project_mean_zero(vertex_vectors(len(V), 1, 2))
    info, z = run(driver, C, b, 64)
    assert info["n"] == len(V) - 1
    assert info["levels"] <= 12 and info["max_front"] <= 256
    assert np.linalg.norm(C @ z - b) <= 1e-9 * np.linalg.norm(b)


def test_leaf_of_one_vertex(driver):
    # leaf size 1: the dissection goes down until no level splits a set
    V, F = small_mesh("torus13x7", seed=1)
    C = O.cotan_laplacian(V, F)
    b = O.project_mean_zero(vertex_vectors(len(V), 1, 1))
    info, z = run(driver, C, b, 1)
    assert info["nnode"] >= 2
    assert np.linalg.norm(C @ z - b) <= 1e-12 * np.linalg.norm(b)


def test_long_separators_become_chains(driver):
    # an icosphere of level 6 (40,962 vertices) has separators whose fronts
    # are too wide for one panel: they are split into chains of supernodes,
    # and the factorisation through the chained tree still solves exactly
    from synth import icosphere
    V, F = icosphere(6)
    C = O.cotan_laplacian(V, F)
    b = O.project_mean_zero(vertex_vectors(len(V), 2, 5))
    info, z = run(driver, C, b, 64)
    assert info["n"] == len(V) - 1
    assert info["levels"] > 12            # the chains deepen the tree
    ref = O.poisson_solve(C, b)
    assert np.linalg.norm(O.project_mean_zero(z) - ref) <= 1e-10 * np.linalg.norm(ref)
