"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics (closed forms, invariants, exact identities, brute force).

Each test is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails it; the mutation tests
at the end plant such slips in the oracle and check that a pin catches them.
"""
import numpy as np
import pytest

from oracle import tp_oracle as O
from synth import icosphere, small_mesh, torus, linked_tori

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


# ---------------------------------------------------------------------------
# energy, Eq. 10
# ---------------------------------------------------------------------------

def test_energy_tetrahedron_closed_form():
    # regular tetrahedron (+-1,+-1,+-1 with even sign count): barycenters at
    # radius 1/sqrt(3) with radial normals, so K = (2/sqrt3)^-6 = 27/64 for all
    # 12 ordered pairs; every face has area 2 sqrt(3): E = 12 * 27/64 * 12.
    V, F = small_mesh("tetra")
    assert O.energy(V, F) == pytest.approx(60.75, rel=1e-14)


def test_energy_octahedron_closed_form():
    # octahedron: 8 faces of area sqrt(3)/2, barycenters on a sphere of radius
    # 1/sqrt(3), K = 27/64 for each of the 56 ordered pairs.
    V, F = small_mesh("octa")
    assert O.energy(V, F) == pytest.approx(56 * 27 / 64 * 0.75, rel=1e-14)


@pytest.mark.parametrize("p", [6.0, 4.5, 3.0])
def test_energy_icosahedron_inscribed_sphere(p):
    # all barycenters of the regular icosahedron lie on one sphere (radius rho)
    # with radial normals: |P d| = |d|^2 / (2 rho), so K = (2 rho)^-p exactly
    # and E = (2 rho)^-p ((sum a)^2 - sum a^2).
    V, F = icosphere(0)
    X, N, a = O.face_geometry(V, F)
    rho = np.linalg.norm(X, axis=1)
    assert np.ptp(rho) < 1e-14
    expect = (2 * rho[0]) ** (-p) * (a.sum() ** 2 - np.sum(a * a))
    assert O.energy(V, F, p) == pytest.approx(expect, rel=1e-13)


def test_energy_sphere_limit_second_order():
    # smooth energy of the unit sphere: k = (2R)^-p and E = (4 pi R^2)^2 (2R)^-p
    # = pi^2/4 at p=6, R=1. Midpoint quadrature on icospheres converges to it;
    # the error falls by ~4 per level (O(h^2), the upper end of the O(h)..O(h^2)
    # range the consistency study of §8.1 reports).
    errs = []
    for lvl in range(1, 5):
        V, F = icosphere(lvl)
        errs.append(abs(O.energy(V, F) - np.pi ** 2 / 4) / (np.pi ** 2 / 4))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.5 < r < 4.5 for r in ratios), ratios
    assert errs[-1] < 5e-3


# Energies of the unperturbed unit icospheres of levels 1-4 at p = 6 (midpoint
# subdivision of the regular icosahedron, projected to R = 1), to six digits.
# They come from an evaluation of Eq. 10 written separately from this oracle
# before it existed; they pin the absolute level of E (a uniform factor, a
# wrong area weight or a wrong exponent shifts them), which the convergence
# ratio of the test above cannot see.
ICOSPHERE_ENERGIES_P6 = {1: 3.07657, 2: 2.61306, 3: 2.50407, 4: 2.47678}


@pytest.mark.parametrize("lvl", [1, 2, 3, 4])
def test_energy_unit_icospheres_stored_values(lvl):
    V, F = icosphere(lvl)
    assert O.energy(V, F) == pytest.approx(ICOSPHERE_ENERGIES_P6[lvl], abs=6e-6)


def test_energy_rigid_invariance_and_scaling():
    V, F = small_mesh("ico2", seed=3)
    E = O.energy(V, F)
    R = _rot(11)
    assert O.energy(V @ R.T + np.array([0.3, -2.0, 5.0]), F) == pytest.approx(E, rel=1e-12)
    for p in (6.0, 4.5):
        lam = 1.7
        # units m^{2n-p} = m^{4-p} (§2.1)
        assert O.energy(lam * V, F, p) == pytest.approx(lam ** (4 - p) * O.energy(V, F, p), rel=1e-12)


def test_energy_rows_brute_force():
    # pure-Python double loop on a tiny mesh (independent of the chunked sum)
    V, F = small_mesh("ico1", seed=5)
    X, N, a = O.face_geometry(V, F)
    E = 0.0
    for S in range(len(F)):
        for T in range(len(F)):
            if S == T:
                continue
            d = X[S] - X[T]
            E += abs(float(N[S] @ d)) ** 6 / float(d @ d) ** 6 * a[S] * a[T]
    assert O.energy(V, F) == pytest.approx(E, rel=1e-13)


# ---------------------------------------------------------------------------
# differential
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mesh,p", [("ico2", 6.0), ("torus12x6", 6.0), ("ico1", 4.5)])
def test_differential_central_differences(mesh, p):
    V, F = small_mesh(mesh, seed=9)
    g = O.differential(V, F, p)
    rng = np.random.default_rng(303)
    h = 1e-6
    for _ in range(8):
        dv = rng.standard_normal(V.shape)
        dv /= np.linalg.norm(dv)
        fd = (O.energy(V + h * dv, F, p) - O.energy(V - h * dv, F, p)) / (2 * h)
        assert np.sum(g * dv) == pytest.approx(fd, rel=2e-7, abs=1e-9 * np.abs(g).sum())


def test_differential_invariances():
    V, F = small_mesh("ico2", seed=4)
    g = O.differential(V, F)
    scale = np.abs(g).max()
    assert np.abs(g.sum(axis=0)).max() < 1e-12 * scale * len(V)           # translations
    assert np.abs(np.cross(V, g).sum(axis=0)).max() < 1e-12 * scale * len(V)  # rotations
    R = _rot(2)
    assert np.allclose(O.differential(V @ R.T, F), g @ R.T, rtol=0, atol=1e-12 * scale)
    lam = 0.6
    assert np.allclose(O.differential(lam * V, F), lam ** (3 - 6) * g, rtol=1e-11, atol=0)


def test_differential_sampled_vertices_match_full():
    V, F = small_mesh("torus12x6", seed=1)
    g = O.differential(V, F)
    idx = [0, 7, 33, len(V) - 1]
    assert np.allclose(O.differential_at_vertices(V, F, idx), g[idx], rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# operators: Algorithm 1 / Eq. 11-13 against the kernel-matrix form (App. A)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mesh", ["ico1", "torus8x4"])
@pytest.mark.parametrize("kind", ["L", "B", "B0"])
def test_pairwise_assembly_equals_kernel_matrix_form(mesh, kind):
    V, F = small_mesh(mesh, seed=2)
    s = O.sobolev_s(6.0)
    sigma = 2.0 - s if kind == "L" else s - 1.0
    M1 = O.assemble_pairwise(V, F, kind, sigma)
    M2 = O.operator_matrix(V, F, kind)
    assert np.abs(M1 - M2).max() <= 1e-12 * np.abs(M1).max()


@pytest.mark.parametrize("op", ["A", "B", "B0", "L"])
def test_operator_nullspace_symmetry_psd(op):
    V, F = small_mesh("ico2", seed=6)
    M = O.operator_matrix(V, F, op)
    m = np.abs(M).max()
    assert np.abs(M @ np.ones(len(V))).max() < 1e-12 * m * len(V)
    assert np.abs(M - M.T).max() < 1e-12 * m
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.min() > -1e-12 * m
    assert np.sum(ev < 1e-10 * ev.max()) == 1        # only the constants


@pytest.mark.parametrize("op,expo", [("A", 2 - 2 * (5 / 3)), ("L", 2 * (5 / 3) - 2)])
def test_operator_scaling_and_rotation(op, expo):
    V, F = small_mesh("ico1", seed=8)
    u = np.random.default_rng(101).standard_normal((len(V), 3))
    y = O.apply_operator(V, F, u, op)
    lam = 1.9
    assert np.allclose(O.apply_operator(lam * V, F, u, op), lam ** expo * y, rtol=1e-11, atol=0)
    R = _rot(4)
    assert np.allclose(O.apply_operator(V @ R.T + 1.0, F, u, op), y, rtol=1e-11,
                       atol=1e-12 * np.abs(y).max())


def test_discrete_derivative_reproduces_linear_functions():
    # item of §3.2.1 read as the P1 gradient: for u_i = c . f_i the per-face
    # gradient is the tangential part (I - N N^T) c
    V, F = small_mesh("ico2", seed=1)
    c = np.array([0.3, -1.2, 2.0])
    Du = O.D_apply(V, F, (V @ c)[:, None])[:, :, 0]
    N = O.face_geometry(V, F)[1]
    expect = c[None, :] - (N @ c)[:, None] * N
    assert np.allclose(Du, expect, atol=1e-12)


# ---------------------------------------------------------------------------
# cotan Laplacian and Poisson solve (§5.2)
# ---------------------------------------------------------------------------

def test_cotan_flat_grid_is_five_point_stencil():
    n = 6
    xs, ys = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    V = np.stack([xs.ravel(), ys.ravel(), np.zeros(n * n)], 1)
    F = []
    for i in range(n - 1):
        for j in range(n - 1):
            a, b, c, d = i * n + j, (i + 1) * n + j, (i + 1) * n + j + 1, i * n + j + 1
            F += [[a, b, c], [a, c, d]]
    C = O.cotan_laplacian(V, np.array(F)).toarray()
    k = 2 * n + 2                                    # interior vertex (2,2)
    row = np.zeros(n * n)
    row[k] = 4
    for m in (k - 1, k + 1, k - n, k + n):
        row[m] = -1
    assert np.allclose(C[k], row, atol=1e-14)


def test_cotan_dirichlet_energy_identity():
    # u^T C u = sum_S a_S |grad u|_S|^2 (stiffness matrix of P1 elements)
    V, F = small_mesh("torus10x5", seed=3)
    C = O.cotan_laplacian(V, F)
    u = np.random.default_rng(0).standard_normal(len(V))
    a = O.face_geometry(V, F)[2]
    grad = O.D_apply(V, F, u[:, None])[:, :, 0]
    assert float(u @ (C @ u)) == pytest.approx(float(np.sum(a * np.sum(grad ** 2, 1))), rel=1e-12)
    assert np.abs(C @ np.ones(len(V))).max() < 1e-12


def test_poisson_solve_residual():
    V, F = small_mesh("ico2", seed=3)
    C = O.cotan_laplacian(V, F)
    b = O.project_mean_zero(np.random.default_rng(1).standard_normal((len(V), 3)))
    z = O.poisson_solve(C, b)
    assert np.abs(C @ z - b).max() < 1e-10 * np.abs(b).max()
    assert np.abs(z.mean(0)).max() < 1e-13


# ---------------------------------------------------------------------------
# constraints (§7.1)
# ---------------------------------------------------------------------------

def test_constraint_closed_forms():
    V, F = small_mesh("tetra")
    assert O.total_volume(V, F) == pytest.approx(8.0 / 3.0, rel=1e-14)
    assert O.total_area(V, F) == pytest.approx(4 * 2 * np.sqrt(3), rel=1e-14)
    V, F = small_mesh("octa")
    assert O.total_volume(V, F) == pytest.approx(4.0 / 3.0, rel=1e-14)
    assert O.total_area(V, F) == pytest.approx(4 * np.sqrt(3), rel=1e-14)


def test_constraint_gradients_central_differences():
    V, F = small_mesh("ico2", seed=12)
    ga, gv = O.area_gradient(V, F), O.volume_gradient(V, F)
    rng = np.random.default_rng(7)
    h = 1e-6
    for _ in range(5):
        dv = rng.standard_normal(V.shape)
        fa = (O.total_area(V + h * dv, F) - O.total_area(V - h * dv, F)) / (2 * h)
        fv = (O.total_volume(V + h * dv, F) - O.total_volume(V - h * dv, F)) / (2 * h)
        assert np.sum(ga * dv) == pytest.approx(fa, rel=1e-7)
        assert np.sum(gv * dv) == pytest.approx(fv, rel=1e-7)


# ---------------------------------------------------------------------------
# constrained step (§3.3, §5.3)
# ---------------------------------------------------------------------------

def test_saddle_and_schur_directions_agree():
    V, F = small_mesh("ico1", seed=5)
    x, g = O.descent_direction(V, F)
    xs, Z, S = O.schur_direction(V, F)
    assert np.abs(x - xs).max() < 1e-9 * np.abs(x).max()
    J = np.stack([O.area_gradient(V, F).ravel(), O.volume_gradient(V, F).ravel()])
    assert np.abs(J @ x.ravel()).max() < 1e-12 * np.abs(J).max() * np.abs(x).max() * len(V)
    assert np.abs(x.sum(0)).max() < 1e-12 * np.abs(x).max() * len(V)
    assert np.sum(g * x) < 0                       # descent


def test_step_decreases_energy_and_projects():
    V, F = small_mesh("ico2", seed=13)
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    r = O.precond_step(V, F, A0, V0)
    assert r["E1"] < r["E0"]
    f1 = V + r["tau"] * r["x"]
    before = np.abs(O.constraint_values(f1, F, A0, V0)).max()
    after = np.abs(O.constraint_values(r["f_new"], F, A0, V0)).max()
    assert after < 0.2 * before


def test_repeated_projection_converges_linearly():
    # §3.3.2: the correction may be repeated; with the Jacobian of f each
    # repeat shrinks the violation by a constant factor
    V, F = small_mesh("ico2", seed=8)
    A0, V0 = O.total_area(V, F), O.total_volume(V, F)
    viol = []
    for k in range(4):
        r = O.precond_step(V, F, A0, V0, fixed_tau=0.25, proj_iters=k)
        viol.append(np.abs(O.constraint_values(r["f_new"], F, A0, V0) / [A0, V0]).max())
    assert all(viol[i + 1] < 0.1 * viol[i] for i in range(3)), viol


def test_linked_tori_generator_gap():
    # the two tubes (r = 0.25) have centre lines at distance >= 1, so no
    # vertex of one torus comes closer than ~0.5 to the other's vertices
    V, F = linked_tori(40, 10, 1.0, 0.25, 1.0)
    n = len(V) // 2
    d = np.linalg.norm(V[:n, None, :] - V[None, n:, :], axis=-1)
    assert d.min() > 0.45


# ---------------------------------------------------------------------------
# mutation checks: plant a slip in the oracle, a pin must fail
# ---------------------------------------------------------------------------

def test_pin_catches_halved_area_adjoint(monkeypatch):
    V, F = small_mesh("ico1", seed=9)
    orig = O.face_adjoints

    def broken(f, faces, p=6.0, rows=None):
        gX, gN, ga = orig(f, faces, p, rows)
        return gX, gN, 0.5 * ga             # drop the reverse half of dE/da
    monkeypatch.setattr(O, "face_adjoints", broken)
    g = O.differential(V, F)
    dv = np.random.default_rng(0).standard_normal(V.shape)
    h = 1e-6
    fd = (O.energy(V + h * dv, F) - O.energy(V - h * dv, F)) / (2 * h)
    assert abs(np.sum(g * dv) - fd) > 1e-3 * abs(fd)


def test_pin_catches_wrong_kernel_exponent():
    V, F = small_mesh("ico1", seed=2)
    s = O.sobolev_s(6.0)
    M1 = O.assemble_pairwise(V, F, "B", s - 1.0 + 0.1)      # wrong sigma
    M2 = O.operator_matrix(V, F, "B")
    assert np.abs(M1 - M2).max() > 1e-3 * np.abs(M2).max()


def test_pin_catches_transposed_low_order_kernel(monkeypatch):
    # using k_2(X_S,P_S;X_T) twice instead of the symmetrised pair breaks the
    # symmetry pin
    V, F = small_mesh("ico1", seed=3)
    orig = O._kernel_rows

    def broken(X, N, S, kind, expo):
        if kind != "low":
            return orig(X, N, S, kind, expo)
        nf = len(X)
        d = X[S, None, :] - X[None, :, :]
        r2 = np.sum(d * d, axis=-1)
        self_pair = S[:, None] == np.arange(nf)[None, :]
        r2 = np.where(self_pair, 1.0, r2)
        uS = np.einsum("sk,stk->st", N[S], d)
        h = r2 ** (-0.5 * expo) * (2 * uS * uS) / (2.0 * r2 * r2)
        return np.where(self_pair, 0.0, h)
    monkeypatch.setattr(O, "_kernel_rows", broken)
    M = O.operator_matrix(V, F, "B0")
    assert np.abs(M - M.T).max() > 1e-6 * np.abs(M).max()


@pytest.mark.parametrize("op", ["A", "B", "B0", "L"])
def test_sampled_operator_rows_match_full(op):
    V, F = small_mesh("torus10x5", seed=4)
    u = np.random.default_rng(3).standard_normal((len(V), 3))
    y = O.apply_operator(V, F, u, op)
    idx = [0, 11, 27, len(V) - 1]
    assert np.allclose(O.apply_operator_at_vertices(V, F, u, op, idx), y[idx], rtol=1e-12,
                       atol=1e-12 * np.abs(y).max())
