"""FP64 CPU oracle for the tangent-point surface-flow hot path.

TEST INFRASTRUCTURE ONLY. This module is the plain, slow, obviously correct
restatement of what the GPU library computes. Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import it; the library never
does, and it never imports the library.

Every function cites the passage of "Repulsive Surfaces" (Yu, Brakensiek,
Schumacher, Crane 2021) it follows. Equations are numbered in order of
appearance: Eq. 9 discrete kernel, Eq. 10 discrete energy, Eq. 11 pairwise
L^sigma entries, Eq. 12/13 high/low-order summands, Eq. 14 saddle problem,
Eq. 15 projection saddle problem, Eq. 16 Barnes-Hut energy, Eq. 17 Schur
complement, Eq. 18 projected direction, Eq. 19 Schur correction.

Conventions: positions f are float64 [nv,3]; faces int [nf,3] counter-
clockwise; all arithmetic is float64; pair sums run over ordered pairs
S != T (the diagonal term is 0/0 and is excluded, as in the (1 - delta_ST)
factor of the kernel matrices of §5.1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

CHUNK = 256


# ---------------------------------------------------------------------------
# §3.1 face geometry
# ---------------------------------------------------------------------------

def face_geometry(f, faces):
    """Barycenter X_S, unit normal N_S and area a_S of every face (§3.1:
    barycenters and areas of Eq. 9/10; the normal projector is P_S = N_S N_S^T,
    §2.1)."""
    fi, fj, fk = f[faces[:, 0]], f[faces[:, 1]], f[faces[:, 2]]
    X = (fi + fj + fk) / 3.0
    n = np.cross(fj - fi, fk - fi)
    nn = np.linalg.norm(n, axis=1)
    return X, n / nn[:, None], 0.5 * nn


def sobolev_s(p, n=2):
    """Sobolev order s = 2 - n/p of the energy (§2.3)."""
    return 2.0 - n / p


# ---------------------------------------------------------------------------
# §3.1 discrete energy, Eq. 9 and Eq. 10
# ---------------------------------------------------------------------------

def tp_kernel(X, N, Y, p):
    """K_p(X, P; Y) = |P (X - Y)|^p / |X - Y|^{2p} with P = N N^T (Eq. 9, and
    its rewriting in §4.1). Broadcasts over leading axes."""
    d = X - Y
    r2 = np.sum(d * d, axis=-1)
    u = np.abs(np.sum(N * d, axis=-1))
    return u ** p / r2 ** p


def energy_rows(f, faces, p=6.0, targets=None):
    """Row sums E_S = sum_{T != S} K(S,T) a_S a_T of Eq. 10 for the given
    target faces (all by default)."""
    X, N, a = face_geometry(f, faces)
    nf = len(faces)
    targets = np.arange(nf) if targets is None else np.asarray(targets)
    out = np.empty(len(targets))
    for c0 in range(0, len(targets), CHUNK):
        S = targets[c0:c0 + CHUNK]
        d = X[S, None, :] - X[None, :, :]
        r2 = np.sum(d * d, axis=-1)
        self_pair = S[:, None] == np.arange(nf)[None, :]
        r2 = np.where(self_pair, 1.0, r2)
        u = np.abs(np.einsum("sk,stk->st", N[S], d))
        K = np.where(self_pair, 0.0, u ** p / r2 ** p)
        out[c0:c0 + CHUNK] = a[S] * (K @ a)
    return out


def energy(f, faces, p=6.0):
    """Discrete tangent-point energy, Eq. 10, ordered pairs S != T."""
    return float(np.sum(energy_rows(f, faces, p)))


# ---------------------------------------------------------------------------
# §3.1 differential (chain rule through X_S, N_S, a_S)
# ---------------------------------------------------------------------------

def face_adjoints(f, faces, p=6.0, rows=None):
    """Per-face partial derivatives of Eq. 10 with respect to the face data:
    gX = dE/dX_S, gN = dE/dN_S (N_S treated as a free vector), ga = dE/da_S.

    Face S enters Eq. 10 twice: as the first argument of K(S,T) (its
    barycenter, normal and area) and as the second argument of K(T,S) (its
    barycenter and area). With d = X_S - X_T, u = N.d and
    K = |u|^p / |d|^{2p}:
        dK/dd = p |u|^{p-2} u |d|^{-2p} N - 2 p K d / |d|^2,
        dK/dN = p |u|^{p-2} u |d|^{-2p} d.
    """
    X, N, a = face_geometry(f, faces)
    nf = len(faces)
    rows = np.arange(nf) if rows is None else np.asarray(rows)
    gX = np.zeros((len(rows), 3))
    gN = np.zeros((len(rows), 3))
    ga = np.zeros(len(rows))
    for c0 in range(0, len(rows), CHUNK):
        S = rows[c0:c0 + CHUNK]
        d = X[S, None, :] - X[None, :, :]                 # d_ST = X_S - X_T
        r2 = np.sum(d * d, axis=-1)
        self_pair = S[:, None] == np.arange(nf)[None, :]
        r2 = np.where(self_pair, 1.0, r2)
        w = np.where(self_pair, 0.0, 1.0)
        uS = np.einsum("sk,stk->st", N[S], d)             # N_S . d_ST
        uT = np.einsum("tk,stk->st", N, d)                # N_T . d_ST
        r2p = r2 ** p
        KST = w * np.abs(uS) ** p / r2p
        KTS = w * np.abs(uT) ** p / r2p
        cS = w * p * np.abs(uS) ** (p - 2.0) * uS / r2p   # p|u|^{p-2}u/|d|^{2p}
        cT = w * p * np.abs(uT) ** (p - 2.0) * uT / r2p
        aT = a[None, :]
        # forward role: E_ST = K(S,T) a_S a_T, derivative wrt X_S is +dK/dd
        fwd = cS[..., None] * N[S][:, None, :] - (2.0 * p * KST / r2)[..., None] * d
        # reverse role: E_TS = K(T,S) a_T a_S with d_TS = -d_ST and normal N_T;
        # derivative wrt X_S is -dK/dd(d_TS) = cT N_T - 2p K(T,S) d_ST/|d|^2
        rev = cT[..., None] * N[None, :, :] - (2.0 * p * KTS / r2)[..., None] * d
        gX[c0:c0 + CHUNK] = a[S][:, None] * np.einsum("st,stk->sk", aT, fwd + rev)
        gN[c0:c0 + CHUNK] = a[S][:, None] * np.einsum("st,stk->sk", aT * cS, d)
        ga[c0:c0 + CHUNK] = (KST + KTS) @ a
    return gX, gN, ga


def faces_to_vertices(f, faces, gX, gN, ga, rows=None):
    """Chain rule from face adjoints to vertex positions (§3.1).

    X = (f_i+f_j+f_k)/3; n = (f_j-f_i) x (f_k-f_i); a = |n|/2; N = n/|n|.
    dN = (I - N N^T) dn / |n|, da = N.dn / 2, so gN.dN + ga da = w.dn with
    w = (I - N N^T) gN / |n| + ga N / 2, and dn = de1 x e2 + e1 x de2.
    Returns the per-face corner gradients [nf,3,3] (rows: corners i,j,k).
    """
    F = faces if rows is None else faces[rows]
    fi, fj, fk = f[F[:, 0]], f[F[:, 1]], f[F[:, 2]]
    e1, e2 = fj - fi, fk - fi
    n = np.cross(e1, e2)
    nn = np.linalg.norm(n, axis=1)
    N = n / nn[:, None]
    tang = gN - np.sum(gN * N, axis=1, keepdims=True) * N
    w = tang / nn[:, None] + 0.5 * ga[:, None] * N
    gj = np.cross(e2, w)
    gk = np.cross(w, e1)
    gi = -(gj + gk)
    third = gX / 3.0
    return np.stack([gi + third, gj + third, gk + third], axis=1)


def differential(f, faces, p=6.0):
    """dE/df of Eq. 10, shape [nv,3]."""
    gX, gN, ga = face_adjoints(f, faces, p)
    corner = faces_to_vertices(f, faces, gX, gN, ga)
    out = np.zeros_like(f)
    for c in range(3):
        np.add.at(out, faces[:, c], corner[:, c])
    return out


def differential_at_vertices(f, faces, verts, p=6.0):
    """dE/df_v for a sample of vertices v, computed from the adjoints of the
    faces incident to v only (for checks at sizes where the full sum is too
    slow)."""
    verts = np.asarray(verts)
    out = np.zeros((len(verts), 3))
    inc = [np.nonzero(np.any(faces == v, axis=1))[0] for v in verts]
    rows = np.unique(np.concatenate(inc))
    gX, gN, ga = face_adjoints(f, faces, p, rows)
    corner = faces_to_vertices(f, faces, gX, gN, ga, rows)
    pos = {int(r): i for i, r in enumerate(rows)}
    for vi, v in enumerate(verts):
        for S in inc[vi]:
            c = int(np.nonzero(faces[S] == v)[0][0])
            out[vi] += corner[pos[int(S)], c]
    return out


# ---------------------------------------------------------------------------
# §3.2 discrete inner product: hat averages, discrete derivative D
# ---------------------------------------------------------------------------

def hat_average_matrix(faces, nv):
    """F x V sparse matrix of bar-phi_i(S) = 1/3 if i is a vertex of S (§3.2)."""
    nf = len(faces)
    rows = np.repeat(np.arange(nf), 3)
    return sp.csr_matrix((np.full(3 * nf, 1.0 / 3.0), (rows, faces.reshape(-1))),
                         shape=(nf, nv))


def hat_gradients(f, faces):
    """Gradient of the hat function of each corner inside each face (the
    discrete derivative D of §3.2.1, read as the piecewise-linear gradient):
    grad phi_i |_S = N_S x e_i / (2 a_S), e_i the edge opposite corner i taken
    counter-clockwise. Returns [nf, 3 corners, 3]."""
    fi, fj, fk = f[faces[:, 0]], f[faces[:, 1]], f[faces[:, 2]]
    X, N, a = face_geometry(f, faces)
    e = np.stack([fk - fj, fi - fk, fj - fi], axis=1)
    return np.cross(N[:, None, :], e) / (2.0 * a)[:, None, None]


def D_apply(f, faces, v):
    """(D v)(S) = sum_{i in S} v_i grad phi_i|_S; v [nv,k] -> [nf,3,k]."""
    G = hat_gradients(f, faces)
    return np.einsum("sci,sck->sik", G, v[faces])


def D_transpose(f, faces, z, nv):
    """D^T: per-face 3-vectors z [nf,3,k] -> vertices [nv,k]."""
    G = hat_gradients(f, faces)
    out = np.zeros((nv, z.shape[2]))
    for c in range(3):
        np.add.at(out, faces[:, c], np.einsum("si,sik->sk", G[:, c, :], z))
    return out


# ---------------------------------------------------------------------------
# Algorithm 1 / Eq. 11-13: pairwise assembly of L^sigma, B, B0 (small meshes)
# ---------------------------------------------------------------------------

def assemble_pairwise(f, faces, kind, sigma, p=6.0):
    """Dense |V|x|V| matrix by the pair loop of Algorithm 1 over ordered
    distinct face pairs, with the summand of Eq. 11 (kind='L'), Eq. 12
    ('B', vector-valued D phi differences) or Eq. 13 ('B0', extra factor
    K_{f,2}(S,T)). The kernel denominator is |X_S - X_T|^{2 sigma + 2}."""
    nv, nf = len(f), len(faces)
    X, N, a = face_geometry(f, faces)
    G = hat_gradients(f, faces)
    M = np.zeros((nv, nv))
    S, T = np.nonzero(~np.eye(nf, dtype=bool))
    d = X[S] - X[T]
    r2 = np.sum(d * d, axis=1)
    w = a[S] * a[T] / r2 ** (sigma + 1.0)
    if kind == "B0":
        w = w * tp_kernel(X[S], N[S], X[T], 2.0)
    idx = np.concatenate([faces[S], faces[T]], axis=1)          # [npairs, 6]
    if kind in ("L", "B0"):
        c = np.concatenate([np.full((len(S), 3), 1.0 / 3.0),
                            np.full((len(S), 3), -1.0 / 3.0)], axis=1)
        val = w[:, None, None] * c[:, :, None] * c[:, None, :]
    elif kind == "B":
        c = np.concatenate([G[S], -G[T]], axis=1)                # [npairs, 6, 3]
        val = w[:, None, None] * np.einsum("pak,pbk->pab", c, c)
    else:
        raise ValueError(kind)
    np.add.at(M, (np.repeat(idx, 6, axis=1).reshape(-1), np.tile(idx, (1, 6)).reshape(-1)),
              val.reshape(-1))
    return M


# ---------------------------------------------------------------------------
# §5.1.1-5.1.3 and Appendix A: kernel-matrix form of the operators
# ---------------------------------------------------------------------------

def _kernel_rows(X, N, S, kind, expo):
    """Rows S of a kernel matrix H_ST = (1 - delta_ST) h(X_S, P_S; X_T, P_T)
    with |d|^{-expo} singular part; kind 'plain' or 'low' (the symmetrised
    k_2 factor of §5.1.3)."""
    nf = len(X)
    d = X[S, None, :] - X[None, :, :]
    r2 = np.sum(d * d, axis=-1)
    self_pair = S[:, None] == np.arange(nf)[None, :]
    r2 = np.where(self_pair, 1.0, r2)
    h = r2 ** (-0.5 * expo)
    if kind == "low":
        uS = np.einsum("sk,stk->st", N[S], d)
        uT = np.einsum("tk,stk->st", N, d)
        h = h * (uS * uS + uT * uT) / (2.0 * r2 * r2)
    return np.where(self_pair, 0.0, h)


def kernel_apply(X, N, a, W, kind, expo):
    """z = [diag(diag(a)^-1 H a) - H] W for a per-face block W [nf, m]."""
    nf = len(X)
    z = np.empty_like(W)
    for c0 in range(0, nf, CHUNK):
        S = np.arange(c0, min(nf, c0 + CHUNK))
        H = _kernel_rows(X, N, S, kind, expo)
        r = (H @ a) / a[S]
        z[S] = r[:, None] * W[S] - H @ W
    return z


def apply_operator(f, faces, v, op, p=6.0):
    """y = O v for v [nv,k] (each column separately, i.e. O_3 on k columns).

    op 'B'    high-order term, §5.1.2: 2 V^T [..] V v, V = diag(a) D,
              kernel |d|^{-2s};
    op 'B0'   low-order term, §5.1.3 (read with the face-average map U):
              kernel (k_2(X,P;Y) + k_2(Y,Q;X)) / (2 |d|^{2s});
    op 'A'    B + B0 (§2.4);
    op 'L'    L^{2-s} of the preconditioner (§5.2), §5.1.1 with
              sigma = 2 - s, kernel |d|^{-(2 sigma + 2)}.
    """
    nv = len(f)
    X, N, a = face_geometry(f, faces)
    s = sobolev_s(p)
    Ubar = hat_average_matrix(faces, nv)
    y = np.zeros_like(v)
    if op in ("B", "A"):
        W = a[:, None, None] * D_apply(f, faces, v)                 # V v, [nf,3,k]
        nk = v.shape[1]
        z = kernel_apply(X, N, a, W.reshape(len(faces), 3 * nk), "plain", 2.0 * s)
        y += 2.0 * D_transpose(f, faces, a[:, None, None] * z.reshape(-1, 3, nk), nv)
    if op in ("B0", "A"):
        W = a[:, None] * (Ubar @ v)                                 # U v
        z = kernel_apply(X, N, a, W, "low", 2.0 * s)
        y += 2.0 * (Ubar.T @ (a[:, None] * z))
    if op == "L":
        sigma = 2.0 - s
        W = a[:, None] * (Ubar @ v)
        z = kernel_apply(X, N, a, W, "plain", 2.0 * sigma + 2.0)
        y += 2.0 * (Ubar.T @ (a[:, None] * z))
    return y


def operator_matrix(f, faces, op, p=6.0):
    """Dense |V|x|V| matrix of apply_operator (columns = applies to unit
    vectors), for small meshes."""
    nv = len(f)
    return apply_operator(f, faces, np.eye(nv), op, p)


# ---------------------------------------------------------------------------
# §5.2 preconditioner: cotan Laplacian, Poisson solves, L^{2-s}
# ---------------------------------------------------------------------------

def cotan_laplacian(f, faces):
    """Weak (stiffness) cotan Laplacian C of the mesh (§5.2): C_ij =
    -1/2 (cot alpha_ij + cot beta_ij) for edges, C_ii = -sum_j C_ij."""
    nv = len(f)
    I, J, W = [], [], []
    for c in range(3):
        i, j, k = faces[:, c], faces[:, (c + 1) % 3], faces[:, (c + 2) % 3]
        u, w = f[i] - f[k], f[j] - f[k]
        cot = np.sum(u * w, axis=1) / np.linalg.norm(np.cross(u, w), axis=1)
        I += [i, j]
        J += [j, i]
        W += [-0.5 * cot, -0.5 * cot]
    I, J, W = np.concatenate(I), np.concatenate(J), np.concatenate(W)
    off = sp.csr_matrix((W, (I, J)), shape=(nv, nv))
    diag = -np.asarray(off.sum(axis=1)).ravel()
    return (off + sp.diags(diag)).tocsr()


def mesh_components(nv, faces):
    """Connected component of every vertex (through the face edges)."""
    from scipy.sparse.csgraph import connected_components
    I = np.concatenate([faces[:, 0], faces[:, 1], faces[:, 2]])
    J = np.concatenate([faces[:, 1], faces[:, 2], faces[:, 0]])
    adj = sp.csr_matrix((np.ones(len(I)), (I, J)), shape=(nv, nv))
    return connected_components(adj, directed=False)[1]


def project_mean_zero(b, comp=None):
    """Remove the constant component of each column (the nullspace of C and
    of the fractional operators); with `comp` (component labels) the mean
    of each connected component separately (the nullspace of C)."""
    if comp is None:
        return b - b.mean(axis=0, keepdims=True)
    out = b.copy()
    for c in np.unique(comp):
        sel = comp == c
        out[sel] -= out[sel].mean(axis=0, keepdims=True)
    return out


def poisson_solve(C, b, comp=None):
    """Solve C z = b in the mean-zero subspace (exact sparse direct solve:
    the system with the first vertex's row and column removed, then the
    mean removed); with `comp`, per connected component (one vertex of each
    component removed, means per component). b [nv,k]."""
    nv = C.shape[0]
    if comp is None:
        comp = np.zeros(nv, dtype=np.int64)
    b = project_mean_zero(b, comp)
    drop = np.array([np.nonzero(comp == c)[0][0] for c in np.unique(comp)])
    keep = np.setdiff1d(np.arange(nv), drop)
    Cr = C[keep][:, keep].tocsc()
    z = np.zeros_like(b)
    lu = spla.splu(Cr)
    for c in range(b.shape[1]):
        z[keep, c] = lu.solve(b[keep, c])
    return project_mean_zero(z, comp)


def pinned_poisson_solve(C, b, pins):
    """Poisson solve with vertex pins appended to the Laplacian (§7.2: the
    pin rows and columns added to the integer Laplacian): the first block of
    the solution of [C S^T; S 0][z; mu] = [b; 0], S the rows of the identity
    at the pinned vertices (one pin fixes all three coordinates, and the
    three coordinates are independent columns of b). b [nv,k]."""
    nv = C.shape[0]
    pins = np.asarray(pins)
    S = sp.csr_matrix((np.ones(len(pins)), (np.arange(len(pins)), pins)), shape=(len(pins), nv))
    K = sp.bmat([[C, S.T], [S, None]]).tocsc()
    lu = spla.splu(K)
    z = np.zeros_like(b)
    for c in range(b.shape[1]):
        rhs = np.concatenate([b[:, c], np.zeros(len(pins))])
        z[:, c] = lu.solve(rhs)[:nv]
    return z


PREC_SELF_WEIGHT = 24.0


def self_term_stiffness(f, faces, sigma, kappa):
    """Within-face term of the L^sigma double integral that the pairwise
    discretization of §5.1.1 (ordered pairs S != T, face averages) leaves
    out. For a piecewise-linear u the pairs (x, y) inside one face S give
    int_{SxS} (grad u . (x - y))^2 / |x - y|^{2 sigma + 2}, which is
    |grad u_S|^2 times a constant times a_S^{2 - sigma}; summed over the faces
    this is the P1 stiffness matrix with face weights w_S = kappa a_S^{1-sigma}:
        G_ij = sum_S w_S a_S grad phi_i . grad phi_j
    (the cotan matrix of the face-weighted cotangents). kappa is a design
    constant of the preconditioner."""
    nv = len(f)
    X, N, a = face_geometry(f, faces)
    G = hat_gradients(f, faces)
    w = kappa * a ** (1.0 - sigma)
    I, J, Wv = [], [], []
    for i in range(3):
        for j in range(3):
            I.append(faces[:, i])
            J.append(faces[:, j])
            Wv.append(w * a * np.sum(G[:, i] * G[:, j], axis=1))
    return sp.csr_matrix((np.concatenate(Wv), (np.concatenate(I), np.concatenate(J))), shape=(nv, nv))


def precond_apply(f, faces, b, p=6.0, pins=None, self_weight=PREC_SELF_WEIGHT):
    """Preconditioner of §5.2: C^+ L^{2-s} C^+ b (the two integer Laplacians
    are the cotan stiffness matrix; all vectors kept mean-zero). The forward
    fractional operator is L^{2-s} plus its within-face term
    (self_term_stiffness, weight self_weight; 0 gives L^{2-s} of §5.1.1
    alone). With vertex pins (§7.2) the pin rows are appended to both
    Laplacian solves (pinned_poisson_solve) and nothing is projected: the
    pins remove the nullspace."""
    C = cotan_laplacian(f, faces)
    comp = mesh_components(len(f), faces)
    sigma = 2.0 - sobolev_s(p)
    G = self_term_stiffness(f, faces, sigma, self_weight) if self_weight else None

    def middle(z):
        y = apply_operator(f, faces, z, "L", p)
        return y + G @ z if G is not None else y

    if pins is not None and len(pins):
        z = pinned_poisson_solve(C, b, pins)
        return pinned_poisson_solve(C, middle(z), pins)
    z = poisson_solve(C, b, comp)
    z = project_mean_zero(middle(z), comp)
    return poisson_solve(C, z, comp)


# ---------------------------------------------------------------------------
# §7.1 constraints
# ---------------------------------------------------------------------------

def total_area(f, faces):
    """sum_T a_f(T) (§7.1.3)."""
    return float(np.sum(face_geometry(f, faces)[2]))


def area_gradient(f, faces):
    """d(total area)/df_i = 1/2 sum_{S ni i} N_S x e_i (§7.1.3)."""
    fi, fj, fk = f[faces[:, 0]], f[faces[:, 1]], f[faces[:, 2]]
    N = face_geometry(f, faces)[1]
    out = np.zeros_like(f)
    for c, e in enumerate((fk - fj, fi - fk, fj - fi)):
        np.add.at(out, faces[:, c], 0.5 * np.cross(N, e))
    return out


def total_volume(f, faces):
    """(1/6) sum_{ijk} f_i . (f_j x f_k) (§7.1.4)."""
    fi, fj, fk = f[faces[:, 0]], f[faces[:, 1]], f[faces[:, 2]]
    return float(np.sum(fi * np.cross(fj, fk)) / 6.0)


def volume_gradient(f, faces):
    """d(volume)/df_i = (1/6) sum_{(i,j,k) in F} f_j x f_k (§7.1.4)."""
    out = np.zeros_like(f)
    for c in range(3):
        i, j, k = faces[:, c], faces[:, (c + 1) % 3], faces[:, (c + 2) % 3]
        np.add.at(out, i, np.cross(f[j], f[k]) / 6.0)
    return out


# ---------------------------------------------------------------------------
# §3.3 and §5.3: constrained descent direction, line search, projection
# ---------------------------------------------------------------------------

def _constraint_rows(f, faces, use_area, use_volume):
    rows = []
    if use_area:
        rows.append(area_gradient(f, faces).reshape(-1))
    if use_volume:
        rows.append(volume_gradient(f, faces).reshape(-1))
    if not rows:
        return np.zeros((0, 3 * len(f)))
    return np.array(rows)


def _barycenter_rows(nv, comp=None):
    """Jacobian of the fixed-barycenter constraint read as |V| copies of I_3
    (§7.1.1), one row per coordinate, in the [nv,3] row-major ordering; with
    several components, one barycenter per component (3 rows each, copies of
    I_3 over that component's vertices)."""
    if comp is None:
        comp = np.zeros(nv, dtype=np.int64)
    labels = np.unique(comp)
    J = np.zeros((3 * len(labels), 3 * nv))
    for k, lab in enumerate(labels):
        vs = np.nonzero(comp == lab)[0]
        for c in range(3):
            J[3 * k + c, 3 * vs + c] = 1.0
    return J


def _pin_rows(nv, pins):
    """Jacobian of the vertex pins Phi_P(f) = f(i) - f_0(i) (§7.1.2): per
    pinned vertex, a copy of I_3 in the block of that vertex."""
    J = np.zeros((3 * len(pins), 3 * nv))
    for k, i in enumerate(pins):
        for c in range(3):
            J[3 * k + c, 3 * i + c] = 1.0
    return J


def _positional_rows(nv, pins, comp=None):
    """The linear positional rows of the step: the barycenter rows (per
    component), or the pin rows when pins are given (a pin removes the
    nullspace, so the barycenter constraint is then not needed, §7.1.2)."""
    if pins is not None and len(pins):
        return _pin_rows(nv, pins)
    return _barycenter_rows(nv, comp)


def saddle_matrix(f, faces, use_area=True, use_volume=True, p=6.0, pins=None, willmore=0.0):
    """[A_3 dPhi^T; dPhi 0] of Eq. 14 with the barycenter rows (§7.1.1), or
    the vertex pin rows (§7.1.2, included in the matrix as in §7.2), plus
    area and volume rows; A_3 = A (x) I_3 on the [nv,3] ordering. With a
    Willmore weight w, w C M^{-1} C is added to A (the H^2 term of §7.3.5)."""
    nv = len(f)
    A = operator_matrix(f, faces, "A", p)
    if willmore:
        A = A + willmore * willmore_metric(f, faces)
    A3 = np.kron(A, np.eye(3))
    J = np.concatenate([_positional_rows(nv, pins, mesh_components(nv, faces)),
                        _constraint_rows(f, faces, use_area, use_volume)], axis=0)
    m = J.shape[0]
    M = np.zeros((3 * nv + m, 3 * nv + m))
    M[:3 * nv, :3 * nv] = A3
    M[:3 * nv, 3 * nv:] = J.T
    M[3 * nv:, :3 * nv] = J
    return M, J


def _total_energy(f, faces, p, obstacle, willmore=0.0):
    """E of Eq. 10 plus, when `obstacle` = (f_O, faces_O, weight) is given,
    the static-obstacle term of §7.3.2 (obstacle_energy), plus willmore
    times the Willmore energy of §7.3.5."""
    E = energy(f, faces, p)
    if obstacle is not None:
        E += obstacle_energy(f, faces, obstacle[0], obstacle[1], p, obstacle[2])
    if willmore:
        E += willmore * willmore_energy(f, faces)
    return E


def _total_differential(f, faces, p, obstacle, willmore=0.0):
    g = differential(f, faces, p)
    if obstacle is not None:
        g = g + obstacle_differential(f, faces, obstacle[0], obstacle[1], p, obstacle[2])
    if willmore:
        g = g + willmore * willmore_differential(f, faces)
    return g


def descent_direction(f, faces, use_area=True, use_volume=True, p=6.0, obstacle=None, pins=None,
                      willmore=0.0):
    """x of Eq. 14: [A_3 dPhi^T; dPhi 0][x; lambda] = [-dE; 0], solved
    densely. Returns (x [nv,3], g = dE [nv,3]). With an obstacle (see
    _total_energy) dE is the differential of the sum: the obstacle term is
    one more energy in the flow, the metric A is unchanged."""
    nv = len(f)
    g = _total_differential(f, faces, p, obstacle, willmore)
    M, J = saddle_matrix(f, faces, use_area, use_volume, p, pins, willmore)
    rhs = np.zeros(M.shape[0])
    rhs[:3 * nv] = -g.reshape(-1)
    sol = np.linalg.solve(M, rhs)
    return sol[:3 * nv].reshape(nv, 3), g


def schur_direction(f, faces, use_area=True, use_volume=True, p=6.0, pins=None):
    """The same direction via the Schur complement of §5.3 (Eq. 17, Eq. 18)
    with A_3^{-1} applied in the subspace of zero mean per component (where
    the barycenter rows are satisfied), g = dE, Z = A_3^{-1} dPhi^T:
        x = -(A^{-1} g - Z (dPhi Z)^{-1} dPhi A^{-1} g).
    With pins, the pin rows stay in the matrix (§7.2): A_3^{-1} is the solve
    of the pinned saddle system, i.e. A restricted to the free vertices with
    zero pinned rows, and only area and volume go through the Schur
    complement."""
    nv = len(f)
    g = differential(f, faces, p)
    A = operator_matrix(f, faces, "A", p)
    if pins is not None and len(pins):
        free = np.setdiff1d(np.arange(nv), np.asarray(pins))
        AFFi = np.linalg.inv(A[np.ix_(free, free)])

        def Ainv3(w):
            out = np.zeros((nv, 3))
            out[free] = AFFi @ w.reshape(nv, 3)[free]
            return out.reshape(-1)
    else:
        # inverse on the subspace of zero mean per component: P A P plus the
        # projector onto the constants is invertible and maps that subspace
        # to itself
        comp = mesh_components(nv, faces)
        P = project_mean_zero(np.eye(nv), comp)
        Ainv = np.linalg.inv(P @ A @ P + (np.eye(nv) - P))
        Ainv3 = lambda w: project_mean_zero(Ainv @ project_mean_zero(w.reshape(nv, 3), comp), comp).reshape(-1)
    J = _constraint_rows(f, faces, use_area, use_volume)
    Ag = Ainv3(g.reshape(-1))
    Z = np.stack([Ainv3(row) for row in J], axis=1)
    S = J @ Z                                   # -(M/A), Eq. 17
    x = -(Ag - Z @ np.linalg.solve(S, J @ Ag))
    return x.reshape(nv, 3), Z, S


def barycenter_motion(f, faces, g):
    """The translation added to the descent direction when the barycenter may
    float (the barycenter-motion option of §7.1.1): minus the average of the
    L^2 gradient g over the vertices, weighted by the vertex areas (the lumped
    mass), per connected component. Returns [nv,3]."""
    comp = mesh_components(len(f), faces)
    m = lumped_mass(f, faces)
    out = np.zeros_like(f)
    for c in np.unique(comp):
        sel = comp == c
        out[sel] = -(m[sel, None] * g[sel]).sum(axis=0) / m[sel].sum()
    return out


def constraint_values(f, faces, A0, V0, use_area=True, use_volume=True):
    vals = []
    if use_area:
        vals.append(total_area(f, faces) - A0)
    if use_volume:
        vals.append(total_volume(f, faces) - V0)
    return np.array(vals)


def precond_step(f, faces, A0, V0, use_area=True, use_volume=True, p=6.0,
                 tau0=1.0, armijo_c=1e-4, shrink=0.5, ls_max=30, fixed_tau=None, proj_iters=1,
                 obstacle=None, pins=None, willmore=0.0, free_barycenter=False, tau0_disp=0.0):
    """One constrained descent step (§3, steps 1-5; §5.4 with exact solves):
    direction by Eq. 14, Armijo backtracking from tau0 (E(f + tau x) <=
    E(f) + c tau dE.x), then corrective projections by Eq. 15 with the
    left-hand side of Eq. 14 (Jacobian at f) and Phi at the current point;
    §3.3.2 says one suffices and allows repeats (proj_iters). With
    `obstacle` = (f_O, faces_O, weight) the energy is E of Eq. 10 plus the
    static-obstacle term of §7.3.2. With `pins` (vertex indices) the pin rows
    replace the barycenter rows; the pinned positions f_0 are those of f, so
    Phi_P = 0 at the start and every row of the projection's right-hand side
    for a pin is 0. With a Willmore weight w the energy gains w E_W and the
    matrix w C M^{-1} C (§7.3.5). With free_barycenter the direction gains
    barycenter_motion (§7.1.1). With tau0_disp > 0 the line search starts
    from min(tau0, tau0_disp h / max_v |x_v|), h = sqrt(total area / #faces)
    (a first trial that moves no vertex by more than tau0_disp face sizes; the
    paper leaves the initial step open).
    Returns dict(f_new, x, tau, E0, E1, h)."""
    nv = len(f)
    x, g = descent_direction(f, faces, use_area, use_volume, p, obstacle, pins, willmore)
    if free_barycenter:
        x = x + barycenter_motion(f, faces, g)
    E0 = _total_energy(f, faces, p, obstacle, willmore)
    slope = float(np.sum(g * x))
    if fixed_tau is not None:
        tau = fixed_tau
    else:
        tau = tau0
        if tau0_disp > 0.0:
            h = np.sqrt(total_area(f, faces) / len(faces))
            xmax = float(np.sqrt(np.max(np.sum(x * x, axis=1))))
            if xmax > 0.0:
                tau = min(tau, tau0_disp * h / xmax)
        for _ in range(ls_max):
            if _total_energy(f + tau * x, faces, p, obstacle, willmore) <= E0 + armijo_c * tau * slope:
                break
            tau *= shrink
    f1 = f + tau * x
    M, J = saddle_matrix(f, faces, use_area, use_volume, p, pins, willmore)
    npos = _positional_rows(nv, pins, mesh_components(nv, faces)).shape[0]
    f2 = f1
    h = np.zeros_like(f)
    for _ in range(proj_iters):
        rhs = np.zeros(M.shape[0])
        if pins is not None and len(pins):
            rhs[3 * nv:3 * nv + npos] = -(f2[pins] - f[pins]).reshape(-1)
        rhs[3 * nv + npos:] = -constraint_values(f2, faces, A0, V0, use_area, use_volume)
        dh = np.linalg.solve(M, rhs)[:3 * nv].reshape(nv, 3)
        f2 = f2 + dh
        h = h + dh
    return dict(f_new=f2, x=x, tau=tau, E0=E0, E1=_total_energy(f2, faces, p, obstacle, willmore), h=h,
                slope=slope)


def apply_operator_at_vertices(f, faces, v, op, verts, p=6.0):
    """Rows y[verts] of apply_operator, with the kernel-matrix rows computed
    only for the faces incident to those vertices (for checks at sizes where
    the full product is too slow). Same formulas as apply_operator."""
    nv = len(f)
    verts = np.asarray(verts)
    X, N, a = face_geometry(f, faces)
    s = sobolev_s(p)
    G = hat_gradients(f, faces)
    vbar = (v[faces[:, 0]] + v[faces[:, 1]] + v[faces[:, 2]]) / 3.0        # [nf,k]
    inc = [np.nonzero(np.any(faces == u, axis=1))[0] for u in verts]
    rows = np.unique(np.concatenate(inc))
    pos = {int(r): i for i, r in enumerate(rows)}
    zV = zU = None
    if op in ("B", "A"):
        W = a[:, None, None] * D_apply(f, faces, v)
        Wf = W.reshape(len(faces), -1)
        H = _kernel_rows(X, N, rows, "plain", 2.0 * s)
        zV = (((H @ a) / a[rows])[:, None] * Wf[rows] - H @ Wf).reshape(len(rows), 3, -1)
    if op in ("B0", "A", "L"):
        W = a[:, None] * vbar
        if op == "L":
            H = _kernel_rows(X, N, rows, "plain", 2.0 * (2.0 - s) + 2.0)
        else:
            H = _kernel_rows(X, N, rows, "low", 2.0 * s)
        zU = ((H @ a) / a[rows])[:, None] * W[rows] - H @ W
    out = np.zeros((len(verts), v.shape[1]))
    for vi, u in enumerate(verts):
        for S in inc[vi]:
            c = int(np.nonzero(faces[S] == u)[0][0])
            r = pos[int(S)]
            if zV is not None:
                out[vi] += 2.0 * a[S] * np.einsum("i,ik->k", G[S, c], zV[r])
            if zU is not None:
                out[vi] += 2.0 * a[S] * zU[r] / 3.0
    return out


# ---------------------------------------------------------------------------
# §4 Barnes-Hut: BVH over the faces, approximate energy and differential
# ---------------------------------------------------------------------------
#
# Tree (the paper leaves the BVH construction open; this is the definition the
# library also uses): faces sorted by the 30-bit Morton code of their
# barycenter, measured in the frame of the vertex bounding-box centre and
# quantised to 1024 cells per axis over the barycenters' bounding box, ties
# by face index; leaves are runs of `leaf` consecutive sorted faces; a node
# over n leaves has a left child over ceil(n/2) leaves; nodes are numbered in
# pre-order. Node data: a_I = sum a_T, X_I = sum a_T X_T / a_I, the bounding
# box of the node's triangle vertices, and the radius r_I = max |v - X_I|
# over the vertices of the node's faces (§4.1: radius from the barycenter).
# Admissibility (§4.1, read with theta): max(r_S, r_I)^2 < theta^2 dist^2 of
# the two boxes, decided in FP32 like the kernel; an inadmissible leaf is
# summed exactly (T != S).

def _spread10(v):
    v = v.astype(np.uint64) & 0x3FF
    v = (v | (v << 16)) & 0x030000FF
    v = (v | (v << 8)) & 0x0300F00F
    v = (v | (v << 4)) & 0x030C30C3
    v = (v | (v << 2)) & 0x09249249
    return v


def bvh_build(f, faces, leaf=8, order=None):
    """Sorted face order, pre-order node table and node data (dict). With
    `order` given, that face order is kept and only the node data come from
    f (a refit of a tree built on other positions)."""
    X, N, a = face_geometry(f, faces)
    c = 0.5 * (f.min(axis=0) + f.max(axis=0))
    Xr = (f[faces[:, 0]] + f[faces[:, 1]] + f[faces[:, 2]]) / 3.0 - c
    lo, hi = Xr.min(axis=0), Xr.max(axis=0)
    ext = hi - lo
    q = np.zeros_like(Xr, dtype=np.int64)
    for k in range(3):
        if ext[k] > 0:
            q[:, k] = np.clip(np.floor((Xr[:, k] - lo[k]) * (1024.0 / ext[k])), 0, 1023).astype(np.int64)
    code = (_spread10(q[:, 0]) << 2) | (_spread10(q[:, 1]) << 1) | _spread10(q[:, 2])
    nf = len(faces)
    if order is None:
        order = np.lexsort((np.arange(nf), code))
    else:
        order = np.asarray(order)
    nleaf = (nf + leaf - 1) // leaf
    first, count, skip, isleaf, right = [], [], [], [], []

    def rec(lo_, hi_):
        nid = len(first)
        n = hi_ - lo_
        first.append(lo_ * leaf)
        count.append(min(hi_ * leaf, nf) - lo_ * leaf)
        skip.append(nid + 2 * n - 1)
        isleaf.append(n == 1)
        right.append(-1)
        if n > 1:
            nl = (n + 1) // 2
            rec(lo_, lo_ + nl)
            right[nid] = len(first)
            rec(lo_ + nl, hi_)
        return nid

    import sys
    sys.setrecursionlimit(max(10000, sys.getrecursionlimit()))
    rec(0, nleaf)
    first, count = np.array(first), np.array(count)
    nn = len(first)
    # node data, bottom-up: leaves from their faces, inner nodes from children
    isleaf = np.array(isleaf)
    right = np.array(right)
    vx = f[faces] - c                                   # [nf,3,3] vertices in the frame
    aI = np.zeros(nn)
    XI = np.zeros((nn, 3))
    box_lo = np.zeros((nn, 3))
    box_hi = np.zeros((nn, 3))
    rI = np.zeros(nn)
    lv = np.nonzero(isleaf)[0]
    for j in range(leaf):                               # leaves: sums over <= leaf faces
        ok = j < count[lv]
        T = order[np.minimum(first[lv] + j, nf - 1)]
        w = np.where(ok, a[T], 0.0)
        aI[lv] += w
        XI[lv] += w[:, None] * Xr[T]
    XI[lv] /= aI[lv][:, None]
    box_lo[lv], box_hi[lv] = np.inf, -np.inf
    for j in range(leaf):
        ok = j < count[lv]
        T = order[np.minimum(first[lv] + j, nf - 1)]
        v = vx[T]                                       # [nleaf,3,3]
        box_lo[lv] = np.where(ok[:, None], np.minimum(box_lo[lv], v.min(axis=1)), box_lo[lv])
        box_hi[lv] = np.where(ok[:, None], np.maximum(box_hi[lv], v.max(axis=1)), box_hi[lv])
        dist = np.sqrt(((v - XI[lv][:, None, :]) ** 2).sum(axis=2)).max(axis=1)
        rI[lv] = np.where(ok, np.maximum(rI[lv], dist), rI[lv])
    depth = np.zeros(nn, dtype=np.int64)
    inner = np.nonzero(~isleaf)[0]
    for nid in inner:                                   # pre-order: parents first
        depth[nid + 1] = depth[right[nid]] = depth[nid] + 1
    for d in range(depth.max(), -1, -1):
        ids = inner[depth[inner] == d]
        L, R = ids + 1, right[ids]
        aI[ids] = aI[L] + aI[R]
        XI[ids] = (aI[L][:, None] * XI[L] + aI[R][:, None] * XI[R]) / aI[ids][:, None]
        box_lo[ids] = np.minimum(box_lo[L], box_lo[R])
        box_hi[ids] = np.maximum(box_hi[L], box_hi[R])
    # exact radii of the inner nodes: max over the vertices of their faces
    for d in range(depth.max() + 1):
        ids = inner[depth[inner] == d]
        if len(ids) == 0:
            continue
        cnt = count[ids]
        starts = np.concatenate([[0], np.cumsum(cnt)[:-1]])       # segment starts
        seg = np.repeat(np.arange(len(ids)), cnt)                  # node of each entry
        fidx = np.repeat(first[ids] - starts, cnt) + np.arange(cnt.sum())   # sorted face positions
        v = vx[order[fidx]]                                        # [m,3,3]
        dist = np.sqrt(((v - XI[ids][seg][:, None, :]) ** 2).sum(axis=2)).max(axis=1)
        rI[ids] = np.maximum.reduceat(dist, starts)
    # target faces: their own boxes and radii
    fbox_lo, fbox_hi = vx.min(axis=1), vx.max(axis=1)
    fr2 = ((vx - Xr[:, None, :]) ** 2).sum(axis=2).max(axis=1)
    return dict(order=order, first=first, count=count, skip=np.array(skip), leaf=isleaf,
                right=right, a=aI, X=XI, lo=box_lo, hi=box_hi, r=rI, Xr=Xr, c=c,
                fbox_lo=fbox_lo, fbox_hi=fbox_hi, fr2=fr2)


def _admissible(T, S, nodes, theta):
    """FP32 admissibility of node(s) `nodes` for target face(s) S."""
    f32 = np.float32
    alo, ahi = T["fbox_lo"][S].astype(f32), T["fbox_hi"][S].astype(f32)
    nlo, nhi = T["lo"][nodes].astype(f32), T["hi"][nodes].astype(f32)
    g = np.maximum(np.maximum(nlo - ahi, alo - nhi), f32(0))
    d2 = (g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1]) + g[:, 2] * g[:, 2]
    mr2 = np.maximum(T["fr2"][S].astype(f32), (T["r"][nodes] * T["r"][nodes]).astype(f32))
    return mr2 < f32(theta * theta) * d2


def bh_interactions(f, faces, theta, leaf=8, targets=None, tree=None):
    """Interaction lists of Eq. 16: far (target face, node) pairs and near
    (target face, source face) pairs, by a breadth-first traversal of all
    targets at once."""
    T = tree if tree is not None else bvh_build(f, faces, leaf)
    nf = len(faces)
    S = np.arange(nf) if targets is None else np.asarray(targets)
    cur_s, cur_n = S.copy(), np.zeros(len(S), dtype=np.int64)
    far_s, far_n, near_s, near_t = [], [], [], []
    while len(cur_s):
        adm = _admissible(T, cur_s, cur_n, theta)
        far_s.append(cur_s[adm])
        far_n.append(cur_n[adm])
        rest_s, rest_n = cur_s[~adm], cur_n[~adm]
        lf = T["leaf"][rest_n]
        # inadmissible leaves: exact pairs with their faces
        ls, ln = rest_s[lf], rest_n[lf]
        for j in range(leaf):
            ok = j < T["count"][ln]
            src = T["order"][np.minimum(T["first"][ln] + j, nf - 1)]
            keep = ok & (src != ls)
            near_s.append(ls[keep])
            near_t.append(src[keep])
        # inner nodes: descend to both children
        is_, in_ = rest_s[~lf], rest_n[~lf]
        cur_s = np.concatenate([is_, is_])
        cur_n = np.concatenate([in_ + 1, T["right"][in_]])
    cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0, dtype=np.int64)
    return T, dict(far_s=cat(far_s), far_n=cat(far_n), near_s=cat(near_s), near_t=cat(near_t))


def bh_energy_rows(f, faces, theta, leaf=8, p=6.0, targets=None, order=None):
    """Rows of Eq. 16 for the given targets (all faces by default); `order`:
    the face order of a refit tree (see bvh_build)."""
    X, N, a = face_geometry(f, faces)
    tree = bvh_build(f, faces, leaf, order) if order is not None else None
    T, L = bh_interactions(f, faces, theta, leaf, targets, tree)
    Xr = T["Xr"]
    nf = len(faces)
    rows = np.zeros(nf)
    Kf = tp_kernel(Xr[L["far_s"]], N[L["far_s"]], T["X"][L["far_n"]], p)
    np.add.at(rows, L["far_s"], Kf * a[L["far_s"]] * T["a"][L["far_n"]])
    Kn = tp_kernel(Xr[L["near_s"]], N[L["near_s"]], Xr[L["near_t"]], p)
    np.add.at(rows, L["near_s"], Kn * a[L["near_s"]] * a[L["near_t"]])
    S = np.arange(nf) if targets is None else np.asarray(targets)
    return rows[S], len(L["far_s"]) + len(L["near_s"])


def bh_energy(f, faces, theta, leaf=8, p=6.0, order=None):
    rows, _ = bh_energy_rows(f, faces, theta, leaf, p, order=order)
    return float(rows.sum())


def bh_energy_frozen(f, faces, tree, lists, p=6.0):
    """Barnes-Hut energy of Eq. 16 at positions f with the tree membership and
    the interaction lists of another configuration held fixed (node areas and
    barycenters recomputed from f). Its gradient is the 'full' Barnes-Hut
    differential."""
    X, N, a = face_geometry(f, faces)
    c = tree["c"]
    Xr = X - c
    nn = len(tree["first"])
    aI = np.zeros(nn)
    XI = np.zeros((nn, 3))
    for nid in range(nn):
        Tf = tree["order"][tree["first"][nid]:tree["first"][nid] + tree["count"][nid]]
        aI[nid] = a[Tf].sum()
        XI[nid] = (a[Tf, None] * Xr[Tf]).sum(axis=0) / aI[nid]
    fs, fn, ns, nt = lists["far_s"], lists["far_n"], lists["near_s"], lists["near_t"]
    E = np.sum(tp_kernel(Xr[fs], N[fs], XI[fn], p) * a[fs] * aI[fn])
    E += np.sum(tp_kernel(Xr[ns], N[ns], Xr[nt], p) * a[ns] * a[nt])
    return float(E)


def bvh_node_sums(tree, vals):
    """Sums of per-face rows `vals` [nf, m] over each node's faces."""
    first, count = tree["first"], tree["count"]
    sv = np.asarray(vals)[tree["order"]]
    out = np.zeros((len(first),) + sv.shape[1:])
    for nid in range(len(first)):
        out[nid] = sv[first[nid]:first[nid] + count[nid]].sum(axis=0)
    return out


def bvh_average_projectors(f, faces, tree):
    """Node-average projectors P_I = a_I^-1 sum_{S in I} a_S N_S N_S^T (§5.1.4)."""
    X, N, a = face_geometry(f, faces)
    aP = a[:, None, None] * N[:, :, None] * N[:, None, :]
    return bvh_node_sums(tree, aP) / tree["a"][:, None, None]


def bh_kernel_apply(tree, lists, Xr, N, a, W, kind, expo, Pbar):
    """z = [diag(diag(a)^-1 H~ a) - H~] W, H~ the Barnes-Hut version of the
    kernel matrix of the operator applies (§5.1.1-5.1.3 with the per-target
    admissible sets of §4.1): a far pair (S, node I) contributes
    h(X_S, P_S; X_I, P_I) times the node sums of a and W, with the
    node-average projector P_I in the source-side k_2 (§5.1.4); a near pair
    (S, T) in an inadmissible leaf contributes the exact h(X_S, P_S; X_T, P_T)."""
    nf = len(Xr)
    aW = np.concatenate([a[:, None], W], axis=1)
    nodeS = bvh_node_sums(tree, aW)
    H = np.zeros_like(aW)

    def add(s, Y, Q, src):
        d = Xr[s] - Y
        r2 = np.sum(d * d, axis=1)
        h = r2 ** (-0.5 * expo)
        if kind == "low":
            uS = np.sum(N[s] * d, axis=1)
            Qd = np.einsum("nij,nj->ni", Q, d)
            h = h * (uS * uS + np.sum(Qd * Qd, axis=1)) / (2.0 * r2 * r2)
        np.add.at(H, s, h[:, None] * src)

    fs, fn, ns, nt = lists["far_s"], lists["far_n"], lists["near_s"], lists["near_t"]
    if len(fs):
        add(fs, tree["X"][fn], Pbar[fn], nodeS[fn])
    if len(ns):
        PT = N[nt][:, :, None] * N[nt][:, None, :]
        add(ns, Xr[nt], PT, aW[nt])
    return (H[:, 0] / a)[:, None] * W - H[:, 1:]


def bh_apply_operator(f, faces, v, op, theta, leaf=8, p=6.0):
    """Barnes-Hut version of apply_operator: the same assembly (Appendix A
    form) with every kernel-matrix product taken over the Barnes-Hut
    interaction lists of the energy (§4.1). theta = 0 gives apply_operator."""
    nv = len(f)
    nf = len(faces)
    X, N, a = face_geometry(f, faces)
    s = sobolev_s(p)
    T, L = bh_interactions(f, faces, theta, leaf)
    Xr = T["Xr"]
    Pbar = bvh_average_projectors(f, faces, T)
    Ubar = hat_average_matrix(faces, nv)
    y = np.zeros_like(v)
    if op in ("B", "A"):
        W = a[:, None, None] * D_apply(f, faces, v)
        nk = v.shape[1]
        z = bh_kernel_apply(T, L, Xr, N, a, W.reshape(nf, 3 * nk), "plain", 2.0 * s, Pbar)
        y += 2.0 * D_transpose(f, faces, a[:, None, None] * z.reshape(-1, 3, nk), nv)
    if op in ("B0", "A"):
        W = a[:, None] * (Ubar @ v)
        z = bh_kernel_apply(T, L, Xr, N, a, W, "low", 2.0 * s, Pbar)
        y += 2.0 * (Ubar.T @ (a[:, None] * z))
    if op == "L":
        sigma = 2.0 - s
        W = a[:, None] * (Ubar @ v)
        z = bh_kernel_apply(T, L, Xr, N, a, W, "plain", 2.0 * sigma + 2.0, Pbar)
        y += 2.0 * (Ubar.T @ (a[:, None] * z))
    return y


def bh_differential(f, faces, theta, leaf=8, p=6.0, mode="full"):
    """Barnes-Hut differential (§4.2), shape [nv,3].

    mode 'literal': only the terms where the face is the target S of an
    interaction (the formula printed in §4.2);
    mode 'full': the exact derivative of Eq. 16 with the interaction lists
    fixed -- the target-side terms plus the source-side terms, where a node's
    barycenter X_I = sum a_T X_T / a_I and area a_I = sum a_T pass the
    derivative on to the node's faces."""
    X, N, a = face_geometry(f, faces)
    T, L = bh_interactions(f, faces, theta, leaf)
    Xr = T["Xr"]
    nf = len(faces)
    gX = np.zeros((nf, 3))
    gN = np.zeros((nf, 3))
    ga = np.zeros(nf)

    def side(s, Y, wY):
        d = Xr[s] - Y
        r2 = np.sum(d * d, axis=1)
        u = np.sum(N[s] * d, axis=1)
        K = np.abs(u) ** p / r2 ** p
        cc = p * np.abs(u) ** (p - 2.0) * u / r2 ** p
        dKdd = cc[:, None] * N[s] - (2.0 * p * K / r2)[:, None] * d
        dKdN = cc[:, None] * d
        np.add.at(gX, s, (a[s] * wY)[:, None] * dKdd)
        np.add.at(gN, s, (a[s] * wY)[:, None] * dKdN)
        np.add.at(ga, s, K * wY)
        return -(a[s] * wY)[:, None] * dKdd, a[s] * K     # source side: d/dY, d/dwY

    GYf, QYf = side(L["far_s"], T["X"][L["far_n"]], T["a"][L["far_n"]])
    GYn, QYn = side(L["near_s"], Xr[L["near_t"]], a[L["near_t"]])
    if mode == "full":
        np.add.at(gX, L["near_t"], GYn)
        np.add.at(ga, L["near_t"], QYn)
        nn = len(T["first"])
        G = np.zeros((nn, 3))
        Q = np.zeros(nn)
        np.add.at(G, L["far_n"], GYf)
        np.add.at(Q, L["far_n"], QYf)
        for nid in np.nonzero(np.any(G != 0, axis=1) | (Q != 0))[0]:
            Tf = T["order"][T["first"][nid]:T["first"][nid] + T["count"][nid]]
            gX[Tf] += (a[Tf] / T["a"][nid])[:, None] * G[nid]
            ga[Tf] += Q[nid] + (Xr[Tf] - T["X"][nid]) @ G[nid] / T["a"][nid]
    elif mode != "literal":
        raise ValueError(mode)
    corner = faces_to_vertices(f, faces, gX, gN, ga)
    out = np.zeros_like(f)
    for cidx in range(3):
        np.add.at(out, faces[:, cidx], corner[:, cidx])
    return out


# ---------------------------------------------------------------------------
# §7.3.2 static obstacles
# ---------------------------------------------------------------------------

def obstacle_potential(x, fO, facesO, p=6.0, grad=False):
    """Potential of a static obstacle mesh at points x [m,3] (§7.3.2):
        E_obs(x) = sum_{S in F_O} |f_O(S) - x|^{-p} a_O(S),
    f_O(S) the barycenter and a_O(S) the area of obstacle face S (the face
    data of §3.1), p the tangent-point exponent. With grad=True also returns
        dE_obs/dx = p sum_S a_O(S) |f_O(S) - x|^{-p-2} (f_O(S) - x)   [m,3]."""
    Y, _, aO = face_geometry(fO, facesO)
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    phi = np.zeros(len(x))
    g = np.zeros((len(x), 3))
    step = max(1, 2 ** 22 // max(1, len(Y)))
    for i0 in range(0, len(x), step):
        d = Y[None, :, :] - x[i0:i0 + step, None, :]
        r2 = np.sum(d * d, axis=2)
        w = aO[None, :] * r2 ** (-0.5 * p)
        phi[i0:i0 + step] = w.sum(axis=1)
        if grad:
            g[i0:i0 + step] = p * np.einsum("ij,ijk->ik", w / r2, d)
    return (phi, g) if grad else phi


def obstacle_energy_rows(f, faces, fO, facesO, p=6.0, weight=1.0):
    """Per-face obstacle terms weight * a_T * E_obs(X_T). Reading: the
    potential E_obs of §7.3.2 is a density over the surface, integrated with
    the same one-point (barycenter) rule per face as Eq. 10, and scaled by
    a user weight."""
    X, _, a = face_geometry(f, faces)
    return weight * a * obstacle_potential(X, fO, facesO, p)


def obstacle_energy(f, faces, fO, facesO, p=6.0, weight=1.0):
    return float(obstacle_energy_rows(f, faces, fO, facesO, p, weight).sum())


def obstacle_differential(f, faces, fO, facesO, p=6.0, weight=1.0):
    """d/df of obstacle_energy, shape [nv,3]: face adjoints
    gX_T = weight a_T dE_obs/dx(X_T), ga_T = weight E_obs(X_T), gN_T = 0,
    through the chain rule of §3.1 (faces_to_vertices)."""
    X, _, a = face_geometry(f, faces)
    phi, g = obstacle_potential(X, fO, facesO, p, grad=True)
    gX = weight * a[:, None] * g
    ga = weight * phi
    corner = faces_to_vertices(f, faces, gX, np.zeros_like(gX), ga)
    out = np.zeros_like(f)
    for c in range(3):
        np.add.at(out, faces[:, c], corner[:, c])
    return out


def _admissible_point(T, xr, nodes, theta):
    """FP32 admissibility of node(s) for point target(s) xr (tree frame): the
    test of §4.1 with a point in place of the target face (radius 0, box the
    point itself)."""
    f32 = np.float32
    x = xr.astype(f32)
    nlo, nhi = T["lo"][nodes].astype(f32), T["hi"][nodes].astype(f32)
    g = np.maximum(np.maximum(nlo - x, x - nhi), f32(0))
    d2 = (g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1]) + g[:, 2] * g[:, 2]
    r2 = (T["r"][nodes] * T["r"][nodes]).astype(f32)
    return r2 < f32(theta * theta) * d2


def bh_obstacle_potential(x, fO, facesO, theta, leaf=8, p=6.0, grad=False):
    """Barnes-Hut approximation of obstacle_potential (§7.3.2 with §4.1): a
    BVH over the obstacle's faces; a node I admissible for x contributes
    a_I |X_I - x|^{-p} (X_I its area-weighted barycenter, a_I its area),
    inadmissible leaves are summed face by face. Returns (phi, g, count) with
    count the interactions evaluated."""
    T = bvh_build(fO, facesO, leaf)
    YO, _, aO = face_geometry(fO, facesO)
    Yr = T["Xr"]
    xr = np.atleast_2d(np.asarray(x, dtype=np.float64)) - T["c"]
    m = len(xr)
    nfo = len(facesO)
    phi = np.zeros(m)
    g = np.zeros((m, 3))
    count = 0

    def add(s, Y, w):
        d = Y - xr[s]
        r2 = np.sum(d * d, axis=1)
        t = w * r2 ** (-0.5 * p)
        np.add.at(phi, s, t)
        if grad:
            np.add.at(g, s, (p * t / r2)[:, None] * d)

    cur_s, cur_n = np.arange(m), np.zeros(m, dtype=np.int64)
    while len(cur_s):
        adm = _admissible_point(T, xr[cur_s], cur_n, theta)
        add(cur_s[adm], T["X"][cur_n[adm]], T["a"][cur_n[adm]])
        count += int(adm.sum())
        rest_s, rest_n = cur_s[~adm], cur_n[~adm]
        lf = T["leaf"][rest_n]
        ls, ln = rest_s[lf], rest_n[lf]
        for j in range(leaf):
            ok = j < T["count"][ln]
            src = T["order"][np.minimum(T["first"][ln] + j, nfo - 1)]
            add(ls[ok], Yr[src[ok]], aO[src[ok]])
            count += int(ok.sum())
        is_, in_ = rest_s[~lf], rest_n[~lf]
        cur_s = np.concatenate([is_, is_])
        cur_n = np.concatenate([in_ + 1, T["right"][in_]])
    return phi, g, count


def bh_obstacle_energy(f, faces, fO, facesO, theta, leaf=8, p=6.0, weight=1.0):
    """obstacle_energy with the Barnes-Hut potential; also returns dE/df
    (exact derivative of the approximation with the interaction lists fixed:
    the obstacle is static, so only the surface side moves) and the count."""
    X, _, a = face_geometry(f, faces)
    phi, g, count = bh_obstacle_potential(X, fO, facesO, theta, leaf, p, grad=True)
    gX = weight * a[:, None] * g
    corner = faces_to_vertices(f, faces, gX, np.zeros_like(gX), weight * phi)
    dE = np.zeros_like(f)
    for c in range(3):
        np.add.at(dE, faces[:, c], corner[:, c])
    return float(np.sum(weight * a * phi)), dE, count


# ---------------------------------------------------------------------------
# §7.3.5 Willmore energy and its H^2 inner product term
# ---------------------------------------------------------------------------

def lumped_mass(f, faces):
    """Lumped mass of every vertex: a third of the area of each face around
    it (the diagonal mass matrix M of §7.3.5)."""
    a = face_geometry(f, faces)[2]
    m = np.zeros(len(f))
    for c in range(3):
        np.add.at(m, faces[:, c], a / 3.0)
    return m


def willmore_energy(f, faces):
    """E_W = f^T C M^{-1} C f (§7.3.5, summed over the three coordinate
    columns of f), C the cotan stiffness matrix, M the lumped mass."""
    C = cotan_laplacian(f, faces)
    h = C @ f
    return float(np.sum(h * h / lumped_mass(f, faces)[:, None]))


def willmore_differential(f, faces):
    """dE_W/df, shape [nv,3]. With h = C f, m the lumped mass, g = 2 h / m:
        dE_W = g . (C df) + g . (dC f) - sum_i |h_i|^2 / m_i^2 dm_i,
    the first term is C g (C symmetric); in the second, corner k of face S
    opposite the edge (i, j) adds cot(theta_k)/2 (f_i - f_j) to h_i (and the
    opposite to h_j), so it contributes (g_i - g_j).(f_i - f_j)/2 times
    d cot(theta_k); in the third, m_i gains a_S/3 from each face S around i,
    and da_S is the area gradient of §7.1.3."""
    nv = len(f)
    C = cotan_laplacian(f, faces)
    m = lumped_mass(f, faces)
    h = C @ f
    g = 2.0 * h / m[:, None]
    out = C @ g
    q = np.sum(h * h, axis=1) / (m * m)
    X, N, a = face_geometry(f, faces)
    for c in range(3):
        k, i, j = faces[:, c], faces[:, (c + 1) % 3], faces[:, (c + 2) % 3]
        u, v = f[i] - f[k], f[j] - f[k]
        w = np.cross(u, v)
        s = np.linalg.norm(w, axis=1)
        nhat = w / s[:, None]
        cot = np.sum(u * v, axis=1) / s
        # d cot / du, d cot / dv (u, v the edges from corner k)
        dcu = v / s[:, None] - (cot / s)[:, None] * np.cross(v, nhat)
        dcv = u / s[:, None] - (cot / s)[:, None] * np.cross(nhat, u)
        coef = 0.5 * np.sum((g[i] - g[j]) * (f[i] - f[j]), axis=1)
        np.add.at(out, i, coef[:, None] * dcu)
        np.add.at(out, j, coef[:, None] * dcv)
        np.add.at(out, k, -coef[:, None] * (dcu + dcv))
    # mass term: dm_i = sum_S da_S / 3
    fi, fj, fk = f[faces[:, 0]], f[faces[:, 1]], f[faces[:, 2]]
    qS = (q[faces[:, 0]] + q[faces[:, 1]] + q[faces[:, 2]]) / 3.0
    for c, e in enumerate((fk - fj, fi - fk, fj - fi)):
        np.add.at(out, faces[:, c], -qS[:, None] * 0.5 * np.cross(N, e))
    return out


def willmore_metric(f, faces):
    """The H^2 inner product term C M^{-1} C of §7.3.5 (dense, per coordinate)."""
    C = cotan_laplacian(f, faces).toarray()
    return C @ (C / lumped_mass(f, faces)[:, None])
