// Willmore energy and its H^2 inner product term (§7.3.5).
//
//   E_W = f^T C M^{-1} C f   (summed over the three coordinate columns),
// C the cotan stiffness matrix, M the lumped mass (a third of the area of
// each face around a vertex). With h = C f, m the lumped mass, g = 2 h / m:
//   dE_W = C g                                  (C df term, C symmetric)
//        + sum over face corners k opposite the edge (i, j):
//            (g_i - g_j).(f_i - f_j) / 2  d cot(theta_k)
//        - sum_S (da_S / 3) sum_{i in S} |h_i|^2 / m_i^2   (mass term)
// (corner k adds cot(theta_k)/2 (f_i - f_j) to h_i and the opposite to h_j).
// With a weight w set on the mesh, the constrained step minimises
// E + w E_W and adds w C M^{-1} C to the operator it inverts (the H^2 term).
//
// All of it is O(V + F) sparse FP64 work: CSR products on the pattern of C,
// one thread per vertex or per face, corner contributions gathered per
// vertex in a fixed order (deterministic).
#include <cmath>

#include "tp_internal.cuh"

namespace tp {

namespace {

// lumped mass of each vertex from the faces around it
__global__ void k_wm_mass(const int* __restrict__ vf_ptr, const int* __restrict__ vf_idx, const d4* __restrict__ f64a,
                          int nv, double* __restrict__ mass) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double s = 0.0;
    for (int e = vf_ptr[v]; e < vf_ptr[v + 1]; ++e) s += f64a[vf_idx[e] / 3].w;
    mass[v] = s / 3.0;
}

// y[v][j] = (acc ? y[v][j] : 0) + alpha * rs[v] * sum_e val[e] x[col[e]][j]
// (rs = nullptr: 1), k columns
__global__ void k_wm_spmv(const int* __restrict__ rowptr, const int* __restrict__ col, const double* __restrict__ val,
                          int nv, int k, const double* __restrict__ x, const double* __restrict__ rs, double alpha,
                          int acc, double* __restrict__ y) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nv * k) return;
    const int v = (int)(i / k), j = (int)(i % k);
    double s = 0.0;
    for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) s += val[e] * x[(size_t)col[e] * k + j];
    s *= alpha;
    if (rs) s *= rs[v];
    y[i] = acc ? y[i] + s : s;
}

// per vertex: e = |h|^2 / m, g = 2 h / m, q = |h|^2 / m^2
__global__ void k_wm_vertex(const double* __restrict__ h, const double* __restrict__ mass, int nv,
                            double* __restrict__ e, double* __restrict__ g, double* __restrict__ q) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const double m = mass[v];
    const double hx = h[3 * v], hy = h[3 * v + 1], hz = h[3 * v + 2];
    const double h2 = hx * hx + hy * hy + hz * hz;
    e[v] = h2 / m;
    q[v] = h2 / (m * m);
    g[3 * v] = 2.0 * hx / m;
    g[3 * v + 1] = 2.0 * hy / m;
    g[3 * v + 2] = 2.0 * hz / m;
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// per-face corner contributions [nf][3 corners][3] of the cotangent and
// mass terms of dE_W
__global__ void k_wm_corners(const double* __restrict__ pos, const int* __restrict__ faces, int nf,
                             const double* __restrict__ g, const double* __restrict__ q,
                             double* __restrict__ corner) {
    const int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S >= nf) return;
    int id[3];
    double P[3][3], G[3][3], out[3][3];
    for (int c = 0; c < 3; ++c) {
        id[c] = faces[3 * S + c];
        for (int t = 0; t < 3; ++t) {
            P[c][t] = pos[3 * id[c] + t];
            G[c][t] = g[3 * id[c] + t];
            out[c][t] = 0.0;
        }
    }
    // cotangent terms: corner c opposite the edge (c+1, c+2)
    for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        double u[3], v[3], w[3], n[3], vxn[3], nxu[3];
        for (int t = 0; t < 3; ++t) {
            u[t] = P[a][t] - P[c][t];
            v[t] = P[b][t] - P[c][t];
        }
        cross3(u, v, w);
        const double s = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        for (int t = 0; t < 3; ++t) n[t] = w[t] / s;
        const double cot = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / s;
        cross3(v, n, vxn);
        cross3(n, u, nxu);
        double coef = 0.0;
        for (int t = 0; t < 3; ++t) coef += (G[a][t] - G[b][t]) * (P[a][t] - P[b][t]);
        coef *= 0.5;
        for (int t = 0; t < 3; ++t) {
            const double dcu = v[t] / s - cot / s * vxn[t];
            const double dcv = u[t] / s - cot / s * nxu[t];
            out[a][t] += coef * dcu;
            out[b][t] += coef * dcv;
            out[c][t] -= coef * (dcu + dcv);
        }
    }
    // mass term: -(q_0 + q_1 + q_2)/3 times the area gradient 1/2 N x e_c
    {
        double e1[3], e2[3], n[3];
        for (int t = 0; t < 3; ++t) {
            e1[t] = P[1][t] - P[0][t];
            e2[t] = P[2][t] - P[0][t];
        }
        cross3(e1, e2, n);
        const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int t = 0; t < 3; ++t) n[t] /= nn;
        const double qS = (q[id[0]] + q[id[1]] + q[id[2]]) / 3.0;
        for (int c = 0; c < 3; ++c) {
            double e[3], ga[3];
            for (int t = 0; t < 3; ++t) e[t] = P[(c + 2) % 3][t] - P[(c + 1) % 3][t];
            cross3(n, e, ga);
            for (int t = 0; t < 3; ++t) out[c][t] -= qS * 0.5 * ga[t];
        }
    }
    for (int c = 0; c < 3; ++c)
        for (int t = 0; t < 3; ++t) corner[(size_t)S * 9 + 3 * c + t] = out[c][t];
}

__global__ void k_wm_axpy(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b,
                          double w, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += w * (a[i] + b[i]);
}

}  // namespace

namespace {

// workspace of the Willmore terms: mass | 1/mass | h | g | e | q | grad | t (9 columns)
struct WmBufs {
    double *mass, *imass, *h, *g, *e, *q, *grad, *t;
};

int wm_bufs(tp_mesh* m, WmBufs* b) {
    const size_t nv = (size_t)m->nv;
    TP_TRY(ensure(m->wm, sizeof(double) * 24 * nv));
    double* p = m->wm.as<double>();
    b->mass = p;
    b->imass = p + nv;
    b->h = p + 2 * nv;
    b->g = p + 5 * nv;
    b->e = p + 8 * nv;
    b->q = p + 9 * nv;
    b->grad = p + 10 * nv;
    b->t = p + 13 * nv;
    return TP_OK;
}

__global__ void k_wm_inv(const double* __restrict__ mass, int nv, double* __restrict__ imass) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) imass[v] = 1.0 / mass[v];
}

// cotan values and lumped mass of the current positions
int wm_prepare(tp_mesh* m, WmBufs* b, cudaStream_t st) {
    TP_TRY(laplacian_values(m, st));
    TP_TRY(wm_bufs(m, b));
    if (m->wm_valid) return TP_OK;
    const int nb = (m->nv + 255) / 256;
    k_wm_mass<<<nb, 256, 0, st>>>(m->vf_ptr.as<int>(), m->vf_idx.as<int>(), m->f64a.as<d4>(), m->nv, b->mass);
    TP_LAUNCH_CHECK();
    k_wm_inv<<<nb, 256, 0, st>>>(b->mass, m->nv, b->imass);
    TP_LAUNCH_CHECK();
    m->wm_valid = true;
    return TP_OK;
}

int wm_spmv(tp_mesh* m, int k, const double* x, const double* rs, double alpha, bool acc, double* y, cudaStream_t st) {
    const size_t n = (size_t)m->nv * k;
    k_wm_spmv<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->rowptr.as<int>(), m->col.as<int>(), m->val.as<double>(),
                                                           m->nv, k, x, rs, alpha, acc ? 1 : 0, y);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

}  // namespace

// E_W into E_dev (device scalar; may be null) and, with dE_dev, dE += w dE_W
int willmore_eval(tp_mesh* m, double* E_dev, double* dE_dev, double w, cudaStream_t st) {
    WmBufs b;
    TP_TRY(wm_prepare(m, &b, st));
    const int nv = m->nv;
    TP_TRY(wm_spmv(m, 3, m->pos.as<double>(), nullptr, 1.0, false, b.h, st));
    k_wm_vertex<<<(nv + 255) / 256, 256, 0, st>>>(b.h, b.mass, nv, b.e, b.g, b.q);
    TP_LAUNCH_CHECK();
    if (E_dev) TP_TRY(sum_f64(b.e, nv, E_dev, m, st));
    if (dE_dev) {
        TP_TRY(ensure(m->corner, sizeof(double) * 9 * (size_t)m->nf));
        k_wm_corners<<<(m->nf + 255) / 256, 256, 0, st>>>(m->pos.as<double>(), m->faces.as<int>(), m->nf, b.g, b.q,
                                                          m->corner.as<double>());
        TP_LAUNCH_CHECK();
        TP_TRY(corners_to_vertices(m, m->corner.as<double>(), 3, b.grad, st));
        TP_TRY(wm_spmv(m, 3, b.g, nullptr, 1.0, false, b.t, st));
        const size_t n = (size_t)nv * 3;
        k_wm_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dE_dev, b.grad, b.t, w, n);
        TP_LAUNCH_CHECK();
    }
    return TP_OK;
}

// y += w C M^{-1} C v, k <= 9 columns (the H^2 term of the step's operator)
int willmore_operator_add(tp_mesh* m, const double* v, int k, double* y, double w, cudaStream_t st) {
    if (k < 1 || k > 9) return fail(TP_ERR_INVALID_ARG, "willmore: k must be in 1..9");
    WmBufs b;
    TP_TRY(wm_prepare(m, &b, st));
    TP_TRY(wm_spmv(m, k, v, b.imass, 1.0, false, b.t, st));
    return wm_spmv(m, k, b.t, nullptr, w, true, y, st);
}

}  // namespace tp
