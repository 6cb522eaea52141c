// Vertex pins (§7.1.2) as fast positional constraints (§7.2).
//
// A pin fixes a vertex: Phi_P(f) = f(i) - f_0(i), with f_0(i) the vertex's
// position when the step starts, so Phi_P = 0 there and the step must leave
// the vertex where it is. The pin rows are kept inside the matrices instead
// of going through the Schur complement: the saddle system
//     [A S^T; S 0] [x; lambda] = [-g; 0]   (S: identity rows at the pins)
// has x = 0 at the pins and A_FF x_F = -g_F on the free vertices, so the
// Krylov solver works on vectors whose pinned rows are zero (every A product
// and every preconditioner output is masked), and the rows are appended to
// the integer Laplacians of the preconditioner as well: each Poisson solve
// becomes the solve of [C S^T; S 0] [z; mu] = [b; 0].
//
// That pinned Poisson solve reuses the unpinned solver (C^+: per component,
// mean-zero right-hand side and solution) through a capacitance correction.
// With u = C^+ b and W = C^+ S^T (one solve per pin, once per positions),
//     z = u - W mu + sum_c alpha_c 1_c,
// where, per connected component c, the reactions mu_p of its pins balance
// the right-hand side (sum_{p in c} mu_p = sum_{i in c} b_i, so that
// b - S^T mu lies in the range of C) and the constants alpha_c put z to 0 at
// the pins (u_p - (W mu)_p + alpha_c(p) = 0). The (pins + components)
// square system is inverted on the host once per positions; each solve then
// costs the unpinned solve plus three small kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_util.h"
#include "tp_internal.cuh"

namespace tp {

namespace {

constexpr int PIN_K = 9;   // columns per solve

__global__ void k_pin_unit_rhs(const int* __restrict__ idx, int q0, int kb, int nv, double* __restrict__ E) {
    const int j = threadIdx.x;
    if (j < kb) E[(size_t)idx[q0 + j] * kb + j] = 1.0;
}

// W[q0 + j][v] = sol[v][j]
__global__ void k_pin_store_W(const double* __restrict__ sol, int q0, int kb, int nv, double* __restrict__ W) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nv * kb) return;
    const int v = (int)(i / kb), j = (int)(i % kb);
    W[(size_t)(q0 + j) * nv + v] = sol[i];
}

// right-hand side of the small system, per column j:
//   R[q][j] = -u[pin_q][j] (q < np),   R[np + c][j] = sum_{i in c} b[i][j]
// one block per (row of R, column); the component sums run over the
// vertices of the component in a fixed order (deterministic)
__global__ void k_pin_rhs(const double* __restrict__ u, const double* __restrict__ b, int nv, int k,
                          const int* __restrict__ idx, int np, const int* __restrict__ comp,
                          double* __restrict__ R) {
    const int row = blockIdx.x, j = blockIdx.y;
    if (row < np) {
        if (threadIdx.x == 0) R[(size_t)row * k + j] = -u[(size_t)idx[row] * k + j];
        return;
    }
    const int c = row - np;
    __shared__ double red[256];
    double s = 0.0;
    for (int v = threadIdx.x; v < nv; v += blockDim.x)
        if (comp[v] == c) s += b[(size_t)v * k + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) R[(size_t)row * k + j] = red[0];
}

// Y = Minv R (n x n times n x k), one block
__global__ void k_pin_small(const double* __restrict__ Minv, int n, int k, const double* __restrict__ R,
                            double* __restrict__ Y) {
    for (int e = threadIdx.x; e < n * k; e += blockDim.x) {
        const int r = e / k, j = e % k;
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += Minv[(size_t)r * n + q] * R[(size_t)q * k + j];
        Y[e] = s;
    }
}

// z[v][j] = u[v][j] - sum_q W[q][v] mu[q][j] + alpha[comp(v)][j]; exactly 0 at the pins
__global__ void k_pin_update(const double* __restrict__ u, const double* __restrict__ W, int nv, int k, int np,
                             const double* __restrict__ Y, const int* __restrict__ comp,
                             const unsigned char* __restrict__ pinned, double* __restrict__ z) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nv * k) return;
    const int v = (int)(i / k), j = (int)(i % k);
    if (pinned[v]) {
        z[i] = 0.0;
        return;
    }
    double s = u[i] + Y[(size_t)(np + comp[v]) * k + j];
    for (int q = 0; q < np; ++q) s -= W[(size_t)q * nv + v] * Y[(size_t)q * k + j];
    z[i] = s;
}

__global__ void k_zero_rows(const int* __restrict__ idx, int np, int k, double* __restrict__ x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np * k) return;
    x[(size_t)idx[i / k] * k + (i % k)] = 0.0;
}

// W = C^+ S^T for the current positions, and the inverse of the small system
int pins_prepare(tp_mesh* m, const tp_params* p, cudaStream_t st, int* iters) {
    if (m->pin_valid) return TP_OK;
    const int nv = m->nv, np = m->npins, nc = m->pin_ncomp, n = np + nc;
    TP_TRY(ensure(m->pin_W, sizeof(double) * (size_t)np * nv));
    TP_TRY(ensure(m->pin_tmp, sizeof(double) * (size_t)nv * PIN_K * 2));
    double* E = m->pin_tmp.as<double>();
    double* sol = E + (size_t)nv * PIN_K;
    for (int q0 = 0; q0 < np; q0 += PIN_K) {
        const int kb = std::min(PIN_K, np - q0);
        TP_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * (size_t)nv * kb, st));
        k_pin_unit_rhs<<<1, 32, 0, st>>>(m->pin_idx.as<int>(), q0, kb, nv, E);
        TP_LAUNCH_CHECK();
        int it = 0;
        TP_TRY(cg_solve(m, p, E, kb, sol, st, &it));
        if (iters) *iters += it;
        const size_t cnt = (size_t)nv * kb;
        k_pin_store_W<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(sol, q0, kb, nv, m->pin_W.as<double>());
        TP_LAUNCH_CHECK();
    }
    // W_PP to the host (np x np entries, gathered column by column)
    std::vector<double> wpp((size_t)np * np);
    std::vector<double> col(nv);
    for (int q = 0; q < np; ++q) {
        TP_CUDA(cudaMemcpyAsync(col.data(), m->pin_W.as<double>() + (size_t)q * nv, sizeof(double) * nv,
                                cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < np; ++r) wpp[(size_t)r * np + q] = col[m->pin_host[r]];
    }
    // M = [-W_PP  E; E^T  0], E[p][c] = 1 if pin p lies in component c
    std::vector<double> M((size_t)n * n, 0.0), Minv;
    for (int r = 0; r < np; ++r) {
        for (int q = 0; q < np; ++q) M[(size_t)r * n + q] = -wpp[(size_t)r * np + q];
        const int c = m->pin_comp_host[r];
        M[(size_t)r * n + np + c] = 1.0;
        M[(size_t)(np + c) * n + r] = 1.0;
    }
    if (!invert_dense(M, n, Minv)) return fail(TP_ERR_DEGENERATE, "pins: singular pin system (repeated pins?)");
    TP_TRY(ensure(m->pin_Minv, sizeof(double) * (size_t)n * n + sizeof(double) * (size_t)n * PIN_K * 2));
    TP_CUDA(cudaMemcpyAsync(m->pin_Minv.ptr, Minv.data(), sizeof(double) * (size_t)n * n, cudaMemcpyHostToDevice,
                            st));
    TP_CUDA(cudaStreamSynchronize(st));
    m->pin_valid = true;
    return TP_OK;
}

}  // namespace

int pins_set(tp_mesh* m, int n, const int* idx_host, cudaStream_t st) {
    if (n == 0) {
        pins_release(m);
        return TP_OK;
    }
    if (n < 0 || n > TP_MAX_PINS) return fail(TP_ERR_INVALID_ARG, "pins: n must be in 0..64");
    std::vector<int> pins(idx_host, idx_host + n);
    std::vector<int> sorted(pins);
    std::sort(sorted.begin(), sorted.end());
    for (int i = 0; i < n; ++i) {
        if (sorted[i] < 0 || sorted[i] >= m->nv) return fail(TP_ERR_INVALID_ARG, "pins: vertex index out of range");
        if (i > 0 && sorted[i] == sorted[i - 1]) return fail(TP_ERR_INVALID_ARG, "pins: repeated vertex");
    }
    // connected components of the mesh (computed at creation)
    const std::vector<int>& comp = m->comp_host;
    const int nc = m->ncomp;
    std::vector<int> has(nc, 0), pin_comp(n);
    for (int i = 0; i < n; ++i) {
        pin_comp[i] = comp[pins[i]];
        has[pin_comp[i]] = 1;
    }
    for (int c = 0; c < nc; ++c)
        if (!has[c]) return fail(TP_ERR_INVALID_ARG, "pins: every connected component needs at least one pin");
    std::vector<unsigned char> pinned(m->nv, 0);
    for (int i = 0; i < n; ++i) pinned[pins[i]] = 1;
    pins_release(m);
    TP_TRY(ensure(m->pin_idx, sizeof(int) * (size_t)n));
    TP_TRY(ensure(m->pin_vcomp, sizeof(int) * (size_t)m->nv + (size_t)m->nv));
    TP_CUDA(cudaMemcpyAsync(m->pin_idx.ptr, pins.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
    TP_CUDA(cudaMemcpyAsync(m->pin_vcomp.ptr, comp.data(), sizeof(int) * (size_t)m->nv, cudaMemcpyHostToDevice, st));
    TP_CUDA(cudaMemcpyAsync(m->pin_vcomp.as<char>() + sizeof(int) * (size_t)m->nv, pinned.data(), (size_t)m->nv,
                            cudaMemcpyHostToDevice, st));
    TP_CUDA(cudaStreamSynchronize(st));
    m->npins = n;
    m->pin_ncomp = nc;
    m->pin_host = pins;
    m->pin_comp_host = pin_comp;
    m->pin_valid = false;
    return TP_OK;
}

void pins_release(tp_mesh* m) {
    Buf* all[] = {&m->pin_idx, &m->pin_vcomp, &m->pin_W, &m->pin_Minv, &m->pin_tmp};
    for (Buf* b : all) release(*b);
    m->npins = 0;
    m->pin_ncomp = 0;
    m->pin_host.clear();
    m->pin_comp_host.clear();
    m->pin_valid = false;
}

// z = the pinned Poisson solve of b (k columns): [C S^T; S 0] [z; mu] = [b; 0]
int pinned_solve(tp_mesh* m, const tp_params* p, const double* b, int k, double* z, cudaStream_t st, int* iters) {
    if (k < 1 || k > PIN_K) return fail(TP_ERR_INVALID_ARG, "pinned solve: k must be in 1..9");
    TP_TRY(laplacian_values(m, st));
    TP_TRY(pins_prepare(m, p, st, iters));
    const int nv = m->nv, np = m->npins, nc = m->pin_ncomp, n = np + nc;
    TP_TRY(ensure(m->pin_tmp, sizeof(double) * (size_t)nv * PIN_K * 2));
    double* u = m->pin_tmp.as<double>();   // C^+ b
    int it = 0;
    const int s = cg_solve(m, p, b, k, u, st, &it);
    if (iters) *iters += it;
    if (s != TP_OK && s != TP_ERR_NOT_CONVERGED) return s;
    double* R = m->pin_Minv.as<double>() + (size_t)n * n;
    double* Y = R + (size_t)n * PIN_K;
    const int* comp = m->pin_vcomp.as<int>();
    const unsigned char* pinned = (const unsigned char*)(comp + nv);
    k_pin_rhs<<<dim3(n, k), 256, 0, st>>>(u, b, nv, k, m->pin_idx.as<int>(), np, comp, R);
    TP_LAUNCH_CHECK();
    k_pin_small<<<1, 256, 0, st>>>(m->pin_Minv.as<double>(), n, k, R, Y);
    TP_LAUNCH_CHECK();
    const size_t cnt = (size_t)nv * k;
    k_pin_update<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(u, m->pin_W.as<double>(), nv, k, np, Y, comp, pinned,
                                                                z);
    TP_LAUNCH_CHECK();
    return s;
}

// zero the pinned rows (pins) or remove the mean of each connected component
// (no pins: one barycenter per component, §7.1.1): the subspace the step's
// vectors live in
int project_space(tp_mesh* m, double* x, int k, cudaStream_t st) {
    if (m->npins == 0) return m->ncomp == 1 ? project_mean_zero(m, x, k, st) : project_components(m, x, k, st);
    const int cnt = m->npins * k;
    k_zero_rows<<<(cnt + 255) / 256, 256, 0, st>>>(m->pin_idx.as<int>(), m->npins, k, x);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

}  // namespace tp
