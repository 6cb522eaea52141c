// Cotan-Laplacian Poisson solves of the preconditioner (§5.2) and the FP64
// vector kernels of the Krylov solver.
//
// C is the weak (stiffness) cotan Laplacian: C_ij = -1/2 (cot a_ij + cot b_ij)
// on edges, C_ii = -sum_j C_ij. Its CSR pattern is fixed by the topology and
// built once on the host; the values are refreshed on the device from the
// current positions. The solve is Jacobi-preconditioned CG on k columns at
// once (independent scalars per column), right-hand side and solution kept
// in the mean-zero subspace (the constants span the nullspace of C).
//
// One CG iteration is two kernels. The direction update is folded into the
// SpMV through q_new = C z + beta q_old, so that each kernel needs only data
// completed by the previous one. Global scalars are reduced by the last
// block to finish (fence + counter), which sums the per-block partials in a
// fixed order: the iteration is deterministic.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "tp_internal.cuh"

namespace tp {

constexpr int KMAX = 9;
constexpr int CG_T = 256;

// ---------------------------------------------------------------------------
// pattern (host, once per mesh)
// ---------------------------------------------------------------------------

int laplacian_setup(tp_mesh* m) {
    const int nv = m->nv, nf = m->nf;
    std::vector<int> F(3 * (size_t)nf);
    TP_CUDA(cudaMemcpy(F.data(), m->faces.ptr, sizeof(int) * 3 * (size_t)nf, cudaMemcpyDeviceToHost));
    // undirected edge -> opposite corners (face*3+corner)
    std::vector<std::map<int, std::pair<int, int>>> adj(nv);
    for (int S = 0; S < nf; ++S)
        for (int c = 0; c < 3; ++c) {
            int i = F[3 * S + (c + 1) % 3], j = F[3 * S + (c + 2) % 3];
            int opp = 3 * S + c;
            for (int dir = 0; dir < 2; ++dir) {
                int a = dir ? j : i, b = dir ? i : j;
                auto it = adj[a].find(b);
                if (it == adj[a].end())
                    adj[a][b] = {opp, -1};
                else if (it->second.second < 0)
                    it->second.second = opp;
                else
                    return fail(TP_ERR_INVALID_ARG, "non-manifold edge (more than two faces)");
            }
        }
    std::vector<int> rowptr(nv + 1, 0), col, src, diagpos(nv);
    for (int v = 0; v < nv; ++v) {
        adj[v][v] = {-1, -1};  // diagonal
        rowptr[v + 1] = rowptr[v] + (int)adj[v].size();
        for (auto& kv : adj[v]) {
            if (kv.first == v) diagpos[v] = (int)col.size();
            col.push_back(kv.first);
            src.push_back(kv.second.first);
            src.push_back(kv.second.second);
        }
    }
    m->nnz = (int)col.size();
    TP_TRY(ensure(m->rowptr, sizeof(int) * (nv + 1)));
    TP_TRY(ensure(m->col, sizeof(int) * m->nnz));
    TP_TRY(ensure(m->cotsrc, sizeof(int) * 2 * (size_t)m->nnz));
    TP_TRY(ensure(m->diagpos, sizeof(int) * nv));
    TP_TRY(ensure(m->val, sizeof(double) * m->nnz));
    TP_TRY(ensure(m->dinv, sizeof(double) * nv));
    TP_CUDA(cudaMemcpy(m->rowptr.ptr, rowptr.data(), sizeof(int) * (nv + 1), cudaMemcpyHostToDevice));
    TP_CUDA(cudaMemcpy(m->col.ptr, col.data(), sizeof(int) * m->nnz, cudaMemcpyHostToDevice));
    TP_CUDA(cudaMemcpy(m->cotsrc.ptr, src.data(), sizeof(int) * 2 * (size_t)m->nnz, cudaMemcpyHostToDevice));
    TP_CUDA(cudaMemcpy(m->diagpos.ptr, diagpos.data(), sizeof(int) * nv, cudaMemcpyHostToDevice));
    return TP_OK;
}

// cot of the angle at each face corner
__global__ void k_corner_cot(const double* __restrict__ pos, const int* __restrict__ faces, int nf,
                             double* __restrict__ cot) {
    int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S >= nf) return;
    for (int c = 0; c < 3; ++c) {
        int o = faces[3 * S + c], i = faces[3 * S + (c + 1) % 3], j = faces[3 * S + (c + 2) % 3];
        double u[3], w[3];
        for (int q = 0; q < 3; ++q) {
            u[q] = pos[3 * i + q] - pos[3 * o + q];
            w[q] = pos[3 * j + q] - pos[3 * o + q];
        }
        double x[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        cot[3 * S + c] = (u[0] * w[0] + u[1] * w[1] + u[2] * w[2]) /
                         sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    }
}

__global__ void k_lap_values(const int* __restrict__ rowptr, const int* __restrict__ col,
                             const int* __restrict__ src, const double* __restrict__ cot, int nv,
                             double* __restrict__ val, double* __restrict__ dinv) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double sum = 0.0;
    int dpos = -1;
    for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        if (col[e] == v) {
            dpos = e;
            continue;
        }
        double w = 0.0;
        if (src[2 * e] >= 0) w += cot[src[2 * e]];
        if (src[2 * e + 1] >= 0) w += cot[src[2 * e + 1]];
        val[e] = -0.5 * w;
        sum += -0.5 * w;
    }
    val[dpos] = -sum;
    dinv[v] = -sum != 0.0 ? 1.0 / (-sum) : 0.0;
}

int laplacian_values(tp_mesh* m, cudaStream_t st) {
    if (m->lap_valid) return TP_OK;
    TP_TRY(ensure(m->tmpv[7], sizeof(double) * 3 * (size_t)m->nf));
    k_corner_cot<<<(m->nf + 255) / 256, 256, 0, st>>>(m->pos.as<double>(), m->faces.as<int>(), m->nf,
                                                      m->tmpv[7].as<double>());
    TP_LAUNCH_CHECK();
    k_lap_values<<<(m->nv + 255) / 256, 256, 0, st>>>(m->rowptr.as<int>(), m->col.as<int>(),
                                                      m->cotsrc.as<int>(), m->tmpv[7].as<double>(),
                                                      m->nv, m->val.as<double>(), m->dinv.as<double>());
    TP_LAUNCH_CHECK();
    m->lap_valid = true;
    return TP_OK;
}

// ---------------------------------------------------------------------------
// CG state in device memory
// ---------------------------------------------------------------------------

struct CgScalars {
    double rz[KMAX], alpha[KMAX], beta[KMAX], rr[KMAX], bb[KMAX];
    int active[KMAX];
    int done;       // all columns converged (or failed)
    int iters;      // iterations executed
    int counter;    // last-block-done counter
    int pad;
};

// block-wide FP64 sum of per-thread values for k columns; result in sh[c*CG_T]
__device__ __forceinline__ void block_sums(double (*vals)[CG_T], int k) {
    for (int w = CG_T / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < k; ++c) vals[c][threadIdx.x] += vals[c][threadIdx.x + w];
        __syncthreads();
    }
}

// is this the last block to finish? (partials written before the call)
__device__ __forceinline__ bool last_block(int* counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
    __syncthreads();
    return last;
}

// init: r = b, z = D^-1 r, p = z, q = C p ; partial rz, bb, pq
__global__ void k_cg_init(const int* __restrict__ rowptr, const int* __restrict__ col,
                          const double* __restrict__ val, const double* __restrict__ dinv, int nv, int k,
                          const double* b, double* __restrict__ x, double* r,
                          double* __restrict__ z, double* __restrict__ p, double* __restrict__ part,
                          CgScalars* sc) {
    __shared__ double sh[2][KMAX][CG_T];
    int v = blockIdx.x * CG_T + threadIdx.x;
    for (int c = 0; c < k; ++c) {
        double rz = 0.0, bb = 0.0;
        if (v < nv) {
            double bv = b[(size_t)v * k + c];
            double zv = dinv[v] * bv;
            x[(size_t)v * k + c] = 0.0;
            r[(size_t)v * k + c] = bv;
            z[(size_t)v * k + c] = zv;
            p[(size_t)v * k + c] = 0.0;   // p = z + beta p with beta = 0 in the first SpMV pass
            rz = bv * zv;
            bb = bv * bv;
        }
        sh[0][c][threadIdx.x] = rz;
        sh[1][c][threadIdx.x] = bb;
    }
    __syncthreads();
    block_sums(sh[0], k);
    block_sums(sh[1], k);
    if (threadIdx.x == 0)
        for (int c = 0; c < k; ++c) {
            part[(size_t)blockIdx.x * 2 * KMAX + c] = sh[0][c][0];
            part[(size_t)blockIdx.x * 2 * KMAX + KMAX + c] = sh[1][c][0];
        }
    if (last_block(&sc->counter) && threadIdx.x == 0) {
        for (int c = 0; c < k; ++c) {
            double rz = 0.0, bb = 0.0;
            for (int bI = 0; bI < (int)gridDim.x; ++bI) {
                rz += __ldcg(part + (size_t)bI * 2 * KMAX + c);
                bb += __ldcg(part + (size_t)bI * 2 * KMAX + KMAX + c);
            }
            sc->rz[c] = rz;
            sc->bb[c] = bb;
            sc->rr[c] = bb;
            sc->beta[c] = 0.0;
            sc->alpha[c] = 0.0;
            sc->active[c] = bb > 0.0 ? 1 : 0;
        }
        sc->iters = 0;
        int any = 0;
        for (int c = 0; c < k; ++c) any |= sc->active[c];
        sc->done = any ? 0 : 1;
        sc->counter = 0;
    }
}

// p = z + beta p ; q = C z + beta q ; partial p.q ; last block: alpha = rz / pq
__global__ void k_cg_dir(const int* __restrict__ rowptr, const int* __restrict__ col,
                         const double* __restrict__ val, int nv, int k, const double* __restrict__ z,
                         double* __restrict__ p, double* __restrict__ q, double* __restrict__ part,
                         CgScalars* sc) {
    if (sc->done) return;
    __shared__ double sh[KMAX][CG_T];
    int v = blockIdx.x * CG_T + threadIdx.x;
    double cz[KMAX];
    for (int c = 0; c < k; ++c) cz[c] = 0.0;
    if (v < nv)
        for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            double w = val[e];
            const double* zr = z + (size_t)col[e] * k;
            for (int c = 0; c < k; ++c) cz[c] += w * zr[c];
        }
    for (int c = 0; c < k; ++c) {
        double pq = 0.0;
        if (v < nv) {
            double be = sc->beta[c];
            size_t o = (size_t)v * k + c;
            double pv = z[o] + be * p[o];
            double qv = cz[c] + be * q[o];
            if (sc->beta[c] == 0.0) qv = cz[c];  // first pass: q is uninitialised
            p[o] = pv;
            q[o] = qv;
            pq = pv * qv;
        }
        sh[c][threadIdx.x] = pq;
    }
    __syncthreads();
    block_sums(sh, k);
    if (threadIdx.x == 0)
        for (int c = 0; c < k; ++c) part[(size_t)blockIdx.x * 2 * KMAX + c] = sh[c][0];
    if (last_block(&sc->counter) && threadIdx.x == 0) {
        for (int c = 0; c < k; ++c) {
            double pq = 0.0;
            for (int bI = 0; bI < (int)gridDim.x; ++bI) pq += __ldcg(part + (size_t)bI * 2 * KMAX + c);
            sc->alpha[c] = (sc->active[c] && pq > 0.0) ? sc->rz[c] / pq : 0.0;
        }
        sc->counter = 0;
    }
}

// x += alpha p ; r -= alpha q ; z = D^-1 r ; partial r.z, r.r ;
// last block: beta = rz_new / rz, convergence per column
__global__ void k_cg_update(const double* __restrict__ dinv, int nv, int k, double* __restrict__ x,
                            double* __restrict__ r, double* __restrict__ z, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ part, CgScalars* sc,
                            double tol2, int max_iter) {
    if (sc->done) return;
    __shared__ double sh[2][KMAX][CG_T];
    int v = blockIdx.x * CG_T + threadIdx.x;
    for (int c = 0; c < k; ++c) {
        double rz = 0.0, rr = 0.0;
        if (v < nv) {
            size_t o = (size_t)v * k + c;
            double al = sc->alpha[c];
            x[o] += al * p[o];
            double rv = r[o] - al * q[o];
            r[o] = rv;
            double zv = dinv[v] * rv;
            z[o] = zv;
            rz = rv * zv;
            rr = rv * rv;
        }
        sh[0][c][threadIdx.x] = rz;
        sh[1][c][threadIdx.x] = rr;
    }
    __syncthreads();
    block_sums(sh[0], k);
    block_sums(sh[1], k);
    if (threadIdx.x == 0)
        for (int c = 0; c < k; ++c) {
            part[(size_t)blockIdx.x * 2 * KMAX + c] = sh[0][c][0];
            part[(size_t)blockIdx.x * 2 * KMAX + KMAX + c] = sh[1][c][0];
        }
    if (last_block(&sc->counter) && threadIdx.x == 0) {
        int any = 0;
        for (int c = 0; c < k; ++c) {
            double rz = 0.0, rr = 0.0;
            for (int bI = 0; bI < (int)gridDim.x; ++bI) {
                rz += __ldcg(part + (size_t)bI * 2 * KMAX + c);
                rr += __ldcg(part + (size_t)bI * 2 * KMAX + KMAX + c);
            }
            if (sc->active[c]) {
                // a converged column keeps its iterate: zero step from now on
                sc->beta[c] = sc->rz[c] > 0.0 ? rz / sc->rz[c] : 0.0;
                sc->rz[c] = rz;
                sc->rr[c] = rr;
                if (rr <= tol2 * sc->bb[c]) {
                    sc->active[c] = 0;
                    sc->beta[c] = 0.0;
                }
            }
            any |= sc->active[c];
        }
        sc->iters += 1;
        if (!any || sc->iters >= max_iter) sc->done = 1;
        sc->counter = 0;
    }
}

static int i_copy(void* host, const void* dev, cudaStream_t st) {
    TP_CUDA(cudaMemcpyAsync(host, dev, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    return TP_OK;
}

int cg_solve(tp_mesh* m, const tp_params* p, const double* b, int k, double* z_out, cudaStream_t st,
             int* iters) {
    if (k < 1 || k > KMAX) return fail(TP_ERR_INVALID_ARG, "cg: k must be in 1..9");
    TP_TRY(laplacian_values(m, st));
    const int nv = m->nv;
    const size_t n = (size_t)nv * k;
    for (int i = 0; i < 5; ++i) TP_TRY(ensure(m->tmpv[i], sizeof(double) * n));
    double *x = m->tmpv[0].as<double>(), *r = m->tmpv[1].as<double>(), *z = m->tmpv[2].as<double>(),
           *pp = m->tmpv[3].as<double>(), *q = m->tmpv[4].as<double>();
    int nblk = (nv + CG_T - 1) / CG_T;
    TP_TRY(ensure(m->part2, sizeof(double) * 2 * KMAX * (size_t)nblk));
    TP_TRY(ensure(m->scal, sizeof(CgScalars)));
    CgScalars* sc = m->scal.as<CgScalars>();
    TP_CUDA(cudaMemsetAsync(sc, 0, sizeof(CgScalars), st));
    // rhs in the mean-zero subspace
    TP_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    TP_TRY(project_mean_zero(m, r, k, st));
    k_cg_init<<<nblk, CG_T, 0, st>>>(m->rowptr.as<int>(), m->col.as<int>(), m->val.as<double>(),
                                     m->dinv.as<double>(), nv, k, r, x, r, z, pp, m->part2.as<double>(),
                                     sc);
    TP_LAUNCH_CHECK();
    const double tol2 = p->cg_tol * p->cg_tol;
    const int cap = p->cg_max;
    int batch = 32, done = 0, it = 0;
    CgScalars host{};
    ProfScope* ps = new ProfScope(m, PK_CG, 0.0, st);
    while (!done) {
        count_launches(2 * (unsigned long long)batch - 1);
        for (int i = 0; i < batch; ++i) {
            k_cg_dir<<<nblk, CG_T, 0, st>>>(m->rowptr.as<int>(), m->col.as<int>(), m->val.as<double>(),
                                            nv, k, z, pp, q, m->part2.as<double>(), sc);
            k_cg_update<<<nblk, CG_T, 0, st>>>(m->dinv.as<double>(), nv, k, x, r, z, pp, q,
                                               m->part2.as<double>(), sc, tol2, cap);
        }
        if (cudaGetLastError() != cudaSuccess) {
            delete ps;
            return fail(TP_ERR_CUDA, "cg: kernel launch failed");
        }
        if (i_copy(&host, sc, st) != TP_OK) {
            delete ps;
            return TP_ERR_CUDA;
        }
        done = host.done;
        it = host.iters;
        if (batch < 256) batch *= 2;
    }
    delete ps;
    // algorithmic bytes of one iteration: CSR values and columns, row pointers
    // and the inverse diagonal once, the k-column vectors z (read), p and q
    // (read + write), x and r (read + write), z (write), p and q (read)
    m->prof.units[PK_CG] += (double)it * ((double)m->nnz * 12.0 + (double)nv * 12.0 +
                                          (double)nv * k * 8.0 * 12.0);
    if (iters) *iters = it;
    TP_TRY(project_mean_zero(m, x, k, st));
    TP_CUDA(cudaMemcpyAsync(z_out, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    bool conv = true;
    for (int c = 0; c < k; ++c) conv = conv && !host.active[c];
    if (!conv)
        return fail(TP_ERR_NOT_CONVERGED, "cg: iteration cap " + std::to_string(cap) +
                                              " reached, relative residual " +
                                              std::to_string(std::sqrt(host.rr[0] / (host.bb[0] + 1e-300))));
    return TP_OK;
}

// ---------------------------------------------------------------------------
// FP64 vector kernels (deterministic reductions)
// ---------------------------------------------------------------------------

__global__ void k_sub_mean(double* __restrict__ x, int nv, int k, const double* __restrict__ mean) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nv * k) return;
    x[i] -= mean[i % k];
}

int project_mean_zero(tp_mesh* m, double* x, int k, cudaStream_t st) {
    TP_TRY(ensure(m->tmpv[6], sizeof(double) * 64));
    TP_TRY(colsum(m, x, m->nv, k, 1.0 / m->nv, m->tmpv[6].as<double>(), st));
    size_t n = (size_t)m->nv * k;
    k_sub_mean<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, m->nv, k, m->tmpv[6].as<double>());
    TP_LAUNCH_CHECK();
    return TP_OK;
}

constexpr int DOT_T = 256;
constexpr int DOT_MAXV = 64;

struct PtrList {
    const double* p[DOT_MAXV];
};
struct CoefList {
    double c[DOT_MAXV];
};

__global__ void k_multidot(PtrList xs, const double* __restrict__ y, int nvec, size_t n,
                           double* __restrict__ part) {
    __shared__ double sh[DOT_T];
    size_t per = (n + gridDim.x - 1) / gridDim.x;
    size_t i0 = (size_t)blockIdx.x * per, i1 = i0 + per < n ? i0 + per : n;
    for (int j = 0; j < nvec; ++j) {
        double s = 0.0;
        const double* x = xs.p[j];
        for (size_t i = i0 + threadIdx.x; i < i1; i += DOT_T) s += x[i] * y[i];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = DOT_T / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * nvec + j] = sh[0];
        __syncthreads();
    }
}

__global__ void k_multidot_final(const double* __restrict__ part, int nblk, int nvec,
                                 double* __restrict__ out) {
    int j = threadIdx.x;
    if (j >= nvec) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * nvec + j];
    out[j] = s;
}

int dots(tp_mesh* m, const double* const* xs, const double* y, int nvec, size_t n, double* out_host,
         cudaStream_t st) {
    if (nvec < 1 || nvec > DOT_MAXV) return fail(TP_ERR_INVALID_ARG, "dots: too many vectors");
    PtrList pl;
    for (int j = 0; j < nvec; ++j) pl.p[j] = xs[j];
    int nblk = (int)std::min<size_t>((n + 2047) / 2048, (size_t)sm_count() * 2);
    if (nblk < 1) nblk = 1;
    TP_TRY(ensure(m->part2, sizeof(double) * (size_t)nblk * nvec + sizeof(double) * DOT_MAXV));
    double* part = m->part2.as<double>();
    double* out = part + (size_t)nblk * nvec;
    k_multidot<<<nblk, DOT_T, 0, st>>>(pl, y, nvec, n, part);
    TP_LAUNCH_CHECK();
    k_multidot_final<<<1, DOT_MAXV, 0, st>>>(part, nblk, nvec, out);
    TP_LAUNCH_CHECK();
    TP_CUDA(cudaMemcpyAsync(out_host, out, sizeof(double) * nvec, cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    return TP_OK;
}

__global__ void k_lincomb(double* __restrict__ y, PtrList xs, CoefList cf, int nvec, size_t n,
                          double beta) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = beta == 0.0 ? 0.0 : beta * y[i];
    for (int j = 0; j < nvec; ++j) s += cf.c[j] * xs.p[j][i];
    y[i] = s;
}

int lincomb(double* y, const double* const* xs, const double* coef, int nvec, size_t n, double beta,
            cudaStream_t st) {
    if (nvec < 0 || nvec > DOT_MAXV) return fail(TP_ERR_INVALID_ARG, "lincomb: too many vectors");
    PtrList pl;
    CoefList cl;
    for (int j = 0; j < nvec; ++j) {
        pl.p[j] = xs[j];
        cl.c[j] = coef[j];
    }
    k_lincomb<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, pl, cl, nvec, n, beta);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

int axpy(double* y, const double* x, double a, size_t n, cudaStream_t st) {
    const double* xs[1] = {x};
    return lincomb(y, xs, &a, 1, n, 1.0, st);
}

}  // namespace tp
