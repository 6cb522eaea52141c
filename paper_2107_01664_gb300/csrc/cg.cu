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
// The whole solve is one cooperative launch (see k_cg_persistent). The
// direction update is folded into the SpMV through q_new = C z + beta q_old,
// so that one grid barrier separates the two halves of an iteration; the
// global scalars are sums of per-block partials taken in a fixed order, so
// the iteration is deterministic.
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
// persistent CG: the whole solve in one cooperative launch
// ---------------------------------------------------------------------------
//
// Blocks own strided rows; two grid barriers per iteration separate
//   phase A: p = z + beta p, q = C z + beta q, partial p.q      (needs all z)
//   phase B: x += alpha p, r -= alpha q, z = D^-1 r, partial r.z, r.r
// Every block reduces the per-block partials itself, in the same order, so
// all blocks hold bit-identical alpha, beta and convergence decisions and
// leave the loop together. Phase A and phase B partials live in separate
// buffers, so a block that runs ahead never overwrites partials another
// block is still reading. The barrier spins on a generation counter with a
// clock budget; when the budget runs out the kernel records TP_ERR_TIMEOUT
// and every block returns.

struct CgCtl {
    unsigned count;        // barrier arrivals
    unsigned gen;          // barrier generation
    int err;               // 0 ok, 1 barrier timeout
    int iters;             // iterations done
    int active[KMAX];      // per column: 1 = not yet converged
    double rr[KMAX], bb[KMAX];
};

__device__ __forceinline__ bool grid_barrier(CgCtl* ctl, unsigned nblk) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &ctl->gen;
        unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(&ctl->count, 1u) == nblk - 1) {
            ctl->count = 0;
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
            ok = 1;
        } else {
            long long t0 = clock64();
            ok = 1;
            while (*vgen == g) {
                if (*(volatile int*)&ctl->err) { ok = 0; break; }
                if (clock64() - t0 > (1LL << 32)) {   // ~2 s at 2 GHz
                    atomicExch(&ctl->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// block-wide sums of up to 2*KMAX per-thread values (vals[j][t]) -> vals[j][0]
template <int NTH>
__device__ __forceinline__ void block_reduce(double (*vals)[NTH], int nval) {
    for (int w = NTH / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < nval; ++j) vals[j][threadIdx.x] += vals[j][threadIdx.x + w];
        __syncthreads();
    }
}

constexpr int PCG_T = 128;

// sums over blocks of per-block partials part[bI * ld + j], j < nval: every
// thread loads a strided subset, then a fixed-order tree in shared memory.
// Result in sh[j][0]; identical in every block (same data, same order).
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int ld, int nval,
                                                unsigned nblk, double (*sh)[PCG_T]) {
    __syncthreads();
    for (int j = 0; j < nval; ++j) {
        double a = 0.0;
        for (unsigned bI = threadIdx.x; bI < nblk; bI += PCG_T) a += __ldcg(part + (size_t)bI * ld + j);
        sh[j][threadIdx.x] = a;
    }
    __syncthreads();
    block_reduce<PCG_T>(sh, nval);
}

__global__ void __launch_bounds__(PCG_T)
k_cg_persistent(const int* __restrict__ rowptr, const int* __restrict__ col, const double* __restrict__ val,
                const double* __restrict__ dinv, int nv, int k, const double* __restrict__ b,
                double* __restrict__ x, double* __restrict__ r, double* __restrict__ z, double* __restrict__ p,
                double* __restrict__ q, double* __restrict__ partA /* [grid][KMAX] */,
                double* __restrict__ partB /* [grid][2*KMAX] */, CgCtl* ctl, double tol2, int max_iter) {
    __shared__ double sh[2 * KMAX][PCG_T];
    __shared__ double s_alpha[KMAX], s_beta[KMAX], s_rz[KMAX], s_bb[KMAX];
    __shared__ int s_active[KMAX], s_done;
    const unsigned nblk = gridDim.x;
    const int stride = gridDim.x * PCG_T;
    // ---- init: x = 0, r = b, z = D^-1 r, p = q = 0 ; partial r.z, b.b
    for (int j = 0; j < 2 * k; ++j) sh[j][threadIdx.x] = 0.0;
    for (int v = blockIdx.x * PCG_T + threadIdx.x; v < nv; v += stride)
        for (int c = 0; c < k; ++c) {
            size_t o = (size_t)v * k + c;
            double bv = b[o], zv = dinv[v] * bv;
            x[o] = 0.0;
            r[o] = bv;
            z[o] = zv;
            p[o] = 0.0;
            q[o] = 0.0;
            sh[c][threadIdx.x] += bv * zv;
            sh[k + c][threadIdx.x] += bv * bv;
        }
    __syncthreads();
    block_reduce<PCG_T>(sh, 2 * k);
    if (threadIdx.x == 0)
        for (int j = 0; j < 2 * k; ++j) partB[(size_t)blockIdx.x * 2 * KMAX + j] = sh[j][0];
    if (!grid_barrier(ctl, nblk)) return;
    reduce_partials(partB, 2 * KMAX, 2 * k, nblk, sh);
    if (threadIdx.x < k) {
        int c = threadIdx.x;
        double rz = sh[c][0], bb = sh[k + c][0];
        s_rz[c] = rz;
        s_bb[c] = bb;
        s_beta[c] = 0.0;
        s_active[c] = bb > 0.0 ? 1 : 0;
        if (blockIdx.x == 0) {
            ctl->bb[c] = bb;
            ctl->rr[c] = bb;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int c = 0; c < k; ++c) any |= s_active[c];
        s_done = any ? 0 : 1;
    }
    __syncthreads();
    int it = 0;
    while (!s_done) {
        // ---- phase A
        for (int j = 0; j < k; ++j) sh[j][threadIdx.x] = 0.0;
        for (int v = blockIdx.x * PCG_T + threadIdx.x; v < nv; v += stride) {
            double cz[KMAX];
#pragma unroll
            for (int c = 0; c < KMAX; ++c) cz[c] = 0.0;
            for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                double w = val[e];
                const double* zr = z + (size_t)col[e] * k;
#pragma unroll
                for (int c = 0; c < KMAX; ++c)
                    if (c < k) cz[c] += w * __ldcg(zr + c);
            }
#pragma unroll
            for (int c = 0; c < KMAX; ++c)
                if (c < k) {
                    size_t o = (size_t)v * k + c;
                    double be = s_beta[c];
                    double pv = __ldcg(z + o) + be * p[o];
                    double qv = cz[c] + be * q[o];
                    p[o] = pv;
                    q[o] = qv;
                    sh[c][threadIdx.x] += pv * qv;
                }
        }
        __syncthreads();
        block_reduce<PCG_T>(sh, k);
        if (threadIdx.x == 0)
            for (int c = 0; c < k; ++c) partA[(size_t)blockIdx.x * KMAX + c] = sh[c][0];
        if (!grid_barrier(ctl, nblk)) return;
        reduce_partials(partA, KMAX, k, nblk, sh);
        if (threadIdx.x < k) {
            int c = threadIdx.x;
            double pq = sh[c][0];
            s_alpha[c] = (s_active[c] && pq > 0.0) ? s_rz[c] / pq : 0.0;
        }
        __syncthreads();
        // ---- phase B
        for (int j = 0; j < 2 * k; ++j) sh[j][threadIdx.x] = 0.0;
        for (int v = blockIdx.x * PCG_T + threadIdx.x; v < nv; v += stride)
            for (int c = 0; c < k; ++c) {
                size_t o = (size_t)v * k + c;
                double al = s_alpha[c];
                x[o] += al * p[o];
                double rv = r[o] - al * q[o];
                r[o] = rv;
                double zv = dinv[v] * rv;
                z[o] = zv;
                sh[c][threadIdx.x] += rv * zv;
                sh[k + c][threadIdx.x] += rv * rv;
            }
        __syncthreads();
        block_reduce<PCG_T>(sh, 2 * k);
        if (threadIdx.x == 0)
            for (int j = 0; j < 2 * k; ++j) partB[(size_t)blockIdx.x * 2 * KMAX + j] = sh[j][0];
        if (!grid_barrier(ctl, nblk)) return;
        ++it;
        reduce_partials(partB, 2 * KMAX, 2 * k, nblk, sh);
        if (threadIdx.x < k) {
            int c = threadIdx.x;
            double rz = sh[c][0], rr = sh[k + c][0];
            if (s_active[c]) {
                s_beta[c] = s_rz[c] > 0.0 ? rz / s_rz[c] : 0.0;
                s_rz[c] = rz;
                if (blockIdx.x == 0) ctl->rr[c] = rr;
                if (rr <= tol2 * s_bb[c]) {
                    s_active[c] = 0;
                    s_beta[c] = 0.0;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int any = 0;
            for (int c = 0; c < k; ++c) any |= s_active[c];
            s_done = (!any || it >= max_iter) ? 1 : 0;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x < k) ctl->active[threadIdx.x] = s_active[threadIdx.x];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->iters = it;
}

static int cg_grid(int nv) {
    static int cached_dev = -1, cached_max = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_persistent, PCG_T, 0);
        cached_max = per_sm * sm_count();
        cached_dev = dev;
    }
    int want = (nv + PCG_T - 1) / PCG_T;
    int g = want < cached_max ? want : cached_max;
    return g < 1 ? 1 : g;
}

int cg_solve(tp_mesh* m, const tp_params* p, const double* b, int k, double* z_out, cudaStream_t st,
             int* iters) {
    if (k < 1 || k > KMAX) return fail(TP_ERR_INVALID_ARG, "cg: k must be in 1..9");
    TP_TRY(laplacian_values(m, st));
    const int nv = m->nv;
    const size_t n = (size_t)nv * k;
    for (int i = 0; i < 6; ++i) TP_TRY(ensure(m->tmpv[i], sizeof(double) * n));
    double *x = m->tmpv[0].as<double>(), *r = m->tmpv[1].as<double>(), *z = m->tmpv[2].as<double>(),
           *pp = m->tmpv[3].as<double>(), *q = m->tmpv[4].as<double>(), *bp = m->tmpv[5].as<double>();
    const int grid = cg_grid(nv);
    TP_TRY(ensure(m->scal, 16 + sizeof(CgCtl) + sizeof(double) * 3 * KMAX * (size_t)grid));
    CgCtl* ctl = m->scal.as<CgCtl>();
    double* partA = (double*)(m->scal.as<char>() + ((sizeof(CgCtl) + 15) / 16) * 16);
    double* partB = partA + (size_t)KMAX * grid;
    TP_CUDA(cudaMemsetAsync(ctl, 0, sizeof(CgCtl), st));
    // rhs in the mean-zero subspace
    TP_CUDA(cudaMemcpyAsync(bp, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    TP_TRY(project_mean_zero(m, bp, k, st));
    const double tol2 = p->cg_tol * p->cg_tol;
    int cap = p->cg_max;
    const int* rowptr = m->rowptr.as<int>();
    const int* colp = m->col.as<int>();
    const double* valp = m->val.as<double>();
    const double* dinv = m->dinv.as<double>();
    int nvv = nv, kk = k;
    void* args[] = {(void*)&rowptr, (void*)&colp, (void*)&valp, (void*)&dinv, (void*)&nvv, (void*)&kk,
                    (void*)&bp, (void*)&x, (void*)&r, (void*)&z, (void*)&pp, (void*)&q, (void*)&partA,
                    (void*)&partB, (void*)&ctl, (void*)&tol2, (void*)&cap};
    CgCtl host{};
    {
        ProfScope ps(m, PK_CG, 0.0, st);
        TP_CUDA(cudaLaunchCooperativeKernel((void*)k_cg_persistent, dim3(grid), dim3(PCG_T), args, 0, st));
        TP_LAUNCH_CHECK();
    }
    TP_CUDA(cudaMemcpyAsync(&host, ctl, sizeof(CgCtl), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    if (host.err) return fail(TP_ERR_TIMEOUT, "cg: grid barrier timed out");
    const int it = host.iters;
    if (iters) *iters = it;
    // algorithmic bytes of one iteration: CSR values and columns, row pointers
    // and the inverse diagonal, the k-column vectors z (read twice), p and q
    // (read + write), x and r (read + write), z (write), p and q (read)
    m->prof.units[PK_CG] += (double)it * ((double)m->nnz * 12.0 + (double)nv * 12.0 +
                                          (double)nv * k * 8.0 * 13.0);
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
