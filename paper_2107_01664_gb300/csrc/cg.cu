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
#include <mutex>
#include <vector>

#include "tp_internal.cuh"

namespace tp {

constexpr int KMAX = 9;

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
// within-face term of the preconditioner's L^{2-s}: the P1 stiffness with
// face weights w_S = kappa a_S^{1-sigma}, i.e. the cotan matrix of the
// cotangents scaled by the weight of their face (same CSR pattern as C)
// ---------------------------------------------------------------------------

__global__ void k_corner_cot_weighted(const double* __restrict__ cot, const d4* __restrict__ f64a, int nf,
                                      double kappa, double expo, double* __restrict__ wcot) {
    const int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S >= nf) return;
    const double w = kappa * pow(f64a[S].w, expo);
    for (int c = 0; c < 3; ++c) wcot[3 * S + c] = w * cot[3 * S + c];
}

// y[v][j] += sum_e val[e] x[col[e]][j], k columns
__global__ void k_csr_add(const int* __restrict__ rowptr, const int* __restrict__ col,
                          const double* __restrict__ val, int nv, int k, const double* __restrict__ x,
                          double* __restrict__ y) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nv * k) return;
    const int v = (int)(i / k), j = (int)(i % k);
    double s = 0.0;
    for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) s += val[e] * x[(size_t)col[e] * k + j];
    y[i] += s;
}

int self_term_add(tp_mesh* m, const tp_params* p, const double* x, int k, double* y, cudaStream_t st) {
    const double kappa = p->prec_self_weight;
    if (!(kappa > 0.0)) return TP_OK;
    const double sigma = 2.0 - (2.0 - 2.0 / p->p);   // 2 - s, s = 2 - 2/p
    if (!m->gself_valid || m->gself_kappa != kappa || m->gself_sigma != sigma) {
        TP_TRY(ensure(m->tmpv[7], sizeof(double) * 6 * (size_t)m->nf));
        TP_TRY(ensure(m->gval, sizeof(double) * (size_t)m->nnz + sizeof(double) * m->nv));
        double* cot = m->tmpv[7].as<double>();
        double* wcot = cot + 3 * (size_t)m->nf;
        k_corner_cot<<<(m->nf + 255) / 256, 256, 0, st>>>(m->pos.as<double>(), m->faces.as<int>(), m->nf, cot);
        TP_LAUNCH_CHECK();
        k_corner_cot_weighted<<<(m->nf + 255) / 256, 256, 0, st>>>(cot, m->f64a.as<d4>(), m->nf, kappa,
                                                                   1.0 - sigma, wcot);
        TP_LAUNCH_CHECK();
        k_lap_values<<<(m->nv + 255) / 256, 256, 0, st>>>(m->rowptr.as<int>(), m->col.as<int>(),
                                                          m->cotsrc.as<int>(), wcot, m->nv, m->gval.as<double>(),
                                                          m->gval.as<double>() + m->nnz);
        TP_LAUNCH_CHECK();
        m->gself_valid = true;
        m->gself_kappa = kappa;
        m->gself_sigma = sigma;
    }
    const size_t n = (size_t)m->nv * k;
    k_csr_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->rowptr.as<int>(), m->col.as<int>(),
                                                           m->gval.as<double>(), m->nv, k, x, y);
    TP_LAUNCH_CHECK();
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
//
// Vector type V: double (FP64 path) or float (FP32 path: matrix and vectors
// in FP32, which GB300 runs 64x faster than FP64). The inner products are
// accumulated in FP64 in both cases: products of FP32 values are exact in
// FP64, summed per thread, then by warp shuffles and across warps in a
// fixed order.

struct CgCtl {
    unsigned count;        // barrier arrivals
    unsigned gen;          // barrier generation
    int err;               // 0 ok, 1 barrier timeout
    int iters;             // iterations done
    int active[KMAX];      // per column: 1 = not yet converged
    int gdone[KMAX];       // per column group: 1 = all its columns converged (or the cap hit)
    double rr[KMAX], bb[KMAX];
    unsigned long long trace[10];  // per-phase cycles of block 0 (only with TP_CG_TRACE)
};

#ifdef TP_CG_TRACE
#define CG_STAMP(slot)                                                        \
    do {                                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0) {                            \
            long long now_ = clock64();                                       \
            tr[slot] += (unsigned long long)(now_ - tlast);                   \
            tlast = now_;                                                     \
        }                                                                     \
    } while (0)
#else
#define CG_STAMP(slot) \
    do {               \
    } while (0)
#endif

// arrive with release semantics, then poll with acquire loads; the last
// arrival resets the counter and publishes the next generation
__device__ __forceinline__ bool grid_barrier(CgCtl* ctl, unsigned nblk) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        unsigned g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&ctl->gen) : "memory");
        unsigned prev;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&ctl->count) : "memory");
        ok = 1;
        if (prev == nblk - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&ctl->count) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->gen) : "memory");
        } else {
            long long t0 = clock64();
            unsigned cur;
            for (int spins = 0;; ++spins) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&ctl->gen) : "memory");
                if (cur != g) break;
                if (spins > 64) {
                    if (*(volatile int*)&ctl->err) { ok = 0; break; }
                    if (clock64() - t0 > (1LL << 32)) {   // ~2 s at 2 GHz
                        atomicExch(&ctl->err, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

constexpr int PCG_T = 128;
constexpr int PCG_W = PCG_T / 32;
constexpr int CGRP = 3;   // columns per block (column group)

// Warp-level folding butterfly over NV values held by every lane: at each
// level a lane keeps half of its values and adds the partner's matching
// half, so P values (NV padded to a power of two) cost P-1 additions instead
// of P log2(32). Lane L ends with the sum over the warp of value base(L).
template <int NV>
struct Fold {
    static constexpr int P = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : 32;
};

template <int NV>
__device__ __forceinline__ double warp_fold(const double* v, int& base) {
    constexpr int P = Fold<NV>::P;
    double x[P];
#pragma unroll
    for (int j = 0; j < P; ++j) x[j] = j < NV ? v[j] : 0.0;
    const int lane = threadIdx.x & 31;
    base = 0;
    int c = P;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (c > 1) {
            const int h = c / 2;
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < P / 2; ++j) {
                if (j < h) {
                    // send the half I give away, receive the partner's copy of the half I keep
                    double give = up ? x[j] : x[j + h];
                    double got = __shfl_xor_sync(0xffffffffu, give, o);
                    x[j] = (up ? x[j + h] : x[j]) + got;
                }
            }
            if (up) base += h;
            c = h;
        } else {
            x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
        }
    }
    return x[0];
}

// block sums of NV per-thread values, written to out[0..NV) (shared); the
// same order in every block
template <int NV>
__device__ __forceinline__ void block_sum(const double* v, double (*wsum)[PCG_W], double* out) {
    int base = 0;
    double x = warp_fold<NV>(v, base);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // lanes holding the same base carry equal sums; the lowest one writes
    constexpr int P = Fold<NV>::P;
    const bool writer = (lane & (32 / P - 1)) == 0;
    if (writer && base < NV) wsum[base][w] = x;
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < PCG_W; ++i) s += wsum[threadIdx.x][i];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// sums over nbx blocks of partials part[bI * ld + off + j], j < NV
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int ld, int off, unsigned nbx,
                                                double (*wsum)[PCG_W], double* out) {
    double v[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = 0.0;
    for (unsigned bI = threadIdx.x; bI < nbx; bI += PCG_T)
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] += __ldcg(part + (size_t)bI * ld + off + j);
    block_sum<NV>(v, wsum, out);
}

// Block (bx, g) owns rows bx*PCG_T + t (strided) and columns 3g .. 3g+2 of
// the K-column solve. Partials: partA[bx][c] = p.q, partB[bx][c] = r.z,
// partB[bx][K + c] = r.r. alpha of a block's columns needs only its group's
// p.q; every block reduces all columns' r.z and r.r, so the convergence of
// all columns, and with it the exit from the loop, is decided identically
// everywhere.
template <typename V, int K>
__global__ void __launch_bounds__(PCG_T)
k_cg_persistent(const int* __restrict__ rowptr, const int* __restrict__ col, const V* __restrict__ val,
                const V* __restrict__ dinv, int nv, const double* __restrict__ b,
                V* __restrict__ x, V* __restrict__ r, V* __restrict__ z, V* __restrict__ p,
                V* __restrict__ q, double* __restrict__ partA /* [gridDim.x][KMAX] */,
                double* __restrict__ partB /* [gridDim.x][2*KMAX] */, CgCtl* ctl, double tol2, int max_iter) {
    constexpr int k = K;
    constexpr int NG = (K + CGRP - 1) / CGRP;
    __shared__ double wsum[2 * KMAX][PCG_W];
    __shared__ double red[2 * KMAX];
    __shared__ V s_alpha[KMAX], s_beta[KMAX];
    __shared__ double s_rz[KMAX], s_bb[KMAX];
    __shared__ int s_active[KMAX], s_done;
    const unsigned nbx = gridDim.x, nblk = gridDim.x * gridDim.y;
    const int g = blockIdx.y;
    const int c0 = g * CGRP;
    const int nc = (c0 + CGRP <= K) ? CGRP : K - c0;   // columns of this block
    const int stride = gridDim.x * PCG_T;
    const int row0 = blockIdx.x * PCG_T + threadIdx.x;
    double acc[2 * CGRP];
#ifdef TP_CG_TRACE
    unsigned long long tr[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    long long tlast = clock64();
#endif
    (void)NG;
    // ---- init: x = 0, r = b, z = D^-1 r, p = q = 0 ; partial r.z, b.b
#pragma unroll
    for (int j = 0; j < 2 * CGRP; ++j) acc[j] = 0.0;
    for (int v = row0; v < nv; v += stride)
#pragma unroll
        for (int cc = 0; cc < CGRP; ++cc)
            if (cc < nc) {
                const size_t o = (size_t)v * k + c0 + cc;
                V bv = (V)b[o], zv = dinv[v] * bv;
                x[o] = V(0);
                r[o] = bv;
                z[o] = zv;
                p[o] = V(0);
                q[o] = V(0);
                acc[cc] += (double)bv * (double)zv;
                acc[CGRP + cc] += (double)bv * (double)bv;
            }
    block_sum<2 * CGRP>(acc, wsum, red);
    if (threadIdx.x < nc) {
        partB[(size_t)blockIdx.x * 2 * KMAX + c0 + threadIdx.x] = red[threadIdx.x];
        partB[(size_t)blockIdx.x * 2 * KMAX + K + c0 + threadIdx.x] = red[CGRP + threadIdx.x];
    }
    if (!grid_barrier(ctl, nblk)) return;
    // own columns: r.z and b.b
    reduce_partials<CGRP>(partB, 2 * KMAX, c0, nbx, wsum, red);
    reduce_partials<CGRP>(partB, 2 * KMAX, K + c0, nbx, wsum, red + CGRP);
    if (threadIdx.x < nc) {
        const int c = c0 + threadIdx.x;
        const double rz = red[threadIdx.x], bb = red[CGRP + threadIdx.x];
        s_rz[c] = rz;
        s_bb[c] = bb;
        s_beta[c] = V(0);
        s_active[c] = bb > 0.0 ? 1 : 0;
        if (blockIdx.x == 0) {
            ctl->bb[c] = bb;
            ctl->rr[c] = bb;
        }
    }
    __syncthreads();
    int it = 0;
    CG_STAMP(9);
    // Loop exit: each group publishes gdone[g] after its r.r test (block 0 of
    // the group writes it); every block reads all groups' flags after the next
    // barrier, so all blocks leave at the same point. A group that finished
    // earlier idles with alpha = beta = 0.
    for (;;) {
        // ---- phase A: p = z + beta p ; q = C z + beta q (own columns) ; p.q
#pragma unroll
        for (int j = 0; j < CGRP; ++j) acc[j] = 0.0;
        for (int v = row0; v < nv; v += stride) {
            V cz[CGRP];
#pragma unroll
            for (int cc = 0; cc < CGRP; ++cc) cz[cc] = V(0);
            const int e0 = rowptr[v], e1 = rowptr[v + 1];
            for (int e = e0; e < e1; ++e) {
                const V w = val[e];
                const V* zr = z + (size_t)col[e] * k + c0;
#pragma unroll
                for (int cc = 0; cc < CGRP; ++cc)
                    if (cc < nc) cz[cc] += w * __ldcg(zr + cc);
            }
#pragma unroll
            for (int cc = 0; cc < CGRP; ++cc)
                if (cc < nc) {
                    const size_t o = (size_t)v * k + c0 + cc;
                    const V be = s_beta[c0 + cc];
                    const V pv = __ldcg(z + o) + be * p[o];
                    const V qv = cz[cc] + be * q[o];
                    p[o] = pv;
                    q[o] = qv;
                    acc[cc] += (double)pv * (double)qv;
                }
        }
        CG_STAMP(0);
        block_sum<CGRP>(acc, wsum, red);
        if (threadIdx.x < nc) partA[(size_t)blockIdx.x * KMAX + c0 + threadIdx.x] = red[threadIdx.x];
        CG_STAMP(1);
        if (!grid_barrier(ctl, nblk)) return;
        CG_STAMP(2);
        if (it > 0) {
            // flags published before this barrier: identical in every block
            if (threadIdx.x == 0) {
                int all = 1;
                for (int gg = 0; gg < (int)gridDim.y; ++gg) all &= ((volatile int*)ctl->gdone)[gg];
                s_done = all;
            }
            __syncthreads();
            if (s_done) break;
        }
        reduce_partials<CGRP>(partA, KMAX, c0, nbx, wsum, red);   // own group's p.q
        if (threadIdx.x < nc) {
            const int c = c0 + threadIdx.x;
            const double pq = red[threadIdx.x];
            s_alpha[c] = (V)((s_active[c] && pq > 0.0) ? s_rz[c] / pq : 0.0);
        }
        __syncthreads();
        CG_STAMP(3);
        // ---- phase B: x += alpha p ; r -= alpha q ; z = D^-1 r ; r.z, r.r
#pragma unroll
        for (int j = 0; j < 2 * CGRP; ++j) acc[j] = 0.0;
        for (int v = row0; v < nv; v += stride) {
            const V dv = dinv[v];
#pragma unroll
            for (int cc = 0; cc < CGRP; ++cc)
                if (cc < nc) {
                    const size_t o = (size_t)v * k + c0 + cc;
                    const V al = s_alpha[c0 + cc];
                    x[o] += al * p[o];
                    const V rv = r[o] - al * q[o];
                    r[o] = rv;
                    const V zv = dv * rv;
                    z[o] = zv;
                    acc[cc] += (double)rv * (double)zv;
                    acc[CGRP + cc] += (double)rv * (double)rv;
                }
        }
        CG_STAMP(4);
        block_sum<2 * CGRP>(acc, wsum, red);
        if (threadIdx.x < nc) {
            partB[(size_t)blockIdx.x * 2 * KMAX + c0 + threadIdx.x] = red[threadIdx.x];
            partB[(size_t)blockIdx.x * 2 * KMAX + K + c0 + threadIdx.x] = red[CGRP + threadIdx.x];
        }
        CG_STAMP(5);
        if (!grid_barrier(ctl, nblk)) return;
        CG_STAMP(6);
        ++it;
        reduce_partials<CGRP>(partB, 2 * KMAX, c0, nbx, wsum, red);          // own r.z
        reduce_partials<CGRP>(partB, 2 * KMAX, K + c0, nbx, wsum, red + CGRP);  // own r.r
        if (threadIdx.x < nc) {
            const int c = c0 + threadIdx.x;
            const double rz = red[threadIdx.x], rr = red[CGRP + threadIdx.x];
            if (s_active[c]) {
                s_beta[c] = (V)(s_rz[c] > 0.0 ? rz / s_rz[c] : 0.0);
                s_rz[c] = rz;
                if (blockIdx.x == 0) ctl->rr[c] = rr;
                if (rr <= tol2 * s_bb[c]) {
                    s_active[c] = 0;
                    s_beta[c] = V(0);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && blockIdx.x == 0) {
            int any = 0;
            for (int cc = 0; cc < nc; ++cc) any |= s_active[c0 + cc];
            ((volatile int*)ctl->gdone)[g] = (!any || it >= max_iter) ? 1 : 0;
        }
        CG_STAMP(7);
    }
#ifdef TP_CG_TRACE
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        for (int i = 0; i < 10; ++i) ctl->trace[i] = tr[i];
#endif
    if (blockIdx.x == 0 && threadIdx.x < nc) ctl->active[c0 + threadIdx.x] = s_active[c0 + threadIdx.x];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ctl->iters = it;
}

// FP32 copies of the matrix values and the inverse diagonal
__global__ void k_to_f32(const double* __restrict__ a, int n, float* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)a[i];
}

// x (vector type V) -> FP64 output
template <typename V>
__global__ void k_to_f64(const V* __restrict__ a, size_t n, double* __restrict__ out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)a[i];
}

// blocks along the rows for a K-column solve: all rows covered when the
// co-resident capacity allows, and never more than the device holds at once
template <typename V, int K>
static int cg_grid(int nv) {
    static int cached_dev = -1, cached_max = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_persistent<V, K>, PCG_T, 0);
        cached_max = per_sm * sm_count();
        cached_dev = dev;
    }
    constexpr int NG = (K + CGRP - 1) / CGRP;
    int want = (nv + PCG_T - 1) / PCG_T;
    int cap = cached_max / NG;
    int g = want < cap ? want : cap;
    return g < 1 ? 1 : g;
}

template <typename V>
struct CgLaunch {
    const void* fn;
    int grid;    // blocks along the rows
    int groups;  // column groups
};

template <typename V, int K>
static CgLaunch<V> cg_pick(int nv) {
    return CgLaunch<V>{(const void*)k_cg_persistent<V, K>, cg_grid<V, K>(nv), (K + CGRP - 1) / CGRP};
}

template <typename V>
static CgLaunch<V> cg_select(int k, int nv) {
    switch (k) {
        case 1: return cg_pick<V, 1>(nv);
        case 2: return cg_pick<V, 2>(nv);
        case 3: return cg_pick<V, 3>(nv);
        case 4: return cg_pick<V, 4>(nv);
        case 5: return cg_pick<V, 5>(nv);
        case 6: return cg_pick<V, 6>(nv);
        case 7: return cg_pick<V, 7>(nv);
        case 8: return cg_pick<V, 8>(nv);
        default: return cg_pick<V, 9>(nv);
    }
}

template <typename V>
static int cg_run(tp_mesh* m, const tp_params* p, const double* b, int k, double* z_out, cudaStream_t st,
                  int* iters) {
    const int nv = m->nv;
    const size_t n = (size_t)nv * k;
    for (int i = 0; i < 6; ++i) TP_TRY(ensure(m->tmpv[i], sizeof(double) * n));
    V *x = m->tmpv[0].as<V>(), *r = m->tmpv[1].as<V>(), *z = m->tmpv[2].as<V>(), *pp = m->tmpv[3].as<V>(),
      *q = m->tmpv[4].as<V>();
    double* bp = m->tmpv[5].as<double>();
    const V* valp;
    const V* dinv;
    if (sizeof(V) == 8) {
        valp = (const V*)m->val.ptr;
        dinv = (const V*)m->dinv.ptr;
    } else {
        TP_TRY(ensure(m->val32, sizeof(float) * ((size_t)m->nnz + nv)));
        float* v32 = m->val32.as<float>();
        k_to_f32<<<(m->nnz + 255) / 256, 256, 0, st>>>(m->val.as<double>(), m->nnz, v32);
        TP_LAUNCH_CHECK();
        k_to_f32<<<(nv + 255) / 256, 256, 0, st>>>(m->dinv.as<double>(), nv, v32 + m->nnz);
        TP_LAUNCH_CHECK();
        valp = (const V*)v32;
        dinv = (const V*)(v32 + m->nnz);
    }
    const CgLaunch<V> L = cg_select<V>(k, nv);
    const int grid = L.grid;
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
    int nvv = nv;
    void* args[] = {(void*)&rowptr, (void*)&colp, (void*)&valp, (void*)&dinv, (void*)&nvv,
                    (void*)&bp, (void*)&x, (void*)&r, (void*)&z, (void*)&pp, (void*)&q, (void*)&partA,
                    (void*)&partB, (void*)&ctl, (void*)&tol2, (void*)&cap};
    CgCtl host{};
    {
        // One persistent grid at a time per process: two cooperative grids
        // sized to the whole GPU, launched from two meshes on two streams,
        // could each hold part of the SMs while waiting for the rest.
        static std::mutex coop_mutex;
        std::lock_guard<std::mutex> lock(coop_mutex);
        {
            ProfScope ps(m, PK_CG, 0.0, st);
            TP_CUDA(cudaLaunchCooperativeKernel(L.fn, dim3(grid, L.groups), dim3(PCG_T), args, 0, st));
            TP_LAUNCH_CHECK();
        }
        TP_CUDA(cudaMemcpyAsync(&host, ctl, sizeof(CgCtl), cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
    }
    if (host.err) return fail(TP_ERR_TIMEOUT, "cg: grid barrier timed out");
    const int it = host.iters;
    if (iters) *iters = it;
    // algorithmic bytes of one iteration: CSR values (V) and columns, row
    // pointers and the inverse diagonal, the k-column vectors z (read twice),
    // p and q (read + write), x and r (read + write), z (write), p, q (read)
    const double vb = sizeof(V);
    m->prof.units[PK_CG] += (double)it * ((double)m->nnz * (4.0 + vb) + (double)nv * (4.0 + vb) +
                                          (double)nv * k * vb * 13.0);
    double* xo = m->tmpv[5].as<double>();   // b is no longer needed
    if (sizeof(V) == 8) {
        xo = (double*)x;
    } else {
        k_to_f64<V><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, xo);
        TP_LAUNCH_CHECK();
    }
    TP_TRY(project_mean_zero(m, xo, k, st));
    TP_CUDA(cudaMemcpyAsync(z_out, xo, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    bool conv = true;
    for (int c = 0; c < k; ++c) conv = conv && !host.active[c];
    if (!conv)
        return fail(TP_ERR_NOT_CONVERGED, "cg: iteration cap " + std::to_string(cap) +
                                              " reached, relative residual " +
                                              std::to_string(std::sqrt(host.rr[0] / (host.bb[0] + 1e-300))));
    return TP_OK;
}

// per-phase cycle counts of block 0 from the last solve (filled only in a
// build with TP_CG_TRACE; zeros otherwise)
int cg_trace(tp_mesh* m, unsigned long long out[10]) {
    for (int i = 0; i < 10; ++i) out[i] = 0;
    if (!m->scal.ptr) return TP_OK;
    CgCtl h{};
    TP_CUDA(cudaMemcpy(&h, m->scal.ptr, sizeof(CgCtl), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 10; ++i) out[i] = h.trace[i];
    return TP_OK;
}

int cg_solve(tp_mesh* m, const tp_params* p, const double* b, int k, double* z_out, cudaStream_t st,
             int* iters, bool deferred) {
    if (k < 1 || k > KMAX) return fail(TP_ERR_INVALID_ARG, "cg: k must be in 1..9");
    TP_TRY(laplacian_values(m, st));
    if (p->poisson_solver == TP_POISSON_CHOLESKY) {
        bool used = false;
        TP_TRY(chol_solve(m, p, b, k, z_out, st, iters, &used, deferred));
        if (used) return TP_OK;
    }
    // FP64 vectors in both precision modes: with FP32 vectors the Jacobi-CG
    // iteration stalls above a 1e-6 relative residual on rough meshes
    return cg_run<double>(m, p, b, k, z_out, st, iters);
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
constexpr int DOT_MAXV = 128;
constexpr int DOT_CH = 8;   // dot products accumulated per pass over the elements
constexpr int DOT_PAIRS_MAX = 512;
constexpr int DOT_SL_MAX = 64;   // element slices of k_multidot

struct PtrList {
    const double* p[DOT_MAXV];
};
struct CoefList {
    double c[DOT_MAXV];
};

// Block (b, e) takes the DOT_CH pairs j0 = b DOT_CH, ... over the elements of
// slice e (gridDim.y slices): part[e][j] = sum over the slice of
// xs[j][i] * ys[j][i]. The block sums fold across the warp (P-1 additions
// for P values) and then across warps, always in the same order.
__global__ void __launch_bounds__(DOT_T)
k_multidot(PtrList xs, PtrList ys, int nvec, size_t n, double* __restrict__ part, double* __restrict__ out,
           unsigned* __restrict__ ticket) {
    __shared__ double wsum[DOT_CH][DOT_T / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j0 = blockIdx.x * DOT_CH;
    const int nsl = gridDim.y;
    const size_t per = (n + nsl - 1) / nsl;
    const size_t i0 = (size_t)blockIdx.y * per, i1 = i0 + per < n ? i0 + per : n;
    {
        double acc[DOT_CH];
#pragma unroll
        for (int c = 0; c < DOT_CH; ++c) acc[c] = 0.0;
#pragma unroll 2
        for (size_t i = i0 + threadIdx.x; i < i1; i += DOT_T) {
#pragma unroll
            for (int c = 0; c < DOT_CH; ++c)
                if (j0 + c < nvec) acc[c] += xs.p[j0 + c][i] * ys.p[j0 + c][i];
        }
        // folding butterfly: lane L ends with the warp sum of value (L / 4) % 8
        int base = 0, cnt = DOT_CH;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (cnt > 1) {
                const int h = cnt / 2;
                const bool up = (lane & o) != 0;
#pragma unroll
                for (int c = 0; c < DOT_CH / 2; ++c)
                    if (c < h) {
                        double give = up ? acc[c] : acc[c + h];
                        double got = __shfl_xor_sync(0xffffffffu, give, o);
                        acc[c] = (up ? acc[c + h] : acc[c]) + got;
                    }
                if (up) base += h;
                cnt = h;
            } else {
                acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
            }
        }
        if ((lane & (32 / DOT_CH - 1)) == 0) wsum[base][w] = acc[0];
        __syncthreads();
        if (threadIdx.x < DOT_CH && j0 + threadIdx.x < nvec) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < DOT_T / 32; ++q) s += wsum[threadIdx.x][q];
            part[(size_t)blockIdx.y * nvec + j0 + threadIdx.x] = s;
        }
    }
    // the last block to finish adds the block sums in block order (the
    // result does not depend on which block that is) and resets the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // pair j's slices in four quarters of DOT_SL_MAX / 4 (one thread each,
    // its loads issued before the first addition), then the quarters in order
    __shared__ double fin[4 * DOT_MAXV];
    constexpr int QS = DOT_SL_MAX / 4;
    for (int id = threadIdx.x; id < 4 * nvec; id += DOT_T) {
        const int j = id >> 2, e0 = (id & 3) * QS;
        double v[QS];
#pragma unroll
        for (int e = 0; e < QS; ++e) v[e] = e0 + e < nsl ? __ldcg(part + (size_t)(e0 + e) * nvec + j) : 0.0;
        double s = 0.0;
#pragma unroll
        for (int e = 0; e < QS; ++e) s += v[e];
        fin[id] = s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nvec; j += DOT_T)
        out[j] = ((fin[4 * j] + fin[4 * j + 1]) + fin[4 * j + 2]) + fin[4 * j + 3];
    if (threadIdx.x == 0) *ticket = 0u;
}

// element slices of the dot kernels: about 512 elements per block (two per
// thread and pair, so that a thread's loads are in flight together), at most
// eight blocks per SM over all pair chunks, at most DOT_SL_MAX
static int dot_slices(size_t n, int nvec) {
    const int chunks = (nvec + DOT_CH - 1) / DOT_CH;
    const long want = (long)((n + 511) / 512);
    const long cap = std::max(1L, std::min<long>(DOT_SL_MAX, 8L * sm_count() / chunks));
    return (int)std::max(1L, std::min(want, cap));
}

// out_host[j] = xs[j] . ys[j] (FP64, n elements each), one host sync
int dot_pairs(tp_mesh* m, const double* const* xs, const double* const* ys, int nvec, size_t n, double* out_host,
              cudaStream_t st) {
    if (nvec < 1 || nvec > DOT_PAIRS_MAX) return fail(TP_ERR_INVALID_ARG, "dots: too many vectors");
    TP_TRY(ensure(m->part2, sizeof(double) * ((size_t)DOT_SL_MAX * DOT_MAXV + DOT_PAIRS_MAX)));
    double* part = m->part2.as<double>();
    unsigned* tk = nullptr;
    TP_TRY(mesh_tickets(m, &tk, st));
    double* out = part + (size_t)DOT_SL_MAX * DOT_MAXV;
    for (int j0 = 0; j0 < nvec; j0 += DOT_MAXV) {
        const int nc = std::min(DOT_MAXV, nvec - j0);
        PtrList px, py;
        for (int j = 0; j < nc; ++j) {
            px.p[j] = xs[j0 + j];
            py.p[j] = ys[j0 + j];
        }
        const dim3 grid((nc + DOT_CH - 1) / DOT_CH, dot_slices(n, nc));
        k_multidot<<<grid, DOT_T, 0, st>>>(px, py, nc, n, part, out + j0, tk + TICKET_DOTS);
        TP_LAUNCH_CHECK();
    }
    TP_CUDA(cudaMemcpyAsync(out_host, out, sizeof(double) * nvec, cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    return TP_OK;
}

// as dot_pairs, the results left in device memory out_dev [nvec] (no host
// synchronisation)
int dot_pairs_dev(tp_mesh* m, const double* const* xs, const double* const* ys, int nvec, size_t n, double* out_dev,
                  cudaStream_t st) {
    if (nvec < 1 || nvec > DOT_PAIRS_MAX) return fail(TP_ERR_INVALID_ARG, "dots: too many vectors");
    TP_TRY(ensure(m->part2, sizeof(double) * ((size_t)DOT_SL_MAX * DOT_MAXV + DOT_PAIRS_MAX)));
    double* part = m->part2.as<double>();
    unsigned* tk = nullptr;
    TP_TRY(mesh_tickets(m, &tk, st));
    for (int j0 = 0; j0 < nvec; j0 += DOT_MAXV) {
        const int nc = std::min(DOT_MAXV, nvec - j0);
        PtrList px, py;
        for (int j = 0; j < nc; ++j) {
            px.p[j] = xs[j0 + j];
            py.p[j] = ys[j0 + j];
        }
        const dim3 grid((nc + DOT_CH - 1) / DOT_CH, dot_slices(n, nc));
        k_multidot<<<grid, DOT_T, 0, st>>>(px, py, nc, n, part, out_dev + j0, tk + TICKET_DOTS);
        TP_LAUNCH_CHECK();
    }
    return TP_OK;
}

int dots(tp_mesh* m, const double* const* xs, const double* y, int nvec, size_t n, double* out_host,
         cudaStream_t st) {
    std::vector<const double*> ys(nvec, y);
    return dot_pairs(m, xs, ys.data(), nvec, n, out_host, st);
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

constexpr int LC_MAXS = 4;
struct LcSys {
    double* out[LC_MAXS];
    const double* y[LC_MAXS];
    double scale[LC_MAXS];
};

// blockIdx.y = system; the same operation order as k_lincomb (beta y first,
// then the vectors in order), then the scale
__global__ void k_lincomb_sys(PtrList xs, CoefList cf, const double* __restrict__ coef_dev, LcSys L, int nvec,
                              size_t n, double beta) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n) return;
    double acc = beta == 0.0 ? 0.0 : beta * L.y[s][i];
    for (int l = 0; l < nvec; ++l) {
        const double c = coef_dev ? -coef_dev[s * nvec + l] : cf.c[s * nvec + l];
        acc += c * xs.p[s * nvec + l][i];
    }
    L.out[s][i] = L.scale[s] == 1.0 ? acc : L.scale[s] * acc;
}

int lincomb_sys(int ns, double* const* out, const double* const* y, const double* const* xs, int nvec,
                const double* coef_dev, const double* coef_host, const double* scale, double beta, size_t n,
                cudaStream_t st) {
    if (ns < 1 || ns > LC_MAXS || nvec < 0 || ns * nvec > DOT_MAXV)
        return fail(TP_ERR_INVALID_ARG, "lincomb_sys: too many vectors");
    PtrList pl;
    CoefList cl;
    LcSys L;
    for (int j = 0; j < ns * nvec; ++j) {
        pl.p[j] = xs[j];
        cl.c[j] = coef_host ? coef_host[j] : 0.0;
    }
    for (int s = 0; s < ns; ++s) {
        L.out[s] = out[s];
        L.y[s] = y[s];
        L.scale[s] = scale ? scale[s] : 1.0;
    }
    k_lincomb_sys<<<dim3((unsigned)((n + 255) / 256), ns), 256, 0, st>>>(pl, cl, coef_dev, L, nvec, n, beta);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

int axpy(double* y, const double* x, double a, size_t n, cudaStream_t st) {
    const double* xs[1] = {x};
    return lincomb(y, xs, &a, 1, n, 1.0, st);
}

}  // namespace tp
