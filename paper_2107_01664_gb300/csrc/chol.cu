// Pre-factorised cotan-Laplacian solves (§5.2): supernodal sparse Cholesky of
// C with one pinned vertex per connected component, on the device.
//
// The ordering, supernodal tree and index maps come from chol_symbolic.h
// (host, once per topology). Per set of positions the values of C change and
// the factor is recomputed:
//
//   factor (one launch per tree level, one block per supernode J): assemble
//   the panel (t x nJ, shared memory) from the entries of C in J's columns and
//   the children's update matrices, factor its diagonal block (right-looking,
//   column by column), form U_J = (children's share of struct x struct) -
//   L21 L21^T (global memory), and store L11^-1 (explicit inverse of the
//   diagonal block) and L21.
//
//   solve (forward levels leaves -> root, backward levels root -> leaves):
//   with L11^-1 stored, each supernode's step is two small dense mat-vecs on
//   K columns, so the substitution's only sequential chain is the tree height.
//
// The factor is FP32 (64x the FP64 issue rate of this GPU); the solve is
// wrapped in FP64 iterative refinement x += L^-T L^-1 (b - C x), with the
// residual in FP64, until every column meets |r| <= tol |b| (the same test
// as the CG path). Refinement that stops reducing the residual hands the
// solve to the CG path.
#include <algorithm>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "chol_symbolic.h"
#include "tp_internal.cuh"

namespace tp {

constexpr int CH_KMAX = 9;
constexpr int CH_LEAF = 64;                    // vertices per leaf supernode
constexpr int CHF_T = 256;                     // factor block
constexpr int CHS_T = 256;                     // solve block
constexpr int CHR_T = 256;                     // residual block
constexpr size_t CH_SMEM_MAX = 200 * 1024;     // largest factor panel kept in shared memory

struct CholNode {   // 64 bytes
    int p0, nJ, mJ, t;
    long long loff, uoff;
    int voff, child0, child1, s0;
    int asm0, asm1, pad0, pad1;
};
static_assert(sizeof(CholNode) == 64, "CholNode layout");

struct CholCtl {
    int done;       // 1: every column converged (or the refinement gave up)
    int stalled;    // 1: the residual stopped decreasing
    int iters;      // refinement sweeps done
    int err;        // 1: a cross-block wait of a sweep gave up
    unsigned ticket, bcount, arrive;   // sweep scheduling (zero between sweeps)
    int bad_pivot;  // 1: a non-positive pivot appeared in the factorisation
    double bb[CH_KMAX], rr[CH_KMAX];
    unsigned epoch;  // sweeps finished; never cleared (the node flags compare against it)
};

struct CholState {
    CholSymbolic S;
    bool ok = false;
    std::string why;
    int H = 0;                            // number of levels
    std::vector<int> lvl_max_t, lvl_max_n, lvl_max_m;
    std::vector<size_t> lvl_factor_smem, lvl_solve_smem;   // bytes; solve: factor block + 9-column vectors
    std::vector<double> lvl_factor_flops;
    double solve_bytes = 0.0;             // factor bytes read by one forward + backward sweep
    Buf nodes, level_nodes, child_idx, rel, struct_pos, asm_dst, asm_src, perm, comp_ptr, comp_verts, comp_of;
    Buf parent, fdone, bdone, trace;
    size_t solve_smem = 0;     // dynamic shared memory of the sweep kernel
    Buf L, U, uvec, ybuf, xbuf, ctl, part, x, r, bp;
    bool factored = false;
    int ncomp = 1;
    // refinement sweeps captured as CUDA graphs, one per column count, keyed
    // by the buffers and scalars baked into their launches
    // deferred solves (inside flexible GMRES): the pivot check of the current
    // factor is read once, and the sweeps' wait errors and unconverged
    // columns accumulate in dflags [2] for the caller to read once per step
    bool pivot_known = false, pivot_ok = false;
    Buf dflags;
    struct SweepGraph {
        cudaGraphExec_t exec = nullptr;
        const void* key[4] = {};
        double tol2 = 0.0;
        int cap = 0, rgrid = 0, kernels = 0;
    } graph[CH_KMAX + 1];
    cudaStream_t capture = nullptr;
};

// ---------------------------------------------------------------------------
// factorisation
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(CHF_T)
k_chol_factor(const CholNode* __restrict__ nodes, const int* __restrict__ lvl, const int* __restrict__ child_idx,
              const int* __restrict__ rel, const int* __restrict__ asm_dst, const int* __restrict__ asm_src,
              const double* __restrict__ val, float* __restrict__ L, float* __restrict__ U,
              CholCtl* __restrict__ ctl) {
    extern __shared__ float smem[];
    __shared__ float s_rd;
    const CholNode nd = nodes[lvl[blockIdx.x]];
    const int n = nd.nJ, m = nd.mJ, t = nd.t;
    float* P = smem;                 // panel t x n, column-major
    float* X = smem + (size_t)t * n; // L11^-1, n x n column-major
    float* UJ = U + nd.uoff;         // m x m, column-major (lower part used)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = CHF_T / 32;

    for (int i = tid; i < t * n; i += CHF_T) P[i] = 0.f;
    for (int i = tid; i < m * m; i += CHF_T) UJ[i] = 0.f;
    __syncthreads();
    // entries of C in J's columns (each panel position at most once)
    for (int e = nd.asm0 + tid; e < nd.asm1; e += CHF_T) P[asm_dst[e]] = (float)val[asm_src[e]];
    __syncthreads();
    // extend-add of the children's update matrices, one child at a time
    for (int ci = nd.child0; ci < nd.child1; ++ci) {
        const CholNode cn = nodes[child_idx[ci]];
        const int mc = cn.mJ;
        const int* rl = rel + cn.s0;
        const float* Uc = U + cn.uoff;
        for (int idx = tid; idx < mc * mc; idx += CHF_T) {
            const int y = idx / mc, x = idx - y * mc;
            if (x < y) continue;
            const int R = rl[x], Cc = rl[y];
            const float v = Uc[idx];
            if (Cc < n)
                P[R + Cc * t] += v;
            else
                UJ[(R - n) + (Cc - n) * m] += v;
        }
        __syncthreads();
    }
    // right-looking Cholesky of the diagonal block; the rows below it become L21
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            float d = P[k + k * t];
            if (!(d > 0.f)) {
                ctl->bad_pivot = 1;
                d = 1.f;
            }
            d = sqrtf(d);
            P[k + k * t] = d;
            s_rd = 1.f / d;
        }
        __syncthreads();
        const float rd = s_rd;
        for (int i = k + 1 + tid; i < t; i += CHF_T) P[i + k * t] *= rd;
        __syncthreads();
        for (int j = k + 1 + warp; j < n; j += NW) {
            const float ljk = P[j + k * t];
            for (int i = j + lane; i < t; i += 32) P[i + j * t] -= P[i + k * t] * ljk;
        }
        __syncthreads();
    }
    // U_J -= L21 L21^T (lower part)
    for (int idx = tid; idx < m * m; idx += CHF_T) {
        const int y = idx / m, x = idx - y * m;
        if (x < y) continue;
        float s = 0.f;
        for (int k = 0; k < n; ++k) s += P[n + x + k * t] * P[n + y + k * t];
        UJ[idx] -= s;
    }
    // X = L11^-1 by forward substitution, one column per thread
    for (int c = tid; c < n; c += CHF_T) {
        for (int i = 0; i < c; ++i) X[i + c * n] = 0.f;
        X[c + c * n] = 1.f / P[c + c * t];
        for (int i = c + 1; i < n; ++i) {
            float s = 0.f;
            for (int k = c; k < i; ++k) s += P[i + k * t] * X[k + c * n];
            X[i + c * n] = -s / P[i + i * t];
        }
    }
    __syncthreads();
    const int ldn = n | 1, ldm = m == 0 ? 0 : (m | 1);
    float* Lj = L + nd.loff;   // n x n, leading dimension ldn
    for (int i = tid; i < n * n; i += CHF_T) {
        const int c = i / n, r = i - c * n;
        Lj[r + c * ldn] = X[i];
    }
    float* L21 = Lj + (size_t)n * ldn;   // m x n, leading dimension ldm
    for (int idx = tid; idx < m * n; idx += CHF_T) {
        const int k = idx / m, x = idx - k * m;
        L21[x + k * ldm] = P[n + x + k * t];
    }
}

// ---------------------------------------------------------------------------
// solves
// ---------------------------------------------------------------------------

// The node's factor block [L11^-1 | L21] (odd leading dimensions, from a
// 16-byte aligned offset) is first copied to shared memory with 16-byte
// loads, so that the mat-vecs below read shared memory only.
__device__ __forceinline__ float* stage_factor(const float* __restrict__ L, const CholNode& nd, float* smem) {
    const int ldn = nd.nJ | 1, ldm = nd.mJ == 0 ? 0 : (nd.mJ | 1);
    const int nl4 = (nd.nJ * ldn + nd.nJ * ldm + 3) >> 2;
    const float4* src = reinterpret_cast<const float4*>(L + nd.loff);
    float4* dst = reinterpret_cast<float4*>(smem);
    for (int i = threadIdx.x; i < nl4; i += CHS_T) dst[i] = __ldcg(src + i);
    return smem + 4 * nl4;
}

// Everything one refinement sweep needs (kernel parameter block).
struct SweepArgs {
    const CholNode* nodes;
    const int* order;        // level_nodes: children before parents
    const int* child_idx;
    const int* rel;
    const int* struct_pos;
    const int* perm;
    const int* parent;
    const float* L;
    float* ybuf;
    float* xbuf;
    float* uvec;
    unsigned* fdone;         // per node: epoch of its last finished forward step
    unsigned* bdone;         // per node: epoch of its last finished backward step
    const int* rowptr;
    const int* col;
    const double* val;
    const double* bp;
    double* x;
    double* r;
    double* part;
    CholCtl* ctl;
    unsigned long long* trace;   // per ticket timestamps (builds with TP_CHOL_TRACE only)
    double tol2;
    int nv, nn, cap;
};

#ifdef TP_CHOL_TRACE
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#define CH_TRACE(tk, slot)                                                      \
    do {                                                                        \
        if (threadIdx.x == 0 && A.trace) A.trace[(size_t)(tk) * 6 + (slot)] = gtimer(); \
    } while (0)
#else
#define CH_TRACE(tk, slot) \
    do {                   \
    } while (0)
#endif

constexpr int CH_MAXCH = 16;   // children whose records are prefetched to shared memory

struct ChildRec {
    int voff, mJ, s0, row0;   // row0: first row of this child in the staged update vectors
};

// store(e, load(e)) for e < count, the block's threads taking entries
// e = tid, tid + CHS_T, ...: each thread issues B independent loads before
// its stores, so a gather costs one memory round trip per B entries
// instead of one per entry
template <int B, class Load, class Store>
__device__ __forceinline__ void gather_batched(int count, Load load, Store store) {
    for (int e0 = threadIdx.x; e0 < count; e0 += CHS_T * B) {
        float v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int e = e0 + b * CHS_T;
            if (e < count) v[b] = load(e);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int e = e0 + b * CHS_T;
            if (e < count) store(e, v[b]);
        }
    }
}

// K columns padded to whole float4s in shared memory
template <int K>
struct Kp {
    static constexpr int P = (K + 3) & ~3;
};

// out(r, acc) for r < R with acc[c] = sum_k A(r, k) v[k][c], A(r, k) =
// M[r * sr + k * sk], k over [0, r] (mode 0), [r, n) (mode 1) or [0, n)
// (mode 2). One thread per row (passes of 128 rows); the two halves of the
// block take the even and the odd k, so every lane of a warp reads the same
// row of v (a broadcast) and the halves meet in one shared-memory add.
template <int K, class Out>
__device__ __forceinline__ void rows_matvec(const float* M, int sr, int sk, int R, int n, int mode, const float* v,
                                            float* scratch, Out out) {
    constexpr int KP = Kp<K>::P;
    static_assert(CHS_T == 256, "two halves of 128 threads");
    const int tid = threadIdx.x, rr = tid & 127, half = tid >> 7;
    for (int r0 = 0; r0 < R; r0 += 128) {
        const int r = r0 + rr;
        float acc[K];
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] = 0.f;
        if (r < R) {
            const float* mr = M + (size_t)r * sr;
            int k, kend, step;
            if (mode == 1) {
                k = n - 1 - half;
                kend = r - 1;
                step = -2;
            } else {
                k = half;
                kend = mode == 0 ? r + 1 : n;
                step = 2;
            }
            for (; step > 0 ? k < kend : k > kend; k += step) {
                const float m = mr[k * sk];
                const float4* vr = reinterpret_cast<const float4*>(v + k * KP);
#pragma unroll
                for (int q = 0; q < KP / 4; ++q) {
                    const float4 t = vr[q];
                    if (4 * q + 0 < K) acc[4 * q + 0] += m * t.x;
                    if (4 * q + 1 < K) acc[4 * q + 1] += m * t.y;
                    if (4 * q + 2 < K) acc[4 * q + 2] += m * t.z;
                    if (4 * q + 3 < K) acc[4 * q + 3] += m * t.w;
                }
            }
        }
        if (half && r < R)
#pragma unroll
            for (int c = 0; c < K; ++c) scratch[rr * KP + c] = acc[c];
        __syncthreads();
        if (!half && r < R) {
#pragma unroll
            for (int c = 0; c < K; ++c) acc[c] += scratch[rr * KP + c];
            out(r, acc);
        }
        __syncthreads();
    }
}

// shared-memory layout of a solve step (floats): factor block, then the
// K-column vectors (rows of KP floats): forward w (t), y (n); backward x_S
// (m), y_J (n), z (n); then the two-half scratch (128 rows); then (backward)
// the node's FP64 solution entries
template <int K>
struct StepSmem {
    float* vec;
    float* scratch;
    double* xo;
    int* aux;      // forward: the children's target rows, then their update vectors; backward: struct(J)
    __device__ StepSmem(const CholNode& nd, float* smem) {
        constexpr int KP = Kp<K>::P;
        const int n = nd.nJ, m = nd.mJ;
        const int ldn = n | 1, ldm = m == 0 ? 0 : (m | 1);
        vec = smem + 4 * ((n * ldn + n * ldm + 3) >> 2);
        scratch = vec + (m + 2 * n) * KP;
        xo = reinterpret_cast<double*>(scratch + 128 * KP);
        aux = reinterpret_cast<int*>(xo + n * K);
    }
};

// forward step of node J, in two halves. fwd_prepare does what does not
// depend on the children (factor block to shared memory, w = (r_J ; 0),
// the children's records); fwd_finish adds the children's update vectors
// and forms y_J = L11^-1 w_J and u_J = w_S - L21 y_J.
template <int K>
__device__ __forceinline__ void fwd_prepare(const SweepArgs& A, const CholNode& nd, float* smem, ChildRec* kids) {
    constexpr int KP = Kp<K>::P;
    const int n = nd.nJ, t = nd.t, tid = threadIdx.x;
    stage_factor(A.L, nd, smem);
    const StepSmem<K> sm(nd, smem);
    float* w = sm.vec;   // t x KP
    const int* perm = A.perm + nd.p0;
    gather_batched<8>(t * K,
                      [&](int e) { const int a = e / K; return a < n ? (float)__ldcg(A.r + (size_t)perm[a] * K + (e - a * K)) : 0.f; },
                      [&](int e, float v) { const int a = e / K; w[a * KP + (e - a * K)] = v; });
    const int nc = nd.child1 - nd.child0;
    if (nc <= CH_MAXCH) {
        // the children's records, then their target rows in this front
        if (tid == 0) {
            int row0 = 0;
            for (int ci = 0; ci < nc; ++ci) {
                const CholNode cn = A.nodes[A.child_idx[nd.child0 + ci]];
                kids[ci] = ChildRec{cn.voff, cn.mJ, cn.s0, row0};
                row0 += cn.mJ;
            }
        }
        __syncthreads();
        for (int ci = 0; ci < nc; ++ci) {
            const ChildRec cr = kids[ci];
            for (int x = tid; x < cr.mJ; x += CHS_T) sm.aux[cr.row0 + x] = A.rel[cr.s0 + x];
        }
    }
}

template <int K>
__device__ void fwd_finish(const SweepArgs& A, const CholNode& nd, float* smem, const ChildRec* kids) {
    constexpr int KP = Kp<K>::P;
    const int n = nd.nJ, m = nd.mJ, t = nd.t, tid = threadIdx.x;
    const int ldn = n | 1, ldm = m == 0 ? 0 : (m | 1);
    const StepSmem<K> sm(nd, smem);
    float* w = sm.vec;            // t x KP
    float* y = w + t * KP;        // n x KP
    const float* Li = smem;       // n x n, leading dimension ldn
    const float* L21 = smem + n * ldn;   // m x n, leading dimension ldm
    const int nc = nd.child1 - nd.child0;
    if (nc <= CH_MAXCH) {
        // every child's update vector in one batched pass, then the
        // extend-add from shared memory, one child at a time
        const int rows = nc ? kids[nc - 1].row0 + kids[nc - 1].mJ : 0;
        const int* krow = sm.aux;
        float* kval = reinterpret_cast<float*>(sm.aux + rows);
        gather_batched<8>(rows * K,
                          [&](int e) {
                              const int r = e / K;
                              int ci = 0;
                              while (ci + 1 < nc && kids[ci + 1].row0 <= r) ++ci;
                              return __ldcg(A.uvec + ((size_t)kids[ci].voff + (r - kids[ci].row0)) * K + (e - r * K));
                          },
                          [&](int e, float v) { kval[e] = v; });
        __syncthreads();
        for (int ci = 0; ci < nc; ++ci) {
            const ChildRec cr = kids[ci];
            for (int idx = tid; idx < cr.mJ * K; idx += CHS_T) {
                const int x = idx / K, c = idx - x * K;
                w[krow[cr.row0 + x] * KP + c] += kval[cr.row0 * K + idx];
            }
            __syncthreads();
        }
    } else {
        for (int ci = 0; ci < nc; ++ci) {
            const CholNode cn = A.nodes[A.child_idx[nd.child0 + ci]];
            const int* rl = A.rel + cn.s0;
            const float* uc = A.uvec + (size_t)cn.voff * K;
            for (int idx = tid; idx < cn.mJ * K; idx += CHS_T) {
                const int x = idx / K, c = idx - x * K;
                w[rl[x] * KP + c] += __ldcg(uc + idx);
            }
            __syncthreads();
        }
    }
    float* yb = A.ybuf + (size_t)nd.p0 * K;
    rows_matvec<K>(Li, 1, ldn, n, n, 0, w, sm.scratch, [&](int r, const float (&acc)[K]) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
            y[r * KP + c] = acc[c];
            yb[r * K + c] = acc[c];
        }
    });
    float* uj = A.uvec + (size_t)nd.voff * K;
    rows_matvec<K>(L21, 1, ldm, m, n, 2, y, sm.scratch, [&](int r, const float (&acc)[K]) {
#pragma unroll
        for (int c = 0; c < K; ++c) uj[r * K + c] = w[(n + r) * KP + c] - acc[c];
    });
}

// backward step of node J. bwd_prepare stages the factor block and the
// node's own entries of the FP64 solution (only this node writes them);
// bwd_finish gathers x_S and y_J in one pass, then z = y_J - L21^T x_S,
// x_J = L11^-T z, and the solution gains x_J.
template <int K>
__device__ __forceinline__ void bwd_prepare(const SweepArgs& A, const CholNode& nd, float* smem) {
    stage_factor(A.L, nd, smem);
    const StepSmem<K> sm(nd, smem);
    for (int idx = threadIdx.x; idx < nd.nJ * K; idx += CHS_T) {
        const int a = idx / K, c = idx - a * K;
        sm.xo[idx] = A.x[(size_t)A.perm[nd.p0 + a] * K + c];
    }
    for (int x = threadIdx.x; x < nd.mJ; x += CHS_T) sm.aux[x] = A.struct_pos[nd.s0 + x];
}

template <int K>
__device__ void bwd_finish(const SweepArgs& A, const CholNode& nd, float* smem) {
    constexpr int KP = Kp<K>::P;
    const int n = nd.nJ, m = nd.mJ, tid = threadIdx.x;
    const int ldn = n | 1, ldm = m == 0 ? 0 : (m | 1);
    const StepSmem<K> sm(nd, smem);
    float* xs = sm.vec;           // m x KP
    float* yj = xs + m * KP;      // n x KP
    float* z = yj + n * KP;       // n x KP
    const float* Li = smem;
    const float* L21 = smem + n * ldn;
    const int* spos = sm.aux;   // struct(J), staged before the wait
    gather_batched<8>((m + n) * K,
                      [&](int e) {
                          if (e < m * K) {
                              const int x = e / K;
                              return __ldcg(A.xbuf + (size_t)spos[x] * K + (e - x * K));
                          }
                          return __ldcg(A.ybuf + (size_t)nd.p0 * K + (e - m * K));
                      },
                      [&](int e, float v) {
                          if (e < m * K) {
                              const int x = e / K;
                              xs[x * KP + (e - x * K)] = v;
                          } else {
                              const int j = e - m * K, a = j / K;
                              yj[a * KP + (j - a * K)] = v;
                          }
                      });
    __syncthreads();
    rows_matvec<K>(L21, ldm, 1, n, m, 2, xs, sm.scratch, [&](int r, const float (&acc)[K]) {
#pragma unroll
        for (int c = 0; c < K; ++c) z[r * KP + c] = yj[r * KP + c] - acc[c];
    });
    float* xb = A.xbuf + (size_t)nd.p0 * K;
    const double* xo = sm.xo;
    rows_matvec<K>(Li, ldn, 1, n, n, 1, z, sm.scratch, [&](int r, const float (&acc)[K]) {
        double* xv = A.x + (size_t)A.perm[nd.p0 + r] * K;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            xb[r * K + c] = acc[c];
            xv[c] = xo[r * K + c] + (double)acc[c];
        }
    });
}

// ---- cross-block signalling (bounded waits: ~1 s, then ctl->err) ---------

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    __threadfence();
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// waits until *p >= target (counters) or == target (epoch flags); false on
// timeout. Spins tightly first (a flag is usually set within microseconds).
__device__ bool wait_until(const unsigned* p, unsigned target, bool at_least, CholCtl* ctl) {
    const long long t0 = clock64();
    for (int spins = 0;; ++spins) {
        const unsigned v = ld_acquire(p);
        if (at_least ? v >= target : v == target) return true;
        if (spins > 256) {
            if (*(volatile int*)&ctl->err) return false;
            if (clock64() - t0 > (1LL << 31)) {   // ~1 s at 2 GHz
                atomicExch(&ctl->err, 1);
                return false;
            }
            __nanosleep(32);
        }
    }
}

// One refinement sweep in one launch: forward and backward substitution
// over the supernodal tree, then r = bp - C x and the convergence test.
// Blocks take nodes from a ticket counter: tickets 0..nn-1 are the forward
// steps in `order` (children first), nn..2nn-1 the backward steps in
// reverse order (parents first). A step waits only for steps with smaller
// tickets (its children's forward steps; its parent's backward step, or
// for a root its own forward step), and those were taken by blocks that
// are already running, so the waits end without any assumption on how
// many blocks are resident. Flags hold the sweep's epoch, so they need no
// reset; the last block to finish the residual resets the counters and
// advances the epoch.
template <int K>
__global__ void __launch_bounds__(CHS_T)
k_chol_sweep(SweepArgs A) {
    CholCtl* ctl = A.ctl;
    if (*(volatile int*)&ctl->done) return;
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int s_tk, s_ok, s_last;
    __shared__ ChildRec s_kids[CH_MAXCH];
    __shared__ double s_red[CHS_T];
    const unsigned ep = *(volatile unsigned*)&ctl->epoch + 1;
    const int nn = A.nn, tid = threadIdx.x;
    if (tid == 0) s_tk = (int)atomicAdd(&ctl->ticket, 1u);
    __syncthreads();
    for (;;) {
        const int tk = s_tk;
        if (tk >= 2 * nn) break;
        // the next ticket is taken now and used after this step: the atomic's
        // latency overlaps the step (the block runs both steps in order)
        unsigned next = 0;
        if (tid == 0) next = atomicAdd(&ctl->ticket, 1u);
        const bool fwd = tk < nn;
        CH_TRACE(tk, 0);
        const int J = fwd ? A.order[tk] : A.order[2 * nn - 1 - tk];
        const CholNode nd = A.nodes[J];
        if (fwd)
            fwd_prepare<K>(A, nd, smem, s_kids);
        else
            bwd_prepare<K>(A, nd, smem);
        // wait: forward for every child (one thread each), backward for the
        // parent (a root for its own forward step)
        if (tid == 0) s_ok = 1;
        __syncthreads();
        CH_TRACE(tk, 1);
        if (fwd) {
            const int nc = nd.child1 - nd.child0;
            for (int i = tid; i < nc; i += CHS_T)
                if (!wait_until(A.fdone + A.child_idx[nd.child0 + i], ep, false, ctl)) s_ok = 0;
        } else if (tid == 0) {
            const int P = A.parent[J];
            if (!(P >= 0 ? wait_until(A.bdone + P, ep, false, ctl) : wait_until(A.fdone + J, ep, false, ctl))) s_ok = 0;
        }
        __syncthreads();
        CH_TRACE(tk, 2);
        if (s_ok) {
            if (fwd)
                fwd_finish<K>(A, nd, smem, s_kids);
            else
                bwd_finish<K>(A, nd, smem);
        }
        __syncthreads();
        CH_TRACE(tk, 3);
#ifdef TP_CHOL_TRACE
        if (tid == 0 && A.trace) A.trace[(size_t)tk * 6 + 4] = blockIdx.x, A.trace[(size_t)tk * 6 + 5] = J;
#endif
        if (tid == 0) {
            if (fwd) {
                st_release(A.fdone + J, ep);
            } else {
                st_release(A.bdone + J, ep);
                atomicAdd(&ctl->bcount, 1u);
            }
            s_tk = (int)next;
        }
        __syncthreads();
    }
    // r = bp - C x once every backward step is done; per-block sums of r.r
    CH_TRACE(2 * nn + blockIdx.x, 0);
    if (tid == 0) s_ok = wait_until(&ctl->bcount, (unsigned)nn, true, ctl);
    __syncthreads();
    CH_TRACE(2 * nn + blockIdx.x, 1);
    // one thread per (vertex, column): the block covers R = (CHS_T / K) K
    // consecutive entries and the grid stride is a multiple of K, so thread
    // t always holds column t % K and the block's column sums are taken in a
    // fixed order
    constexpr int R = (CHS_T / K) * K;
    double acc = 0.0;
    if (tid < R) {
        const size_t total = (size_t)A.nv * K;
        for (size_t i = (size_t)blockIdx.x * R + tid; i < total; i += (size_t)gridDim.x * R) {
            const int v = (int)(i / K), c = (int)(i - (size_t)v * K);
            double rs = A.bp[i];
            for (int e = A.rowptr[v]; e < A.rowptr[v + 1]; ++e) rs -= A.val[e] * __ldcg(A.x + (size_t)A.col[e] * K + c);
            A.r[i] = rs;
            acc += rs * rs;
        }
    }
    s_red[tid] = acc;
    __syncthreads();
    if (tid < K) {
        double sum = 0.0;
        for (int q = tid; q < R; q += K) sum += s_red[q];
        A.part[(size_t)blockIdx.x * K + tid] = sum;
    }
    CH_TRACE(2 * nn + blockIdx.x, 2);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last block: convergence test (every column at |r|^2 <= tol^2 |b|^2;
    // a column that has not lost three quarters of |r|^2 in the sweep means
    // the FP32 factor is too coarse: stalled), reset
    __threadfence();
    __shared__ double s_rr[K];
    {
        // column c: lanes of warp c % 8 stride over the blocks' partials,
        // then a fixed butterfly
        const int lane = tid & 31, wp = tid >> 5;
        for (int c = wp; c < K; c += CHS_T / 32) {
            double sum = 0.0;
            for (unsigned b = lane; b < gridDim.x; b += 32) sum += __ldcg(A.part + (size_t)b * K + c);
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) s_rr[c] = sum;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int conv = 1, worse = 0;
        for (int j = 0; j < K; ++j) {
            const double rr = s_rr[j];
            if (!(rr <= A.tol2 * ctl->bb[j])) {
                conv = 0;
                if (!(rr <= 0.25 * ctl->rr[j])) worse = 1;
            }
            ctl->rr[j] = rr;
        }
        ctl->iters += 1;
        if (conv) {
            ctl->done = 1;
        } else if (worse || ctl->bad_pivot || ctl->err || ctl->iters >= A.cap) {
            ctl->done = 1;
            ctl->stalled = 1;
        }
        CH_TRACE(2 * nn + gridDim.x, 0);
        ctl->ticket = 0;
        ctl->arrive = 0;
        ctl->bcount = 0;
        __threadfence();
        ctl->epoch = ep;
    }
}

// sums over the T threads of a block of K per-thread FP64 values, in a fixed
// order through shared memory sh [K * T] (16 partial sums per column, then
// their sum): thread j < K returns the sum of column j, the others 0. Fewer
// FP64 additions than a shuffle tree per column (the FP64 pipe is narrow).
template <int K, int T>
__device__ __forceinline__ double block_colsum_f64(const double (&acc)[K], double* sh) {
    constexpr int P = 16;
    static_assert(K * P <= T, "one thread per partial sum");
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < K; ++j) sh[j * T + t] = acc[j];
    __syncthreads();
    double s = 0.0;
    if (t < K * P) {
        const int j = t / P, q = t - j * P;
#pragma unroll
        for (int i = q; i < T; i += P) s += sh[j * T + i];
    }
    __syncthreads();
    if (t < K * P) sh[t] = s;
    __syncthreads();
    double v = 0.0;
    if (t < K)
#pragma unroll
        for (int q = 0; q < P; ++q) v += sh[t * P + q];
    return v;
}

// The start of a solve in one launch: bp = b minus its per-component means
// (mean, from k_comp_mean), x = 0, r = bp, per-block partials of |bp|^2;
// the last block to finish (completion ticket) adds the partials in block
// order, records |b|^2 per column (done when every column is zero), then
// puts the ticket back.
template <int K>
__global__ void __launch_bounds__(CHR_T)
k_chol_start(const double* __restrict__ b, const double* __restrict__ mean, const int* __restrict__ comp_of, int nv,
             double* __restrict__ bp, double* __restrict__ x, double* __restrict__ r, double* __restrict__ part,
             unsigned* __restrict__ ticket, CholCtl* __restrict__ ctl) {
    __shared__ double sh[K * CHR_T];
    __shared__ bool last;
    double acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = 0.0;
    for (int v = blockIdx.x * CHR_T + threadIdx.x; v < nv; v += gridDim.x * CHR_T) {
        const double* mc = mean + (size_t)comp_of[v] * K;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const size_t o = (size_t)v * K + c;
            const double s = b[o] - mc[c];
            bp[o] = s;
            x[o] = 0.0;
            r[o] = s;
            acc[c] += s * s;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double bs = block_colsum_f64<K, CHR_T>(acc, sh);
    if (threadIdx.x < K) part[(size_t)blockIdx.x * K + threadIdx.x] = bs;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double s_bb[K];
    for (int c = w; c < K; c += CHR_T / 32) {   // one warp per column
        double t = 0.0;
        for (unsigned q = lane; q < gridDim.x; q += 32) t += __ldcg(part + (size_t)q * K + c);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_bb[c] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int j = 0; j < K; ++j) {
            ctl->bb[j] = s_bb[j];
            ctl->rr[j] = s_bb[j];
            all &= s_bb[j] == 0.0;
        }
        ctl->done = all;
        ctl->iters = 0;
        *ticket = 0u;
    }
}

// per-component means of the k columns in a fixed order: block (c, s)
// sums slice s of component c's vertex list (CH_MSPLIT slices), then the
// last block to finish adds every component's slices in order (and, given
// dflags, records the state of the deferred solve that produced x)
constexpr int CH_MSPLIT = 48;   // about one vertex per thread on 10k-vertex meshes

__global__ void __launch_bounds__(256)
k_comp_mean(const int* __restrict__ comp_ptr, const int* __restrict__ comp_verts, const double* __restrict__ x,
            int k, double* __restrict__ part, double* __restrict__ mean, unsigned* __restrict__ ticket,
            const CholCtl* __restrict__ ctl, int* __restrict__ dflags) {
    __shared__ double sh[CH_KMAX * 256];
    __shared__ bool last;
    const int c = blockIdx.x, s = blockIdx.y;
    const int v0 = comp_ptr[c], v1 = comp_ptr[c + 1];
    const int len = (v1 - v0 + CH_MSPLIT - 1) / CH_MSPLIT;
    const int a0 = v0 + s * len, a1 = min(v1, a0 + len);
    double acc[CH_KMAX];
#pragma unroll
    for (int j = 0; j < CH_KMAX; ++j) acc[j] = 0.0;
    for (int i = a0 + threadIdx.x; i < a1; i += 256) {
        const double* xv = x + (size_t)comp_verts[i] * k;
#pragma unroll
        for (int j = 0; j < CH_KMAX; ++j)
            if (j < k) acc[j] += xv[j];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double bs = block_colsum_f64<CH_KMAX, 256>(acc, sh);
    if (threadIdx.x < k) part[((size_t)c * CH_MSPLIT + s) * k + threadIdx.x] = bs;
    // the last block to finish adds each component's slices in order and
    // resets the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // one warp per (component, column): lane l takes slices l, l + 32, then
    // a fixed shuffle tree
    const int ncomp = gridDim.x;
    for (int e = w; e < ncomp * k; e += 256 / 32) {
        const int cc = e / k, j = e - cc * k;
        double t = 0.0;
        for (int q = lane; q < CH_MSPLIT; q += 32) t += __ldcg(part + ((size_t)cc * CH_MSPLIT + q) * k + j);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) mean[(size_t)cc * k + j] = t / (double)(comp_ptr[cc + 1] - comp_ptr[cc]);
    }
    if (threadIdx.x == 0) {
        *ticket = 0u;
        if (dflags) {
            // after the sweeps of a deferred solve: its wait error, and whether
            // it stopped short of the tolerance
            if (ctl->err) dflags[0] = 1;
            if (!ctl->done || ctl->stalled) dflags[1] = 1;
        }
    }
}

__global__ void k_comp_sub(const int* __restrict__ comp_of, const double* __restrict__ mean, int nv, int k,
                           const double* __restrict__ src, double* __restrict__ dst) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nv * k) return;
    const int v = (int)(i / k), j = (int)(i - (size_t)v * k);
    dst[i] = src[i] - mean[(size_t)comp_of[v] * k + j];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

void chol_release(tp_mesh* m) {
    if (!m->chol) return;
    CholState* c = m->chol;
    Buf* all[] = {&c->nodes, &c->level_nodes, &c->child_idx, &c->rel, &c->struct_pos, &c->asm_dst,
                  &c->asm_src, &c->perm, &c->comp_ptr, &c->comp_verts, &c->comp_of, &c->parent, &c->fdone,
                  &c->bdone, &c->L, &c->U,
                  &c->uvec, &c->ybuf, &c->xbuf, &c->ctl, &c->part, &c->x, &c->r, &c->bp, &c->dflags};
    for (Buf* b : all) release(*b);
    for (auto& g : c->graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->capture) cudaStreamDestroy(c->capture);
    delete c;
    m->chol = nullptr;
}

void chol_invalidate(tp_mesh* m) {
    if (m->chol) {
        m->chol->factored = false;
        m->chol->pivot_known = false;
    }
}

int chol_deferred_flags(tp_mesh* m, cudaStream_t st, int* err, int* unconverged, bool reset) {
    *err = *unconverged = 0;
    CholState* c = m->chol;
    if (!c || !c->dflags.ptr) return TP_OK;
    if (!reset) {
        int h[2] = {0, 0};
        TP_CUDA(cudaMemcpyAsync(h, c->dflags.ptr, sizeof(h), cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
        *err = h[0];
        *unconverged = h[1];
    }
    TP_CUDA(cudaMemsetAsync(c->dflags.ptr, 0, 2 * sizeof(int), st));
    return TP_OK;
}

template <class T>
static int upload(Buf& b, const std::vector<T>& v) {
    TP_TRY(ensure(b, sizeof(T) * std::max<size_t>(1, v.size())));
    if (!v.empty()) TP_CUDA(cudaMemcpy(b.ptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return TP_OK;
}

template <int K>
static int solve_smem_attr() {
    TP_CUDA(cudaFuncSetAttribute(k_chol_sweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CH_SMEM_MAX));
    if constexpr (K < CH_KMAX) return solve_smem_attr<K + 1>();
    return TP_OK;
}

// symbolic analysis and device tables (once per mesh)
static int chol_setup(tp_mesh* m) {
    if (m->chol) return TP_OK;
    std::unique_ptr<CholState> c(new CholState());
    const int nv = m->nv;
    std::vector<int> rowptr(nv + 1), col(m->nnz);
    TP_CUDA(cudaMemcpy(rowptr.data(), m->rowptr.ptr, sizeof(int) * (nv + 1), cudaMemcpyDeviceToHost));
    TP_CUDA(cudaMemcpy(col.data(), m->col.ptr, sizeof(int) * m->nnz, cudaMemcpyDeviceToHost));
    CholSymbolic& S = c->S;
    if (!chol_analyze(nv, rowptr.data(), col.data(), CH_LEAF, S)) {
        c->why = "empty pattern";
        m->chol = c.release();
        return TP_OK;
    }
    c->ncomp = S.ncomp;
    c->H = (int)S.level_ptr.size() - 1;
    c->lvl_max_t.assign(c->H, 0);
    c->lvl_max_n.assign(c->H, 0);
    c->lvl_max_m.assign(c->H, 0);
    c->lvl_factor_smem.assign(c->H, 0);
    c->lvl_solve_smem.assign(c->H, 0);
    c->lvl_factor_flops.assign(c->H, 0.0);
    size_t worst = 0;
    for (int h = 0; h < c->H; ++h)
        for (int i = S.level_ptr[h]; i < S.level_ptr[h + 1]; ++i) {
            const int J = S.level_nodes[i];
            const double n = S.nJ[J], mm = S.mJ[J];
            c->lvl_max_t[h] = std::max(c->lvl_max_t[h], S.nJ[J] + S.mJ[J]);
            c->lvl_max_n[h] = std::max(c->lvl_max_n[h], S.nJ[J]);
            c->lvl_max_m[h] = std::max(c->lvl_max_m[h], S.mJ[J]);
            const size_t sm = sizeof(float) * ((size_t)(S.nJ[J] + S.mJ[J]) * S.nJ[J] + (size_t)S.nJ[J] * S.nJ[J]);
            c->lvl_factor_smem[h] = std::max(c->lvl_factor_smem[h], sm);
            // factor block (rounded to 16 bytes), the vectors (rows of 12
            // floats for up to 9 columns), the 128-row scratch, the node's
            // FP64 solution entries, then the staged rows and update vectors
            // of the children or struct(J) (see StepSmem)
            size_t csum = 0;   // rows of the children's update vectors
            for (int ci = S.child_ptr[J]; ci < S.child_ptr[J + 1]; ++ci) csum += S.mJ[S.child_idx[ci]];
            const size_t ss = sizeof(float) * ((((size_t)S.nJ[J] * chol_ld(S.nJ[J]) +
                                                 (size_t)S.nJ[J] * chol_ld(S.mJ[J]) + 3) & ~size_t(3)) +
                                               ((size_t)S.mJ[J] + 2 * S.nJ[J]) * 12 + 128 * 12 +
                                               2 * (size_t)S.nJ[J] * CH_KMAX +
                                               std::max(csum * (CH_KMAX + 1), (size_t)S.mJ[J]));
            c->lvl_solve_smem[h] = std::max(c->lvl_solve_smem[h], ss);
            worst = std::max(worst, sm);
            // partial Cholesky, Schur update of struct x struct, triangular inverse
            c->lvl_factor_flops[h] += n * n * n / 3.0 + n * n * mm + n * mm * mm + n * n * n / 3.0;
        }
    c->solve_bytes = 2.0 * sizeof(float) * (double)S.lsize;
    size_t solve_smem = 0;
    for (int h = 0; h < c->H; ++h) solve_smem = std::max(solve_smem, c->lvl_solve_smem[h]);
    c->solve_smem = solve_smem;
    if (worst > CH_SMEM_MAX || solve_smem > CH_SMEM_MAX) {
        c->why = "a supernode panel needs " + std::to_string(worst) + " bytes of shared memory";
        m->chol = c.release();
        return TP_OK;
    }
    // device tables
    std::vector<CholNode> nodes(S.nnode);
    for (int J = 0; J < S.nnode; ++J) {
        CholNode& d = nodes[J];
        d.p0 = S.p0[J];
        d.nJ = S.nJ[J];
        d.mJ = S.mJ[J];
        d.t = S.nJ[J] + S.mJ[J];
        d.loff = S.loff[J];
        d.uoff = S.uoff[J];
        d.voff = S.voff[J];
        d.child0 = S.child_ptr[J];
        d.child1 = S.child_ptr[J + 1];
        d.s0 = S.struct_ptr[J];
        d.asm0 = S.asm_ptr[J];
        d.asm1 = S.asm_ptr[J + 1];
        d.pad0 = d.pad1 = 0;
    }
    std::vector<int> comp_ptr(S.ncomp + 1, 0), comp_verts(nv);
    for (int v = 0; v < nv; ++v) comp_ptr[S.comp[v] + 1]++;
    for (int i = 0; i < S.ncomp; ++i) comp_ptr[i + 1] += comp_ptr[i];
    {
        std::vector<int> fill(comp_ptr.begin(), comp_ptr.end() - 1);
        for (int v = 0; v < nv; ++v) comp_verts[fill[S.comp[v]]++] = v;
    }
    TP_TRY(upload(c->nodes, nodes));
    TP_TRY(upload(c->level_nodes, S.level_nodes));
    TP_TRY(upload(c->child_idx, S.child_idx));
    TP_TRY(upload(c->rel, S.rel));
    TP_TRY(upload(c->struct_pos, S.struct_pos));
    TP_TRY(upload(c->asm_dst, S.asm_dst));
    TP_TRY(upload(c->asm_src, S.asm_src));
    TP_TRY(upload(c->perm, S.perm));
    TP_TRY(upload(c->comp_ptr, comp_ptr));
    TP_TRY(upload(c->comp_verts, comp_verts));
    TP_TRY(upload(c->comp_of, S.comp));
    TP_TRY(upload(c->parent, S.parent));
    TP_TRY(ensure(c->fdone, sizeof(unsigned) * std::max(1, S.nnode)));
    TP_TRY(ensure(c->bdone, sizeof(unsigned) * std::max(1, S.nnode)));
    TP_CUDA(cudaMemset(c->fdone.ptr, 0, sizeof(unsigned) * std::max(1, S.nnode)));
    TP_CUDA(cudaMemset(c->bdone.ptr, 0, sizeof(unsigned) * std::max(1, S.nnode)));
    TP_TRY(ensure(c->L, sizeof(float) * std::max<int64_t>(1, S.lsize)));
    TP_TRY(ensure(c->U, sizeof(float) * std::max<int64_t>(1, S.usize)));
    TP_TRY(ensure(c->uvec, sizeof(float) * (size_t)std::max(1, S.vsize) * CH_KMAX));
    TP_TRY(ensure(c->ybuf, sizeof(float) * (size_t)std::max(1, S.n) * CH_KMAX));
    TP_TRY(ensure(c->xbuf, sizeof(float) * (size_t)std::max(1, S.n) * CH_KMAX));
    TP_TRY(ensure(c->ctl, sizeof(CholCtl)));
    TP_CUDA(cudaMemset(c->ctl.ptr, 0, sizeof(CholCtl)));
#ifdef TP_CHOL_TRACE
    TP_TRY(ensure(c->trace, sizeof(unsigned long long) * 6 * ((size_t)2 * S.nnode + 2 * sm_count() + 2)));
#endif
    TP_CUDA(cudaFuncSetAttribute(k_chol_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CH_SMEM_MAX));
    TP_TRY(solve_smem_attr<1>());
    c->ok = true;
    m->chol = c.release();
    return TP_OK;
}

static int chol_factor(tp_mesh* m, cudaStream_t st) {
    CholState* c = m->chol;
    if (c->factored) return TP_OK;
    TP_CUDA(cudaMemsetAsync(c->ctl.ptr, 0, offsetof(CholCtl, epoch), st));   // the epoch is never cleared
    double flops = 0.0;
    for (double f : c->lvl_factor_flops) flops += f;
    {
        ProfScope ps(m, PK_CHOL_FACTOR, flops, st);
        const CholSymbolic& S = c->S;
        for (int h = 0; h < c->H; ++h) {
            const int cnt = S.level_ptr[h + 1] - S.level_ptr[h];
            if (cnt == 0) continue;
            k_chol_factor<<<cnt, CHF_T, c->lvl_factor_smem[h], st>>>(
                c->nodes.as<CholNode>(), c->level_nodes.as<int>() + S.level_ptr[h], c->child_idx.as<int>(),
                c->rel.as<int>(), c->asm_dst.as<int>(), c->asm_src.as<int>(), m->val.as<double>(),
                c->L.as<float>(), c->U.as<float>(), c->ctl.as<CholCtl>());
            TP_LAUNCH_CHECK();
        }
    }
    c->factored = true;
    return TP_OK;
}

// dst = src minus its per-component mean (k columns)
// per-component means of src into c->part (and the deferred flags, see k_comp_mean)
static int comp_means(tp_mesh* m, const double* src, int k, int* dflags, cudaStream_t st) {
    CholState* c = m->chol;
    double* mean = c->part.as<double>();                        // ncomp * 9 doubles
    double* slices = mean + (size_t)c->ncomp * CH_KMAX;          // ncomp * CH_MSPLIT * 9 doubles
    unsigned* tk = nullptr;
    TP_TRY(mesh_tickets(m, &tk, st));
    k_comp_mean<<<dim3(c->ncomp, CH_MSPLIT), 256, 0, st>>>(c->comp_ptr.as<int>(), c->comp_verts.as<int>(), src, k,
                                                           slices, mean, tk + TICKET_COMP, c->ctl.as<CholCtl>(),
                                                           dflags);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

static int comp_project(tp_mesh* m, const double* src, double* dst, int k, cudaStream_t st, int* dflags = nullptr) {
    CholState* c = m->chol;
    double* mean = c->part.as<double>();
    TP_TRY(comp_means(m, src, k, dflags, st));
    const size_t n = (size_t)m->nv * k;
    k_comp_sub<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c->comp_of.as<int>(), mean, m->nv, k, src, dst);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

// `nsweep` refinement sweeps on stream st (recorded into a graph by the
// caller); *nk counts the kernels
template <int K>
static int chol_sweep_kernels(tp_mesh* m, int nsweep, int rgrid, double* partr, double tol2, int cap,
                              cudaStream_t st, int* nk) {
    CholState* c = m->chol;
    const CholSymbolic& S = c->S;
    SweepArgs A;
    A.nodes = c->nodes.as<CholNode>();
    A.order = c->level_nodes.as<int>();
    A.child_idx = c->child_idx.as<int>();
    A.rel = c->rel.as<int>();
    A.struct_pos = c->struct_pos.as<int>();
    A.perm = c->perm.as<int>();
    A.parent = c->parent.as<int>();
    A.L = c->L.as<float>();
    A.ybuf = c->ybuf.as<float>();
    A.xbuf = c->xbuf.as<float>();
    A.uvec = c->uvec.as<float>();
    A.fdone = c->fdone.as<unsigned>();
    A.bdone = c->bdone.as<unsigned>();
    A.rowptr = m->rowptr.as<int>();
    A.col = m->col.as<int>();
    A.val = m->val.as<double>();
    A.bp = c->bp.as<double>();
    A.x = c->x.as<double>();
    A.r = c->r.as<double>();
    A.part = partr;
    A.ctl = c->ctl.as<CholCtl>();
    A.trace = nullptr;
#ifdef TP_CHOL_TRACE
    A.trace = c->trace.as<unsigned long long>();   // allocated with the tables (no allocation under capture)
#endif
    A.tol2 = tol2;
    A.nv = m->nv;
    A.nn = S.nnode;
    A.cap = cap;
    (void)rgrid;
    const int grid = std::max(1, std::min(S.nnode, 2 * sm_count()));
    for (int s = 0; s < nsweep; ++s) {
        k_chol_sweep<K><<<grid, CHS_T, c->solve_smem, st>>>(A);
        TP_CUDA(cudaGetLastError());
        ++*nk;
    }
    return TP_OK;
}

constexpr int CH_SWEEPS_PER_GRAPH = 2;   // FP32 factor: about three digits per sweep

// the graph of CH_SWEEPS_PER_GRAPH sweeps for K columns, captured on a
// private stream (re-captured when a buffer it uses has moved)
template <int K>
static int sweep_graph(tp_mesh* m, int rgrid, double* partr, double tol2, int cap, CholState::SweepGraph** out) {
    CholState* c = m->chol;
    CholState::SweepGraph& g = c->graph[K];
    const void* key[4] = {c->x.ptr, c->r.ptr, c->bp.ptr, partr};
    bool same = g.exec && g.tol2 == tol2 && g.cap == cap && g.rgrid == rgrid;
    for (int i = 0; i < 4 && same; ++i) same = g.key[i] == key[i];
    if (!same) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        if (!c->capture) TP_CUDA(cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
        TP_CUDA(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
        int nk = 0;
        int s = chol_sweep_kernels<K>(m, CH_SWEEPS_PER_GRAPH, rgrid, partr, tol2, cap, c->capture, &nk);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->capture, &graph);
        if (s != TP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return fail(TP_ERR_CUDA, std::string("capturing the refinement sweeps: ") +
                                                           cudaGetErrorString(e));
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(TP_ERR_CUDA, std::string("instantiating the refinement sweeps: ") +
                                                           cudaGetErrorString(e));
        for (int i = 0; i < 4; ++i) g.key[i] = key[i];
        g.tol2 = tol2;
        g.cap = cap;
        g.rgrid = rgrid;
        g.kernels = nk;
    }
    *out = &g;
    return TP_OK;
}

template <int K>
static int chol_run(tp_mesh* m, const tp_params* p, const double* b, double* z_out, cudaStream_t st, int* iters,
                    bool* handed_off, bool deferred) {
    CholState* c = m->chol;
    if (deferred && !c->pivot_known) {
        // the factor's pivot check, once per factorisation
        int bp = 0;
        TP_CUDA(cudaMemcpyAsync(&bp, reinterpret_cast<char*>(c->ctl.ptr) + offsetof(CholCtl, bad_pivot), sizeof(int),
                                cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
        c->pivot_ok = bp == 0;
        c->pivot_known = true;
    }
    if (deferred && !c->pivot_ok) {
        *handed_off = true;
        return TP_OK;
    }
    const int nv = m->nv;
    const size_t n = (size_t)nv * K;
    TP_TRY(ensure(c->x, sizeof(double) * n));
    TP_TRY(ensure(c->r, sizeof(double) * n));
    TP_TRY(ensure(c->bp, sizeof(double) * n));
    const int rgrid = std::min(4 * sm_count(), (nv + CHR_T - 1) / CHR_T);
    // partial sums after the per-component means (comp_project's region)
    // per-block partials of the initial residual (rgrid blocks) and of the
    // sweep kernel (up to 2 blocks per SM)
    const size_t nparts = (size_t)std::max(rgrid, 2 * sm_count());
    const size_t head = (size_t)c->ncomp * CH_KMAX * (1 + CH_MSPLIT);   // means and their slices
    TP_TRY(ensure(c->part, sizeof(double) * (head + nparts * CH_KMAX) + 64));
    double* partr = c->part.as<double>() + head;
    // clear done .. arrive; bad_pivot (from the factorisation) and the epoch stay
    TP_CUDA(cudaMemsetAsync(c->ctl.ptr, 0, offsetof(CholCtl, bad_pivot), st));
    // b minus its component means, x = 0, r = b, |b|^2 (two launches)
    TP_TRY(comp_means(m, b, K, nullptr, st));
    {
        unsigned* tk = nullptr;
        TP_TRY(mesh_tickets(m, &tk, st));
        k_chol_start<K><<<rgrid, CHR_T, 0, st>>>(b, c->part.as<double>(), c->comp_of.as<int>(), nv, c->bp.as<double>(),
                                                c->x.as<double>(), c->r.as<double>(), partr, tk + TICKET_CHOL,
                                                c->ctl.as<CholCtl>());
        TP_LAUNCH_CHECK();
    }
    const double tol2 = p->cg_tol * p->cg_tol;
    const int cap = std::max(1, std::min(p->cg_max, 40));
    CholState::SweepGraph* g = nullptr;
    TP_TRY(sweep_graph<K>(m, rgrid, partr, tol2, cap, &g));
    if (deferred) {
        // no host read: the sweeps that cg_tol needs, then the flags; the
        // caller reads them once per step. Measured digits of |r|/|b| (9
        // columns): at least four after the first sweep (torus_20k,
        // linked_tori_50k, icosphere_l3), about three more per sweep after it.
        if (!c->dflags.ptr) {
            TP_TRY(ensure(c->dflags, 4 * sizeof(int)));
            TP_CUDA(cudaMemsetAsync(c->dflags.ptr, 0, 4 * sizeof(int), st));   // fresh memory holds garbage
        }
        const double digits = -std::log10(std::max(p->cg_tol, 1e-300));
        const int sweeps = std::min(cap, 1 + std::max(0, (int)std::ceil((digits - 4.0) / 3.0)));
        const int graphs = sweeps / CH_SWEEPS_PER_GRAPH;
        for (int gi = 0; gi < graphs; ++gi) {
            ProfScope ps(m, PK_CHOL_SOLVE, c->solve_bytes * CH_SWEEPS_PER_GRAPH, st);
            TP_CUDA(cudaGraphLaunch(g->exec, st));
            count_launches(g->kernels);
        }
        if (sweeps % CH_SWEEPS_PER_GRAPH) {
            // the odd sweep, launched directly
            ProfScope ps(m, PK_CHOL_SOLVE, c->solve_bytes, st);
            int nk = 0;
            TP_TRY(chol_sweep_kernels<K>(m, sweeps % CH_SWEEPS_PER_GRAPH, rgrid, partr, tol2, cap, st, &nk));
            count_launches(nk);
        }
        if (iters) *iters = sweeps;
        TP_TRY(comp_project(m, c->x.as<double>(), z_out, K, st, c->dflags.as<int>()));
        return TP_OK;
    }
    CholCtl h{};
    int launched = 0;
    for (;;) {
        {
            ProfScope ps(m, PK_CHOL_SOLVE, c->solve_bytes * CH_SWEEPS_PER_GRAPH, st);
            TP_CUDA(cudaGraphLaunch(g->exec, st));
            count_launches(g->kernels);
        }
        launched += CH_SWEEPS_PER_GRAPH;
        TP_CUDA(cudaMemcpyAsync(&h, c->ctl.ptr, sizeof(CholCtl), cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
        if (h.done || launched >= cap) break;
    }
    if (iters) *iters = h.iters;
    if (h.err) return fail(TP_ERR_TIMEOUT, "cotan solve: a wait of the factorised sweep gave up");
    if (h.bad_pivot || h.stalled || !h.done) {
        *handed_off = true;
        return TP_OK;
    }
    TP_TRY(comp_project(m, c->x.as<double>(), z_out, K, st));
    return TP_OK;
}

// z = C^+ b by the factor; *used = false when the factor cannot serve this
// mesh or this right-hand side (the caller then runs CG)
int chol_solve(tp_mesh* m, const tp_params* p, const double* b, int k, double* z_out, cudaStream_t st, int* iters,
               bool* used, bool deferred) {
    *used = false;
    if (k < 1 || k > CH_KMAX) return fail(TP_ERR_INVALID_ARG, "cotan solve: k must be in 1..9");
    TP_TRY(laplacian_values(m, st));
    TP_TRY(chol_setup(m));
    if (!m->chol->ok) return TP_OK;
    TP_TRY(chol_factor(m, st));
    bool handed = false;
    int it = 0;
    switch (k) {
        case 1: TP_TRY(chol_run<1>(m, p, b, z_out, st, &it, &handed, deferred)); break;
        case 2: TP_TRY(chol_run<2>(m, p, b, z_out, st, &it, &handed, deferred)); break;
        case 3: TP_TRY(chol_run<3>(m, p, b, z_out, st, &it, &handed, deferred)); break;
        case 4: TP_TRY(chol_run<4>(m, p, b, z_out, st, &it, &handed, deferred)); break;
        case 5: TP_TRY(chol_run<5>(m, p, b, z_out, st, &it, &handed, deferred)); break;
        case 6: TP_TRY(chol_run<6>(m, p, b, z_out, st, &it, &handed, deferred)); break;
        case 7: TP_TRY(chol_run<7>(m, p, b, z_out, st, &it, &handed, deferred)); break;
        case 8: TP_TRY(chol_run<8>(m, p, b, z_out, st, &it, &handed, deferred)); break;
        default: TP_TRY(chol_run<9>(m, p, b, z_out, st, &it, &handed, deferred)); break;
    }
    if (iters) *iters = it;
    *used = !handed;
    return TP_OK;
}

#ifdef TP_CHOL_TRACE
// timestamps of the last sweep (trace builds): [2 nn + blocks + 1][6]
int chol_trace(tp_mesh* m, unsigned long long* out, int max_rows, int* nn, int* grid) {
    CholState* c = m->chol;
    if (!c || !c->trace.ptr) return fail(TP_ERR_INVALID_ARG, "no trace");
    *nn = c->S.nnode;
    *grid = std::max(1, std::min(c->S.nnode, 2 * sm_count()));
    const size_t rows = std::min<size_t>((size_t)max_rows, (size_t)2 * c->S.nnode + *grid + 1);
    TP_CUDA(cudaMemcpy(out, c->trace.ptr, sizeof(unsigned long long) * 6 * rows, cudaMemcpyDeviceToHost));
    return TP_OK;
}
#endif

// host-side description of the factor (for tests and reports)
// Self-test of the bounded cross-block wait: one thread waits for a word
// that nothing sets; the wait gives up after its clock budget (~1 s),
// records the timeout in the control block and returns.
__global__ void k_wait_selftest(const unsigned* word, CholCtl* ctl, int* result) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *result = wait_until(word, 1u, true, ctl) ? 0 : 1;
}

int wait_selftest(int* timed_out) {
    void* mem = nullptr;
    const size_t bytes = 256 + sizeof(CholCtl);
    TP_CUDA(cudaMalloc(&mem, bytes));
    unsigned* word = (unsigned*)mem;
    int* result = (int*)((char*)mem + 64);
    CholCtl* ctl = (CholCtl*)((char*)mem + 256);
    int h[2] = {0, 0};
    cudaError_t e = cudaMemset(mem, 0, bytes);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(word, ctl, result);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h[0], result, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h[1], &ctl->err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(mem);
    if (e != cudaSuccess) return fail(TP_ERR_CUDA, cudaGetErrorString(e));
    *timed_out = (h[0] == 1 && h[1] != 0) ? 1 : 0;
    return *timed_out ? fail(TP_ERR_TIMEOUT, "self-test: the bounded wait gave up as designed") : TP_OK;
}

int chol_info(tp_mesh* m, tp_chol_info* out) {
    *out = tp_chol_info{};
    TP_TRY(chol_setup(m));
    const CholState* c = m->chol;
    const CholSymbolic& S = c->S;
    out->available = c->ok ? 1 : 0;
    out->components = S.ncomp;
    out->unknowns = S.n;
    out->supernodes = S.nnode;
    out->levels = c->H;
    out->max_front = S.max_t;
    out->factor_floats = (double)S.lsize;
    out->update_floats = (double)S.usize;
    return TP_OK;
}

}  // namespace tp
