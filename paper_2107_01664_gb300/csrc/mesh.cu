// Mesh state: face geometry (X_S, N_S, a_S and hat gradients), the
// face-corner -> vertex gather, copies and deterministic FP64 sums.
#include <cmath>
#include <cstring>

#include "host_util.h"
#include <mutex>

#include "tp_internal.cuh"

namespace tp {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

static thread_local tp_ctx* g_current_ctx = nullptr;

tp_ctx*& current_ctx() { return g_current_ctx; }

tp_ctx* default_ctx(int device) {
    static std::mutex mu;
    static tp_ctx* ctxs[64] = {nullptr};
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!ctxs[device]) {
        ctxs[device] = new tp_ctx();
        ctxs[device]->device = device;
        ctxs[device]->is_default = true;
    }
    return ctxs[device];
}

static void ctx_free(tp_ctx* c, void* ptr, size_t bytes) {
    if (!ptr) return;
    if (c && c->custom) {
        // the caller's allocator may hand the block to other work at once:
        // the work that used it must be over (cudaFree gives this itself)
        cudaDeviceSynchronize();
        c->al.free(ptr, bytes, c->device, c->al.user);
    } else {
        cudaFree(ptr);
    }
    if (c) c->in_use -= (long long)bytes;
}

int ensure(Buf& b, size_t bytes) {
    if (bytes <= b.bytes && b.ptr) return TP_OK;
    ctx_free(b.ctx, b.ptr, b.bytes);
    b.ptr = nullptr;
    b.bytes = 0;
    b.ctx = nullptr;
    size_t want = bytes < 256 ? 256 : (bytes + 255) / 256 * 256;
    tp_ctx* c = current_ctx();
    if (c && c->custom) {
        b.ptr = c->al.alloc(want, c->device, c->al.user);
        if (!b.ptr)
            return fail(TP_ERR_OOM, "the context's allocator returned NULL for " + std::to_string(want) + " bytes");
        if (reinterpret_cast<uintptr_t>(b.ptr) % 256 != 0) {
            c->al.free(b.ptr, want, c->device, c->al.user);
            b.ptr = nullptr;
            return fail(TP_ERR_INVALID_ARG, "the context's allocator returned memory not aligned to 256 bytes");
        }
    } else {
        cudaError_t e = cudaMalloc(&b.ptr, want);
        if (e != cudaSuccess) {
            b.ptr = nullptr;
            cudaGetLastError();
            return fail(TP_ERR_OOM, std::string("cudaMalloc(") + std::to_string(want) +
                                        "): " + cudaGetErrorString(e));
        }
    }
    b.bytes = want;
    b.ctx = c;
    if (c) {
        const long long now = (c->in_use += (long long)want);
        long long pk = c->peak.load();
        while (now > pk && !c->peak.compare_exchange_weak(pk, now)) {
        }
    }
    return TP_OK;
}

void release(Buf& b) {
    ctx_free(b.ctx, b.ptr, b.bytes);
    b.ptr = nullptr;
    b.bytes = 0;
    b.ctx = nullptr;
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 132;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 132;
    }
    return cached[dev];
}

int copy_in(void* dst, const void* src, size_t bytes, int ptr_kind, cudaStream_t st) {
    if (bytes == 0) return TP_OK;
    TP_CUDA(cudaMemcpyAsync(dst, src, bytes,
                            ptr_kind == TP_PTR_HOST ? cudaMemcpyHostToDevice
                                                    : cudaMemcpyDeviceToDevice,
                            st));
    return TP_OK;
}

int copy_out(void* dst, const void* src, size_t bytes, int ptr_kind, cudaStream_t st) {
    if (bytes == 0) return TP_OK;
    TP_CUDA(cudaMemcpyAsync(dst, src, bytes,
                            ptr_kind == TP_PTR_HOST ? cudaMemcpyDeviceToHost
                                                    : cudaMemcpyDeviceToDevice,
                            st));
    if (ptr_kind == TP_PTR_HOST) TP_CUDA(cudaStreamSynchronize(st));
    return TP_OK;
}

// ---------------------------------------------------------------------------
// deterministic column sums of a row-major [n][k] FP64 array (k <= 64)
// ---------------------------------------------------------------------------

static constexpr int kSumThreads = 256;

// Block b sums rows [b * rows_per_block, ...) of every column into
// part[b][c]: thread t < (256 / k) k reads the flat elements t, t + (256 / k) k,
// ... of the block's rows (coalesced; all of one column), then eight partial
// sums per column and their sum in a fixed order. The last block to finish
// (completion ticket) adds the block sums the same way, in block order, into
// out[c] (times scale) and puts the ticket back to zero, so the result does
// not depend on which block finished last. k <= 64.
__device__ __forceinline__ double colsum_fold(double* sh, int k, int per, double s) {
    const int t = threadIdx.x;
    const int np = per < 8 ? per : 8;          // partial sums per column
    sh[t] = s;
    __syncthreads();
    double s1 = 0.0;
    if (t < np * k) {
        const int c = t % k, q = t / k;
        for (int i = q; i < per; i += np) s1 += sh[i * k + c];
    }
    __syncthreads();
    if (t < np * k) sh[t] = s1;
    __syncthreads();
    double v = 0.0;
    if (t < k)
        for (int q = 0; q < np; ++q) v += sh[q * k + t];
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(256)
k_colsum(const double* __restrict__ x, long n, int k, int rows_per_block, double* __restrict__ part,
         double scale, double* __restrict__ out, unsigned* __restrict__ ticket) {
    __shared__ double sh[kSumThreads];
    __shared__ bool last;
    const int t = threadIdx.x;
    const int per = kSumThreads / k, tk = per * k;
    const long r0 = (long)blockIdx.x * rows_per_block;
    const long r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
    double s = 0.0;
    if (t < tk) {
        const long e1 = r1 * k;
#pragma unroll 4
        for (long e = r0 * k + t; e < e1; e += tk) s += x[e];
    }
    const double v = colsum_fold(sh, k, per, s);
    if (t < k) part[(long)blockIdx.x * k + t] = v;
    if (t == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // block sums: thread t < tk takes blocks t / k, t / k + per, ... of column t % k
    const int nblk = gridDim.x;
    double sb = 0.0;
    if (t < tk)
        for (int b = t / k; b < nblk; b += per) sb += __ldcg(part + (long)b * k + t % k);
    const double tot = colsum_fold(sh, k, per, sb);
    if (t < k) out[t] = tot * scale;
    if (t == 0) *ticket = 0u;
}

// completion tickets of the fused reductions, zero between launches (the
// last block of a launch puts its ticket back)
int mesh_tickets(tp_mesh* m, unsigned** out, cudaStream_t st) {
    if (!m->tickets.ptr) {
        TP_TRY(ensure(m->tickets, TICKET_COUNT * sizeof(unsigned)));
        TP_CUDA(cudaMemsetAsync(m->tickets.ptr, 0, TICKET_COUNT * sizeof(unsigned), st));
    }
    *out = m->tickets.as<unsigned>();
    return TP_OK;
}

// column sums (times `scale`) of x [n][k] into out_dev [k]; uses m->part2
int colsum(tp_mesh* m, const double* x, long n, int k, double scale, double* out_dev,
                  cudaStream_t st) {
    if (k < 1 || k > 64) return fail(TP_ERR_INVALID_ARG, "colsum: 1 to 64 columns");
    // about 2,048 elements per block (8 per thread), at most two blocks per SM
    long nb = (n * k + 2047) / 2048;
    const long cap = 2L * sm_count();
    int nblk = (int)(nb < 1 ? 1 : (nb > cap ? cap : nb));
    int rpb = (int)((n + nblk - 1) / nblk);
    if (rpb < 1) rpb = 1;
    TP_TRY(ensure(m->part2, sizeof(double) * (size_t)nblk * k));
    unsigned* tk = nullptr;
    TP_TRY(mesh_tickets(m, &tk, st));
    k_colsum<<<nblk, kSumThreads, 0, st>>>(x, n, k, rpb, m->part2.as<double>(), scale, out_dev, tk + TICKET_COLSUM);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

int sum_f64(const double* x, int n, double* out_dev, tp_mesh* m, cudaStream_t st) {
    return colsum(m, x, n, 1, 1.0, out_dev, st);
}

// ---------------------------------------------------------------------------
// face geometry, §3.1 / §3.2.1
// ---------------------------------------------------------------------------

__global__ void k_face_geom(const double* __restrict__ pos, const int* __restrict__ faces, int nf,
                            const double* __restrict__ center, float4* __restrict__ f32a,
                            float4* __restrict__ f32b, float4* __restrict__ f32c, d4* __restrict__ f64a,
                            d4* __restrict__ f64b, double* __restrict__ fgrad, int* __restrict__ err) {
    int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S >= nf) return;
    int i = faces[3 * S], j = faces[3 * S + 1], k = faces[3 * S + 2];
    double pi[3], pj[3], pk[3];
    for (int c = 0; c < 3; ++c) {
        pi[c] = pos[3 * i + c];
        pj[c] = pos[3 * j + c];
        pk[c] = pos[3 * k + c];
    }
    double e1[3] = {pj[0] - pi[0], pj[1] - pi[1], pj[2] - pi[2]};
    double e2[3] = {pk[0] - pi[0], pk[1] - pi[1], pk[2] - pi[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                   e1[0] * e2[1] - e1[1] * e2[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    bool ok = nn > 0.0 && isfinite(nn);
    for (int c = 0; c < 3; ++c) ok = ok && isfinite(pi[c]) && isfinite(pj[c]) && isfinite(pk[c]);
    if (!ok) {
        atomicOr(err, 1);
        nn = 1.0;
    }
    double a = 0.5 * nn;
    double N[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
    double X[3];
    for (int c = 0; c < 3; ++c) X[c] = (pi[c] + pj[c] + pk[c]) / 3.0 - center[c];
    f64a[S] = d4{X[0], X[1], X[2], a};
    f64b[S] = d4{N[0], N[1], N[2], 0.0};
    f32a[S] = make_float4((float)X[0], (float)X[1], (float)X[2], (float)a);
    f32c[S] = make_float4((float)(X[0] - (double)(float)X[0]), (float)(X[1] - (double)(float)X[1]),
                          (float)(X[2] - (double)(float)X[2]), 0.0f);
    f32b[S] = make_float4((float)N[0], (float)N[1], (float)N[2], 0.0f);
    // hat gradients: grad phi_c = N x e_c / (2a), e_c the edge opposite corner c
    const double* P[3] = {pi, pj, pk};
    for (int c = 0; c < 3; ++c) {
        const double* p1 = P[(c + 1) % 3];
        const double* p2 = P[(c + 2) % 3];
        double e[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
        double g[3] = {N[1] * e[2] - N[2] * e[1], N[2] * e[0] - N[0] * e[2],
                       N[0] * e[1] - N[1] * e[0]};
        for (int q = 0; q < 3; ++q) fgrad[9 * S + 3 * c + q] = g[q] / (2.0 * a);
    }
}

// bounding box of the vertices: per-block min/max, then the centre (lo+hi)/2
__global__ void k_pos_bbox_partial(const double* __restrict__ pos, int nv, double* __restrict__ part) {
    __shared__ double lo[3][256], hi[3][256];
    double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
    for (int i = blockIdx.x * 256 + threadIdx.x; i < nv; i += gridDim.x * 256)
        for (int c = 0; c < 3; ++c) {
            l[c] = fmin(l[c], pos[3 * i + c]);
            h[c] = fmax(h[c], pos[3 * i + c]);
        }
    for (int c = 0; c < 3; ++c) {
        lo[c][threadIdx.x] = l[c];
        hi[c][threadIdx.x] = h[c];
    }
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) {
                lo[c][threadIdx.x] = fmin(lo[c][threadIdx.x], lo[c][threadIdx.x + w]);
                hi[c][threadIdx.x] = fmax(hi[c][threadIdx.x], hi[c][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            part[6 * blockIdx.x + c] = lo[c][0];
            part[6 * blockIdx.x + 3 + c] = hi[c][0];
        }
}

__global__ void k_pos_bbox_center(const double* __restrict__ part, int nblk, double* __restrict__ center) {
    if (threadIdx.x != 0) return;
    double half[3];
    for (int c = 0; c < 3; ++c) {
        double l = 1e300, h = -1e300;
        for (int b = 0; b < nblk; ++b) {
            l = fmin(l, part[6 * b + c]);
            h = fmax(h, part[6 * b + 3 + c]);
        }
        center[c] = 0.5 * (l + h);
        half[c] = 0.5 * (h - l);
    }
    // source tiles closer than R/16 to a target block (R = half diagonal of
    // the bounding box) take the compensated barycenter difference: beyond
    // it the FP32 rounding of the barycenters perturbs |d| by < 2^-19
    double R2 = half[0] * half[0] + half[1] * half[1] + half[2] * half[2];
    center[3] = R2 / 256.0;
}

// bounding box of the FP32 barycenters of each tile of 128 consecutive faces
__global__ void k_tile_boxes(const float4* __restrict__ f32a, int nf, float4* __restrict__ box) {
    __shared__ float lo[3][128], hi[3][128];
    int S = blockIdx.x * 128 + threadIdx.x;
    float4 x = S < nf ? f32a[S] : f32a[blockIdx.x * 128];
    lo[0][threadIdx.x] = hi[0][threadIdx.x] = x.x;
    lo[1][threadIdx.x] = hi[1][threadIdx.x] = x.y;
    lo[2][threadIdx.x] = hi[2][threadIdx.x] = x.z;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) {
                lo[c][threadIdx.x] = fminf(lo[c][threadIdx.x], lo[c][threadIdx.x + w]);
                hi[c][threadIdx.x] = fmaxf(hi[c][threadIdx.x], hi[c][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        box[2 * blockIdx.x] = make_float4(lo[0][0], lo[1][0], lo[2][0], 0.f);
        box[2 * blockIdx.x + 1] = make_float4(hi[0][0], hi[1][0], hi[2][0], 0.f);
    }
}

// connected components through the face edges (host_util.h)
int components_setup(tp_mesh* m, const std::vector<int>& F) {
    const int nv = m->nv;
    const int nc = label_components(nv, F, m->comp_host);
    m->ncomp = nc;
    std::vector<int> ptr(nc + 1, 0), verts(nv);
    for (int v = 0; v < nv; ++v) ptr[m->comp_host[v] + 1]++;
    for (int c = 0; c < nc; ++c) ptr[c + 1] += ptr[c];
    {
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int v = 0; v < nv; ++v) verts[fill[m->comp_host[v]]++] = v;
    }
    TP_TRY(ensure(m->vcomp, sizeof(int) * (size_t)nv));
    TP_TRY(ensure(m->comp_ptr, sizeof(int) * (size_t)(nc + 1)));
    TP_TRY(ensure(m->comp_verts, sizeof(int) * (size_t)nv));
    TP_CUDA(cudaMemcpy(m->vcomp.ptr, m->comp_host.data(), sizeof(int) * (size_t)nv, cudaMemcpyHostToDevice));
    TP_CUDA(cudaMemcpy(m->comp_ptr.ptr, ptr.data(), sizeof(int) * (size_t)(nc + 1), cudaMemcpyHostToDevice));
    TP_CUDA(cudaMemcpy(m->comp_verts.ptr, verts.data(), sizeof(int) * (size_t)nv, cudaMemcpyHostToDevice));
    return TP_OK;
}

// mean[c][j] of column j over component c (one block per (c, j), fixed order)
__global__ void k_comp_mean(const int* __restrict__ ptr, const int* __restrict__ verts, const double* __restrict__ x,
                            int k, double* __restrict__ mean) {
    const int c = blockIdx.x, j = blockIdx.y;
    __shared__ double red[256];
    double s = 0.0;
    for (int e = ptr[c] + threadIdx.x; e < ptr[c + 1]; e += blockDim.x) s += x[(size_t)verts[e] * k + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[(size_t)c * k + j] = red[0] / (double)(ptr[c + 1] - ptr[c]);
}

__global__ void k_comp_remove(const int* __restrict__ vcomp, int nv, int k, const double* __restrict__ mean,
                              double* __restrict__ x) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nv * k) return;
    x[i] -= mean[(size_t)vcomp[i / k] * k + (i % k)];
}

int project_components(tp_mesh* m, double* x, int k, cudaStream_t st) {
    TP_TRY(ensure(m->part2, sizeof(double) * (size_t)m->ncomp * k));
    double* mean = m->part2.as<double>();
    k_comp_mean<<<dim3(m->ncomp, k), 256, 0, st>>>(m->comp_ptr.as<int>(), m->comp_verts.as<int>(), x, k, mean);
    TP_LAUNCH_CHECK();
    const size_t n = (size_t)m->nv * k;
    k_comp_remove<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->vcomp.as<int>(), m->nv, k, mean, x);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

int refresh_geometry(tp_mesh* m, cudaStream_t st) {
    // reference frame: centre of the vertices' bounding box (exact in FP64),
    // so that the FP32 face table holds barycenters relative to the mesh
    {
        int nblk = (m->nv + 255) / 256;
        if (nblk > 256) nblk = 256;
        TP_TRY(ensure(m->part2, sizeof(double) * 6 * (size_t)nblk));
        k_pos_bbox_partial<<<nblk, 256, 0, st>>>(m->pos.as<double>(), m->nv, m->part2.as<double>());
        TP_LAUNCH_CHECK();
        k_pos_bbox_center<<<1, 32, 0, st>>>(m->part2.as<double>(), nblk, m->center.as<double>());
        TP_LAUNCH_CHECK();
    }
    TP_CUDA(cudaMemsetAsync(m->errflag.ptr, 0, sizeof(int) * 4, st));
    int nb = (m->nf + 255) / 256;
    k_face_geom<<<nb, 256, 0, st>>>(m->pos.as<double>(), m->faces.as<int>(), m->nf,
                                    m->center.as<double>(), m->f32a.as<float4>(),
                                    m->f32b.as<float4>(), m->f32c.as<float4>(), m->f64a.as<d4>(),
                                    m->f64b.as<d4>(), m->fgrad.as<double>(), m->errflag.as<int>());
    TP_LAUNCH_CHECK();
    {
        int ntiles = (m->nf + 127) / 128;
        TP_TRY(ensure(m->tilebox, sizeof(float4) * 2 * (size_t)ntiles));
        k_tile_boxes<<<ntiles, 128, 0, st>>>(m->f32a.as<float4>(), m->nf, m->tilebox.as<float4>());
        TP_LAUNCH_CHECK();
    }
    TP_TRY(obstacle_frame(m, st));   // the frame moved with the positions
    int err = 0;
    TP_CUDA(cudaMemcpyAsync(&err, m->errflag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    m->lap_valid = false;
    m->gself_valid = false;
    m->wm_valid = false;
    m->pin_valid = false;
    chol_invalidate(m);
    m->bvh_valid = false;
    if (err) return fail(TP_ERR_DEGENERATE, "zero-area face or non-finite position");
    return TP_OK;
}

// ---------------------------------------------------------------------------
// face corners -> vertices (deterministic CSR gather, no atomics)
// ---------------------------------------------------------------------------

// one thread per (vertex, column): the vertex's corners in CSR order (a fixed
// order), the 9 threads of a vertex reading one corner row together
__global__ void k_gather(const double* __restrict__ corner, const int* __restrict__ vf_ptr,
                         const int* __restrict__ vf_idx, int nv, int k, double* __restrict__ y) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nv * k) return;
    const int v = (int)(t / k), c = (int)(t - (long)v * k);
    const int e0 = vf_ptr[v], e1 = vf_ptr[v + 1];
    double s = 0.0;
    for (int e = e0; e < e1; ++e) s += corner[(long)vf_idx[e] * k + c];
    y[t] = s;
}

int corners_to_vertices(tp_mesh* m, const double* corner, int k, double* y, cudaStream_t st) {
    const long n = (long)m->nv * k;
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_gather<<<nb, 256, 0, st>>>(corner, m->vf_ptr.as<int>(), m->vf_idx.as<int>(), m->nv, k, y);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

}  // namespace tp

// ---------------------------------------------------------------------------
// launch counting and per-mesh kernel statistics
// ---------------------------------------------------------------------------

#include <atomic>

namespace tp {

static std::atomic<unsigned long long> g_launches{0};

void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }

ProfScope::ProfScope(tp_mesh* m_, int key_, double units, cudaStream_t st_) : m(m_), key(key_), st(st_) {
    Profiler& P = m->prof;
    P.launches[key] += 1;
    P.units[key] += units;
    if (!P.on) return;
    for (cudaEvent_t* e : {&e0, &e1}) {
        if (!P.pool.empty()) {
            *e = P.pool.back();
            P.pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            *e = nullptr;
        }
    }
    if (e0) cudaEventRecord(e0, st);
}

ProfScope::~ProfScope() {
    if (!e0 || !e1) return;
    cudaEventRecord(e1, st);
    m->prof.pending.push_back({key, {e0, e1}});
}

void prof_release(tp_mesh* m) {
    Profiler& P = m->prof;
    for (auto& pe : P.pending) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (auto e : P.pool) cudaEventDestroy(e);
    P.pending.clear();
    P.pool.clear();
}

}  // namespace tp
