// tp_energy_noalloc: the direct energy for callers that cannot allocate
// device memory.
//
// Some callers are not allowed to call cudaMalloc: plug-ins running inside a
// host program that owns the device allocator and forbids side allocations,
// and real-time loops that must not block on the allocator's locks or risk an
// out-of-memory failure in the middle of a run. This entry point computes the
// same quantity as tp_energy with theta = 0 (Eq. 10, ordered pairs, FP32 pair
// terms, compensated sums, FP64 reduction) from caller-owned device arrays,
// and keeps every intermediate in one fixed static device array of this file.
//
// The static array is sized for NA_MAX_FACES faces (5,767,232 bytes, 5.5 MiB)
// and is held by every GPU that loads the library until the process exits.
// Every call shares it: calls whose kernels overlap on the GPU (two streams,
// two host threads) race and must be serialised by the caller. The array
// keeps the last call's contents. The only entry that must start at zero,
// the bad-index flag, is cleared by the first kernel of each call; every
// other entry a call reads was written earlier in the same call.
#include <mutex>

#include "tp_internal.cuh"

namespace {

constexpr int NA_MAX_FACES = 32768;   // largest mesh accepted
constexpr int NA_T = 128;             // threads per block = faces per source tile
constexpr int NA_MAX_SPLIT = 16;      // source splits of the pair kernel
constexpr int NA_CH = 32;             // sources per FP32 run before the compensated add

struct NoAllocScratch {
    float4 xa[NA_MAX_FACES];   // X - c (hi), a
    float4 xl[NA_MAX_FACES];   // low parts of X - c
    float4 nn[NA_MAX_FACES];   // unit normal
    double part[NA_MAX_SPLIT * NA_MAX_FACES];
    double center[4];
    int bad_index;             // set when a face names a vertex outside 0..nv-1
    int pad[7];
};

static_assert(sizeof(NoAllocScratch) == 5767232, "the size stated in tp.h and the file comment");

// the scratch of every call (see the file comment for its sharing rules)
static __device__ __align__(256) unsigned char g_scratch[sizeof(NoAllocScratch)];

// device address of g_scratch per device, looked up once per device and
// context (a context created again, after cudaDeviceReset for instance, loads
// the module again and may place the array elsewhere)
std::mutex g_setup_mutex;
void* g_scratch_addr[64] = {nullptr};
void* g_scratch_ctx[64] = {nullptr};

// the current driver context (an opaque handle), through the runtime's
// driver entry point so that the library does not link libcuda itself
typedef int (*CtxGetCurrentFn)(void**);
void* current_context() {
    static CtxGetCurrentFn fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(f);
        else
            cudaGetLastError();
        looked_up = true;
    }
    void* ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

__global__ void k_na_center(const double* __restrict__ pos, int nv, NoAllocScratch* sc) {
    __shared__ double lo[3][NA_T], hi[3][NA_T];
    double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
    for (int v = threadIdx.x; v < nv; v += NA_T)
        for (int c = 0; c < 3; ++c) {
            l[c] = fmin(l[c], pos[3 * v + c]);
            h[c] = fmax(h[c], pos[3 * v + c]);
        }
    for (int c = 0; c < 3; ++c) {
        lo[c][threadIdx.x] = l[c];
        hi[c][threadIdx.x] = h[c];
    }
    __syncthreads();
    for (int w = NA_T / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) {
                lo[c][threadIdx.x] = fmin(lo[c][threadIdx.x], lo[c][threadIdx.x + w]);
                hi[c][threadIdx.x] = fmax(hi[c][threadIdx.x], hi[c][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 3) sc->center[threadIdx.x] = 0.5 * (lo[threadIdx.x][0] + hi[threadIdx.x][0]);
    if (threadIdx.x == 0) sc->bad_index = 0;   // the first kernel of a call clears the flag
}

__global__ void k_na_faces(const double* __restrict__ pos, int nv, const int* __restrict__ faces, int nf,
                           NoAllocScratch* sc) {
    int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S >= nf) return;
    const int id[3] = {faces[3 * S], faces[3 * S + 1], faces[3 * S + 2]};
    if (id[0] < 0 || id[0] >= nv || id[1] < 0 || id[1] >= nv || id[2] < 0 || id[2] >= nv) {
        // an index out of range: flagged (the result becomes NaN) and the face
        // is not read (zero area and normal, so the pair kernel stays in bounds)
        sc->bad_index = 1;
        sc->xa[S] = make_float4(0.f, 0.f, 0.f, 0.f);
        sc->xl[S] = sc->xa[S];
        sc->nn[S] = sc->xa[S];
        return;
    }
    double P[3][3];
    for (int cr = 0; cr < 3; ++cr)
        for (int c = 0; c < 3; ++c) P[cr][c] = pos[3 * id[cr] + c];
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = P[1][c] - P[0][c];
        e2[c] = P[2][c] - P[0][c];
    }
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double inv = len > 0.0 ? 1.0 / len : 0.0;
    double X[3];
    for (int c = 0; c < 3; ++c) X[c] = (P[0][c] + P[1][c] + P[2][c]) / 3.0 - sc->center[c];
    float hx = (float)X[0], hy = (float)X[1], hz = (float)X[2];
    sc->xa[S] = make_float4(hx, hy, hz, (float)(0.5 * len));
    sc->xl[S] = make_float4((float)(X[0] - (double)hx), (float)(X[1] - (double)hy), (float)(X[2] - (double)hz), 0.f);
    sc->nn[S] = make_float4((float)(n[0] * inv), (float)(n[1] * inv), (float)(n[2] * inv), 0.f);
}

__device__ __forceinline__ float na_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float na_pow(float x, float y) {
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y * l));
    return r;
}

// rows of Eq. 10 without the a_S factor, per source split
template <bool P6>
__global__ void __launch_bounds__(NA_T) k_na_pairs(NoAllocScratch* sc, int nf, int tiles_per_split, float halfp) {
    __shared__ float4 sx[NA_T], sl[NA_T];
    const int t = blockIdx.x * NA_T + threadIdx.x;
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), Al = A, N = A;
    if (t < nf) {
        A = sc->xa[t];
        Al = sc->xl[t];
        N = sc->nn[t];
    }
    float s = 0.f, comp = 0.f;
    const int ntiles = (nf + NA_T - 1) / NA_T;
    const int k0 = blockIdx.y * tiles_per_split, k1 = min(k0 + tiles_per_split, ntiles);
    for (int tile = k0; tile < k1; ++tile) {
        const int src = tile * NA_T + threadIdx.x;
        __syncthreads();
        sx[threadIdx.x] = src < nf ? sc->xa[src] : make_float4(0.f, 0.f, 0.f, 0.f);
        sl[threadIdx.x] = src < nf ? sc->xl[src] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        for (int c = 0; c < NA_T; c += NA_CH) {
            float run = 0.f;
            for (int q = 0; q < NA_CH; ++q) {
                const float4 X = sx[c + q], L = sl[c + q];
                const float dx = (A.x - X.x) + (Al.x - L.x), dy = (A.y - X.y) + (Al.y - L.y),
                            dz = (A.z - X.z) + (Al.z - L.z);
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-18f)));
                const float ir2 = na_rcp(r2);
                const float tt = (N.x * dx + N.y * dy + N.z * dz) * ir2;
                const float qq = tt * tt;                      // (N.d)^2 / |d|^4; 0 for the self pair
                const float K = P6 ? qq * qq * qq : na_pow(qq, halfp);
                run = fmaf(K, X.w, run);
            }
            const float y = run - comp, tsum = s + y;   // Kahan
            comp = (tsum - s) - y;
            s = tsum;
        }
    }
    if (t < nf) sc->part[(size_t)blockIdx.y * NA_MAX_FACES + t] = (double)s - (double)comp;
}

// E = sum_S a_S sum_splits part, in one block, fixed order
__global__ void k_na_sum(const NoAllocScratch* sc, int nf, int nsplit, double* __restrict__ E) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int S = threadIdx.x; S < nf; S += blockDim.x) {
        double r = 0.0;
        for (int k = 0; k < nsplit; ++k) r += sc->part[(size_t)k * NA_MAX_FACES + S];
        acc += (double)sc->xa[S].w * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    // a face with a vertex index out of range makes the result a quiet NaN
    if (threadIdx.x == 0) *E = sc->bad_index ? __longlong_as_double(0x7ff8000000000000ll) : red[0];
}

}  // namespace

extern "C" int tp_energy_noalloc(const double* pos, int nv, const int32_t* faces, int nf, double p, double* E,
                                 void* stream) {
    using tp::fail;
    tp::set_error("");
    if (!pos || !faces || !E) return fail(TP_ERR_INVALID_ARG, "tp_energy_noalloc: NULL pointer");
    if (nv < 3 || nf < 1) return fail(TP_ERR_INVALID_ARG, "tp_energy_noalloc: need nv >= 3 and nf >= 1");
    if (nf > NA_MAX_FACES)
        return fail(TP_ERR_INVALID_ARG, "tp_energy_noalloc: " + std::to_string(nf) + " faces exceed the maximum of " +
                                            std::to_string(NA_MAX_FACES) + " (use tp_mesh_create and tp_energy)");
    if (nv > 3 * NA_MAX_FACES) return fail(TP_ERR_INVALID_ARG, "tp_energy_noalloc: too many vertices");
    if (!(p > 2.0)) return fail(TP_ERR_INVALID_ARG, "tp_energy_noalloc: p must be > 2");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return fail(TP_ERR_CUDA, "tp_energy_noalloc: no current CUDA device");
    // an error left by earlier work of this thread is reported as such, not
    // as a failure of this call's launches
    {
        cudaError_t prior = cudaGetLastError();
        if (prior != cudaSuccess)
            return fail(TP_ERR_CUDA, std::string("tp_energy_noalloc: an earlier CUDA error is pending: ") +
                                         cudaGetErrorString(prior));
    }
    NoAllocScratch* sc = nullptr;
    {
        // first call on this device (and context): look up the device address
        // of the static array, with this device current (host code cannot use
        // g_scratch's name as a device address)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        void* ctx = current_context();
        if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr)
                return fail(TP_ERR_CUDA, std::string("tp_energy_noalloc: cudaGetSymbolAddress failed: ") +
                                             cudaGetErrorString(e));
            g_scratch_addr[dev] = ptr;
            g_scratch_ctx[dev] = ctx;
        }
        sc = static_cast<NoAllocScratch*>(g_scratch_addr[dev]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int ntiles = (nf + NA_T - 1) / NA_T;
    const int bx = ntiles;
    int nsplit = (tp::sm_count() * 8 + bx - 1) / bx;
    if (nsplit > NA_MAX_SPLIT) nsplit = NA_MAX_SPLIT;
    if (nsplit > ntiles) nsplit = ntiles;
    if (nsplit < 1) nsplit = 1;
    const int tps = (ntiles + nsplit - 1) / nsplit;
    nsplit = (ntiles + tps - 1) / tps;
    auto launched = [](const char* what) -> int {
        tp::count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return fail(TP_ERR_CUDA, std::string("tp_energy_noalloc: launch of ") + what + " failed: " +
                                         cudaGetErrorString(e));
        return TP_OK;
    };
    k_na_center<<<1, NA_T, 0, st>>>(pos, nv, sc);
    TP_TRY(launched("k_na_center"));
    k_na_faces<<<(nf + 255) / 256, 256, 0, st>>>(pos, nv, faces, nf, sc);
    TP_TRY(launched("k_na_faces"));
    if (p == 6.0)
        k_na_pairs<true><<<dim3(bx, nsplit), NA_T, 0, st>>>(sc, nf, tps, 3.0f);
    else
        k_na_pairs<false><<<dim3(bx, nsplit), NA_T, 0, st>>>(sc, nf, tps, (float)(0.5 * p));
    TP_TRY(launched("k_na_pairs"));
    k_na_sum<<<1, 1024, 0, st>>>(sc, nf, nsplit, E);
    TP_TRY(launched("k_na_sum"));
    return TP_OK;
}
