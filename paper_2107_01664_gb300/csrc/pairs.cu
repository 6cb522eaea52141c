// Direct all-pairs kernels of the hot path (N-body tiles):
//   energy rows of Eq. 10 (§3.1),
//   face adjoints of the differential of Eq. 10 (§3.1, both roles of a face),
//   kernel-matrix products of §5.1.1-5.1.3 / Appendix A for A, B, B0, L^{2-s}.
//
// Every thread owns TT target faces held in registers; a block of NT
// threads streams tiles of NT source faces through shared memory. The grid
// is (target blocks) x (source splits) so that small meshes still fill the
// GPU; each (block, split) writes per-target partial sums that a combine
// kernel adds in a fixed order (deterministic results). In the FP32 path
// the pair terms are FP32, each run of CH consecutive sources is summed in
// FP32 and the runs are added with Kahan compensation; partials and the
// final per-face combination are FP64. The FP64 path runs the same kernels
// with double arithmetic.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "tp_internal.cuh"

namespace tp {

constexpr int NT = 128;  // threads per block = sources per shared-memory tile
constexpr int CH = 32;   // sources per FP32 run before the compensated add

template <typename T> struct V4T;
template <> struct V4T<float> { using type = float4; };
template <> struct V4T<double> { using type = d4; };

template <typename T> __device__ __forceinline__ typename V4T<T>::type v4zero();
template <> __device__ __forceinline__ float4 v4zero<float>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ d4 v4zero<double>() { return d4{0.0, 0.0, 0.0, 0.0}; }

// ---- elementary functions (FP32: single MUFU instructions) --------------

__device__ __forceinline__ float rcp_(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }

__device__ __forceinline__ float lg2_(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// x^y for x >= 0 (x = 0 gives 0 for y > 0)
__device__ __forceinline__ float pow_(float x, float y) { return ex2_(y * lg2_(x)); }
__device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }

// smallest |d|^2 treated as a real pair; the self pair has d = 0 exactly
template <typename T> __device__ __forceinline__ T tiny_r2();
template <> __device__ __forceinline__ float tiny_r2<float>() { return 1e-18f; }
template <> __device__ __forceinline__ double tiny_r2<double>() { return 1e-150; }

// |d|^2 + tiny as one FMA chain: keeps 1/|d|^4 finite for the self pair
// (d = 0, where every term below is 0 * finite = 0) without a separate clamp;
// for real pairs the offset is below 1e-12 of |d|^2 at |d| > 1e-3
template <typename T> __device__ __forceinline__ T r2_eps(T dx, T dy, T dz) {
    return fma(dx, dx, fma(dy, dy, fma(dz, dz, tiny_r2<T>())));
}

// ---- packed FP32 arithmetic on float pairs (one f32x2 instruction, IEEE per lane)
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2add(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2b(float a) { return make_float2(a, a); }

// two floats as one packed pair register (lane 0 = a)
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}

// Energy term (p = 6) for two targets against one source, all on packed
// pair registers: p + ((N.d)^2 / |d|^4)^3 a per lane, d = X_target - X_s,
// |d|^2 with the tiny offset in the FMA chain (as r2_eps). t* / n* hold the
// two targets' barycenters and normals, s* the source broadcast to both
// lanes, eps the offset in both lanes.
__device__ __forceinline__ unsigned long long energy2_p6(unsigned long long tx, unsigned long long ty,
                                                         unsigned long long tz, unsigned long long nx,
                                                         unsigned long long ny, unsigned long long nz,
                                                         unsigned long long sx, unsigned long long sy,
                                                         unsigned long long sz, unsigned long long sa,
                                                         unsigned long long eps, unsigned long long p) {
    unsigned long long out;
    asm("{\n\t.reg .b64 dx, dy, dz, r2, ir2, t, q, q3;\n\t.reg .f32 lo, hi;\n\t"
        "sub.rn.f32x2 dx, %1, %7;\n\t"
        "sub.rn.f32x2 dy, %2, %8;\n\t"
        "sub.rn.f32x2 dz, %3, %9;\n\t"
        "fma.rn.f32x2 r2, dz, dz, %11;\n\t"
        "fma.rn.f32x2 r2, dy, dy, r2;\n\t"
        "fma.rn.f32x2 r2, dx, dx, r2;\n\t"
        "mov.b64 {lo, hi}, r2;\n\t"
        "rcp.approx.ftz.f32 lo, lo;\n\t"
        "rcp.approx.ftz.f32 hi, hi;\n\t"
        "mov.b64 ir2, {lo, hi};\n\t"
        "mul.rn.f32x2 t, %6, dz;\n\t"
        "fma.rn.f32x2 t, %5, dy, t;\n\t"
        "fma.rn.f32x2 t, %4, dx, t;\n\t"
        "mul.rn.f32x2 t, t, ir2;\n\t"
        "mul.rn.f32x2 q, t, t;\n\t"
        "mul.rn.f32x2 q3, q, q;\n\t"
        "mul.rn.f32x2 q3, q3, q;\n\t"
        "fma.rn.f32x2 %0, q3, %10, %12;\n\t}"
        : "=l"(out)
        : "l"(tx), "l"(ty), "l"(tz), "l"(nx), "l"(ny), "l"(nz), "l"(sx), "l"(sy), "l"(sz), "l"(sa), "l"(eps),
          "l"(p));
    return out;
}

// ---- compensated accumulators -------------------------------------------

template <typename T> struct Acc;
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {  // Kahan
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// ---- near-pair precision ---------------------------------------------------
// FP32 barycenters are stored as hi (float4 .xyz) + lo (the rounding error,
// a second float4). For a source tile whose bounding box lies within the
// near distance of the block's targets, d is formed as (hi_S - hi_T) +
// (lo_S - lo_T), which removes the rounding of the stored barycenters from
// the small differences of near pairs; other tiles use hi_S - hi_T. The
// choice is the same for every thread of the block.

__device__ __forceinline__ void block_box(float lx, float ly, float lz, float hx, float hy, float hz,
                                          float* sbox) {
    __shared__ float wb[NT / 32][6];
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        wb[w][0] = lx; wb[w][1] = ly; wb[w][2] = lz;
        wb[w][3] = hx; wb[w][4] = hy; wb[w][5] = hz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) {
            float l = wb[0][c], h = wb[0][3 + c];
            for (int i = 1; i < NT / 32; ++i) {
                l = fminf(l, wb[i][c]);
                h = fmaxf(h, wb[i][3 + c]);
            }
            sbox[c] = l;
            sbox[3 + c] = h;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ bool tile_near(const float4* __restrict__ tbox, int tile, const float* sbox,
                                          float thr2) {
    float4 lo = tbox[2 * tile], hi = tbox[2 * tile + 1];
    float gx = fmaxf(fmaxf(lo.x - sbox[3], sbox[0] - hi.x), 0.f);
    float gy = fmaxf(fmaxf(lo.y - sbox[4], sbox[1] - hi.y), 0.f);
    float gz = fmaxf(fmaxf(lo.z - sbox[5], sbox[2] - hi.z), 0.f);
    return gx * gx + gy * gy + gz * gz < thr2;
}

// ---- launch geometry ------------------------------------------------------

struct Grid {
    int bx, nsplit, tiles_per_split;
};

// resident blocks per SM of a kernel (cached per kernel and device)
static int resident_per_sm(const void* fn, int threads, size_t dyn_smem = 0) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(fn, dev);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (dyn_smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;   // the kernel cannot be launched with this much shared memory
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, dyn_smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    cache[key] = n;
    return n;
}

// Source splits. Each block of a target row takes tiles_per_split source
// tiles, and the grid runs in waves of (resident blocks per SM x SMs), so
// the kernel time goes like waves x tiles_per_split. The split count
// minimises that, plus a small charge per split for the partial sums the
// FP64 combine reads (a split's partials cost about a twentieth of a tile).
static Grid make_grid(int nt, int nf, int tt, int per_sm) {
    Grid g;
    g.bx = (nt + NT * tt - 1) / (NT * tt);
    if (g.bx < 1) g.bx = 1;
    const int ntiles = (nf + NT - 1) / NT;
    const long slots = (long)std::max(1, per_sm) * sm_count();
    double best = 1e300;
    g.tiles_per_split = ntiles;
    g.nsplit = 1;
    for (int ns = 1; ns <= std::min(ntiles, 64); ++ns) {
        const int tps = (ntiles + ns - 1) / ns;
        const int nsp = (ntiles + tps - 1) / tps;
        const long waves = ((long)g.bx * nsp + slots - 1) / slots;
        const double cost = (double)waves * tps + 0.05 * nsp;
        if (cost < best - 1e-9) {
            best = cost;
            g.tiles_per_split = tps;
            g.nsplit = nsp;
        }
    }
    return g;
}

// ===========================================================================
// energy rows, Eq. 10: sum_{T != S} K(S,T) a_T  (times a_S in the combine)
// ===========================================================================

template <typename T, bool P6>
__device__ __forceinline__ T energy_term(T dx, T dy, T dz, T nx, T ny, T nz, T halfp) {
    T ir2 = rcp_(r2_eps(dx, dy, dz));
    T t = (nx * dx + ny * dy + nz * dz) * ir2;  // N.d / |d|^2
    T qq = t * t;                                 // (N.d)^2 / |d|^4
    return P6 ? qq * qq * qq : pow_(qq, halfp);
}

template <typename T, bool P6, int TT>
__global__ void __launch_bounds__(NT)
k_energy(const typename V4T<T>::type* __restrict__ fa, const typename V4T<T>::type* __restrict__ fb,
         const float4* __restrict__ flo, const float4* __restrict__ tbox, const double* __restrict__ center,
         int nf, const int* __restrict__ tlist, int nt, int tiles_per_split, T halfp,
         double* __restrict__ part) {
    using V4 = typename V4T<T>::type;
    constexpr bool F32 = sizeof(T) == 4;
    // packed path (FP32, p = 6): sources also staged broadcast to pairs
    constexpr bool PACK = F32 && P6 && TT % 2 == 0;
    __shared__ V4 sh[NT];
    __shared__ float4 shl[F32 ? NT : 1];
    __shared__ ulonglong2 shp[PACK ? 2 * NT : 1];
    __shared__ float sbox[6];
    T tx[TT], ty[TT], tz[TT], nx[TT], ny[TT], nz[TT];
    float lx[TT], ly[TT], lz[TT];
    int tid[TT];
    float bl[3] = {3e38f, 3e38f, 3e38f}, bh[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int j = 0; j < TT; ++j) {
        int t = blockIdx.x * NT * TT + j * NT + threadIdx.x;
        tid[j] = t;
        lx[j] = ly[j] = lz[j] = 0.f;
        if (t < nt) {
            int S = tlist ? tlist[t] : t;
            V4 A = fa[S], B = fb[S];
            tx[j] = A.x; ty[j] = A.y; tz[j] = A.z;
            nx[j] = B.x; ny[j] = B.y; nz[j] = B.z;
            if (F32) {
                float4 L = flo[S];
                lx[j] = L.x; ly[j] = L.y; lz[j] = L.z;
                bl[0] = fminf(bl[0], (float)A.x); bl[1] = fminf(bl[1], (float)A.y); bl[2] = fminf(bl[2], (float)A.z);
                bh[0] = fmaxf(bh[0], (float)A.x); bh[1] = fmaxf(bh[1], (float)A.y); bh[2] = fmaxf(bh[2], (float)A.z);
            }
        } else {  // idle slot: zero normal gives zero terms
            tx[j] = ty[j] = tz[j] = T(0);
            nx[j] = ny[j] = nz[j] = T(0);
        }
    }
    float thr2 = 0.f;
    if (F32) {
        block_box(bl[0], bl[1], bl[2], bh[0], bh[1], bh[2], sbox);
        thr2 = (float)center[3];
    }
    Acc<T> acc[TT];
    unsigned long long TX[PACK ? TT / 2 : 1], TY[PACK ? TT / 2 : 1], TZ[PACK ? TT / 2 : 1];
    unsigned long long NX[PACK ? TT / 2 : 1], NY[PACK ? TT / 2 : 1], NZ[PACK ? TT / 2 : 1];
    unsigned long long EPS = 0ull;
    if constexpr (PACK) {
#pragma unroll
        for (int jj = 0; jj < TT / 2; ++jj) {
            TX[jj] = pk2((float)tx[2 * jj], (float)tx[2 * jj + 1]);
            TY[jj] = pk2((float)ty[2 * jj], (float)ty[2 * jj + 1]);
            TZ[jj] = pk2((float)tz[2 * jj], (float)tz[2 * jj + 1]);
            NX[jj] = pk2((float)nx[2 * jj], (float)nx[2 * jj + 1]);
            NY[jj] = pk2((float)ny[2 * jj], (float)ny[2 * jj + 1]);
            NZ[jj] = pk2((float)nz[2 * jj], (float)nz[2 * jj + 1]);
        }
        EPS = pk2(1e-18f, 1e-18f);
    }
    const int ntiles = (nf + NT - 1) / NT;
    const int k0 = blockIdx.y * tiles_per_split;
    const int k1 = min(k0 + tiles_per_split, ntiles);
    for (int tile = k0; tile < k1; ++tile) {
        const bool near = F32 && tile_near(tbox, tile, sbox, thr2);
        int src = tile * NT + threadIdx.x;
        __syncthreads();
        const V4 sv = src < nf ? fa[src] : v4zero<T>();   // zero area pads the tail
        sh[threadIdx.x] = sv;
        if constexpr (PACK) {
            shp[2 * threadIdx.x] = make_ulonglong2(pk2((float)sv.x, (float)sv.x), pk2((float)sv.y, (float)sv.y));
            shp[2 * threadIdx.x + 1] = make_ulonglong2(pk2((float)sv.z, (float)sv.z), pk2((float)sv.w, (float)sv.w));
        }
        if (near) shl[threadIdx.x] = src < nf ? flo[src] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        for (int c = 0; c < NT; c += CH) {
            T pt[TT];
#pragma unroll
            for (int j = 0; j < TT; ++j) pt[j] = T(0);
            if (near) {
#pragma unroll 4
                for (int q = 0; q < CH; ++q) {
                    V4 s = sh[c + q];
                    float4 l = shl[c + q];
#pragma unroll
                    for (int j = 0; j < TT; ++j) {
                        T dx = (tx[j] - s.x) + (T)(lx[j] - l.x);
                        T dy = (ty[j] - s.y) + (T)(ly[j] - l.y);
                        T dz = (tz[j] - s.z) + (T)(lz[j] - l.z);
                        pt[j] = fma(energy_term<T, P6>(dx, dy, dz, nx[j], ny[j], nz[j], halfp), s.w, pt[j]);
                    }
                }
            } else if constexpr (PACK) {
                // two targets per packed instruction
                unsigned long long P[TT / 2];
#pragma unroll
                for (int jj = 0; jj < TT / 2; ++jj) P[jj] = 0ull;
#pragma unroll 8
                for (int q = 0; q < CH; ++q) {
                    const ulonglong2 u0 = shp[2 * (c + q)], u1 = shp[2 * (c + q) + 1];
#pragma unroll
                    for (int jj = 0; jj < TT / 2; ++jj)
                        P[jj] = energy2_p6(TX[jj], TY[jj], TZ[jj], NX[jj], NY[jj], NZ[jj], u0.x, u0.y, u1.x, u1.y,
                                           EPS, P[jj]);
                }
#pragma unroll
                for (int jj = 0; jj < TT / 2; ++jj) {
                    const float2 v = upk2(P[jj]);
                    pt[2 * jj] = v.x;
                    pt[2 * jj + 1] = v.y;
                }
            } else {
#pragma unroll 8
                for (int q = 0; q < CH; ++q) {
                    V4 s = sh[c + q];
#pragma unroll
                    for (int j = 0; j < TT; ++j)
                        pt[j] = fma(energy_term<T, P6>(tx[j] - s.x, ty[j] - s.y, tz[j] - s.z, nx[j], ny[j],
                                                       nz[j], halfp),
                                    s.w, pt[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < TT; ++j) acc[j].add(pt[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < TT; ++j)
        if (tid[j] < nt) part[(size_t)blockIdx.y * nt + tid[j]] = acc[j].value();
}

__global__ void k_energy_combine(const double* __restrict__ part, int nsplit, int nt,
                                 const int* __restrict__ tlist, const d4* __restrict__ f64a,
                                 double* __restrict__ rows) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int S = tlist ? tlist[t] : t;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += part[(size_t)k * nt + t];
    rows[t] = f64a[S].w * s;
}

template <typename T>
static int launch_energy(tp_mesh* m, const tp_params* p, const int32_t* tl, int nt, double* rows,
                         cudaStream_t st) {
    using V4 = typename V4T<T>::type;
    constexpr int TT = sizeof(T) == 4 ? 4 : 2;
    Grid g = make_grid(nt, m->nf, TT, resident_per_sm((const void*)k_energy<T, true, TT>, NT));
    TP_TRY(ensure(m->part, sizeof(double) * (size_t)g.nsplit * nt));
    const V4* fa = (const V4*)(sizeof(T) == 4 ? m->f32a.ptr : m->f64a.ptr);
    const V4* fb = (const V4*)(sizeof(T) == 4 ? m->f32b.ptr : m->f64b.ptr);
    dim3 grid(g.bx, g.nsplit);
    const double units = (double)nt * (m->nf - 1);
    m->pairs += units;
    {
        ProfScope ps(m, PK_ENERGY, units, st);
        if (p->p == 6.0)
            k_energy<T, true, TT><<<grid, NT, 0, st>>>(fa, fb, m->f32c.as<float4>(), m->tilebox.as<float4>(),
                                                       m->center.as<double>(), m->nf, tl, nt,
                                                       g.tiles_per_split, T(3), m->part.as<double>());
        else
            k_energy<T, false, TT><<<grid, NT, 0, st>>>(fa, fb, m->f32c.as<float4>(), m->tilebox.as<float4>(),
                                                        m->center.as<double>(), m->nf, tl, nt,
                                                        g.tiles_per_split, T(0.5 * p->p), m->part.as<double>());
        TP_LAUNCH_CHECK();
    }
    k_energy_combine<<<(nt + 255) / 256, 256, 0, st>>>(m->part.as<double>(), g.nsplit, nt, tl,
                                                       m->f64a.as<d4>(), rows);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

int energy_rows_direct(tp_mesh* m, const tp_params* p, const int32_t* tl, int nt, double* rows,
                       cudaStream_t st) {
    if (nt == 0) return TP_OK;
    return p->precision == TP_PREC_FP64 ? launch_energy<double>(m, p, tl, nt, rows, st)
                                        : launch_energy<float>(m, p, tl, nt, rows, st);
}

// ===========================================================================
// differential of Eq. 10: face adjoints in both roles of each face
//   with d = X_S - X_T, u_S = N_S.d, u_T = N_T.d, q = u^2/|d|^4,
//   K = q^{p/2}, c = q^{p/2-1} u / |d|^4  (= |u|^{p-2} u / |d|^{2p}):
//   dE/dX_S = a_S sum_T a_T [p c_S N_S + p c_T N_T - 2p (K_ST + K_TS) d/|d|^2]
//   dE/dN_S = a_S sum_T a_T p c_S d
//   dE/da_S = sum_T a_T (K_ST + K_TS)
// accumulators: 0 sum a c_S | 1-3 sum a c_S d | 4-6 sum a c_T N_T |
//               7-9 sum a (K_ST+K_TS) d/|d|^2 | 10 sum a (K_ST+K_TS) | 11 sum a K_ST
// ===========================================================================

constexpr int NADJ = 12;

template <typename T, bool P6>
__device__ __forceinline__ void diff_term(T dx, T dy, T dz, T nx, T ny, T nz, T at, T mx, T my, T mz, T hm1,
                                          T* pt) {
    T ir2 = rcp_(r2_eps(dx, dy, dz));
    T tS = (nx * dx + ny * dy + nz * dz) * ir2;   // u_S / |d|^2
    T tT = (mx * dx + my * dy + mz * dz) * ir2;   // u_T / |d|^2
    T qS = tS * tS, qT = tT * tT;
    T mS = P6 ? qS * qS : pow_(qS, hm1);
    T mT = P6 ? qT * qT : pow_(qT, hm1);
    T KS = mS * qS, KT = mT * qT;
    T w = (at * mS) * (tS * ir2);                 // a_T q_S^{p/2-1} u_S / |d|^4
    T v = (at * mT) * (tT * ir2);
    T kS = at * KS;
    T ks = fma(at, KT, kS);
    T kd = ks * ir2;
    pt[0] += w;
    pt[1] = fma(w, dx, pt[1]);
    pt[2] = fma(w, dy, pt[2]);
    pt[3] = fma(w, dz, pt[3]);
    pt[4] = fma(v, mx, pt[4]);
    pt[5] = fma(v, my, pt[5]);
    pt[6] = fma(v, mz, pt[6]);
    pt[7] = fma(kd, dx, pt[7]);
    pt[8] = fma(kd, dy, pt[8]);
    pt[9] = fma(kd, dz, pt[9]);
    pt[10] += ks;
    pt[11] += kS;
}

// diff_term (p = 6) for two targets (lanes) against one source, packed;
// pt[i] holds accumulator i of both targets
__device__ __forceinline__ void diff_pair_p6(float2 dx, float2 dy, float2 dz, float2 nx, float2 ny, float2 nz, float at,
                                             float mx, float my, float mz, float2* pt) {
    const float2 r2 = f2fma(dx, dx, f2fma(dy, dy, f2fma(dz, dz, f2b(tiny_r2<float>()))));
    const float2 ir2 = make_float2(rcp_(r2.x), rcp_(r2.y));
    const float2 tS = f2mul(f2fma(nx, dx, f2fma(ny, dy, f2mul(nz, dz))), ir2);
    const float2 tT = f2mul(f2fma(f2b(mx), dx, f2fma(f2b(my), dy, f2mul(f2b(mz), dz))), ir2);
    const float2 qS = f2mul(tS, tS), qT = f2mul(tT, tT);
    const float2 mS = f2mul(qS, qS), mT = f2mul(qT, qT);
    const float2 A = f2b(at);
    const float2 w = f2mul(f2mul(A, mS), f2mul(tS, ir2));
    const float2 v = f2mul(f2mul(A, mT), f2mul(tT, ir2));
    const float2 kS = f2mul(A, f2mul(mS, qS));
    const float2 ks = f2fma(A, f2mul(mT, qT), kS);
    const float2 kd = f2mul(ks, ir2);
    pt[0] = f2add(pt[0], w);
    pt[1] = f2fma(w, dx, pt[1]);
    pt[2] = f2fma(w, dy, pt[2]);
    pt[3] = f2fma(w, dz, pt[3]);
    pt[4] = f2fma(v, f2b(mx), pt[4]);
    pt[5] = f2fma(v, f2b(my), pt[5]);
    pt[6] = f2fma(v, f2b(mz), pt[6]);
    pt[7] = f2fma(kd, dx, pt[7]);
    pt[8] = f2fma(kd, dy, pt[8]);
    pt[9] = f2fma(kd, dz, pt[9]);
    pt[10] = f2add(pt[10], ks);
    pt[11] = f2add(pt[11], kS);
}

template <typename T, bool P6, int TT>
__global__ void __launch_bounds__(NT)
k_diff(const typename V4T<T>::type* __restrict__ fa, const typename V4T<T>::type* __restrict__ fb,
       const float4* __restrict__ flo, const float4* __restrict__ tbox, const double* __restrict__ center,
       int nf, int tiles_per_split, T hm1, double* __restrict__ part) {
    using V4 = typename V4T<T>::type;
    constexpr bool F32 = sizeof(T) == 4;
    __shared__ V4 sa[NT];
    __shared__ V4 sb[NT];
    __shared__ float4 shl[F32 ? NT : 1];
    __shared__ float sbox[6];
    const int nt = nf;
    T tx[TT], ty[TT], tz[TT], nx[TT], ny[TT], nz[TT];
    float lx[TT], ly[TT], lz[TT];
    int tid[TT];
    float bl[3] = {3e38f, 3e38f, 3e38f}, bh[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int j = 0; j < TT; ++j) {
        int t = blockIdx.x * NT * TT + j * NT + threadIdx.x;
        tid[j] = t;
        lx[j] = ly[j] = lz[j] = 0.f;
        if (t < nt) {
            V4 A = fa[t], B = fb[t];
            tx[j] = A.x; ty[j] = A.y; tz[j] = A.z;
            nx[j] = B.x; ny[j] = B.y; nz[j] = B.z;
            if (F32) {
                float4 L = flo[t];
                lx[j] = L.x; ly[j] = L.y; lz[j] = L.z;
                bl[0] = fminf(bl[0], (float)A.x); bl[1] = fminf(bl[1], (float)A.y); bl[2] = fminf(bl[2], (float)A.z);
                bh[0] = fmaxf(bh[0], (float)A.x); bh[1] = fmaxf(bh[1], (float)A.y); bh[2] = fmaxf(bh[2], (float)A.z);
            }
        } else {
            tx[j] = ty[j] = tz[j] = T(0);
            nx[j] = ny[j] = nz[j] = T(0);
        }
    }
    float thr2 = 0.f;
    if (F32) {
        block_box(bl[0], bl[1], bl[2], bh[0], bh[1], bh[2], sbox);
        thr2 = (float)center[3];
    }
    Acc<T> acc[TT][NADJ];
    const int ntiles = (nf + NT - 1) / NT;
    const int k0 = blockIdx.y * tiles_per_split;
    const int k1 = min(k0 + tiles_per_split, ntiles);
    for (int tile = k0; tile < k1; ++tile) {
        const bool near = F32 && tile_near(tbox, tile, sbox, thr2);
        int src = tile * NT + threadIdx.x;
        __syncthreads();
        sa[threadIdx.x] = src < nf ? fa[src] : v4zero<T>();
        sb[threadIdx.x] = src < nf ? fb[src] : v4zero<T>();
        if (near) shl[threadIdx.x] = src < nf ? flo[src] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        for (int c = 0; c < NT; c += CH) {
            T pt[TT][NADJ];
#pragma unroll
            for (int j = 0; j < TT; ++j)
#pragma unroll
                for (int i = 0; i < NADJ; ++i) pt[j][i] = T(0);
            if (near) {
#pragma unroll 2
                for (int q = 0; q < CH; ++q) {
                    V4 s = sa[c + q];
                    V4 n = sb[c + q];
                    float4 l = shl[c + q];
#pragma unroll
                    for (int j = 0; j < TT; ++j)
                        diff_term<T, P6>((tx[j] - s.x) + (T)(lx[j] - l.x), (ty[j] - s.y) + (T)(ly[j] - l.y),
                                         (tz[j] - s.z) + (T)(lz[j] - l.z), nx[j], ny[j], nz[j], s.w, n.x, n.y,
                                         n.z, hm1, pt[j]);
                }
            } else if constexpr (F32 && P6 && TT == 2) {
                // both targets per packed instruction
                float2 p2[NADJ];
#pragma unroll
                for (int i = 0; i < NADJ; ++i) p2[i] = make_float2(0.f, 0.f);
                const float2 TXp = make_float2((float)tx[0], (float)tx[1]), TYp = make_float2((float)ty[0], (float)ty[1]),
                             TZp = make_float2((float)tz[0], (float)tz[1]);
                const float2 NXp = make_float2((float)nx[0], (float)nx[1]), NYp = make_float2((float)ny[0], (float)ny[1]),
                             NZp = make_float2((float)nz[0], (float)nz[1]);
#pragma unroll 4
                for (int q = 0; q < CH; ++q) {
                    const float4 s = reinterpret_cast<const float4&>(sa[c + q]);
                    const float4 n = reinterpret_cast<const float4&>(sb[c + q]);
                    diff_pair_p6(f2sub(TXp, f2b(s.x)), f2sub(TYp, f2b(s.y)), f2sub(TZp, f2b(s.z)), NXp, NYp, NZp, s.w,
                                 n.x, n.y, n.z, p2);
                }
#pragma unroll
                for (int i = 0; i < NADJ; ++i) {
                    pt[0][i] = p2[i].x;
                    pt[1][i] = p2[i].y;
                }
            } else {
#pragma unroll 4
                for (int q = 0; q < CH; ++q) {
                    V4 s = sa[c + q];
                    V4 n = sb[c + q];
#pragma unroll
                    for (int j = 0; j < TT; ++j)
                        diff_term<T, P6>(tx[j] - s.x, ty[j] - s.y, tz[j] - s.z, nx[j], ny[j], nz[j], s.w, n.x,
                                         n.y, n.z, hm1, pt[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < TT; ++j)
#pragma unroll
                for (int i = 0; i < NADJ; ++i) acc[j][i].add(pt[j][i]);
        }
    }
#pragma unroll
    for (int j = 0; j < TT; ++j)
        if (tid[j] < nt)
#pragma unroll
            for (int i = 0; i < NADJ; ++i)
                part[((size_t)blockIdx.y * NADJ + i) * nt + tid[j]] = acc[j][i].value();
}

// adj[S*7 + 0..2] = dE/dX_S, [3..5] = dE/dN_S, [6] = dE/da_S; erow[S] = energy row
__global__ void k_diff_combine(const double* __restrict__ part, int nsplit, int nf, double p,
                               const d4* __restrict__ f64a, const d4* __restrict__ f64b,
                               double* __restrict__ adj, double* __restrict__ erow) {
    int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S >= nf) return;
    double s[NADJ];
    for (int i = 0; i < NADJ; ++i) s[i] = 0.0;
    for (int k = 0; k < nsplit; ++k)
        for (int i = 0; i < NADJ; ++i) s[i] += part[((size_t)k * NADJ + i) * nf + S];
    double a = f64a[S].w;
    d4 N = f64b[S];
    double NS[3] = {N.x, N.y, N.z};
    for (int c = 0; c < 3; ++c) {
        adj[7 * S + c] = a * (p * (s[0] * NS[c] + s[4 + c]) - 2.0 * p * s[7 + c]);
        adj[7 * S + 3 + c] = a * p * s[1 + c];
    }
    adj[7 * S + 6] = s[10];
    if (erow) erow[S] = a * s[11];
}

template <typename T>
static int launch_diff(tp_mesh* m, const tp_params* p, double* adj, double* erow, cudaStream_t st) {
    using V4 = typename V4T<T>::type;
    constexpr int TT = sizeof(T) == 4 ? 2 : 1;
    Grid g = make_grid(m->nf, m->nf, TT, resident_per_sm((const void*)k_diff<T, true, TT>, NT));
    TP_TRY(ensure(m->part, sizeof(double) * (size_t)g.nsplit * NADJ * m->nf));
    const V4* fa = (const V4*)(sizeof(T) == 4 ? m->f32a.ptr : m->f64a.ptr);
    const V4* fb = (const V4*)(sizeof(T) == 4 ? m->f32b.ptr : m->f64b.ptr);
    dim3 grid(g.bx, g.nsplit);
    const double units = (double)m->nf * (m->nf - 1);
    m->pairs += units;
    {
        ProfScope ps(m, PK_DIFF, units, st);
        if (p->p == 6.0)
            k_diff<T, true, TT><<<grid, NT, 0, st>>>(fa, fb, m->f32c.as<float4>(), m->tilebox.as<float4>(),
                                                     m->center.as<double>(), m->nf, g.tiles_per_split, T(2),
                                                     m->part.as<double>());
        else
            k_diff<T, false, TT><<<grid, NT, 0, st>>>(fa, fb, m->f32c.as<float4>(), m->tilebox.as<float4>(),
                                                      m->center.as<double>(), m->nf, g.tiles_per_split,
                                                      T(0.5 * p->p - 1.0), m->part.as<double>());
        TP_LAUNCH_CHECK();
    }
    k_diff_combine<<<(m->nf + 255) / 256, 256, 0, st>>>(m->part.as<double>(), g.nsplit, m->nf,
                                                        p->p, m->f64a.as<d4>(), m->f64b.as<d4>(),
                                                        adj, erow);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

int diff_adjoints_direct(tp_mesh* m, const tp_params* p, double* adj, double* erow,
                         cudaStream_t st) {
    return p->precision == TP_PREC_FP64 ? launch_diff<double>(m, p, adj, erow, st)
                                        : launch_diff<float>(m, p, adj, erow, st);
}

// chain rule from (gX, gN, ga) of a face to its corners (§3.1):
//   X = (f_i+f_j+f_k)/3, n = (f_j-f_i) x (f_k-f_i), a = |n|/2, N = n/|n|;
//   w = (I - N N^T) gN / |n| + ga N / 2;  g_j = e2 x w, g_k = w x e1,
//   g_i = -(g_j + g_k), plus gX/3 on each corner.
__global__ void k_adj_to_corner(const double* __restrict__ pos, const int* __restrict__ faces,
                                int nf, const double* __restrict__ adj, double* __restrict__ corner) {
    int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S >= nf) return;
    int i = faces[3 * S], j = faces[3 * S + 1], k = faces[3 * S + 2];
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = pos[3 * j + c] - pos[3 * i + c];
        e2[c] = pos[3 * k + c] - pos[3 * i + c];
    }
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                   e1[0] * e2[1] - e1[1] * e2[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double N[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
    const double* g = adj + 7 * S;
    double gNn = g[3] * N[0] + g[4] * N[1] + g[5] * N[2];
    double w[3];
    for (int c = 0; c < 3; ++c) w[c] = (g[3 + c] - gNn * N[c]) / nn + 0.5 * g[6] * N[c];
    double gj[3] = {e2[1] * w[2] - e2[2] * w[1], e2[2] * w[0] - e2[0] * w[2],
                    e2[0] * w[1] - e2[1] * w[0]};
    double gk[3] = {w[1] * e1[2] - w[2] * e1[1], w[2] * e1[0] - w[0] * e1[2],
                    w[0] * e1[1] - w[1] * e1[0]};
    for (int c = 0; c < 3; ++c) {
        double third = g[c] / 3.0;
        corner[9 * S + c] = -(gj[c] + gk[c]) + third;
        corner[9 * S + 3 + c] = gj[c] + third;
        corner[9 * S + 6 + c] = gk[c] + third;
    }
}

int adjoints_to_dE(tp_mesh* m, const double* adj, double* dE, cudaStream_t st) {
    TP_TRY(ensure(m->corner, sizeof(double) * 9 * (size_t)m->nf));
    k_adj_to_corner<<<(m->nf + 255) / 256, 256, 0, st>>>(m->pos.as<double>(), m->faces.as<int>(),
                                                         m->nf, adj, m->corner.as<double>());
    TP_LAUNCH_CHECK();
    return corners_to_vertices(m, m->corner.as<double>(), 3, dE, st);
}

// ===========================================================================
// kernel-matrix products, §5.1.1-5.1.3 and Appendix A, KC = 3 or 9 columns
// per pass
//   B : W_V = diag(a) D v (3 x KC per face), h = |d|^{-2s}
//   B0: W_U = diag(a) avg v (KC per face),   h = (k2(S;T)+k2(T;S)) / (2|d|^{2s})
//   L : W_U,                                 h = |d|^{-2(3-s)}   (sigma = 2 - s)
// per target: r = sum_T h a_T and (H W)_S = sum_T h W_T.
// ===========================================================================

// Per source face the pair kernels read one vector X of NA values: [a, W_V]
// (the operators with the high-order part) then [a, W_U] (those with a
// low-order part); accumulator i gains h X[i], with h the high-order kernel
// on the first NH entries and the low-order one on the rest. NH and NA are
// even, so the pairs of packed FP32 arithmetic never straddle the parts.
template <int OP, int KC> struct OpLayout {
    static constexpr bool HIGH = (OP == TP_OP_A || OP == TP_OP_B);
    static constexpr bool USEU = (OP != TP_OP_B);
    static constexpr int NH = HIGH ? 1 + 3 * KC : 0;          // high-order entries [a, W_V]
    static constexpr int NL = USEU ? 1 + KC : 0;              // low-order entries [a, W_U]
    static constexpr int NA = NH + NL;                        // accumulators = X entries
    static constexpr int NW4 = (NA + 3) / 4;                  // X in 4-vectors
    static_assert(NH % 2 == 0 && NA % 2 == 0, "pairs of accumulators stay within a part");
};

// per-face W (FP64 [nf][4*KC]: W_V at q*KC+c, then W_U at 3*KC+c) and its
// padded copy in the pair precision and the operator's layout, for columns
// col0 .. col0+KC-1 of v [nv][k] (missing columns are zero)
template <typename T, int KC>
__global__ void k_face_W(const double* __restrict__ v, int k, int col0, const int* __restrict__ faces,
                         int nf, const d4* __restrict__ f64a, const double* __restrict__ fgrad,
                         int op, double* __restrict__ W64, typename V4T<T>::type* __restrict__ Wp,
                         int nw4) {
    // one thread per face and group of (up to) three columns
    constexpr int CG = KC < 3 ? KC : 3, NCG = (KC + CG - 1) / CG;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int S = t / NCG, g = t - S * NCG;
    if (S >= nf) return;
    const int c0 = g * CG;
    const double a = f64a[S].w;
    double val[3][CG];
    for (int cr = 0; cr < 3; ++cr) {
        const int vi = faces[3 * S + cr];
        for (int c = 0; c < CG; ++c)
            val[cr][c] = (c0 + c < KC && col0 + c0 + c < k) ? v[(size_t)vi * k + col0 + c0 + c] : 0.0;
    }
    double gr[9];
    for (int i = 0; i < 9; ++i) gr[i] = fgrad[9 * S + i];
    double* w64 = W64 + 4 * KC * (size_t)S;
    T* out = reinterpret_cast<T*>(Wp) + (size_t)S * 4 * nw4;
    const bool hi = (op == TP_OP_A || op == TP_OP_B), lo = op != TP_OP_B;
    const int ou = hi ? 1 + 3 * KC : 0;   // start of the low-order block in out
    for (int c = 0; c < CG && c0 + c < KC; ++c) {
        for (int q = 0; q < 3; ++q) {
            double gq = 0.0;
            for (int cr = 0; cr < 3; ++cr) gq += val[cr][c] * gr[3 * cr + q];
            const double wv = a * gq;
            w64[q * KC + c0 + c] = wv;
            if (hi) out[1 + q * KC + c0 + c] = (T)wv;
        }
        const double wu = a * (val[0][c] + val[1][c] + val[2][c]) * (1.0 / 3.0);
        w64[3 * KC + c0 + c] = wu;
        if (lo) out[ou + 1 + c0 + c] = (T)wu;
    }
    if (g == 0) {
        if (hi) out[0] = (T)a;
        if (lo) out[ou] = (T)a;
        for (int n = ou + (lo ? 1 + KC : 0); n < 4 * nw4; ++n) out[n] = T(0);
    }
}

// ---- pairs of accumulators ------------------------------------------------
// FP32: packed f32x2 arithmetic (one instruction for two IEEE operations,
// the same results as two scalar ones); FP64: two scalar operations.
template <typename T> struct P2T;
template <> struct P2T<float> { using type = float2; };
template <> struct P2T<double> { using type = double2; };

__device__ __forceinline__ float2 pfma(float a, float2 b, float2 c) {   // a * b + c, a in both lanes
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %2};\n\tmov.b64 rb, {%3, %4};\n\tmov.b64 rc, {%5, %6};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ double2 pfma(double a, double2 b, double2 c) {
    return make_double2(fma(a, b.x, c.x), fma(a, b.y, c.y));
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
// Per-block compensated sums: the chunk sums (32 terms each) of a source
// split are added into Kahan pairs (packed: two accumulators per
// instruction); the splits meet in the FP64 combine.
template <typename T> struct Acc2;
template <> struct Acc2<float> {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 x) {
        const float2 y = psub(x, c);
        const float2 t = padd(s, y);
        c = psub(psub(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value(int lane) const {
        return lane ? (double)s.y - (double)c.y : (double)s.x - (double)c.x;
    }
};
template <> struct Acc2<double> {
    double2 s = make_double2(0.0, 0.0);
    __device__ __forceinline__ void add(double2 x) {
        s.x += x.x;
        s.y += x.y;
    }
    __device__ __forceinline__ double value(int lane) const { return lane ? s.y : s.x; }
};

template <typename T>
__device__ __forceinline__ typename P2T<T>::type p2zero() {
    typename P2T<T>::type z;
    z.x = T(0);
    z.y = T(0);
    return z;
}

// One (target, source) term of the kernel-matrix products on the source's
// vector X (pairs x2[i] = X[2i], X[2i+1]). SELF = the tile may contain the
// target itself (d = 0), whose term must be dropped: the kernels of B and
// L^{2-s} do not vanish at d = 0 by themselves.
template <typename T, int OP, bool SELF, int KC>
__device__ __forceinline__ void apply_term(T dx, T dy, T dz, T nx, T ny, T nz, T mx, T my, T mz,
                                           const typename P2T<T>::type* x2, T s_exp, T l_exp,
                                           typename P2T<T>::type* pt) {
    using L = OpLayout<OP, KC>;
    constexpr bool LOW = (OP == TP_OP_A || OP == TP_OP_B0);
    T r2 = r2_eps(dx, dy, dz);
    if (OP == TP_OP_L) {
        T h = pow_(r2, -l_exp);
        if (SELF) h = r2 > T(2) * tiny_r2<T>() ? h : T(0);
#pragma unroll
        for (int i = 0; i < L::NA / 2; ++i) pt[i] = pfma(h, x2[i], pt[i]);
    } else {
        T hB = pow_(r2, -s_exp);
        if (SELF) hB = r2 > T(2) * tiny_r2<T>() ? hB : T(0);
#pragma unroll
        for (int i = 0; i < L::NH / 2; ++i) pt[i] = pfma(hB, x2[i], pt[i]);
        if (LOW) {
            T ir2 = rcp_(r2);
            T tS = (nx * dx + ny * dy + nz * dz) * ir2;
            T tT = (mx * dx + my * dy + mz * dz) * ir2;
            T h0 = T(0.5) * fma(tS, tS, tT * tT) * hB;   // (k2(S;T) + k2(T;S)) / 2 * |d|^{-2s}
#pragma unroll
            for (int i = L::NH / 2; i < L::NA / 2; ++i) pt[i] = pfma(h0, x2[i], pt[i]);
        }
    }
}

template <typename T, int OP, int TT, int KC>
__global__ void __launch_bounds__(NT)
k_apply(const typename V4T<T>::type* __restrict__ fa, const typename V4T<T>::type* __restrict__ fb,
        const float4* __restrict__ flo, const float4* __restrict__ tbox, const double* __restrict__ center,
        const typename V4T<T>::type* __restrict__ Wp, int nf, int tiles_per_split, T s_exp,
        T l_exp, double* __restrict__ part) {
    using V4 = typename V4T<T>::type;
    using L = OpLayout<OP, KC>;
    constexpr bool LOW = (OP == TP_OP_A || OP == TP_OP_B0);
    constexpr bool F32 = sizeof(T) == 4;
    __shared__ V4 sa[NT];
    __shared__ V4 sb[LOW ? NT : 1];
    __shared__ V4 sw[NT * L::NW4];
    __shared__ float4 shl[F32 ? NT : 1];
    __shared__ float sbox[6];
    T tx[TT], ty[TT], tz[TT], nx[TT], ny[TT], nz[TT];
    float lx[TT], ly[TT], lz[TT];
    int tid[TT];
    float bl[3] = {3e38f, 3e38f, 3e38f}, bh[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int j = 0; j < TT; ++j) {
        const int t = blockIdx.x * NT * TT + j * NT + threadIdx.x;
        tid[j] = t;
        tx[j] = ty[j] = tz[j] = nx[j] = ny[j] = nz[j] = T(0);
        lx[j] = ly[j] = lz[j] = 0.f;
        if (t < nf) {
            V4 A = fa[t];
            tx[j] = A.x; ty[j] = A.y; tz[j] = A.z;
            if (LOW) {
                V4 B = fb[t];
                nx[j] = B.x; ny[j] = B.y; nz[j] = B.z;
            }
            if (F32) {
                float4 Lo = flo[t];
                lx[j] = Lo.x; ly[j] = Lo.y; lz[j] = Lo.z;
                bl[0] = fminf(bl[0], (float)A.x); bl[1] = fminf(bl[1], (float)A.y); bl[2] = fminf(bl[2], (float)A.z);
                bh[0] = fmaxf(bh[0], (float)A.x); bh[1] = fmaxf(bh[1], (float)A.y); bh[2] = fmaxf(bh[2], (float)A.z);
            }
        }
    }
    float thr2 = 0.f;
    if (F32) {
        block_box(bl[0], bl[1], bl[2], bh[0], bh[1], bh[2], sbox);
        thr2 = (float)center[3];
    }
    using P2 = typename P2T<T>::type;
    constexpr int NP = L::NA / 2;   // accumulator pairs
    Acc2<T> acc[TT][NP];
    const int ntiles = (nf + NT - 1) / NT;
    const int k0 = blockIdx.y * tiles_per_split;
    const int k1 = min(k0 + tiles_per_split, ntiles);
    for (int tile = k0; tile < k1; ++tile) {
        // tiles holding this block's own targets (self pairs) or lying near them
        // take the careful path: compensated differences and the self-pair test
        const bool diag = tile >= (int)blockIdx.x * TT && tile < ((int)blockIdx.x + 1) * TT;
        const bool near = F32 && tile_near(tbox, tile, sbox, thr2);
        int src = tile * NT + threadIdx.x;
        __syncthreads();
        sa[threadIdx.x] = src < nf ? fa[src] : v4zero<T>();
        if (LOW) sb[threadIdx.x] = src < nf ? fb[src] : v4zero<T>();
        if (near) shl[threadIdx.x] = src < nf ? flo[src] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = threadIdx.x; i < NT * L::NW4; i += NT) {
            int f = tile * NT + i / L::NW4;
            sw[i] = f < nf ? Wp[(size_t)tile * NT * L::NW4 + i] : v4zero<T>();
        }
        __syncthreads();
        for (int c = 0; c < NT; c += CH) {
            P2 pt[TT][NP];
#pragma unroll
            for (int j = 0; j < TT; ++j)
#pragma unroll
                for (int i = 0; i < NP; ++i) pt[j][i] = p2zero<T>();
            if (near || diag) {
                for (int q = 0; q < CH; ++q) {
                    const int jj = c + q;
                    V4 s = sa[jj];
                    float4 l = near ? shl[jj] : make_float4(0.f, 0.f, 0.f, 0.f);
                    P2 wv[2 * L::NW4];
#pragma unroll
                    for (int i = 0; i < L::NW4; ++i) {
                        V4 x = sw[jj * L::NW4 + i];
                        wv[2 * i].x = x.x; wv[2 * i].y = x.y; wv[2 * i + 1].x = x.z; wv[2 * i + 1].y = x.w;
                    }
                    T mx = 0, my = 0, mz = 0;
                    if (LOW) {
                        V4 n = sb[jj];
                        mx = n.x; my = n.y; mz = n.z;
                    }
#pragma unroll
                    for (int j = 0; j < TT; ++j)
                        apply_term<T, OP, true, KC>((tx[j] - s.x) + (T)(lx[j] - l.x), (ty[j] - s.y) + (T)(ly[j] - l.y),
                                                    (tz[j] - s.z) + (T)(lz[j] - l.z), nx[j], ny[j], nz[j], mx,
                                                    my, mz, wv, s_exp, l_exp, pt[j]);
                }
            } else {
#pragma unroll 2
                for (int q = 0; q < CH; ++q) {
                    const int jj = c + q;
                    V4 s = sa[jj];
                    P2 wv[2 * L::NW4];
#pragma unroll
                    for (int i = 0; i < L::NW4; ++i) {
                        V4 x = sw[jj * L::NW4 + i];
                        wv[2 * i].x = x.x; wv[2 * i].y = x.y; wv[2 * i + 1].x = x.z; wv[2 * i + 1].y = x.w;
                    }
                    T mx = 0, my = 0, mz = 0;
                    if (LOW) {
                        V4 n = sb[jj];
                        mx = n.x; my = n.y; mz = n.z;
                    }
#pragma unroll
                    for (int j = 0; j < TT; ++j)
                        apply_term<T, OP, false, KC>(tx[j] - s.x, ty[j] - s.y, tz[j] - s.z, nx[j], ny[j], nz[j],
                                                     mx, my, mz, wv, s_exp, l_exp, pt[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < TT; ++j)
#pragma unroll
                for (int i = 0; i < NP; ++i) acc[j][i].add(pt[j][i]);
        }
    }
#pragma unroll
    for (int j = 0; j < TT; ++j)
        if (tid[j] < nf)
#pragma unroll
            for (int i = 0; i < L::NA; ++i)
                part[((size_t)blockIdx.y * L::NA + i) * nf + tid[j]] = acc[j][i / 2].value(i & 1);
}

// ---- 9-column products with two targets per thread -------------------------
// The FP32 path of the 9-column products (the lockstep solver applies A and
// L^{2-s} to three right-hand sides at once) takes two targets per thread.
// The kernel value of a (target, source) pair is evaluated for both targets
// in packed f32x2 arithmetic, from source geometry staged pre-broadcast in
// shared memory ({x,x}, {y,y}, ...), and each source vector X is read from
// shared memory once for both targets. The per-chunk FP32 sums stay in
// registers; the Kahan pairs that carry them across chunks live in shared
// memory (one float4 {s.x, s.y, c.x, c.y} per thread, target and accumulator
// pair), which keeps the registers for the two targets' chunk sums. Tiles
// near the block's targets or holding them take the careful scalar path of
// k_apply (compensated differences, self-pair test). Partial sums leave as
// FP32 Kahan pairs (s, c), one per split.

constexpr int WT = 2;   // targets per thread of the wide kernel

// packed kernel values of one source for two targets (lanes): hB = |d|^{-2s}
// (= (|d|^2)^{-s}), h0 = (k2(S;T) + k2(T;S)) / 2 * hB (LOW operators), hL =
// |d|^{-2(3-s)} (operator L, returned in hB). t* / n*: the two targets'
// barycenters and normals; s* / m*: the source's barycenter and normal in both
// lanes; eps: the |d|^2 offset; ne: minus the exponent; half: 0.5 in both lanes.
// d = X_target - X_source as packed pairs; with COMP (tiles near the block's
// targets) plus the difference of the low parts of the barycenters,
// (hi_T - hi_S) + (lo_T - lo_S), as in the scalar careful path
template <bool COMP>
__device__ __forceinline__ void wide_diff2(unsigned long long tx, unsigned long long ty, unsigned long long tz,
                                           unsigned long long sx, unsigned long long sy, unsigned long long sz,
                                           unsigned long long lx, unsigned long long ly, unsigned long long lz,
                                           unsigned long long ux, unsigned long long uy, unsigned long long uz,
                                           unsigned long long& dx, unsigned long long& dy, unsigned long long& dz) {
    if constexpr (COMP) {
        asm("{\n\t.reg .b64 ex, ey, ez;\n\t"
            "sub.rn.f32x2 %0, %3, %6;\n\t"
            "sub.rn.f32x2 %1, %4, %7;\n\t"
            "sub.rn.f32x2 %2, %5, %8;\n\t"
            "sub.rn.f32x2 ex, %9, %12;\n\t"
            "sub.rn.f32x2 ey, %10, %13;\n\t"
            "sub.rn.f32x2 ez, %11, %14;\n\t"
            "add.rn.f32x2 %0, %0, ex;\n\t"
            "add.rn.f32x2 %1, %1, ey;\n\t"
            "add.rn.f32x2 %2, %2, ez;\n\t}"
            : "=l"(dx), "=l"(dy), "=l"(dz)
            : "l"(tx), "l"(ty), "l"(tz), "l"(sx), "l"(sy), "l"(sz), "l"(lx), "l"(ly), "l"(lz), "l"(ux), "l"(uy),
              "l"(uz));
    } else {
        asm("sub.rn.f32x2 %0, %3, %6;\n\t"
            "sub.rn.f32x2 %1, %4, %7;\n\t"
            "sub.rn.f32x2 %2, %5, %8;"
            : "=l"(dx), "=l"(dy), "=l"(dz)
            : "l"(tx), "l"(ty), "l"(tz), "l"(sx), "l"(sy), "l"(sz));
    }
}

template <bool LOW>
__device__ __forceinline__ void wide_kernel2(unsigned long long dx_, unsigned long long dy_, unsigned long long dz_,
                                             unsigned long long nx, unsigned long long ny, unsigned long long nz,
                                             unsigned long long mx, unsigned long long my, unsigned long long mz,
                                             unsigned long long eps, unsigned long long ne, unsigned long long half,
                                             unsigned long long& hb, unsigned long long& h0) {
    if constexpr (LOW) {
        asm("{\n\t.reg .b64 dx, dy, dz, r2, lg, ir2, ts, tt;\n\t.reg .f32 lo, hi;\n\t"
            "mov.b64 dx, %2;\n\t"
            "mov.b64 dy, %3;\n\t"
            "mov.b64 dz, %4;\n\t"
            "fma.rn.f32x2 r2, dz, dz, %14;\n\t"
            "fma.rn.f32x2 r2, dy, dy, r2;\n\t"
            "fma.rn.f32x2 r2, dx, dx, r2;\n\t"
            "mov.b64 {lo, hi}, r2;\n\t"
            "lg2.approx.ftz.f32 lo, lo;\n\t"
            "lg2.approx.ftz.f32 hi, hi;\n\t"
            "mov.b64 lg, {lo, hi};\n\t"
            "mul.rn.f32x2 lg, lg, %15;\n\t"
            "mov.b64 {lo, hi}, lg;\n\t"
            "ex2.approx.ftz.f32 lo, lo;\n\t"
            "ex2.approx.ftz.f32 hi, hi;\n\t"
            "mov.b64 %0, {lo, hi};\n\t"
            "mov.b64 {lo, hi}, r2;\n\t"
            "rcp.approx.ftz.f32 lo, lo;\n\t"
            "rcp.approx.ftz.f32 hi, hi;\n\t"
            "mov.b64 ir2, {lo, hi};\n\t"
            "mul.rn.f32x2 ts, %7, dz;\n\t"
            "fma.rn.f32x2 ts, %6, dy, ts;\n\t"
            "fma.rn.f32x2 ts, %5, dx, ts;\n\t"
            "mul.rn.f32x2 ts, ts, ir2;\n\t"
            "mul.rn.f32x2 tt, %13, dz;\n\t"
            "fma.rn.f32x2 tt, %12, dy, tt;\n\t"
            "fma.rn.f32x2 tt, %11, dx, tt;\n\t"
            "mul.rn.f32x2 tt, tt, ir2;\n\t"
            "mul.rn.f32x2 tt, tt, tt;\n\t"
            "fma.rn.f32x2 tt, ts, ts, tt;\n\t"
            "mul.rn.f32x2 tt, tt, %16;\n\t"
            "mul.rn.f32x2 %1, tt, %0;\n\t}"
            : "=l"(hb), "=l"(h0)
            : "l"(dx_), "l"(dy_), "l"(dz_), "l"(nx), "l"(ny), "l"(nz), "l"(0ull), "l"(0ull), "l"(0ull), "l"(mx),
              "l"(my), "l"(mz), "l"(eps), "l"(ne), "l"(half));
    } else {
        asm("{\n\t.reg .b64 dx, dy, dz, r2, lg;\n\t.reg .f32 lo, hi;\n\t"
            "mov.b64 dx, %1;\n\t"
            "mov.b64 dy, %2;\n\t"
            "mov.b64 dz, %3;\n\t"
            "fma.rn.f32x2 r2, dz, dz, %7;\n\t"
            "fma.rn.f32x2 r2, dy, dy, r2;\n\t"
            "fma.rn.f32x2 r2, dx, dx, r2;\n\t"
            "mov.b64 {lo, hi}, r2;\n\t"
            "lg2.approx.ftz.f32 lo, lo;\n\t"
            "lg2.approx.ftz.f32 hi, hi;\n\t"
            "mov.b64 lg, {lo, hi};\n\t"
            "mul.rn.f32x2 lg, lg, %8;\n\t"
            "mov.b64 {lo, hi}, lg;\n\t"
            "ex2.approx.ftz.f32 lo, lo;\n\t"
            "ex2.approx.ftz.f32 hi, hi;\n\t"
            "mov.b64 %0, {lo, hi};\n\t}"
            : "=l"(hb)
            : "l"(dx_), "l"(dy_), "l"(dz_), "l"(0ull), "l"(0ull), "l"(0ull), "l"(eps), "l"(ne));
        h0 = 0ull;
    }
}

// shared memory of the wide kernel (float4 units): broadcast geometry
// [NT][3], broadcast low parts [NT][2], source vectors [NT][NW4], Kahan pairs
// [NP][WT][NT]
template <int OP>
constexpr size_t wide_smem_bytes() {
    using L = OpLayout<OP, 9>;
    return sizeof(float4) * ((size_t)NT * 3 + 2 * NT + (size_t)NT * L::NW4 + (size_t)(L::NA / 2) * WT * NT);
}

// chunk of CHW sources of the wide kernel on the packed path: both targets'
// kernel values at once, then the accumulations (COMP: compensated d)
template <int OP, bool COMP, int CHW>
__device__ __forceinline__ void wide_chunk(const float4* sg, const float4* sl, const float4* sw, int c0,
                                           unsigned long long TX, unsigned long long TY, unsigned long long TZ,
                                           unsigned long long LX, unsigned long long LY, unsigned long long LZ,
                                           unsigned long long NXp, unsigned long long NYp, unsigned long long NZp,
                                           unsigned long long EPS, unsigned long long NE, unsigned long long HALF,
                                           float2 (&pt)[WT][OpLayout<OP, 9>::NA / 2]) {
    using L = OpLayout<OP, 9>;
    constexpr bool LOW = (OP == TP_OP_A || OP == TP_OP_B0);
    constexpr int NP = L::NA / 2;
    constexpr int NW4 = L::NW4;
    const ulonglong2* sg2 = reinterpret_cast<const ulonglong2*>(sg);
    const ulonglong2* sl2 = reinterpret_cast<const ulonglong2*>(sl);
#pragma unroll 2
    for (int q = 0; q < CHW; ++q) {
        const int jj = c0 + q;
        const ulonglong2 u0 = sg2[3 * jj], u1 = sg2[3 * jj + 1];
        unsigned long long dx, dy, dz, HB, H0;
        if constexpr (COMP) {
            const ulonglong2 v0 = sl2[2 * jj], v1 = sl2[2 * jj + 1];
            wide_diff2<true>(TX, TY, TZ, u0.x, u0.y, u1.x, LX, LY, LZ, v0.x, v0.y, v1.x, dx, dy, dz);
        } else {
            wide_diff2<false>(TX, TY, TZ, u0.x, u0.y, u1.x, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, dx, dy, dz);
        }
        if constexpr (LOW) {
            const ulonglong2 u2 = sg2[3 * jj + 2];
            wide_kernel2<true>(dx, dy, dz, NXp, NYp, NZp, u2.x, u2.y, u1.y, EPS, NE, HALF, HB, H0);
        } else {
            wide_kernel2<false>(dx, dy, dz, NXp, NYp, NZp, 0ull, 0ull, 0ull, EPS, NE, HALF, HB, H0);
        }
        const float2 hb = upk2(HB), h0 = upk2(H0);
        float2 x2[2 * NW4];
#pragma unroll
        for (int i = 0; i < NW4; ++i) {
            const float4 x = sw[jj * NW4 + i];
            x2[2 * i] = make_float2(x.x, x.y);
            x2[2 * i + 1] = make_float2(x.z, x.w);
        }
        if (OP == TP_OP_L) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                pt[0][i] = pfma(hb.x, x2[i], pt[0][i]);
                pt[1][i] = pfma(hb.y, x2[i], pt[1][i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < L::NH / 2; ++i) {
                pt[0][i] = pfma(hb.x, x2[i], pt[0][i]);
                pt[1][i] = pfma(hb.y, x2[i], pt[1][i]);
            }
            if (LOW) {
#pragma unroll
                for (int i = L::NH / 2; i < NP; ++i) {
                    pt[0][i] = pfma(h0.x, x2[i], pt[0][i]);
                    pt[1][i] = pfma(h0.y, x2[i], pt[1][i]);
                }
            }
        }
    }
}

template <int OP, int CHW>
__global__ void __launch_bounds__(NT, 2)
k_apply_wide(const float4* __restrict__ fa, const float4* __restrict__ fb, const float4* __restrict__ flo,
             const float4* __restrict__ tbox, const double* __restrict__ center, const float4* __restrict__ Wp,
             int nf, int tiles_per_split, float s_exp, float l_exp, float2* __restrict__ part) {
    using L = OpLayout<OP, 9>;
    constexpr bool LOW = (OP == TP_OP_A || OP == TP_OP_B0);
    constexpr int NP = L::NA / 2;
    constexpr int NW4 = L::NW4;
    extern __shared__ float4 wsm[];
    float4* sg = wsm;                        // broadcast geometry: {x,x,y,y} {z,z,nz,nz} {nx,nx,ny,ny}
    float4* sl = sg + 3 * NT;                // broadcast low parts (near tiles): {lx,lx,ly,ly} {lz,lz,0,0}
    float4* sw = sl + 2 * NT;                // source vectors X
    float4* kah = sw + NT * NW4;             // Kahan pairs {s.x, s.y, c.x, c.y}
    __shared__ float sbox[6];
    const int tid = threadIdx.x;
    float tx[WT], ty[WT], tz[WT], nx[WT], ny[WT], nz[WT], lx[WT], ly[WT], lz[WT];
    int tg[WT];
    float bl[3] = {3e38f, 3e38f, 3e38f}, bh[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int j = 0; j < WT; ++j) {
        const int t = blockIdx.x * NT * WT + j * NT + tid;
        tg[j] = t;
        tx[j] = ty[j] = tz[j] = nx[j] = ny[j] = nz[j] = 0.f;
        lx[j] = ly[j] = lz[j] = 0.f;
        if (t < nf) {
            const float4 A = fa[t];
            tx[j] = A.x; ty[j] = A.y; tz[j] = A.z;
            if (LOW) {
                const float4 B = fb[t];
                nx[j] = B.x; ny[j] = B.y; nz[j] = B.z;
            }
            const float4 Lo = flo[t];
            lx[j] = Lo.x; ly[j] = Lo.y; lz[j] = Lo.z;
            bl[0] = fminf(bl[0], A.x); bl[1] = fminf(bl[1], A.y); bl[2] = fminf(bl[2], A.z);
            bh[0] = fmaxf(bh[0], A.x); bh[1] = fmaxf(bh[1], A.y); bh[2] = fmaxf(bh[2], A.z);
        }
    }
    block_box(bl[0], bl[1], bl[2], bh[0], bh[1], bh[2], sbox);
    const float thr2 = (float)center[3];
    const unsigned long long TX = pk2(tx[0], tx[1]), TY = pk2(ty[0], ty[1]), TZ = pk2(tz[0], tz[1]);
    const unsigned long long LX = pk2(lx[0], lx[1]), LY = pk2(ly[0], ly[1]), LZ = pk2(lz[0], lz[1]);
    const unsigned long long NXp = pk2(nx[0], nx[1]), NYp = pk2(ny[0], ny[1]), NZp = pk2(nz[0], nz[1]);
    const unsigned long long EPS = pk2(tiny_r2<float>(), tiny_r2<float>());
    const float nexp = OP == TP_OP_L ? -l_exp : -s_exp;
    const unsigned long long NE = pk2(nexp, nexp), HALF = pk2(0.5f, 0.5f);
#pragma unroll
    for (int i = 0; i < NP * WT; ++i) kah[i * NT + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int ntiles = (nf + NT - 1) / NT;
    const int k0 = blockIdx.y * tiles_per_split;
    const int k1 = min(k0 + tiles_per_split, ntiles);
    for (int tile = k0; tile < k1; ++tile) {
        const bool diag = tile >= (int)blockIdx.x * WT && tile < ((int)blockIdx.x + 1) * WT;
        const bool near = tile_near(tbox, tile, sbox, thr2);
        const int src = tile * NT + tid;
        __syncthreads();
        {
            // sources past the end sit far away with zero vectors: finite zero terms
            const float4 A = src < nf ? fa[src] : make_float4(1e18f, 0.f, 0.f, 0.f);
            const float4 B = (LOW && src < nf) ? fb[src] : make_float4(0.f, 0.f, 0.f, 0.f);
            sg[3 * tid] = make_float4(A.x, A.x, A.y, A.y);
            sg[3 * tid + 1] = make_float4(A.z, A.z, B.z, B.z);
            sg[3 * tid + 2] = make_float4(B.x, B.x, B.y, B.y);
            if (near || diag) {
                const float4 l = src < nf ? flo[src] : make_float4(0.f, 0.f, 0.f, 0.f);
                sl[2 * tid] = make_float4(l.x, l.x, l.y, l.y);
                sl[2 * tid + 1] = make_float4(l.z, l.z, 0.f, 0.f);
            }
        }
        for (int i = tid; i < NT * NW4; i += NT) {
            const int f = tile * NT + i / NW4;
            sw[i] = f < nf ? Wp[(size_t)tile * NT * NW4 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        for (int c = 0; c < NT; c += CHW) {
            float2 pt[WT][NP];
#pragma unroll
            for (int j = 0; j < WT; ++j)
#pragma unroll
                for (int i = 0; i < NP; ++i) pt[j][i] = make_float2(0.f, 0.f);
            if (diag) {
                // tiles holding the block's own targets: scalar careful path with
                // the self-pair test
                for (int q = 0; q < CHW; ++q) {
                    const int jj = c + q;
                    const float4 g0 = sg[3 * jj], g1 = sg[3 * jj + 1], g2 = sg[3 * jj + 2];
                    const float4 l0 = sl[2 * jj], l1 = sl[2 * jj + 1];
                    float2 wv[2 * NW4];
#pragma unroll
                    for (int i = 0; i < NW4; ++i) {
                        const float4 x = sw[jj * NW4 + i];
                        wv[2 * i] = make_float2(x.x, x.y);
                        wv[2 * i + 1] = make_float2(x.z, x.w);
                    }
#pragma unroll
                    for (int j = 0; j < WT; ++j)
                        apply_term<float, OP, true, 9>((tx[j] - g0.x) + (lx[j] - l0.x), (ty[j] - g0.z) + (ly[j] - l0.z),
                                                       (tz[j] - g1.x) + (lz[j] - l1.x), nx[j], ny[j], nz[j], g2.x,
                                                       g2.z, g1.z, wv, s_exp, l_exp, pt[j]);
                }
            } else if (near) {
                wide_chunk<OP, true, CHW>(sg, sl, sw, c, TX, TY, TZ, LX, LY, LZ, NXp, NYp, NZp, EPS, NE, HALF, pt);
            } else {
                wide_chunk<OP, false, CHW>(sg, sl, sw, c, TX, TY, TZ, LX, LY, LZ, NXp, NYp, NZp, EPS, NE, HALF, pt);
            }
            // chunk sums into the Kahan pairs in shared memory
#pragma unroll
            for (int j = 0; j < WT; ++j)
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    float4& k = kah[(i * WT + j) * NT + tid];
                    const float4 kv = k;
                    const float2 s = make_float2(kv.x, kv.y), cc = make_float2(kv.z, kv.w);
                    const float2 y = psub(pt[j][i], cc);
                    const float2 t = padd(s, y);
                    const float2 cn = psub(psub(t, s), y);
                    k = make_float4(t.x, t.y, cn.x, cn.y);
                }
        }
    }
#pragma unroll
    for (int j = 0; j < WT; ++j)
        if (tg[j] < nf)
#pragma unroll
            for (int a = 0; a < L::NA; ++a) {
                const float4 kv = kah[((a / 2) * WT + j) * NT + tid];
                part[((size_t)blockIdx.y * L::NA + a) * nf + tg[j]] =
                    (a & 1) ? make_float2(kv.y, kv.w) : make_float2(kv.x, kv.z);
            }
}

// sums over the source splits of the wide kernel's partial Kahan pairs, one
// thread per (accumulator, face): the values s_k and -c_k of the splits in a
// fixed order with FP32 compensation, the result (double)S - (double)C
__global__ void k_split_sum2(const float2* __restrict__ part, int nsplit, int na, int nf, double* __restrict__ out) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)na * nf) return;
    float a = 0.f, ca = 0.f;
#pragma unroll 4
    for (int sp = 0; sp < nsplit; ++sp) {
        const float2 v = part[(size_t)sp * na * nf + idx];
        float y = v.x - ca;
        float t = a + y;
        ca = (t - a) - y;
        a = t;
        y = -v.y - ca;
        t = a + y;
        ca = (t - a) - y;
        a = t;
    }
    out[idx] = (double)a - (double)ca;
}

// The FP64 combine from the split sums of k_split_sum2 (accumulator a of face
// S at sums[a * nf + S]): one thread per (face S, column c), a block per
// SC_FACES faces. Thread (S, c) forms z = (r/a) W_S - (H W)_S for column c,
// then the corner values of the transposed map: 2 a_S grad phi_cr . zV (B)
// and 2 a_S zU / 3 (B0, L). 1/a_S is taken once per face, in shared memory.
constexpr int SC_FACES = 32;
template <int OP, int KC>
__global__ void __launch_bounds__(SC_FACES * KC)
k_apply_combine2(const double* __restrict__ sums, int nf, const d4* __restrict__ f64a,
                 const double* __restrict__ fgrad, const double* __restrict__ W64, int k, int col0,
                 double* __restrict__ corner) {
    using L = OpLayout<OP, KC>;
    __shared__ double s_inv[SC_FACES], s_a[SC_FACES];
    const int S0 = blockIdx.x * SC_FACES;
    if (threadIdx.x < SC_FACES && S0 + threadIdx.x < nf) {
        const double a = f64a[S0 + threadIdx.x].w;
        s_a[threadIdx.x] = a;
        s_inv[threadIdx.x] = 1.0 / a;
    }
    __syncthreads();
    const int fl = threadIdx.x / KC, c = threadIdx.x - fl * KC;
    const int S = S0 + fl;
    if (S >= nf || col0 + c >= k) return;
    const double* ps = sums + S;
    const double a = s_a[fl], ia = s_inv[fl];
    const double* W = W64 + 4 * KC * (size_t)S;
    double zV[3] = {0.0, 0.0, 0.0}, zU = 0.0;
    if (L::HIGH) {
        const double r = ps[0] * ia;
#pragma unroll
        for (int q = 0; q < 3; ++q) zV[q] = r * W[q * KC + c] - ps[(size_t)(1 + q * KC + c) * nf];
    }
    if (L::USEU) {
        const double r = ps[(size_t)L::NH * nf] * ia;
        zU = r * W[3 * KC + c] - ps[(size_t)(L::NH + 1 + c) * nf];
    }
    const double* gr = fgrad + 9 * (size_t)S;
#pragma unroll
    for (int cr = 0; cr < 3; ++cr) {
        const double g = gr[3 * cr] * zV[0] + gr[3 * cr + 1] * zV[1] + gr[3 * cr + 2] * zV[2];
        corner[((size_t)S * 3 + cr) * k + col0 + c] = 2.0 * a * (g + zU * (1.0 / 3.0));
    }
}

// per face: z = (r/a) W_S - (H W)_S in FP64, then the corner values of the
// transposed map: 2 a_S grad phi_c . zV (B) and 2 a_S zU / 3 (B0, L)
// (perm != null: the partials are in sorted order, thread t combines face
// perm[t] from partial row t)
template <int OP, int KC>
__global__ void k_apply_combine(const double* __restrict__ part, int nsplit, int nf,
                                const d4* __restrict__ f64a, const double* __restrict__ fgrad,
                                const double* __restrict__ W64, int k, int col0,
                                double* __restrict__ corner, const int* __restrict__ perm) {
    using L = OpLayout<OP, KC>;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf) return;
    const int S = perm ? perm[t] : t;
    double s[L::NA];
    for (int i = 0; i < L::NA; ++i) {
        double x = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) x += part[((size_t)sp * L::NA + i) * nf + t];
        s[i] = x;
    }
    double a = f64a[S].w;
    const double* W = W64 + 4 * KC * (size_t)S;
    double zV[3 * KC], zU[KC];
    for (int i = 0; i < 3 * KC; ++i) zV[i] = 0.0;
    for (int i = 0; i < KC; ++i) zU[i] = 0.0;
    int o = 0;
    if (L::HIGH) {
        double r = s[0] / a;
        for (int i = 0; i < 3 * KC; ++i) zV[i] = r * W[i] - s[1 + i];
        o = 1 + 3 * KC;
    }
    if (L::USEU) {
        double r = s[o] / a;
        for (int c = 0; c < KC; ++c) zU[c] = r * W[3 * KC + c] - s[o + 1 + c];
    }
    for (int cr = 0; cr < 3; ++cr)
        for (int c = 0; c < KC && col0 + c < k; ++c) {
            double g = 0.0;
            for (int q = 0; q < 3; ++q) g += fgrad[9 * S + 3 * cr + q] * zV[q * KC + c];
            corner[((size_t)S * 3 + cr) * k + col0 + c] = 2.0 * a * (g + zU[c] * (1.0 / 3.0));
        }
}

template <typename T, int OP, int KC>
static int launch_apply_op(tp_mesh* m, const tp_params* p, const double* v, int k, double* y,
                           cudaStream_t st) {
    using V4 = typename V4T<T>::type;
    using L = OpLayout<OP, KC>;
    const int nf = m->nf;
    const double s = 2.0 - 2.0 / p->p;       // Sobolev order, §2.3
    const double l_exp = 3.0 - s;            // |d|^{-(2 sigma + 2)} = r2^{-(sigma+1)}, sigma = 2 - s
    constexpr int TT = (sizeof(T) == 4 && KC == 3) ? 2 : 1;
    Grid g = make_grid(nf, nf, TT, resident_per_sm((const void*)k_apply<T, OP, TT, KC>, NT));
    TP_TRY(ensure(m->part, sizeof(double) * (size_t)g.nsplit * L::NA * nf));
    TP_TRY(ensure(m->wv64, sizeof(double) * 4 * KC * (size_t)nf));
    TP_TRY(ensure(m->wv32, sizeof(V4) * L::NW4 * (size_t)nf));
    TP_TRY(ensure(m->corner, sizeof(double) * 3 * (size_t)nf * k));
    const V4* fa = (const V4*)(sizeof(T) == 4 ? m->f32a.ptr : m->f64a.ptr);
    const V4* fb = (const V4*)(sizeof(T) == 4 ? m->f32b.ptr : m->f64b.ptr);
    for (int col0 = 0; col0 < k; col0 += KC) {
        k_face_W<T, KC><<<(nf * ((KC + 2) / 3) + 255) / 256, 256, 0, st>>>(v, k, col0, m->faces.as<int>(), nf,
                                                          m->f64a.as<d4>(), m->fgrad.as<double>(), OP,
                                                          m->wv64.as<double>(), m->wv32.as<V4>(), L::NW4);
        TP_LAUNCH_CHECK();
        dim3 grid(g.bx, g.nsplit);
        {
            const double units = (double)nf * (nf - 1);
            m->pairs += units;
            constexpr int key = OP == TP_OP_A ? PK_APPLY_A : OP == TP_OP_B ? PK_APPLY_B
                              : OP == TP_OP_B0 ? PK_APPLY_B0 : PK_APPLY_L;
            ProfScope ps(m, key, units, st);
            m->prof.cols[key] += KC;
            k_apply<T, OP, TT, KC><<<grid, NT, 0, st>>>(fa, fb, m->f32c.as<float4>(), m->tilebox.as<float4>(),
                                                        m->center.as<double>(), m->wv32.as<V4>(), nf,
                                                        g.tiles_per_split, T(s), T(l_exp), m->part.as<double>());
        }
        TP_LAUNCH_CHECK();
        k_apply_combine<OP, KC><<<(nf + 255) / 256, 256, 0, st>>>(m->part.as<double>(), g.nsplit, nf,
                                                                  m->f64a.as<d4>(), m->fgrad.as<double>(),
                                                                  m->wv64.as<double>(), k, col0,
                                                                  m->corner.as<double>(), nullptr);
        TP_LAUNCH_CHECK();
    }
    return corners_to_vertices(m, m->corner.as<double>(), k, y, st);
}

// FP32, 9 columns: the two-targets-per-thread kernel (k_apply_wide)
// ---------------------------------------------------------------------------
// 9-column A apply with the accumulation on tcgen05 tensor cores
// ---------------------------------------------------------------------------
//
// For a block of 128 targets and a tile of 16 sources the CUDA cores form the
// kernel values h_B(S,T) and h_0(S,T) of the A operator (as apply_term); the
// tensor cores then add H_B X_high and H_0 X_low into accumulators in tensor
// memory (X_high = [a, W_V] (28 columns, padded to N = 32), X_low = [a, W_U]
// (10 columns, padded to N = 16)). FP32 accuracy from TF32 operands by the
// split product H X = Hh Xh + Hh Xl + Hl Xh (hi = the value rounded to TF32,
// lo = the rest; the dropped lo x lo term is 2^-22 of the product). Every
// 128 sources (8 tiles) the FP32 accumulators are read back and added into
// Kahan pairs, as the CUDA-core kernel does per 128-source chunk; two sets of
// accumulators alternate so that the read-back overlaps the next chunk's
// products. Operands are K-major in shared memory without swizzle: core
// matrices of 8 rows x 16 bytes (4 TF32 along K), adjacent along K at 128
// bytes (leading byte offset), row groups at 512 bytes (stride byte offset).
// Source tiles (X split into hi and lo in that layout, plus the sources'
// barycenter hi, lo and normal) are packed once per apply by k_tc_pack and
// copied into a ring of three shared buffers with cp.async.bulk, one tile
// ahead. One thread issues the MMAs; mbarriers order the copies, the MMAs and
// the reuse of the buffers; every wait is bounded by one second (an exhausted
// wait stops all further work of the block, sets *err and writes NaN
// partials).

constexpr int TC_KT = 32;                      // sources per tile (four K = 8 steps)
constexpr int TC_KC = TC_KT / 4;               // core matrices along K
constexpr int TC_CHUNK = 128 / TC_KT;          // tiles per FP32 chunk (128 sources)
constexpr int TC_CW = 16;                      // compute warps: target t = tid & 127, source quarter tid >> 7
constexpr int TC_T = 32 * (TC_CW + 1);         // + one warp that loads tiles and issues the MMAs
// packed source tile (bytes): X high hi / lo (32 x KT), X low hi / lo (16 x KT),
// K-major operands; then the sources' geometry by pairs (2p, 2p + 1), five
// float4 per pair: {x0 x1 y0 y1} {z0 z1 nx0 nx1} {ny0 ny1 nz0 nz1}
// {lx0 lx1 ly0 ly1} {lz0 lz1 0 0} (barycenter hi, normal, barycenter lo)
constexpr int TC_XH = 0, TC_XHL = 32 * TC_KT * 4, TC_XL = 2 * 32 * TC_KT * 4, TC_XLL = TC_XL + 16 * TC_KT * 4;
constexpr int TC_G = TC_XLL + 16 * TC_KT * 4;
constexpr int TC_BOX = TC_G + (TC_KT / 2) * 5 * 16;   // bounding box of the tile's 128-source chunk (2 float4)
constexpr int TC_TILE_BYTES = TC_BOX + 32;            // 13600
constexpr int TC_NX = 4;                       // source tile buffers
constexpr int TC_NH = 3;                       // H operand buffers (tensor memory)
constexpr size_t TC_SMEM = TC_NX * (size_t)TC_TILE_BYTES;
// tensor memory: accumulator sets at columns [0, 64) and [64, 128) (32 high + 16 low used each);
// the H operands of the three tile buffers at [128, 256), [256, 384), [384, 512): H_B hi, H_B lo,
// H_0 hi, H_0 lo, KT = 32 columns each, one row (lane) per target
constexpr int TC_HCOL = 128;
constexpr int TC_TMEM_COLS = 512;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;   // bound of each mbarrier wait (1 s)

// byte offset of element (row, k) of a [rows][KT] K-major operand
__device__ __forceinline__ int tc_cm(int row, int k) {
    return (((row >> 3) * TC_KC + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2);
}
__device__ __forceinline__ float tc_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ unsigned tc_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr) {
    // start >> 4, leading byte offset 128 >> 4, stride byte offset (128 TC_KC) >> 4, version 1, no swizzle
    return (unsigned long long)((addr >> 4) & 0x3fffu) | (8ull << 16) | ((unsigned long long)(8 * TC_KC) << 32) |
           (1ull << 46);
}
__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// the same with A in tensor memory (address a)
__device__ __forceinline__ void tc_mma_t(unsigned d, unsigned a, unsigned long long b, unsigned idesc, int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
                 ::"r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ unsigned long long tc_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for the completion of the mbarrier phase with the given
// parity; false when it gave up, or when an earlier wait of the block did
__device__ __forceinline__ bool tc_try(unsigned mbar, unsigned parity) {
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}
// (a waiting warp sleeps between tries, up to max_ns, instead of taking the
// issue slots of the warps it waits for)
__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity, volatile int* abort, unsigned max_ns = 64) {
    if (tc_try(mbar, parity)) return true;   // the common case: no clock read
    const unsigned long long t0 = tc_now();
    unsigned ns = 16;
    for (;;) {
        __nanosleep(ns);
        if (ns < max_ns) ns <<= 1;
        if (*abort) return false;
        if (tc_try(mbar, parity)) return true;
        if (tc_now() - t0 > TC_WAIT_NS) {
            *abort = 1;
            return false;
        }
    }
}

// one thread per (source, column group of 4, or the geometry): the packed
// tiles; sources past nf: X = 0, geometry parked far away
__global__ void k_tc_pack(const float4* __restrict__ Wp, const float4* __restrict__ fa, const float4* __restrict__ flo,
                          const float4* __restrict__ fb, const float4* __restrict__ tbox, int nf, int ntile,
                          unsigned char* __restrict__ tiles) {
    constexpr int NW4 = OpLayout<TP_OP_A, 9>::NW4;   // 10 float4: [a, W_V (27), a, W_U (9), 0, 0]
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = idx / (NW4 + 1), q = idx - j * (NW4 + 1);
    if (j >= ntile * TC_KT) return;
    unsigned char* T = tiles + (size_t)(j / TC_KT) * TC_TILE_BYTES;
    const int k = j % TC_KT;
    const bool ok = j < nf;
    if (q == NW4) {   // geometry, by pairs of sources
        const float4 S = ok ? fa[j] : make_float4(1e15f, 1e15f, 1e15f, 0.f);
        const float4 Sl = ok ? flo[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 Sn = ok ? fb[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        float* P = reinterpret_cast<float*>(T + TC_G) + (k >> 1) * 20;
        const int e = k & 1;
        P[0 + e] = S.x;   P[2 + e] = S.y;
        P[4 + e] = S.z;   P[6 + e] = Sn.x;
        P[8 + e] = Sn.y;  P[10 + e] = Sn.z;
        P[12 + e] = Sl.x; P[14 + e] = Sl.y;
        P[16 + e] = Sl.z; P[18 + e] = 0.f;
        if (k == 0) {   // the box of the 128-source chunk (k_tile_boxes), for the near-tile test
            float4* B = reinterpret_cast<float4*>(T + TC_BOX);
            const int ch = j >> 7;
            B[0] = tbox[2 * ch];
            B[1] = tbox[2 * ch + 1];
        }
        return;
    }
    const float4 w = ok ? Wp[(size_t)j * NW4 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int a = 4 * q + e;   // accumulator index in [a, W_V, a, W_U]
        if (a >= 38) continue;
        const float hi = tc_tf32(v[e]), lo = v[e] - hi;
        if (a < 28) {
            *reinterpret_cast<float*>(T + TC_XH + tc_cm(a, k)) = hi;
            *reinterpret_cast<float*>(T + TC_XHL + tc_cm(a, k)) = lo;
        } else {
            *reinterpret_cast<float*>(T + TC_XL + tc_cm(a - 28, k)) = hi;
            *reinterpret_cast<float*>(T + TC_XLL + tc_cm(a - 28, k)) = lo;
        }
    }
    if (q == 0) {   // the padding rows: high 28..31, low 10..15
        for (int a = 28; a < 32; ++a) {
            *reinterpret_cast<float*>(T + TC_XH + tc_cm(a, k)) = 0.f;
            *reinterpret_cast<float*>(T + TC_XHL + tc_cm(a, k)) = 0.f;
        }
        for (int a = 10; a < 16; ++a) {
            *reinterpret_cast<float*>(T + TC_XL + tc_cm(a, k)) = 0.f;
            *reinterpret_cast<float*>(T + TC_XLL + tc_cm(a, k)) = 0.f;
        }
    }
}

// Warp-specialised: warps 0..15 form the kernel values (four threads per
// target row, eight sources each, two sources per packed f32x2 instruction)
// into the H buffer of the tile and arrive on its "full" barrier; warp 16
// (one lane) keeps the tile buffers filled with cp.async.bulk, issues the
// 24 MMAs of each tile once its H buffer is full and commits them to the
// buffer's "done" barrier, which frees the H buffer and the tile buffer.
// Barriers: done[2] (per H buffer), full[2] (per H buffer, 16 arrivals),
// tile[3] (per tile buffer, transaction bytes). One block per SM (17 warps);
// a warp reads back the accumulator columns of its quarter of the rows.
__global__ void __maxnreg__(96)
k_apply_tc(const float4* __restrict__ fa, const float4* __restrict__ fb, const float4* __restrict__ flo,
           const float4* __restrict__ tbox, const double* __restrict__ center, const unsigned char* __restrict__ tiles,
           int nf, int ntile, int tiles_per_split, float s_exp, float2* __restrict__ part, int* __restrict__ err) {
    constexpr int NA = OpLayout<TP_OP_A, 9>::NA;   // 38
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) unsigned long long mbar[2 * TC_NH + TC_NX];
    __shared__ unsigned s_taddr;
    __shared__ int s_abort;
    __shared__ float s_wb[4][6];   // bounding boxes of the block's targets, per warp of rows
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp < 4) {
        const int tb = blockIdx.x * 128 + tid;
        float4 A = tb < nf ? fa[tb] : make_float4(3e38f, 3e38f, 3e38f, 0.f);
        float lx = A.x, ly = A.y, lz = A.z;
        if (tb >= nf) A = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
        float hx = A.x, hy = A.y, hz = A.z;
        for (int o = 16; o > 0; o >>= 1) {
            lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
            ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
            lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        }
        if (lane == 0) {
            s_wb[warp][0] = lx; s_wb[warp][1] = ly; s_wb[warp][2] = lz;
            s_wb[warp][3] = hx; s_wb[warp][4] = hy; s_wb[warp][5] = hz;
        }
    }
    const int q0 = blockIdx.y * tiles_per_split, q1 = min(ntile, q0 + tiles_per_split), nt = max(0, q1 - q0);
    unsigned char* Xb = tsm;                    // TC_NX x TC_TILE_BYTES
    const unsigned mb_done = tc_smem(&mbar[0]), mb_full = tc_smem(&mbar[TC_NH]), mb_tile = tc_smem(&mbar[2 * TC_NH]);
    if (warp == TC_CW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&s_taddr)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < TC_NH; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_done + 8 * i));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb_full + 8 * i), "r"(TC_CW));
        }
        for (int i = 0; i < TC_NX; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_tile + 8 * i));
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned taddr = s_taddr;
    volatile int* abort = &s_abort;

    if (warp == TC_CW) {
        // ---- loads and products
        if (lane == 0) {
            auto issue_copy = [&](int q) {   // tile q0 + q into buffer q % TC_NX
                const unsigned mb = mb_tile + 8 * (q % TC_NX);
                const unsigned dst = tc_smem(Xb + (q % TC_NX) * TC_TILE_BYTES);
                const unsigned char* src = tiles + (size_t)(q0 + q) * TC_TILE_BYTES;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(TC_TILE_BYTES)
                             : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(dst), "l"(src), "r"(TC_TILE_BYTES), "r"(mb) : "memory");
            };
            for (int q = 0; q < min(nt, TC_NX); ++q) issue_copy(q);
            const unsigned idH = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
            const unsigned idL = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
            for (int q = 0; q < nt; ++q) {
                const int hb = q % TC_NH;
                if (!tc_wait(mb_full + 8 * hb, (q / TC_NH) & 1, abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int set = (q / TC_CHUNK) & 1;
                const unsigned dH = taddr + (unsigned)(set * 64), dL = dH + 32;
                const unsigned ha = taddr + (unsigned)(TC_HCOL + hb * 128);   // H operands in tensor memory
                const unsigned xbase = tc_smem(Xb + (q % TC_NX) * TC_TILE_BYTES);
#pragma unroll
                for (int kk = 0; kk < TC_KT / 8; ++kk) {
                    const unsigned o = kk * 256;
                    const int acc = ((q % TC_CHUNK) == 0 && kk == 0) ? 0 : 1;
                    const unsigned ka = kk * 8;   // K columns of this step
                    tc_mma_t(dH, ha + 0 * 32 + ka, tc_desc(xbase + TC_XH + o), idH, acc);
                    tc_mma_t(dH, ha + 0 * 32 + ka, tc_desc(xbase + TC_XHL + o), idH, 1);
                    tc_mma_t(dH, ha + 1 * 32 + ka, tc_desc(xbase + TC_XH + o), idH, 1);
                    tc_mma_t(dL, ha + 2 * 32 + ka, tc_desc(xbase + TC_XL + o), idL, acc);
                    tc_mma_t(dL, ha + 2 * 32 + ka, tc_desc(xbase + TC_XLL + o), idL, 1);
                    tc_mma_t(dL, ha + 3 * 32 + ka, tc_desc(xbase + TC_XL + o), idL, 1);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(mb_done + 8 * hb) : "memory");
                // refill the buffer of tile q - 1 with tile q + TC_NX - 1 once its products are done
                if (q >= 1 && q + TC_NX - 1 < nt) {
                    if (!tc_wait(mb_done + 8 * ((q - 1) % TC_NH), ((q - 1) / TC_NH) & 1, abort)) break;
                    issue_copy(q + TC_NX - 1);
                }
            }
        }
    } else {
        // ---- kernel values, read-back of the accumulators
        const int t = tid & 127, sq = tid >> 7;   // row; source quarter of the tile and column group
        const int tg = blockIdx.x * 128 + t;
        const bool tv = tg < nf;
        const float4 T = tv ? fa[tg] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 Tl = tv ? flo[tg] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 Tn = tv ? fb[tg] : make_float4(0.f, 0.f, 0.f, 0.f);
        const unsigned long long TX = pk2(T.x, T.x), TY = pk2(T.y, T.y), TZ = pk2(T.z, T.z);
        const unsigned long long LX = pk2(Tl.x, Tl.x), LY = pk2(Tl.y, Tl.y), LZ = pk2(Tl.z, Tl.z);
        const unsigned long long NX = pk2(Tn.x, Tn.x), NY = pk2(Tn.y, Tn.y), NZ = pk2(Tn.z, Tn.z);
        const unsigned long long EPS = pk2(1e-18f, 1e-18f), NE = pk2(-s_exp, -s_exp), HALF = pk2(0.5f, 0.5f);
        float sbox[6];
        for (int c = 0; c < 3; ++c) {
            sbox[c] = fminf(fminf(s_wb[0][c], s_wb[1][c]), fminf(s_wb[2][c], s_wb[3][c]));
            sbox[3 + c] = fmaxf(fmaxf(s_wb[0][3 + c], s_wb[1][3 + c]), fmaxf(s_wb[2][3 + c], s_wb[3][3 + c]));
        }
        const float thr2 = (float)center[3];
        // accumulator columns 12 sq .. 12 sq + 11 of a set (high 0..31 then low 32..47)
        float ks[12], kc[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) ks[i] = kc[i] = 0.f;
        auto drain = [&](int set) {
            const unsigned base = taddr + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)(set * 64 + 12 * sq);
            unsigned r[12];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                         : "r"(base));
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11])
                         : "r"(base + 8));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 12; ++i) {   // Kahan
                const float y = __uint_as_float(r[i]) - kc[i];
                const float s = ks[i] + y;
                kc[i] = (s - ks[i]) - y;
                ks[i] = s;
            }
        };
        int drained = 0;   // chunks read back
        for (int q = 0; q < nt; ++q) {
            const int hb = q % TC_NH;
            // this tile's sources, and the H buffer of tile q - TC_NH free
            tc_wait(mb_tile + 8 * (q % TC_NX), (q / TC_NX) & 1, abort);
            if (q >= TC_NH) tc_wait(mb_done + 8 * hb, ((q - TC_NH) / TC_NH) & 1, abort);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!*abort) {
                const ulonglong2* G = reinterpret_cast<const ulonglong2*>(Xb + (q % TC_NX) * TC_TILE_BYTES + TC_G);
                const int sg0 = (q0 + q) * TC_KT;
                // tiles on the block's own rows (self pairs) or past nf take the masked path; tiles near
                // the block's targets take the compensated differences (as in k_apply_wide)
                const bool special = (sg0 < (int)blockIdx.x * 128 + 128 && sg0 + TC_KT > (int)blockIdx.x * 128) ||
                                     sg0 + TC_KT > nf;
                const bool near = special || tile_near(reinterpret_cast<const float4*>(Xb + (q % TC_NX) * TC_TILE_BYTES + TC_BOX),
                                                       0, sbox, thr2);
                unsigned long long hBp[4], h0p[4];   // kernel values of sources (2i, 2i + 1) of this thread
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int pp = 4 * sq + i;   // sources 2 pp, 2 pp + 1 of the tile, packed
                    const ulonglong2 Q0 = G[5 * pp], Q1 = G[5 * pp + 1], Q2 = G[5 * pp + 2];
                    unsigned long long dx, dy, dz;
                    if (near) {
                        const ulonglong2 Q3 = G[5 * pp + 3], Q4 = G[5 * pp + 4];
                        wide_diff2<true>(TX, TY, TZ, Q0.x, Q0.y, Q1.x, LX, LY, LZ, Q3.x, Q3.y, Q4.x, dx, dy, dz);
                    } else {
                        wide_diff2<false>(TX, TY, TZ, Q0.x, Q0.y, Q1.x, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, dx, dy, dz);
                    }
                    wide_kernel2<true>(dx, dy, dz, NX, NY, NZ, Q1.y, Q2.x, Q2.y, EPS, NE, HALF, hBp[i], h0p[i]);
                    if (special) {
                        const int s0 = sg0 + 2 * pp, s1 = s0 + 1;
                        const bool on0 = tv && s0 < nf && s0 != tg, on1 = tv && s1 < nf && s1 != tg;
                        const float2 b = upk2(hBp[i]), z = upk2(h0p[i]);
                        hBp[i] = pk2(on0 ? b.x : 0.f, on1 ? b.y : 0.f);
                        h0p[i] = pk2(on0 ? z.x : 0.f, on1 ? z.y : 0.f);
                    }
                }
                // TF32 splits: hi = the value with the 13 mantissa bits below TF32 cleared, lo = value - hi;
                // the thread's 8 K-columns of each operand into its row of tensor memory
                constexpr unsigned long long HI = 0xffffe000ffffe000ull;
                unsigned long long m[4][4];   // [operand][pair]
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const unsigned long long bh = hBp[i] & HI, zh = h0p[i] & HI;
                    unsigned long long bl, zl;
                    asm("sub.rn.f32x2 %0, %2, %4;\n\tsub.rn.f32x2 %1, %3, %5;"
                        : "=l"(bl), "=l"(zl) : "l"(hBp[i]), "l"(h0p[i]), "l"(bh), "l"(zh));
                    m[0][i] = bh; m[1][i] = bl; m[2][i] = zh; m[3][i] = zl;
                }
                const unsigned hrow = taddr + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)(TC_HCOL + hb * 128 + 8 * sq);
#pragma unroll
                for (int op = 0; op < 4; ++op) {
                    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                                 ::"r"(hrow + 32 * op), "r"((unsigned)m[op][0]), "r"((unsigned)(m[op][0] >> 32)),
                                   "r"((unsigned)m[op][1]), "r"((unsigned)(m[op][1] >> 32)), "r"((unsigned)m[op][2]),
                                   "r"((unsigned)(m[op][2] >> 32)), "r"((unsigned)m[op][3]), "r"((unsigned)(m[op][3] >> 32))
                                 : "memory");
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            // the warp's part of H(q) is in tensor memory: ordered before the MMAs
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0 && !*abort) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb_full + 8 * hb)
                                                   : "memory");
            // the previous chunk's accumulators, one tile after its last product was issued: the wait is
            // for tile q - 2, and no later product on that barrier can have completed yet (it needs
            // this warp's arrival for tile q + 1), so its phase is the one waited for
            if ((q % TC_CHUNK) == 1 && q > TC_CHUNK) {
                const bool ok = __all_sync(0xffffffffu, tc_wait(mb_done + 8 * ((q - 2) % TC_NH), ((q - 2) / TC_NH) & 1, abort));
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (ok) drain(drained & 1);
                ++drained;
            }
        }
        // the remaining chunks (their last tiles are among the last three, so no later product
        // shares their barrier phases)
        const int nchunk = (nt + TC_CHUNK - 1) / TC_CHUNK;
        for (; drained < nchunk; ++drained) {
            const int last = min(TC_CHUNK * drained + TC_CHUNK - 1, nt - 1);
            const bool ok = __all_sync(0xffffffffu, tc_wait(mb_done + 8 * (last % TC_NH), (last / TC_NH) & 1, abort));
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok) drain(drained & 1);
        }
        const bool bad = *abort != 0;
        if (tv) {
            const float qnan = __int_as_float(0x7fc00000);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const int c = 12 * sq + i;   // column of the set
                const int a = c < 28 ? c : (c >= 32 && c < 42 ? 28 + (c - 32) : -1);
                if (a < 0) continue;
                part[((size_t)blockIdx.y * NA + a) * nf + tg] = bad ? make_float2(qnan, 0.f) : make_float2(ks[i], kc[i]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(err, 1);
    if (warp == TC_CW) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_TMEM_COLS));
}

// the A apply on 9 columns with tensor-core accumulation (see k_apply_tc)
static int launch_apply_tc(tp_mesh* m, const tp_params* p, const double* v, int k, double* y, cudaStream_t st) {
    using L = OpLayout<TP_OP_A, 9>;
    const int nf = m->nf;
    const double s = 2.0 - 2.0 / p->p;
    static bool carveout_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !carveout_set[dev]) {
        // the whole shared-memory carveout: the kernel needs 172 KB per block
        TP_CUDA(cudaFuncSetAttribute((const void*)k_apply_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        carveout_set[dev] = true;
    }
    const int per_sm = resident_per_sm((const void*)k_apply_tc, TC_T, TC_SMEM);
    if (per_sm < 1) return fail(TP_ERR_CUDA, "k_apply_tc: shared memory per block not available");
    // source splits: blocks = target blocks x splits run in waves of per_sm x SMs; the time goes
    // like waves x (tiles per split + the fixed cost of a block, about 6 tiles)
    const int ntile = (nf + TC_KT - 1) / TC_KT;
    Grid g;
    g.bx = (nf + 127) / 128;
    {
        const long long slots = (long long)per_sm * sm_count();
        long long best = -1;
        for (int ns = 1; ns <= 64 && ns <= ntile; ++ns) {
            const long long tps_ = (ntile + ns - 1) / ns;
            const long long waves = ((long long)g.bx * ns + slots - 1) / slots;
            const long long cost = waves * (tps_ + 6);
            if (best < 0 || cost < best) {
                best = cost;
                g.nsplit = ns;
                g.tiles_per_split = (int)tps_;
            }
        }
    }
    const int tps = g.tiles_per_split;
    TP_TRY(ensure(m->part, sizeof(float2) * (size_t)g.nsplit * L::NA * nf + sizeof(double) * L::NA * (size_t)nf));
    TP_TRY(ensure(m->wv64, sizeof(double) * 4 * 9 * (size_t)nf));
    TP_TRY(ensure(m->wv32, sizeof(float4) * L::NW4 * (size_t)nf));
    TP_TRY(ensure(m->corner, sizeof(double) * 3 * (size_t)nf * k));
    TP_TRY(ensure(m->tcbuf, (size_t)ntile * TC_TILE_BYTES));
    if (!m->tcerr.ptr) {
        TP_TRY(ensure(m->tcerr, 16));
        TP_CUDA(cudaMemsetAsync(m->tcerr.ptr, 0, 16, st));   // fresh memory holds garbage
    }
    int* err = m->tcerr.as<int>();
    const float4* fa = m->f32a.as<float4>();
    const float4* fb = m->f32b.as<float4>();
    const float4* fl = m->f32c.as<float4>();
    for (int col0 = 0; col0 < k; col0 += 9) {
        k_face_W<float, 9><<<(nf * 3 + 255) / 256, 256, 0, st>>>(v, k, col0, m->faces.as<int>(), nf, m->f64a.as<d4>(),
                                                             m->fgrad.as<double>(), TP_OP_A, m->wv64.as<double>(),
                                                             m->wv32.as<float4>(), L::NW4);
        TP_LAUNCH_CHECK();
        const int npack = ntile * TC_KT * (L::NW4 + 1);
        k_tc_pack<<<(npack + 255) / 256, 256, 0, st>>>(m->wv32.as<float4>(), fa, fl, fb, m->tilebox.as<float4>(), nf,
                                                       ntile, m->tcbuf.as<unsigned char>());
        TP_LAUNCH_CHECK();
        {
            const double units = (double)nf * (nf - 1);
            m->pairs += units;
            ProfScope ps(m, PK_APPLY_A, units, st);
            m->prof.cols[PK_APPLY_A] += 9;
            k_apply_tc<<<dim3(g.bx, g.nsplit), TC_T, TC_SMEM, st>>>(fa, fb, fl, m->tilebox.as<float4>(),
                                                                   m->center.as<double>(), m->tcbuf.as<unsigned char>(),
                                                                   nf, ntile, tps, (float)s, m->part.as<float2>(), err);
        }
        TP_LAUNCH_CHECK();
        double* sums = reinterpret_cast<double*>(m->part.as<float2>() + (size_t)g.nsplit * L::NA * nf);
        k_split_sum2<<<(unsigned)(((size_t)L::NA * nf + 255) / 256), 256, 0, st>>>(m->part.as<float2>(), g.nsplit,
                                                                                L::NA, nf, sums);
        TP_LAUNCH_CHECK();
        k_apply_combine2<TP_OP_A, 9><<<(nf + SC_FACES - 1) / SC_FACES, SC_FACES * 9, 0, st>>>(
            sums, nf, m->f64a.as<d4>(), m->fgrad.as<double>(), m->wv64.as<double>(), k, col0, m->corner.as<double>());
        TP_LAUNCH_CHECK();
    }
    return corners_to_vertices(m, m->corner.as<double>(), k, y, st);
}

// the tensor-core wait flag of the mesh's A applies (0 when none gave up), and reset
int apply_tc_error(tp_mesh* m, int* gave_up, cudaStream_t st) {
    *gave_up = 0;
    if (!m->tcerr.ptr) return TP_OK;
    int* err = m->tcerr.as<int>();
    TP_CUDA(cudaMemcpyAsync(gave_up, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    if (*gave_up) TP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    return TP_OK;
}

template <int OP>
static int launch_apply_wide(tp_mesh* m, const tp_params* p, const double* v, int k, double* y, cudaStream_t st) {
    using L = OpLayout<OP, 9>;
    // sources per FP32 chunk sum before the Kahan update: whole tiles for the
    // operators with the high-order part (many accumulators per flush), half
    // tiles for the others
    constexpr int CHW = (OP == TP_OP_A || OP == TP_OP_B) ? 128 : 64;
    const int nf = m->nf;
    const double s = 2.0 - 2.0 / p->p;
    const double l_exp = 3.0 - s;
    const size_t smem = wide_smem_bytes<OP>();
    const int per_sm = resident_per_sm((const void*)k_apply_wide<OP, CHW>, NT, smem);
    if (per_sm < 1) return fail(TP_ERR_CUDA, "k_apply_wide: shared memory per block not available");
    Grid g = make_grid(nf, nf, WT, per_sm);
    TP_TRY(ensure(m->part, sizeof(float2) * (size_t)g.nsplit * L::NA * nf + sizeof(double) * L::NA * (size_t)nf));
    TP_TRY(ensure(m->wv64, sizeof(double) * 4 * 9 * (size_t)nf));
    TP_TRY(ensure(m->wv32, sizeof(float4) * L::NW4 * (size_t)nf));
    TP_TRY(ensure(m->corner, sizeof(double) * 3 * (size_t)nf * k));
    const float4* fa = m->f32a.as<float4>();
    const float4* fb = m->f32b.as<float4>();
    for (int col0 = 0; col0 < k; col0 += 9) {
        k_face_W<float, 9><<<(nf * 3 + 255) / 256, 256, 0, st>>>(v, k, col0, m->faces.as<int>(), nf, m->f64a.as<d4>(),
                                                             m->fgrad.as<double>(), OP, m->wv64.as<double>(),
                                                             m->wv32.as<float4>(), L::NW4);
        TP_LAUNCH_CHECK();
        dim3 grid(g.bx, g.nsplit);
        {
            const double units = (double)nf * (nf - 1);
            m->pairs += units;
            constexpr int key = OP == TP_OP_A ? PK_APPLY_A : OP == TP_OP_B ? PK_APPLY_B
                              : OP == TP_OP_B0 ? PK_APPLY_B0 : PK_APPLY_L;
            ProfScope ps(m, key, units, st);
            m->prof.cols[key] += 9;
            k_apply_wide<OP, CHW><<<grid, NT, smem, st>>>(fa, fb, m->f32c.as<float4>(), m->tilebox.as<float4>(),
                                                          m->center.as<double>(), m->wv32.as<float4>(), nf,
                                                          g.tiles_per_split, (float)s, (float)l_exp,
                                                          m->part.as<float2>());
        }
        TP_LAUNCH_CHECK();
        double* sums = reinterpret_cast<double*>(m->part.as<float2>() + (size_t)g.nsplit * L::NA * nf);
        k_split_sum2<<<(unsigned)(((size_t)L::NA * nf + 255) / 256), 256, 0, st>>>(m->part.as<float2>(), g.nsplit,
                                                                                L::NA, nf, sums);
        TP_LAUNCH_CHECK();
        k_apply_combine2<OP, 9><<<(nf + SC_FACES - 1) / SC_FACES, SC_FACES * 9, 0, st>>>(
            sums, nf, m->f64a.as<d4>(), m->fgrad.as<double>(), m->wv64.as<double>(), k, col0, m->corner.as<double>());
        TP_LAUNCH_CHECK();
    }
    return corners_to_vertices(m, m->corner.as<double>(), k, y, st);
}

template <typename T>
static int launch_apply(tp_mesh* m, const tp_params* p, int op, const double* v, int k, double* y,
                        cudaStream_t st) {
    // 9 columns in one pass share the kernel evaluation; up to 3 columns
    // take the lighter 3-column kernel
    const bool wide = k > 3;
    if (sizeof(T) == 4 && wide) {
        switch (op) {
            case TP_OP_A: return p->tensor_cores ? launch_apply_tc(m, p, v, k, y, st)
                                                 : launch_apply_wide<TP_OP_A>(m, p, v, k, y, st);
            case TP_OP_B: return launch_apply_wide<TP_OP_B>(m, p, v, k, y, st);
            case TP_OP_B0: return launch_apply_wide<TP_OP_B0>(m, p, v, k, y, st);
            case TP_OP_L: return launch_apply_wide<TP_OP_L>(m, p, v, k, y, st);
        }
        return fail(TP_ERR_INVALID_ARG, "unknown operator");
    }
    switch (op) {
        case TP_OP_A: return wide ? launch_apply_op<T, TP_OP_A, 9>(m, p, v, k, y, st)
                                  : launch_apply_op<T, TP_OP_A, 3>(m, p, v, k, y, st);
        case TP_OP_B: return wide ? launch_apply_op<T, TP_OP_B, 9>(m, p, v, k, y, st)
                                  : launch_apply_op<T, TP_OP_B, 3>(m, p, v, k, y, st);
        case TP_OP_B0: return wide ? launch_apply_op<T, TP_OP_B0, 9>(m, p, v, k, y, st)
                                   : launch_apply_op<T, TP_OP_B0, 3>(m, p, v, k, y, st);
        case TP_OP_L: return wide ? launch_apply_op<T, TP_OP_L, 9>(m, p, v, k, y, st)
                                  : launch_apply_op<T, TP_OP_L, 3>(m, p, v, k, y, st);
    }
    return fail(TP_ERR_INVALID_ARG, "unknown operator");
}

// ===========================================================================
// Barnes-Hut operator applies: the kernel-matrix products of §5.1.1-5.1.3
// taken over the admissible sets of §4.1 (the same tree and test as the
// Barnes-Hut energy). An admissible node I contributes h(X_S, P_S; X_I, P_I)
// times the node sums of the source vectors X = [a, W_V, a, W_U]; the
// source-side k_2 of the low-order kernel uses the node-average projector
// P_I = a_I^-1 sum a_T N_T N_T^T (§5.1.4). An inadmissible leaf is summed
// exactly, face by face. The diagonal of [diag(H a / a) - H] uses the same
// approximate row sums, so constants stay in the nullspace.
// ===========================================================================

// sorted copies of the per-face vectors X
template <int NW4>
__global__ void k_sort_X(const float4* __restrict__ Wp, const int* __restrict__ perm, int nf,
                         float4* __restrict__ Ws) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const float4* src = Wp + (size_t)perm[i] * NW4;
    float4* dst = Ws + (size_t)i * NW4;
#pragma unroll
    for (int q = 0; q < NW4; ++q) dst[q] = src[q];
}

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// node sums of X and (PROJ) node-average projectors (upper triangle xx, xy,
// xz, yy, yz, zz in two float4), one depth level per launch, deepest first
template <int NW4, bool PROJ>
__global__ void k_node_X(const BvhNode* __restrict__ node, const int* __restrict__ right,
                         const int* __restrict__ order, int n0, int n1, const float4* __restrict__ Ws,
                         const float4* __restrict__ sa, const float4* __restrict__ sb,
                         float4* __restrict__ nodeX, float4* __restrict__ nodeP) {
    const int k = n0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n1) return;
    const int id = order[k];
    const BvhNode n = node[id];
    float4 acc[NW4];
#pragma unroll
    for (int q = 0; q < NW4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    float P[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (n.leaf) {
        float asum = 0.f;
        for (int i = n.first; i < n.first + n.count; ++i) {
#pragma unroll
            for (int q = 0; q < NW4; ++q) acc[q] = f4add(acc[q], Ws[(size_t)i * NW4 + q]);
            if (PROJ) {
                const float a = sa[i].w;
                const float4 N = sb[i];
                P[0] += a * N.x * N.x; P[1] += a * N.x * N.y; P[2] += a * N.x * N.z;
                P[3] += a * N.y * N.y; P[4] += a * N.y * N.z; P[5] += a * N.z * N.z;
                asum += a;
            }
        }
        if (PROJ)
            for (int c = 0; c < 6; ++c) P[c] /= asum;
    } else {
        const int L = id + 1, R = right[id];
#pragma unroll
        for (int q = 0; q < NW4; ++q) acc[q] = f4add(nodeX[(size_t)L * NW4 + q], nodeX[(size_t)R * NW4 + q]);
        if (PROJ) {
            const float aL = node[L].a, aR = node[R].a, ia = 1.f / (aL + aR);
            const float4 l0 = nodeP[2 * L], l1 = nodeP[2 * L + 1], r0 = nodeP[2 * R], r1 = nodeP[2 * R + 1];
            P[0] = (aL * l0.x + aR * r0.x) * ia; P[1] = (aL * l0.y + aR * r0.y) * ia;
            P[2] = (aL * l0.z + aR * r0.z) * ia; P[3] = (aL * l0.w + aR * r0.w) * ia;
            P[4] = (aL * l1.x + aR * r1.x) * ia; P[5] = (aL * l1.y + aR * r1.y) * ia;
        }
    }
#pragma unroll
    for (int q = 0; q < NW4; ++q) nodeX[(size_t)id * NW4 + q] = acc[q];
    if (PROJ) {
        nodeP[2 * id] = make_float4(P[0], P[1], P[2], P[3]);
        nodeP[2 * id + 1] = make_float4(P[4], P[5], 0.f, 0.f);
    }
}

// Warp-cooperative traversal (as in the Barnes-Hut energy): each lane owns
// one sorted target; the warp walks the pre-order node sequence together and
// a lane is active at node id only when id >= its escape marker. Near pairs
// use the compensated (hi + lo) barycenter differences. The sums per target
// run in FP32 chunks of 32 terms folded into Kahan accumulators, written in
// sorted order for the FP64 combine.
template <int OP, int KC>
__global__ void __launch_bounds__(128)
k_bh_apply(const BvhNode* __restrict__ node, const float4* __restrict__ nodelo, int nnodes,
           const float4* __restrict__ sa, const float4* __restrict__ sb, const float4* __restrict__ sl,
           const FaceBox* __restrict__ fbox, const int* __restrict__ perm, int nf,
           const float4* __restrict__ Ws, const float4* __restrict__ nodeX, const float4* __restrict__ nodeP,
           float theta2, float s_exp, float l_exp, double* __restrict__ part,
           unsigned long long* __restrict__ count) {
    using L = OpLayout<OP, KC>;
    constexpr bool LOW = (OP == TP_OP_A || OP == TP_OP_B0);
    constexpr int NP = L::NA / 2;
    constexpr int NW4 = L::NW4;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = i < nf;
    const int ii = has ? i : 0;
    const float4 A = sa[ii], B = sb[ii], Al = sl[ii];
    const FaceBox fb = fbox[ii];
    int skip = has ? 0 : nnodes;
    float2 pt[NP];
    Acc2<float> acc[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) pt[c] = make_float2(0.f, 0.f);
    int run = 0;
    unsigned nint = 0;
    int id = 0;
    while (id < nnodes) {
        const BvhNode n = node[id];
        bool desc = false;
        if (id >= skip) {
            const float d2 = box_dist2(fb.lox, fb.loy, fb.loz, fb.hix, fb.hiy, fb.hiz, n);
            const float mr2 = fmaxf(fb.r2, n.r2);
            if (mr2 < __fmul_rn(theta2, d2)) {
                const float4 nl = nodelo[id];
                const float dx = (A.x - n.cx) + (Al.x - nl.x), dy = (A.y - n.cy) + (Al.y - nl.y),
                            dz = (A.z - n.cz) + (Al.z - nl.z);
                float2 x2[2 * NW4];
#pragma unroll
                for (int q = 0; q < NW4; ++q) {
                    const float4 x = nodeX[(size_t)id * NW4 + q];
                    x2[2 * q] = make_float2(x.x, x.y);
                    x2[2 * q + 1] = make_float2(x.z, x.w);
                }
                const float r2 = r2_eps(dx, dy, dz);
                if (OP == TP_OP_L) {
                    const float h = pow_(r2, -l_exp);
#pragma unroll
                    for (int c = 0; c < NP; ++c) pt[c] = pfma(h, x2[c], pt[c]);
                } else {
                    const float hB = pow_(r2, -s_exp);
#pragma unroll
                    for (int c = 0; c < L::NH / 2; ++c) pt[c] = pfma(hB, x2[c], pt[c]);
                    if (LOW) {
                        const float4 p0 = nodeP[2 * id], p1 = nodeP[2 * id + 1];
                        const float ir2 = rcp_(r2);
                        const float tS = (B.x * dx + B.y * dy + B.z * dz) * ir2;
                        const float qx = p0.x * dx + p0.y * dy + p0.z * dz;
                        const float qy = p0.y * dx + p0.w * dy + p1.x * dz;
                        const float qz = p0.z * dx + p1.x * dy + p1.y * dz;
                        const float tT2 = (qx * qx + qy * qy + qz * qz) * (ir2 * ir2);   // |P_I d|^2 / |d|^4
                        const float h0 = 0.5f * fmaf(tS, tS, tT2) * hB;
#pragma unroll
                        for (int c = L::NH / 2; c < NP; ++c) pt[c] = pfma(h0, x2[c], pt[c]);
                    }
                }
                ++nint;
                if (++run == 32) {
#pragma unroll
                    for (int c = 0; c < NP; ++c) {
                        acc[c].add(pt[c]);
                        pt[c] = make_float2(0.f, 0.f);
                    }
                    run = 0;
                }
                skip = n.skip;
            } else if (n.leaf) {
                for (int j = n.first; j < n.first + n.count; ++j) {
                    if (j == i) continue;
                    const float4 s = sa[j], l = sl[j], m = sb[j];
                    float2 x2[2 * NW4];
#pragma unroll
                    for (int q = 0; q < NW4; ++q) {
                        const float4 x = Ws[(size_t)j * NW4 + q];
                        x2[2 * q] = make_float2(x.x, x.y);
                        x2[2 * q + 1] = make_float2(x.z, x.w);
                    }
                    apply_term<float, OP, false, KC>((A.x - s.x) + (Al.x - l.x), (A.y - s.y) + (Al.y - l.y),
                                                     (A.z - s.z) + (Al.z - l.z), B.x, B.y, B.z, m.x, m.y, m.z,
                                                     x2, s_exp, l_exp, pt);
                    ++nint;
                }
#pragma unroll
                for (int c = 0; c < NP; ++c) {
                    acc[c].add(pt[c]);
                    pt[c] = make_float2(0.f, 0.f);
                }
                run = 0;
                skip = n.skip;
            } else {
                desc = true;
            }
        }
        id = __any_sync(0xffffffffu, desc) ? id + 1 : n.skip;
    }
#pragma unroll
    for (int c = 0; c < NP; ++c) acc[c].add(pt[c]);
    if (has)   // sorted order: consecutive lanes write consecutive words
#pragma unroll
        for (int c = 0; c < L::NA; ++c) part[(size_t)c * nf + i] = acc[c / 2].value(c & 1);
    if (count && nint) atomicAdd(count, (unsigned long long)nint);
}

// Barnes-Hut operator products from the interaction lists: one warp per
// group of 32 sorted targets, streaming the group's far entries and then its
// near leaves in batches of 32 sources (32 far nodes, or the faces of
// 32 / leaf near leaves). The records of a batch (far: barycenter hi, low
// part, the node's X and projector; near: the face's barycenter, low part,
// normal and W) are copied global -> shared with cp.async, one 16-byte chunk
// per lane and instruction, one batch ahead of their use (two buffers), so
// the gathers of 32 sources are in flight together while the warp evaluates
// the previous batch. Shared layout per warp and buffer: chunk-major
// [chunk][32 sources] float4 (each copy instruction writes 512 contiguous
// bytes; each read is a broadcast), plus the entries' lane masks and the
// near faces' indices. A lane outside an entry's mask, and the self pair,
// get a zero kernel value (the geometric factor h is selected to 0; the other
// factors stay finite at d = 0 thanks to the |d|^2 offset).
template <int OP, int KC> struct BhApplyStage {
    using L = OpLayout<OP, KC>;
    static constexpr bool LOW = (OP == TP_OP_A || OP == TP_OP_B0);
    static constexpr int RF = 2 + L::NW4 + (LOW ? 2 : 0);   // far: c, lo, X[NW4], P[2]
    static constexpr int RN = 2 + (LOW ? 1 : 0) + L::NW4;   // near: c, lo, normal, W[NW4]
    static constexpr int R = RF > RN ? RF : RN;
    static constexpr int BUF = R * 32;                      // float4 per warp and buffer
    static constexpr size_t bytes = sizeof(float4) * 4 * 2 * BUF + sizeof(int) * 4 * 2 * 64;
};

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int OP, int KC>
__global__ void __launch_bounds__(128)
k_bh_apply_list(const float4* __restrict__ node4, const float4* __restrict__ nodelo, const float4* __restrict__ sa,
                const float4* __restrict__ sb, const float4* __restrict__ sl, int nf, BhLists Ls,
                const float4* __restrict__ Ws, const float4* __restrict__ nodeX, const float4* __restrict__ nodeP,
                float s_exp, float l_exp, double* __restrict__ part, unsigned long long* __restrict__ count) {
    using L = OpLayout<OP, KC>;
    using SG = BhApplyStage<OP, KC>;
    constexpr bool LOW = SG::LOW;
    constexpr int NP = L::NA / 2;
    constexpr int NW4 = L::NW4;
    extern __shared__ float4 bsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = blockIdx.x * 4 + w;
    if (g >= Ls.ngroups) return;
    float4* buf0 = bsm + (size_t)w * 2 * SG::BUF;
    int* meta = reinterpret_cast<int*>(bsm + 4 * 2 * SG::BUF) + w * 128;   // [2][mask 32, idx 32]
    const int i = g * BHL_GROUP + lane;
    const bool has = i < nf;
    const int ii = has ? i : 0;
    const float4 A = sa[ii], B = sb[ii], Al = sl[ii];
    // batches: far first, then near (lb leaves of `leaf` faces per batch)
    const int f0 = (int)Ls.far_off[g], f1 = (int)Ls.far_off[g + 1];
    const int n0 = (int)Ls.near_off[g], n1 = (int)Ls.near_off[g + 1];
    const int leaf = Ls.leaf, lb = 32 / leaf, kl = lane / leaf, fi = lane - kl * leaf;
    const int nbf = (f1 - f0 + 31) >> 5, nb = nbf + (n1 - n0 + lb - 1) / lb;
    auto entry = [&](int b) -> int2 {
        if (b < nbf) {
            const int e = f0 + 32 * b + lane;
            return e < f1 ? Ls.far[e] : make_int2(-1, 0);
        }
        const int e = n0 + lb * (b - nbf) + kl;
        return (kl < lb && e < n1) ? Ls.near[e] : make_int2(-1, 0);
    };
    // issue the copies of this lane's source of batch b into buffer b & 1
    auto issue = [&](int b, int2 en) {
        float4* dst = buf0 + (b & 1) * SG::BUF + lane;
        int* mt = meta + (b & 1) * 64;
        if (b < nbf) {
            const bool v = en.x >= 0;
            const int id = v ? en.x : 0;
            cp_async16(dst, node4 + 4 * (size_t)id, v);
            cp_async16(dst + 32, nodelo + id, v);
#pragma unroll
            for (int q = 0; q < NW4; ++q) cp_async16(dst + 32 * (2 + q), nodeX + (size_t)id * NW4 + q, v);
            if (LOW) {
                cp_async16(dst + 32 * (2 + NW4), nodeP + 2 * (size_t)id, v);
                cp_async16(dst + 32 * (3 + NW4), nodeP + 2 * (size_t)id + 1, v);
            }
            mt[lane] = v ? en.y : 0;
            mt[32 + lane] = -1;
        } else {
            const bool v = en.x >= 0 && fi < min(leaf, nf - en.x);
            const int j = v ? en.x + fi : 0;
            cp_async16(dst, sa + j, v);
            cp_async16(dst + 32, sl + j, v);
            if (LOW) cp_async16(dst + 64, sb + j, v);
            constexpr int W0 = LOW ? 3 : 2;
#pragma unroll
            for (int q = 0; q < NW4; ++q) cp_async16(dst + 32 * (W0 + q), Ws + (size_t)j * NW4 + q, v);
            mt[lane] = v ? en.y : 0;
            mt[32 + lane] = v ? j : -1;
        }
        cp_async_commit();
    };
    const unsigned sh = 31u - (unsigned)lane;
    float2 pt[NP];
    Acc2<float> acc[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) pt[c] = make_float2(0.f, 0.f);
    int2 en = entry(0);
    if (nb > 0) issue(0, en);
    en = entry(1);
    for (int b = 0; b < nb; ++b) {
        const bool more = b + 1 < nb;
        if (more) issue(b + 1, en);
        const int2 en2 = entry(b + 2);
        if (more) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncwarp();
        const float4* C = buf0 + (b & 1) * SG::BUF;
        const int* mt = meta + (b & 1) * 64;
        if (b < nbf) {
            const int cnt = min(32, f1 - f0 - 32 * b);
#pragma unroll 4
            for (int k = 0; k < cnt; ++k) {
                const bool on = ((unsigned)mt[k] << sh) >> 31;
                const float4 c = C[k], nl = C[32 + k];
                const float dx = (A.x - c.x) + (Al.x - nl.x), dy = (A.y - c.y) + (Al.y - nl.y),
                            dz = (A.z - c.z) + (Al.z - nl.z);
                float2 x2[2 * NW4];
#pragma unroll
                for (int q = 0; q < NW4; ++q) {
                    const float4 x = C[32 * (2 + q) + k];
                    x2[2 * q] = make_float2(x.x, x.y);
                    x2[2 * q + 1] = make_float2(x.z, x.w);
                }
                const float r2 = r2_eps(dx, dy, dz);
                if (OP == TP_OP_L) {
                    const float h = on ? pow_(r2, -l_exp) : 0.f;
#pragma unroll
                    for (int q = 0; q < NP; ++q) pt[q] = pfma(h, x2[q], pt[q]);
                } else {
                    const float hB = on ? pow_(r2, -s_exp) : 0.f;
#pragma unroll
                    for (int q = 0; q < L::NH / 2; ++q) pt[q] = pfma(hB, x2[q], pt[q]);
                    if (LOW) {
                        const float4 p0 = C[32 * (2 + NW4) + k], p1 = C[32 * (3 + NW4) + k];
                        const float ir2 = rcp_(r2);
                        const float tS = (B.x * dx + B.y * dy + B.z * dz) * ir2;
                        const float qx = p0.x * dx + p0.y * dy + p0.z * dz;
                        const float qy = p0.y * dx + p0.w * dy + p1.x * dz;
                        const float qz = p0.z * dx + p1.x * dy + p1.y * dz;
                        const float tT2 = (qx * qx + qy * qy + qz * qz) * (ir2 * ir2);   // |P_I d|^2 / |d|^4
                        const float h0 = 0.5f * fmaf(tS, tS, tT2) * hB;
#pragma unroll
                        for (int q = L::NH / 2; q < NP; ++q) pt[q] = pfma(h0, x2[q], pt[q]);
                    }
                }
            }
        } else {
            const int cnt = min(lb, n1 - n0 - lb * (b - nbf)) * leaf;
            constexpr int W0 = LOW ? 3 : 2;
#pragma unroll 4
            for (int k = 0; k < cnt; ++k) {
                const bool on = (((unsigned)mt[k] << sh) >> 31) && mt[32 + k] != i;
                const float4 s = C[k], l = C[32 + k];
                const float dx = (A.x - s.x) + (Al.x - l.x), dy = (A.y - s.y) + (Al.y - l.y),
                            dz = (A.z - s.z) + (Al.z - l.z);
                float2 x2[2 * NW4];
#pragma unroll
                for (int q = 0; q < NW4; ++q) {
                    const float4 x = C[32 * (W0 + q) + k];
                    x2[2 * q] = make_float2(x.x, x.y);
                    x2[2 * q + 1] = make_float2(x.z, x.w);
                }
                const float r2 = r2_eps(dx, dy, dz);
                if (OP == TP_OP_L) {
                    const float h = on ? pow_(r2, -l_exp) : 0.f;
#pragma unroll
                    for (int q = 0; q < NP; ++q) pt[q] = pfma(h, x2[q], pt[q]);
                } else {
                    const float hB = on ? pow_(r2, -s_exp) : 0.f;
#pragma unroll
                    for (int q = 0; q < L::NH / 2; ++q) pt[q] = pfma(hB, x2[q], pt[q]);
                    if (LOW) {
                        const float4 m = C[64 + k];
                        const float ir2 = rcp_(r2);
                        const float tS = (B.x * dx + B.y * dy + B.z * dz) * ir2;
                        const float tT = (m.x * dx + m.y * dy + m.z * dz) * ir2;
                        const float h0 = 0.5f * fmaf(tS, tS, tT * tT) * hB;   // (k2(S;T) + k2(T;S)) / 2 |d|^{-2s}
#pragma unroll
                        for (int q = L::NH / 2; q < NP; ++q) pt[q] = pfma(h0, x2[q], pt[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            acc[q].add(pt[q]);
            pt[q] = make_float2(0.f, 0.f);
        }
        __syncwarp();
        en = en2;
    }
    if (has)   // sorted order: consecutive lanes write consecutive words
#pragma unroll
        for (int c = 0; c < L::NA; ++c) part[(size_t)c * nf + i] = acc[c / 2].value(c & 1);
    if (count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(count, Ls.interactions);
}

template <int OP, int KC>
static int launch_bh_apply_op(tp_mesh* m, const tp_params* p, const double* v, int k, double* y,
                              cudaStream_t st) {
    using L = OpLayout<OP, KC>;
    constexpr bool LOW = (OP == TP_OP_A || OP == TP_OP_B0);
    constexpr int NW4 = L::NW4;
    BvhView bv;
    TP_TRY(bvh_view(m, p, st, &bv));
    const int nf = m->nf, nn = bv.nnodes;
    const double s = 2.0 - 2.0 / p->p;
    const double l_exp = 3.0 - s;
    TP_TRY(ensure(m->part, sizeof(double) * (size_t)L::NA * nf));
    TP_TRY(ensure(m->wv64, sizeof(double) * 4 * KC * (size_t)nf));
    TP_TRY(ensure(m->wv32, sizeof(float4) * NW4 * (size_t)nf));
    TP_TRY(ensure(m->corner, sizeof(double) * 3 * (size_t)nf * k));
    TP_TRY(ensure(m->bh_apply_ws, sizeof(float4) * ((size_t)NW4 * nf + (size_t)NW4 * nn + 2 * (size_t)nn)));
    float4* Ws = m->bh_apply_ws.as<float4>();
    float4* nodeX = Ws + (size_t)NW4 * nf;
    float4* nodeP = nodeX + (size_t)NW4 * nn;
    TP_TRY(bh_counter(m, st));
    unsigned long long* cnt = m->bhcount.as<unsigned long long>() + 2;
    BhLists Ls;
    bool lists = false;
    TP_TRY(bh_lists(m, p, st, &Ls, &lists));
    for (int col0 = 0; col0 < k; col0 += KC) {
        k_face_W<float, KC><<<(nf * ((KC + 2) / 3) + 255) / 256, 256, 0, st>>>(v, k, col0, m->faces.as<int>(), nf,
                                                              m->f64a.as<d4>(), m->fgrad.as<double>(), OP,
                                                              m->wv64.as<double>(), m->wv32.as<float4>(), NW4);
        TP_LAUNCH_CHECK();
        k_sort_X<NW4><<<(nf + 255) / 256, 256, 0, st>>>(m->wv32.as<float4>(), bv.perm, nf, Ws);
        TP_LAUNCH_CHECK();
        for (int d = bv.maxdepth; d >= 0; --d) {
            const int n0 = bv.level_off[d], n1 = bv.level_off[d + 1];
            k_node_X<NW4, LOW><<<(n1 - n0 + 127) / 128, 128, 0, st>>>(bv.node, bv.right, bv.level_order, n0, n1,
                                                                     Ws, bv.sa, bv.sb, nodeX, nodeP);
            TP_LAUNCH_CHECK();
        }
        {
            ProfScope ps(m, PK_BH_APPLY, 0.0, st);
            m->prof.cols[PK_BH_APPLY] += KC;
            // (resident_per_sm raises the kernel's dynamic shared memory limit when it needs more than 48 KB)
            if (lists && resident_per_sm((const void*)k_bh_apply_list<OP, KC>, 128, BhApplyStage<OP, KC>::bytes) < 1)
                return fail(TP_ERR_CUDA, "Barnes-Hut apply: shared memory for the staged batches not available");
            if (lists)
                k_bh_apply_list<OP, KC><<<(Ls.ngroups + 3) / 4, 128, BhApplyStage<OP, KC>::bytes, st>>>(
                    reinterpret_cast<const float4*>(bv.node), bv.nodelo, bv.sa, bv.sb, bv.sl, nf, Ls, Ws, nodeX,
                    nodeP, (float)s, (float)l_exp, m->part.as<double>(), cnt);
            else
                k_bh_apply<OP, KC><<<(nf + 127) / 128, 128, 0, st>>>(
                    bv.node, bv.nodelo, nn, bv.sa, bv.sb, bv.sl, bv.fbox, bv.perm, nf, Ws, nodeX, nodeP,
                    (float)(p->theta * p->theta), (float)s, (float)l_exp, m->part.as<double>(), cnt);
        }
        TP_LAUNCH_CHECK();
        k_apply_combine<OP, KC><<<(nf + 255) / 256, 256, 0, st>>>(m->part.as<double>(), 1, nf,
                                                                  m->f64a.as<d4>(), m->fgrad.as<double>(),
                                                                  m->wv64.as<double>(), k, col0,
                                                                  m->corner.as<double>(), bv.perm);
        TP_LAUNCH_CHECK();
    }
    return corners_to_vertices(m, m->corner.as<double>(), k, y, st);
}

int apply_bh(tp_mesh* m, const tp_params* p, int op, const double* v, int k, double* y, cudaStream_t st) {
    if (p->precision != TP_PREC_FP32) return fail(TP_ERR_INVALID_ARG, "Barnes-Hut applies run in FP32 only");
    const bool wide = k > 3;
    switch (op) {
        case TP_OP_A: return wide ? launch_bh_apply_op<TP_OP_A, 9>(m, p, v, k, y, st)
                                  : launch_bh_apply_op<TP_OP_A, 3>(m, p, v, k, y, st);
        case TP_OP_B: return wide ? launch_bh_apply_op<TP_OP_B, 9>(m, p, v, k, y, st)
                                  : launch_bh_apply_op<TP_OP_B, 3>(m, p, v, k, y, st);
        case TP_OP_B0: return wide ? launch_bh_apply_op<TP_OP_B0, 9>(m, p, v, k, y, st)
                                   : launch_bh_apply_op<TP_OP_B0, 3>(m, p, v, k, y, st);
        case TP_OP_L: return wide ? launch_bh_apply_op<TP_OP_L, 9>(m, p, v, k, y, st)
                                  : launch_bh_apply_op<TP_OP_L, 3>(m, p, v, k, y, st);
    }
    return fail(TP_ERR_INVALID_ARG, "unknown operator");
}

int apply_op(tp_mesh* m, const tp_params* p, int op, const double* v, int k, double* y, cudaStream_t st) {
    return p->theta > 0.0 ? apply_bh(m, p, op, v, k, y, st) : apply_direct(m, p, op, v, k, y, st);
}

int apply_direct(tp_mesh* m, const tp_params* p, int op, const double* v, int k, double* y,
                 cudaStream_t st) {
    return p->precision == TP_PREC_FP64 ? launch_apply<double>(m, p, op, v, k, y, st)
                                        : launch_apply<float>(m, p, op, v, k, y, st);
}

}  // namespace tp
