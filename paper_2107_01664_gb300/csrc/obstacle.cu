// Static mesh obstacles (§7.3.2).
//
// An obstacle O is a fixed triangle mesh. Every point x of the moving
// surface feels the potential
//     E_obs(x) = sum_{S in F_O} |f_O(S) - x|^{-p} a_O(S),
// f_O(S) the barycenter and a_O(S) the area of obstacle face S, p the
// tangent-point exponent. The surface integral of the potential is taken
// with the one-point rule of Eq. 10 (the barycenter X_T of each surface
// face, weighted by its area a_T) and scaled by a user weight w:
//     E_O          = w sum_T a_T E_obs(X_T),
//     dE_O/dX_T    = w a_T p sum_S a_O(S) |d|^{-p-2} d,   d = f_O(S) - X_T,
//     dE_O/da_T    = w E_obs(X_T),   dE_O/dN_T = 0,
// and the face adjoints reach the vertices through the chain rule of §3.1.
//
// Direct sums: N-body tiles, surface faces as targets held in registers and
// obstacle faces streamed through shared memory in tiles of NT, with source
// splits for small surfaces; FP32 runs of CH terms added with Kahan
// compensation, FP64 partials and an FP64 combine in a fixed order (the
// FP64 path runs the same kernel in double). Near tiles take the
// compensated (hi + lo) barycenter difference, as the kernels of Eq. 10 do.
// Barnes-Hut (theta > 0, FP32): the obstacle is a mesh of its own whose BVH
// is built once (it never moves); each surface face walks it with the
// admissibility test of §4.1 for a point target (radius 0): an admissible
// node I contributes a_I |X_I - x|^{-p}, inadmissible leaves are summed face
// by face.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "tp_internal.cuh"

namespace tp {

__global__ void k_tile_boxes(const float4* __restrict__ f32a, int nf, float4* __restrict__ box);

namespace {

constexpr int NT = 128;  // threads per block = obstacle faces per shared-memory tile
constexpr int CH = 32;   // sources per FP32 run before the compensated add
constexpr float PAD_X = 1e18f;   // x of the padding sources of the last tile (area 0, far away)

template <typename T> struct V4O;
template <> struct V4O<float> { using type = float4; };
template <> struct V4O<double> { using type = d4; };

__device__ __forceinline__ float orcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double orcp(double x) { return 1.0 / x; }
// x^y for x > 0 (x = inf gives inf)
__device__ __forceinline__ float opow(float x, float y) {
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y * l));
    return r;
}
__device__ __forceinline__ double opow(double x, double y) { return pow(x, y); }

template <typename T> struct OAcc;
template <> struct OAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {  // Kahan
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct OAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// |d|^{-p} for |d|^2 = r2; also returns 1/|d|^2
template <typename T, bool P6>
__device__ __forceinline__ T obs_term(T r2, T halfp, T& ir2) {
    ir2 = orcp(r2);
    return P6 ? ir2 * ir2 * ir2 : opow(ir2, halfp);
}

// two floats as one packed pair register (lane 0 = a), and back
__device__ __forceinline__ unsigned long long opk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 oupk2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}

// p = 6 terms of two targets (one per lane of the packed pair registers)
// against one source broadcast to both lanes, in packed FP32 (f32x2, IEEE
// per lane): d = X_target - f_O(S), k = a_S |d|^-6,
//   e += k;  with the gradient also g += k |d|^-2 d.
__device__ __forceinline__ void obs2_p6(unsigned long long tx, unsigned long long ty, unsigned long long tz,
                                        unsigned long long sx, unsigned long long sy, unsigned long long sz,
                                        unsigned long long sa, unsigned long long& e) {
    asm("{\n\t.reg .b64 dx, dy, dz, r2, ir2, k;\n\t.reg .f32 lo, hi;\n\t"
        "sub.rn.f32x2 dx, %1, %4;\n\t"
        "sub.rn.f32x2 dy, %2, %5;\n\t"
        "sub.rn.f32x2 dz, %3, %6;\n\t"
        "mul.rn.f32x2 r2, dz, dz;\n\t"
        "fma.rn.f32x2 r2, dy, dy, r2;\n\t"
        "fma.rn.f32x2 r2, dx, dx, r2;\n\t"
        "mov.b64 {lo, hi}, r2;\n\t"
        "rcp.approx.ftz.f32 lo, lo;\n\t"
        "rcp.approx.ftz.f32 hi, hi;\n\t"
        "mov.b64 ir2, {lo, hi};\n\t"
        "mul.rn.f32x2 k, ir2, ir2;\n\t"
        "mul.rn.f32x2 k, k, ir2;\n\t"
        "fma.rn.f32x2 %0, k, %7, %0;\n\t}"
        : "+l"(e)
        : "l"(tx), "l"(ty), "l"(tz), "l"(sx), "l"(sy), "l"(sz), "l"(sa));
}
__device__ __forceinline__ void obs2_p6_grad(unsigned long long tx, unsigned long long ty, unsigned long long tz,
                                             unsigned long long sx, unsigned long long sy, unsigned long long sz,
                                             unsigned long long sa, unsigned long long& e, unsigned long long& gx,
                                             unsigned long long& gy, unsigned long long& gz) {
    asm("{\n\t.reg .b64 dx, dy, dz, r2, ir2, k;\n\t.reg .f32 lo, hi;\n\t"
        "sub.rn.f32x2 dx, %4, %7;\n\t"
        "sub.rn.f32x2 dy, %5, %8;\n\t"
        "sub.rn.f32x2 dz, %6, %9;\n\t"
        "mul.rn.f32x2 r2, dz, dz;\n\t"
        "fma.rn.f32x2 r2, dy, dy, r2;\n\t"
        "fma.rn.f32x2 r2, dx, dx, r2;\n\t"
        "mov.b64 {lo, hi}, r2;\n\t"
        "rcp.approx.ftz.f32 lo, lo;\n\t"
        "rcp.approx.ftz.f32 hi, hi;\n\t"
        "mov.b64 ir2, {lo, hi};\n\t"
        "mul.rn.f32x2 k, ir2, ir2;\n\t"
        "mul.rn.f32x2 k, k, ir2;\n\t"
        "mul.rn.f32x2 k, k, %10;\n\t"
        "add.rn.f32x2 %0, %0, k;\n\t"
        "mul.rn.f32x2 k, k, ir2;\n\t"
        "fma.rn.f32x2 %1, k, dx, %1;\n\t"
        "fma.rn.f32x2 %2, k, dy, %2;\n\t"
        "fma.rn.f32x2 %3, k, dz, %3;\n\t}"
        : "+l"(e), "+l"(gx), "+l"(gy), "+l"(gz)
        : "l"(tx), "l"(ty), "l"(tz), "l"(sx), "l"(sy), "l"(sz), "l"(sa));
}

// ---------------------------------------------------------------------------
// obstacle faces in the surface's frame
// ---------------------------------------------------------------------------

// f_O(S) - c (c: the surface's reference frame) from the obstacle's
// positions, in FP64 and as FP32 hi + lo, with the obstacle face areas;
// entry i holds face S = perm[i] (the obstacle's Morton order, so that a
// tile of consecutive entries is a compact patch of the obstacle)
__global__ void k_obs_frame(const double* __restrict__ pos, const int* __restrict__ faces, int nf,
                            const int* __restrict__ perm, const d4* __restrict__ of64a,
                            const double* __restrict__ center, d4* __restrict__ f64a, float4* __restrict__ f32a,
                            float4* __restrict__ f32c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int S = perm[i];
    const double* pi = pos + 3 * faces[3 * S];
    const double* pj = pos + 3 * faces[3 * S + 1];
    const double* pk = pos + 3 * faces[3 * S + 2];
    double X[3];
    for (int c = 0; c < 3; ++c) X[c] = (pi[c] + pj[c] + pk[c]) / 3.0 - center[c];
    const double a = of64a[S].w;
    f64a[i] = d4{X[0], X[1], X[2], a};
    f32a[i] = make_float4((float)X[0], (float)X[1], (float)X[2], (float)a);
    f32c[i] = make_float4((float)(X[0] - (double)(float)X[0]), (float)(X[1] - (double)(float)X[1]),
                          (float)(X[2] - (double)(float)X[2]), 0.f);
}

// squared near distance of the obstacle tiles: a tile closer than R/16 to a
// target block takes the compensated difference, R the larger of the
// surface's half diagonal and the largest obstacle coordinate in the frame
// (beyond it the FP32 rounding of the barycenters perturbs |d| by < 2^-19)
__global__ void k_obs_thr(const float4* __restrict__ box, int ntiles, const double* __restrict__ center,
                          double* __restrict__ thr) {
    __shared__ float red[256];
    float m = 0.f;
    for (int t = threadIdx.x; t < 2 * ntiles; t += blockDim.x) {
        float4 b = box[t];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fabsf(b.z)));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double R = (double)red[0];
        thr[0] = fmax(center[3], 3.0 * R * R / 256.0);
    }
}

// ---------------------------------------------------------------------------
// direct sums
// ---------------------------------------------------------------------------

__device__ __forceinline__ void obs_block_box(float lx, float ly, float lz, float hx, float hy, float hz,
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

// Per target face T (surface order) and source split: accumulator 0 gets
// sum_S a_S |d|^{-p}, accumulators 1..3 (DIFF) sum_S a_S |d|^{-p-2} d with
// d = X_T - f_O(S) (target minus source). FP32 with p = 6 on far tiles:
// two targets per packed f32x2 instruction, the sources staged in shared
// memory already broadcast to both lanes.
template <typename T, bool P6, bool DIFF, int TT>
__global__ void __launch_bounds__(NT)
k_obstacle(const typename V4O<T>::type* __restrict__ ta, const float4* __restrict__ tlo, int nt,
           const typename V4O<T>::type* __restrict__ oa, const float4* __restrict__ olo,
           const float4* __restrict__ obox, const double* __restrict__ thr, int no, int tiles_per_split,
           T halfp, double* __restrict__ part) {
    using V4 = typename V4O<T>::type;
    constexpr bool F32 = sizeof(T) == 4;
    constexpr bool PACK = F32 && P6 && TT % 2 == 0;
    constexpr int NACC = DIFF ? 4 : 1;
    constexpr int TP = PACK ? TT / 2 : 1;
    __shared__ V4 sh[NT];
    __shared__ float4 shl[F32 ? NT : 1];
    __shared__ ulonglong2 shp[PACK ? 2 * NT : 1];
    __shared__ float sbox[6];
    T tx[TT], ty[TT], tz[TT];
    float lx[TT], ly[TT], lz[TT];
    int tid[TT];
    float bl[3] = {3e38f, 3e38f, 3e38f}, bh[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int j = 0; j < TT; ++j) {
        const int t = blockIdx.x * NT * TT + j * NT + threadIdx.x;
        tid[j] = t;
        lx[j] = ly[j] = lz[j] = 0.f;
        tx[j] = ty[j] = tz[j] = T(0);
        if (t < nt) {
            const V4 A = ta[t];
            tx[j] = A.x; ty[j] = A.y; tz[j] = A.z;
            if (F32) {
                const float4 L = tlo[t];
                lx[j] = L.x; ly[j] = L.y; lz[j] = L.z;
                bl[0] = fminf(bl[0], (float)A.x); bl[1] = fminf(bl[1], (float)A.y); bl[2] = fminf(bl[2], (float)A.z);
                bh[0] = fmaxf(bh[0], (float)A.x); bh[1] = fmaxf(bh[1], (float)A.y); bh[2] = fmaxf(bh[2], (float)A.z);
            }
        }
    }
    float thr2 = 0.f;
    if (F32) {
        obs_block_box(bl[0], bl[1], bl[2], bh[0], bh[1], bh[2], sbox);
        thr2 = (float)thr[0];
    }
    unsigned long long TX[TP], TY[TP], TZ[TP];
    if constexpr (PACK) {
#pragma unroll
        for (int jj = 0; jj < TP; ++jj) {
            TX[jj] = opk2((float)tx[2 * jj], (float)tx[2 * jj + 1]);
            TY[jj] = opk2((float)ty[2 * jj], (float)ty[2 * jj + 1]);
            TZ[jj] = opk2((float)tz[2 * jj], (float)tz[2 * jj + 1]);
        }
    }
    OAcc<T> acc[TT][NACC];
    const int ntiles = (no + NT - 1) / NT;
    const int k0 = blockIdx.y * tiles_per_split;
    const int k1 = min(k0 + tiles_per_split, ntiles);
    for (int tile = k0; tile < k1; ++tile) {
        bool near = false;
        if (F32) {
            const float4 lo = obox[2 * tile], hi = obox[2 * tile + 1];
            const float gx = fmaxf(fmaxf(lo.x - sbox[3], sbox[0] - hi.x), 0.f);
            const float gy = fmaxf(fmaxf(lo.y - sbox[4], sbox[1] - hi.y), 0.f);
            const float gz = fmaxf(fmaxf(lo.z - sbox[5], sbox[2] - hi.z), 0.f);
            near = gx * gx + gy * gy + gz * gz < thr2;
        }
        const int src = tile * NT + threadIdx.x;
        __syncthreads();
        V4 sv;
        if (src < no) {
            sv = oa[src];
        } else {
            sv.x = T(PAD_X); sv.y = T(0); sv.z = T(0); sv.w = T(0);
        }
        sh[threadIdx.x] = sv;
        if constexpr (PACK) {
            shp[2 * threadIdx.x] = make_ulonglong2(opk2((float)sv.x, (float)sv.x), opk2((float)sv.y, (float)sv.y));
            shp[2 * threadIdx.x + 1] = make_ulonglong2(opk2((float)sv.z, (float)sv.z), opk2((float)sv.w, (float)sv.w));
        }
        if (near) shl[threadIdx.x] = src < no ? olo[src] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        for (int c = 0; c < NT; c += CH) {
            T pt[TT][NACC];
#pragma unroll
            for (int j = 0; j < TT; ++j)
#pragma unroll
                for (int i = 0; i < NACC; ++i) pt[j][i] = T(0);
            if (near) {
#pragma unroll 4
                for (int q = 0; q < CH; ++q) {
                    const V4 s = sh[c + q];
                    const float4 l = shl[c + q];
#pragma unroll
                    for (int j = 0; j < TT; ++j) {
                        const T dx = (tx[j] - s.x) + (T)(lx[j] - l.x);
                        const T dy = (ty[j] - s.y) + (T)(ly[j] - l.y);
                        const T dz = (tz[j] - s.z) + (T)(lz[j] - l.z);
                        T ir2;
                        const T k = obs_term<T, P6>(fma(dx, dx, fma(dy, dy, dz * dz)), halfp, ir2) * s.w;
                        pt[j][0] += k;
                        if constexpr (DIFF) {
                            const T kg = k * ir2;
                            pt[j][1] = fma(kg, dx, pt[j][1]);
                            pt[j][2] = fma(kg, dy, pt[j][2]);
                            pt[j][3] = fma(kg, dz, pt[j][3]);
                        }
                    }
                }
            } else if constexpr (PACK) {
                unsigned long long P[TP][NACC];
#pragma unroll
                for (int jj = 0; jj < TP; ++jj)
#pragma unroll
                    for (int i = 0; i < NACC; ++i) P[jj][i] = 0ull;
#pragma unroll 8
                for (int q = 0; q < CH; ++q) {
                    const ulonglong2 u0 = shp[2 * (c + q)], u1 = shp[2 * (c + q) + 1];
#pragma unroll
                    for (int jj = 0; jj < TP; ++jj) {
                        if constexpr (DIFF)
                            obs2_p6_grad(TX[jj], TY[jj], TZ[jj], u0.x, u0.y, u1.x, u1.y, P[jj][0], P[jj][1],
                                         P[jj][2], P[jj][3]);
                        else
                            obs2_p6(TX[jj], TY[jj], TZ[jj], u0.x, u0.y, u1.x, u1.y, P[jj][0]);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < TP; ++jj)
#pragma unroll
                    for (int i = 0; i < NACC; ++i) {
                        const float2 v = oupk2(P[jj][i]);
                        pt[2 * jj][i] = v.x;
                        pt[2 * jj + 1][i] = v.y;
                    }
            } else {
#pragma unroll 8
                for (int q = 0; q < CH; ++q) {
                    const V4 s = sh[c + q];
#pragma unroll
                    for (int j = 0; j < TT; ++j) {
                        const T dx = tx[j] - s.x, dy = ty[j] - s.y, dz = tz[j] - s.z;
                        T ir2;
                        const T k = obs_term<T, P6>(fma(dx, dx, fma(dy, dy, dz * dz)), halfp, ir2) * s.w;
                        pt[j][0] += k;
                        if constexpr (DIFF) {
                            const T kg = k * ir2;
                            pt[j][1] = fma(kg, dx, pt[j][1]);
                            pt[j][2] = fma(kg, dy, pt[j][2]);
                            pt[j][3] = fma(kg, dz, pt[j][3]);
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < TT; ++j)
#pragma unroll
                for (int i = 0; i < NACC; ++i) acc[j][i].add(pt[j][i]);
        }
    }
#pragma unroll
    for (int j = 0; j < TT; ++j)
        if (tid[j] < nt)
#pragma unroll
            for (int i = 0; i < NACC; ++i)
                part[((size_t)blockIdx.y * NACC + i) * nt + tid[j]] = acc[j][i].value();
}

// erow[T] (+)= w a_T E_obs(X_T); with DIFF the face adjoints
// adj[7T..7T+2] (+)= w a_T p sum a_S |d|^{-p-2} (f_O(S) - X_T), adj[7T+6] (+)= w E_obs(X_T)
template <bool DIFF>
__global__ void k_obs_combine(const double* __restrict__ part, int nsplit, int nt, double p, double w,
                              const d4* __restrict__ f64a, double* __restrict__ erow, double* __restrict__ adj,
                              int accumulate) {
    constexpr int NACC = DIFF ? 4 : 1;
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= nt) return;
    double s[NACC];
    for (int i = 0; i < NACC; ++i) s[i] = 0.0;
    for (int k = 0; k < nsplit; ++k)
        for (int i = 0; i < NACC; ++i) s[i] += part[((size_t)k * NACC + i) * nt + T];
    const double a = f64a[T].w;
    const double e = w * a * s[0];
    if (erow) erow[T] = accumulate ? erow[T] + e : e;
    if constexpr (DIFF) {
        double* g = adj + 7 * (size_t)T;
        const double cg = -p * w * a;
        if (accumulate) {
            for (int c = 0; c < 3; ++c) g[c] += cg * s[1 + c];
            g[6] += w * s[0];
        } else {
            for (int c = 0; c < 3; ++c) {
                g[c] = cg * s[1 + c];
                g[3 + c] = 0.0;
            }
            g[6] = w * s[0];
        }
    }
}

int resident_blocks(const void* fn) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT, 0) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

// source splits: minimise waves x tiles per split (+ a small charge per split)
void obs_grid(int nt, int no, int tt, int per_sm, int* bx, int* nsplit, int* tps) {
    *bx = std::max(1, (nt + NT * tt - 1) / (NT * tt));
    const int ntiles = (no + NT - 1) / NT;
    const long slots = (long)std::max(1, per_sm) * sm_count();
    double best = 1e300;
    *tps = ntiles;
    *nsplit = 1;
    for (int ns = 1; ns <= std::min(ntiles, 64); ++ns) {
        const int t = (ntiles + ns - 1) / ns;
        const int nsp = (ntiles + t - 1) / t;
        const long waves = ((long)*bx * nsp + slots - 1) / slots;
        const double cost = (double)waves * t + 0.05 * nsp;
        if (cost < best - 1e-9) {
            best = cost;
            *tps = t;
            *nsplit = nsp;
        }
    }
}

template <typename T, bool DIFF>
int launch_obstacle(tp_mesh* m, const tp_params* p, double* erow, double* adj, bool accumulate, cudaStream_t st) {
    using V4 = typename V4O<T>::type;
    constexpr int TT = DIFF ? 2 : 4;
    constexpr int NACC = DIFF ? 4 : 1;
    const int nt = m->nf, no = m->obs->nf;
    const bool p6 = p->p == 6.0;
    const void* fn = p6 ? (const void*)k_obstacle<T, true, DIFF, TT> : (const void*)k_obstacle<T, false, DIFF, TT>;
    int bx, nsplit, tps;
    obs_grid(nt, no, TT, resident_blocks(fn), &bx, &nsplit, &tps);
    TP_TRY(ensure(m->obs_part, sizeof(double) * (size_t)nsplit * NACC * nt));
    const V4* ta = (const V4*)(sizeof(T) == 4 ? m->f32a.ptr : m->f64a.ptr);
    const V4* oa = (const V4*)(sizeof(T) == 4 ? m->obs_f32a.ptr : m->obs_f64a.ptr);
    const dim3 grid(bx, nsplit);
    const double units = (double)nt * no;
    m->pairs += units;
    {
        ProfScope ps(m, PK_OBSTACLE, units, st);
        if (p6)
            k_obstacle<T, true, DIFF, TT><<<grid, NT, 0, st>>>(ta, m->f32c.as<float4>(), nt, oa,
                                                               m->obs_f32c.as<float4>(), m->obs_tilebox.as<float4>(),
                                                               m->obs_thr.as<double>(), no, tps, T(3),
                                                               m->obs_part.as<double>());
        else
            k_obstacle<T, false, DIFF, TT><<<grid, NT, 0, st>>>(ta, m->f32c.as<float4>(), nt, oa,
                                                                m->obs_f32c.as<float4>(), m->obs_tilebox.as<float4>(),
                                                                m->obs_thr.as<double>(), no, tps, T(0.5 * p->p),
                                                                m->obs_part.as<double>());
        TP_LAUNCH_CHECK();
    }
    k_obs_combine<DIFF><<<(nt + 255) / 256, 256, 0, st>>>(m->obs_part.as<double>(), nsplit, nt, p->p, m->obs_weight,
                                                          m->f64a.as<d4>(), erow, adj, accumulate ? 1 : 0);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

// ---------------------------------------------------------------------------
// Barnes-Hut over the obstacle's BVH
// ---------------------------------------------------------------------------

struct KahanObs {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Warp-cooperative stackless walk, one surface face per lane (the scheme of
// the Barnes-Hut energy kernel): the warp visits the pre-order node sequence
// together, a lane is active at node id only when id >= its skip index, and
// the warp descends when any active lane needs to. The target point is the
// face barycenter in the obstacle's frame, x = (f_i + f_j + f_k)/3 - c_O in
// FP64, split into FP32 hi + lo.
template <bool P6, bool DIFF>
__global__ void __launch_bounds__(128)
k_bh_obstacle(const BvhNode* __restrict__ node, const float4* __restrict__ nodelo, int nnodes,
              const float4* __restrict__ sa, const float4* __restrict__ sl,
              const double* __restrict__ pos, const int* __restrict__ faces, const d4* __restrict__ f64a, int nt,
              const double* __restrict__ ocenter, float theta2, float halfp, double p, double w,
              double* __restrict__ erow, double* __restrict__ adj, int accumulate,
              unsigned long long* __restrict__ count) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = t < nt;
    float xh[3] = {0.f, 0.f, 0.f}, xl[3] = {0.f, 0.f, 0.f};
    if (has) {
        const double* pi = pos + 3 * faces[3 * t];
        const double* pj = pos + 3 * faces[3 * t + 1];
        const double* pk = pos + 3 * faces[3 * t + 2];
        for (int c = 0; c < 3; ++c) {
            const double x = (pi[c] + pj[c] + pk[c]) / 3.0 - ocenter[c];
            xh[c] = (float)x;
            xl[c] = (float)(x - (double)xh[c]);
        }
    }
    int skip = has ? 0 : nnodes;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    KahanObs sum[DIFF ? 4 : 1];
    int nint = 0, run = 0;
    int id = 0;
    auto term = [&](float cx, float cy, float cz, float lx, float ly, float lz, float a) {
        const float dx = (xh[0] - cx) + (xl[0] - lx), dy = (xh[1] - cy) + (xl[1] - ly),
                    dz = (xh[2] - cz) + (xl[2] - lz);
        const float ir2 = orcp(dx * dx + dy * dy + dz * dz);
        const float k = (P6 ? ir2 * ir2 * ir2 : opow(ir2, halfp)) * a;
        acc[0] += k;
        if constexpr (DIFF) {
            const float kg = k * ir2;
            acc[1] = fmaf(kg, dx, acc[1]);
            acc[2] = fmaf(kg, dy, acc[2]);
            acc[3] = fmaf(kg, dz, acc[3]);
        }
    };
    auto flush = [&]() {
#pragma unroll
        for (int i = 0; i < (DIFF ? 4 : 1); ++i) {
            sum[i].add(acc[i]);
            acc[i] = 0.f;
        }
        run = 0;
    };
    while (id < nnodes) {
        const BvhNode n = node[id];
        bool desc = false;
        if (id >= skip) {
            const float d2 = box_dist2(xh[0], xh[1], xh[2], xh[0], xh[1], xh[2], n);
            if (n.r2 < __fmul_rn(theta2, d2)) {
                const float4 nl = nodelo[id];
                term(n.cx, n.cy, n.cz, nl.x, nl.y, nl.z, n.a);
                ++nint;
                if (++run == 32) flush();
                skip = n.skip;
            } else if (n.leaf) {
                for (int j = n.first; j < n.first + n.count; ++j) {
                    const float4 s = sa[j], l = sl[j];
                    term(s.x, s.y, s.z, l.x, l.y, l.z, s.w);
                    ++nint;
                }
                flush();
                skip = n.skip;
            } else {
                desc = true;
            }
        }
        id = __any_sync(0xffffffffu, desc) ? id + 1 : n.skip;
    }
    flush();
    if (has) {
        const double a = f64a[t].w;
        const double s0 = sum[0].value();
        const double e = w * a * s0;
        erow[t] = accumulate ? erow[t] + e : e;
        if constexpr (DIFF) {
            double* g = adj + 7 * (size_t)t;
            const double cg = -p * w * a;
            if (accumulate) {
                for (int c = 0; c < 3; ++c) g[c] += cg * sum[1 + c].value();
                g[6] += w * s0;
            } else {
                for (int c = 0; c < 3; ++c) {
                    g[c] = cg * sum[1 + c].value();
                    g[3 + c] = 0.0;
                }
                g[6] = w * s0;
            }
        }
    }
    if (count && nint) atomicAdd(count, (unsigned long long)nint);
}

template <bool DIFF>
int launch_bh_obstacle(tp_mesh* m, const tp_params* p, double* erow, double* adj, bool accumulate,
                       cudaStream_t st) {
    BvhView v;
    TP_TRY(bvh_view(m->obs, p, st, &v));
    TP_TRY(bh_counter(m, st));
    const float theta2 = (float)(p->theta * p->theta);
    const float halfp = (float)(0.5 * p->p);
    unsigned long long* cnt = m->bhcount.as<unsigned long long>() + 3;
    const int nt = m->nf;
    const int g = (nt + 127) / 128;
    ProfScope ps(m, PK_BH_OBSTACLE, 0.0, st);
    if (p->p == 6.0)
        k_bh_obstacle<true, DIFF><<<g, 128, 0, st>>>(v.node, v.nodelo, v.nnodes, v.sa, v.sl, m->pos.as<double>(),
                                                     m->faces.as<int>(), m->f64a.as<d4>(), nt,
                                                     m->obs->center.as<double>(), theta2, halfp, p->p, m->obs_weight,
                                                     erow, adj, accumulate ? 1 : 0, cnt);
    else
        k_bh_obstacle<false, DIFF><<<g, 128, 0, st>>>(v.node, v.nodelo, v.nnodes, v.sa, v.sl, m->pos.as<double>(),
                                                      m->faces.as<int>(), m->f64a.as<d4>(), nt,
                                                      m->obs->center.as<double>(), theta2, halfp, p->p,
                                                      m->obs_weight, erow, adj, accumulate ? 1 : 0, cnt);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

}  // namespace

// Re-express the obstacle's faces in the surface's current frame (after the
// surface's positions, hence its frame, changed, and when an obstacle is set).
int obstacle_frame(tp_mesh* m, cudaStream_t st) {
    if (!m->obs) return TP_OK;
    const int no = m->obs->nf;
    const int ntiles = (no + NT - 1) / NT;
    TP_TRY(ensure(m->obs_f64a, sizeof(d4) * (size_t)no));
    TP_TRY(ensure(m->obs_f32a, sizeof(float4) * (size_t)no));
    TP_TRY(ensure(m->obs_f32c, sizeof(float4) * (size_t)no));
    TP_TRY(ensure(m->obs_tilebox, sizeof(float4) * 2 * (size_t)ntiles));
    TP_TRY(ensure(m->obs_thr, sizeof(double)));
    k_obs_frame<<<(no + 255) / 256, 256, 0, st>>>(m->obs->pos.as<double>(), m->obs->faces.as<int>(), no,
                                                  m->obs_perm.as<int>(), m->obs->f64a.as<d4>(), m->center.as<double>(),
                                                  m->obs_f64a.as<d4>(), m->obs_f32a.as<float4>(),
                                                  m->obs_f32c.as<float4>());
    TP_LAUNCH_CHECK();
    k_tile_boxes<<<ntiles, 128, 0, st>>>(m->obs_f32a.as<float4>(), no, m->obs_tilebox.as<float4>());
    TP_LAUNCH_CHECK();
    k_obs_thr<<<1, 256, 0, st>>>(m->obs_tilebox.as<float4>(), ntiles, m->center.as<double>(),
                                 m->obs_thr.as<double>());
    TP_LAUNCH_CHECK();
    return TP_OK;
}

// Attach obstacle mesh o (owned by m from here on): its Morton order (from
// its BVH) fixes the order of the obstacle's faces in the direct sums.
int obstacle_attach(tp_mesh* m, tp_mesh* o, double weight, cudaStream_t st) {
    obstacle_release(m);
    m->obs = o;
    m->obs_weight = weight;
    tp_params dp;
    tp_params_default(&dp);
    BvhView v;
    int s = bvh_view(o, &dp, st, &v);
    if (s == TP_OK) s = ensure(m->obs_perm, sizeof(int) * (size_t)o->nf);
    if (s == TP_OK && cudaMemcpyAsync(m->obs_perm.ptr, v.perm, sizeof(int) * (size_t)o->nf,
                                      cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        s = fail(TP_ERR_CUDA, "copying the obstacle's face order failed");
    if (s == TP_OK) s = obstacle_frame(m, st);
    if (s != TP_OK) obstacle_release(m);
    return s;
}

int obstacle_terms(tp_mesh* m, const tp_params* p, bool diff, bool accumulate, double* erow, double* adj,
                   cudaStream_t st) {
    if (!m->obs) return TP_OK;
    if (p->theta > 0.0)
        return diff ? launch_bh_obstacle<true>(m, p, erow, adj, accumulate, st)
                    : launch_bh_obstacle<false>(m, p, erow, adj, accumulate, st);
    if (p->precision == TP_PREC_FP64)
        return diff ? launch_obstacle<double, true>(m, p, erow, adj, accumulate, st)
                    : launch_obstacle<double, false>(m, p, erow, adj, accumulate, st);
    return diff ? launch_obstacle<float, true>(m, p, erow, adj, accumulate, st)
                : launch_obstacle<float, false>(m, p, erow, adj, accumulate, st);
}

void obstacle_release(tp_mesh* m) {
    Buf* all[] = {&m->obs_f64a, &m->obs_f32a, &m->obs_f32c, &m->obs_tilebox, &m->obs_thr, &m->obs_part,
                  &m->obs_perm};
    for (Buf* b : all) release(*b);
    if (m->obs) {
        tp_mesh_destroy(m->obs);
        m->obs = nullptr;
    }
    m->obs_weight = 0.0;
}

}  // namespace tp
