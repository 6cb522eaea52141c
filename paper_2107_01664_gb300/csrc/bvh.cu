// Barnes-Hut approximation of the energy (§4.1, Eq. 16) and its
// differential (§4.2) over a BVH built on the GPU.
//
// Tree. Faces are sorted by the 30-bit Morton code of their barycenter
// (ties broken by face index, so the order is unique); runs of `leaf_size`
// consecutive faces form the leaves, and an implicit binary tree over the
// leaves splits every range of n leaves into ceil(n/2) + floor(n/2). Nodes
// are numbered in pre-order, so the left child of node i is i + 1 and the
// first node after the subtree of i (its escape index) is i + 2n - 1: the
// traversal needs no stack. The shape depends only on (nf, leaf_size) and
// is built once per mesh; the Morton order and the node data (area a_I,
// area-weighted barycenter X_I, bounding box of the faces' vertices, radius
// r_I from X_I) are rebuilt bottom-up whenever the positions change. With
// bvh_refit the face order of the last build is kept and only the node data
// are recomputed: any face order gives a valid tree (the admissibility test
// uses the actual boxes and radii), only its quality drifts.
//
// Admissibility of node I for target face S (read with the separation
// parameter theta, which the printed inequality omits):
//     max(r_S, r_I)^2 < theta^2 dist(box_S, box_I)^2,
// box_S the bounding box of triangle S and r_S its radius from X_S. An
// admissible node contributes K(X_S, P_S; X_I) a_S a_I; a leaf that is not
// admissible is summed exactly over its faces (T != S); otherwise the
// traversal descends. theta = 0 never admits a node, which gives the exact
// all-pairs sum.
//
// Differential ("full" mode): the exact derivative of the Barnes-Hut energy
// with the admissible sets held fixed. The target side is accumulated in
// registers. The source side is scattered with FP64 atomics into per-node
// accumulators G_I = sum_S -a_S a_I dK/dd, Q_I = sum_S a_S K (far field) and
// per-face accumulators (near field), then pushed down to the faces through
// X_I = sum a_T X_T / a_I and a_I = sum a_T. "Literal" mode keeps only the
// target-side terms, the formula printed in §4.2.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <vector>

#include "tp_internal.cuh"

namespace tp {

struct NodeShape {  // fixed per mesh
    int first, count, skip, leaf;
};

// ---------------------------------------------------------------------------
// host: implicit tree shape
// ---------------------------------------------------------------------------

static void shape_rec(std::vector<NodeShape>& out, std::vector<int>& depth, std::vector<int>& left,
                      int id, int lo, int hi, int d, int leaf, int nf) {
    int n = hi - lo;
    NodeShape s;
    s.first = lo * leaf;
    s.count = std::min(hi * leaf, nf) - lo * leaf;
    s.skip = id + 2 * n - 1;
    s.leaf = n == 1;
    out[id] = s;
    depth[id] = d;
    if (n == 1) {
        left[id] = -1;
        return;
    }
    int nl = (n + 1) / 2;
    left[id] = id + 1;
    shape_rec(out, depth, left, id + 1, lo, lo + nl, d + 1, leaf, nf);
    shape_rec(out, depth, left, id + 2 * nl, lo + nl, hi, d + 1, leaf, nf);
}

struct BvhHost {
    int leaf = 0, nleaf = 0, nnodes = 0, maxdepth = 0;
    std::vector<int> level_off;  // nodes sorted by depth: offsets per depth
};

// device arrays in m->bvh_tmp: [shape int4 nnodes][right child int][level order int]
static int bvh_shape(tp_mesh* m, int leaf, BvhHost& h) {
    h.leaf = leaf;
    h.nleaf = (m->nf + leaf - 1) / leaf;
    h.nnodes = 2 * h.nleaf - 1;
    std::vector<NodeShape> sh(h.nnodes);
    std::vector<int> depth(h.nnodes), left(h.nnodes);
    shape_rec(sh, depth, left, 0, 0, h.nleaf, 0, leaf, m->nf);
    h.maxdepth = *std::max_element(depth.begin(), depth.end());
    std::vector<int> order(h.nnodes);
    for (int i = 0; i < h.nnodes; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return depth[a] < depth[b]; });
    h.level_off.assign(h.maxdepth + 2, 0);
    for (int i = 0; i < h.nnodes; ++i) h.level_off[depth[i] + 1]++;
    for (int d = 0; d <= h.maxdepth; ++d) h.level_off[d + 1] += h.level_off[d];
    // right child = first node after the left subtree = escape index of the left child
    std::vector<int> right(h.nnodes, -1);
    for (int i = 0; i < h.nnodes; ++i)
        if (!sh[i].leaf) right[i] = sh[i + 1].skip;
    size_t bytes = sizeof(NodeShape) * h.nnodes + sizeof(int) * 2 * (size_t)h.nnodes;
    TP_TRY(ensure(m->bvh_tmp, bytes));
    char* base = m->bvh_tmp.as<char>();
    TP_CUDA(cudaMemcpy(base, sh.data(), sizeof(NodeShape) * h.nnodes, cudaMemcpyHostToDevice));
    TP_CUDA(cudaMemcpy(base + sizeof(NodeShape) * h.nnodes, right.data(), sizeof(int) * h.nnodes,
                       cudaMemcpyHostToDevice));
    TP_CUDA(cudaMemcpy(base + sizeof(NodeShape) * h.nnodes + sizeof(int) * h.nnodes, order.data(),
                       sizeof(int) * h.nnodes, cudaMemcpyHostToDevice));
    return TP_OK;
}


// node buffer layout: [BvhNode nn][d4 nn][float4 nn][double nn]; with 64-,
// 32-, 16- and 8-byte elements in decreasing size every array starts on a
// boundary of its own element size
static_assert(sizeof(BvhNode) == 64, "BvhNode must stay 64 bytes");
static_assert(sizeof(d4) == 32 && alignof(d4) == 32, "d4 must be a 32-byte aligned quad");

struct NodeArrays {
    BvhNode* node;
    d4* node64;      // FP64 barycenter (relative frame) and area
    float4* nodelo;  // low parts of the FP32 barycenter
    double* noder;   // FP64 radius
};

static size_t node_bytes(int nn) {
    return (sizeof(BvhNode) + sizeof(d4) + sizeof(float4) + sizeof(double)) * (size_t)nn;
}

static NodeArrays node_arrays(const tp_mesh* m) {
    NodeArrays a;
    const int nn = m->bvh_nodes;
    a.node = m->bvh_node.as<BvhNode>();
    a.node64 = reinterpret_cast<d4*>(a.node + nn);
    a.nodelo = reinterpret_cast<float4*>(a.node64 + nn);
    a.noder = reinterpret_cast<double*>(a.nodelo + nn);
    return a;
}

// ---------------------------------------------------------------------------
// device: Morton codes, sort, face boxes, node aggregates
// ---------------------------------------------------------------------------

__global__ void k_bbox_partial(const d4* __restrict__ X, int nf, double* __restrict__ part) {
    __shared__ double lo[3][256], hi[3][256];
    double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
    for (int i = blockIdx.x * 256 + threadIdx.x; i < nf; i += gridDim.x * 256) {
        d4 x = X[i];
        double v[3] = {x.x, x.y, x.z};
        for (int c = 0; c < 3; ++c) {
            l[c] = fmin(l[c], v[c]);
            h[c] = fmax(h[c], v[c]);
        }
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

__global__ void k_bbox_final(double* __restrict__ part, int nblk) {
    if (threadIdx.x != 0) return;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int b = 0; b < nblk; ++b)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], part[6 * b + c]);
            hi[c] = fmax(hi[c], part[6 * b + 3 + c]);
        }
    for (int c = 0; c < 3; ++c) {
        part[6 * 1024 + c] = lo[c];
        part[6 * 1024 + 3 + c] = hi[c];
    }
}

__device__ __forceinline__ unsigned spread10(unsigned v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// 30-bit Morton code of the FP64 barycenter, cell = floor((x - lo) / ext * 1024)
__global__ void k_morton(const d4* __restrict__ X, int nf, const double* __restrict__ bb,
                         unsigned long long* __restrict__ keys) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const double lo[3] = {bb[0], bb[1], bb[2]}, hi[3] = {bb[3], bb[4], bb[5]};
    d4 x = X[i];
    double v[3] = {x.x, x.y, x.z};
    unsigned q[3];
    for (int c = 0; c < 3; ++c) {
        double ext = hi[c] - lo[c];
        double t = ext > 0.0 ? __dmul_rn(__dsub_rn(v[c], lo[c]), 1024.0 / ext) : 0.0;
        int qi = (int)floor(t);
        q[c] = (unsigned)(qi < 0 ? 0 : (qi > 1023 ? 1023 : qi));
    }
    unsigned code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    keys[i] = ((unsigned long long)code << 32) | (unsigned)i;
}

// sorted face tables, face boxes and radii
// sort keys that reproduce a given face order (refit): the low 32 bits carry the face
__global__ void k_keys_from_perm(const int* __restrict__ perm, int nf, unsigned long long* __restrict__ keys) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) keys[i] = (unsigned long long)(unsigned)perm[i];
}

__global__ void k_sorted_faces(const unsigned long long* __restrict__ keys, int nf,
                               const double* __restrict__ pos, const int* __restrict__ faces,
                               const double* __restrict__ center, const d4* __restrict__ f64a,
                               const float4* __restrict__ f32a, const float4* __restrict__ f32b,
                               const float4* __restrict__ f32c, int* __restrict__ perm, float4* __restrict__ sa,
                               float4* __restrict__ sb, float4* __restrict__ sl, FaceBox* __restrict__ box) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int S = (int)(keys[i] & 0xffffffffull);
    perm[i] = S;
    sa[i] = f32a[S];
    sb[i] = f32b[S];
    sl[i] = f32c[S];
    d4 X = f64a[S];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, r2 = 0.0;
    for (int cr = 0; cr < 3; ++cr) {
        int v = faces[3 * S + cr];
        double p[3] = {pos[3 * v] - center[0], pos[3 * v + 1] - center[1], pos[3 * v + 2] - center[2]};
        double dx = p[0] - X.x, dy = p[1] - X.y, dz = p[2] - X.z;
        r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], p[c]);
            hi[c] = fmax(hi[c], p[c]);
        }
    }
    box[i] = FaceBox{(float)lo[0], (float)lo[1], (float)lo[2], (float)r2,
                     (float)hi[0], (float)hi[1], (float)hi[2], (float)X.w};
}

// node aggregates, one depth level per launch (deepest first)
__global__ void k_nodes_level(const NodeShape* __restrict__ shape, const int* __restrict__ right,
                              const int* __restrict__ order, int n0, int n1,
                              const int* __restrict__ perm, const double* __restrict__ pos,
                              const int* __restrict__ faces, const double* __restrict__ center,
                              const d4* __restrict__ f64a, const FaceBox* __restrict__ fbox,
                              BvhNode* __restrict__ node, d4* __restrict__ node64, double* __restrict__ noder,
                              float4* __restrict__ nodelo) {
    int k = n0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n1) return;
    int id = order[k];
    NodeShape s = shape[id];
    double a = 0.0, X[3] = {0, 0, 0}, lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300},
           r = 0.0;
    if (s.leaf) {
        for (int i = s.first; i < s.first + s.count; ++i) {
            d4 f = f64a[perm[i]];
            a += f.w;
            X[0] += f.w * f.x;
            X[1] += f.w * f.y;
            X[2] += f.w * f.z;
        }
        for (int c = 0; c < 3; ++c) X[c] /= a;
        for (int i = s.first; i < s.first + s.count; ++i) {
            int S = perm[i];
            FaceBox b = fbox[i];
            lo[0] = fmin(lo[0], (double)b.lox); lo[1] = fmin(lo[1], (double)b.loy); lo[2] = fmin(lo[2], (double)b.loz);
            hi[0] = fmax(hi[0], (double)b.hix); hi[1] = fmax(hi[1], (double)b.hiy); hi[2] = fmax(hi[2], (double)b.hiz);
            for (int cr = 0; cr < 3; ++cr) {
                int v = faces[3 * S + cr];
                double dx = pos[3 * v] - center[0] - X[0], dy = pos[3 * v + 1] - center[1] - X[1],
                       dz = pos[3 * v + 2] - center[2] - X[2];
                r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
            }
        }
    } else {
        int L = id + 1, R = right[id];
        d4 xl = node64[L], xr = node64[R];
        a = xl.w + xr.w;
        X[0] = (xl.w * xl.x + xr.w * xr.x) / a;
        X[1] = (xl.w * xl.y + xr.w * xr.y) / a;
        X[2] = (xl.w * xl.z + xr.w * xr.z) / a;
        BvhNode nl = node[L], nr = node[R];
        lo[0] = fmin(nl.lox, nr.lox); lo[1] = fmin(nl.loy, nr.loy); lo[2] = fmin(nl.loz, nr.loz);
        hi[0] = fmax(nl.hix, nr.hix); hi[1] = fmax(nl.hiy, nr.hiy); hi[2] = fmax(nl.hiz, nr.hiz);
        double rl = noder[L], rr = noder[R];
        double dl = sqrt((xl.x - X[0]) * (xl.x - X[0]) + (xl.y - X[1]) * (xl.y - X[1]) + (xl.z - X[2]) * (xl.z - X[2]));
        double dr = sqrt((xr.x - X[0]) * (xr.x - X[0]) + (xr.y - X[1]) * (xr.y - X[1]) + (xr.z - X[2]) * (xr.z - X[2]));
        r = fmax(dl + rl, dr + rr);
    }
    node64[id] = d4{X[0], X[1], X[2], a};
    noder[id] = r;
    nodelo[id] = make_float4((float)(X[0] - (double)(float)X[0]), (float)(X[1] - (double)(float)X[1]),
                             (float)(X[2] - (double)(float)X[2]), 0.f);
    BvhNode o;
    o.cx = (float)X[0]; o.cy = (float)X[1]; o.cz = (float)X[2]; o.a = (float)a;
    o.lox = (float)lo[0]; o.loy = (float)lo[1]; o.loz = (float)lo[2]; o.r2 = (float)(r * r);
    o.hix = (float)hi[0]; o.hiy = (float)hi[1]; o.hiz = (float)hi[2]; o.pad = 0.f;
    o.first = s.first; o.count = s.count; o.skip = s.skip; o.leaf = s.leaf;
    node[id] = o;
}

// Exact node radii r_I = max |v - X_I| over the vertices of the node's faces.
// Each sorted face walks its root-to-leaf path and raises the radius of every
// node on it; non-negative doubles order like their bit patterns, so a 64-bit
// integer max is exact and independent of the order of the updates.
__global__ void k_node_radius_exact(const int* __restrict__ perm, int nf, int leaf,
                                    const NodeShape* __restrict__ shape, const int* __restrict__ right,
                                    const d4* __restrict__ node64, const double* __restrict__ pos,
                                    const int* __restrict__ faces, const double* __restrict__ center,
                                    unsigned long long* __restrict__ rbits) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int S = perm[i];
    double v[3][3];
    for (int cr = 0; cr < 3; ++cr) {
        int vi = faces[3 * S + cr];
        for (int c = 0; c < 3; ++c) v[cr][c] = pos[3 * vi + c] - center[c];
    }
    const int lf = i / leaf;
    int id = 0;
    for (;;) {
        d4 X = node64[id];
        double d2 = 0.0;
        for (int cr = 0; cr < 3; ++cr) {
            double dx = v[cr][0] - X.x, dy = v[cr][1] - X.y, dz = v[cr][2] - X.z;
            d2 = fmax(d2, dx * dx + dy * dy + dz * dz);
        }
        unsigned long long b = (unsigned long long)__double_as_longlong(sqrt(d2));
        if (b > rbits[id]) atomicMax(rbits + id, b);
        NodeShape sh = shape[id];
        if (sh.leaf) break;
        const int L = id + 1;
        NodeShape sl = shape[L];
        int lfirst = sl.first / leaf, lcount = (sl.skip - L + 1) / 2;
        id = (lf >= lfirst && lf < lfirst + lcount) ? L : right[id];
    }
}

__global__ void k_node_radius_apply(const unsigned long long* __restrict__ rbits, int nn, double* __restrict__ noder,
                                    BvhNode* __restrict__ node) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nn) return;
    double r = __longlong_as_double((long long)rbits[id]);
    noder[id] = r;
    node[id].r2 = (float)(r * r);
}

int bvh_build(tp_mesh* m, const tp_params* p, cudaStream_t st) {
    if (m->bvh_shape_leaf != p->leaf_size) {
        BvhHost h;
        TP_TRY(bvh_shape(m, p->leaf_size, h));
        m->bvh_shape_leaf = h.leaf;
        m->bvh_maxdepth = h.maxdepth;
        m->bvh_nodes = h.nnodes;
        m->bvh_level_off = h.level_off;
        m->bvh_valid = false;
        m->bvh_ordered = false;
    }
    if (m->bvh_valid) return TP_OK;
    BvhHost h;
    h.leaf = m->bvh_shape_leaf;
    h.nnodes = m->bvh_nodes;
    h.maxdepth = m->bvh_maxdepth;
    h.level_off = m->bvh_level_off;
    const int nf = m->nf;
    m->bvh_nodes = h.nnodes;
    m->bvh_leaf = h.leaf;
    // buffers
    size_t sort_bytes = 0;
    cub::DeviceRadixSort::SortKeys((void*)nullptr, sort_bytes, (unsigned long long*)nullptr,
                                   (unsigned long long*)nullptr, nf, 0, 62);
    TP_TRY(ensure(m->bvh_keys, sizeof(unsigned long long) * 2 * (size_t)nf + sizeof(double) * 6 * 1025));
    TP_TRY(ensure(m->bvh_sortws, sort_bytes + 256));
    TP_TRY(ensure(m->bvh_perm, sizeof(int) * (size_t)nf + sizeof(FaceBox) * (size_t)nf));
    TP_TRY(ensure(m->bvh_f32a, sizeof(float4) * (size_t)nf));
    TP_TRY(ensure(m->bvh_f32b, sizeof(float4) * (size_t)nf));
    TP_TRY(ensure(m->bvh_node, node_bytes(h.nnodes)));
    TP_TRY(ensure(m->bvh_f32c, sizeof(float4) * (size_t)nf));
    unsigned long long* kin = m->bvh_keys.as<unsigned long long>();
    unsigned long long* kout = kin + nf;
    double* bpart = (double*)(kout + nf);
    int* perm = m->bvh_perm.as<int>();
    FaceBox* fbox = (FaceBox*)(perm + nf);
    const NodeArrays na = node_arrays(m);
    if ((reinterpret_cast<uintptr_t>(na.node64) & 31) || (reinterpret_cast<uintptr_t>(na.nodelo) & 15) ||
        (reinterpret_cast<uintptr_t>(na.noder) & 7))
        return fail(TP_ERR_CUDA, "bvh: node arrays misaligned");
    BvhNode* node = na.node;
    d4* node64 = na.node64;
    double* noder = na.noder;
    float4* nodelo = na.nodelo;
    const NodeShape* shape = m->bvh_tmp.as<NodeShape>();
    const int* right = (const int*)(shape + h.nnodes);
    const int* order = right + h.nnodes;

    ProfScope ps(m, PK_BVH_BUILD, (double)nf, st);
    if (p->bvh_refit && m->bvh_ordered) {
        // refit: the face order of the last build, node data from the new positions
        k_keys_from_perm<<<(nf + 255) / 256, 256, 0, st>>>(perm, nf, kout);
        TP_LAUNCH_CHECK();
    } else {
        int nblk = std::min(1024, (nf + 255) / 256);
        k_bbox_partial<<<nblk, 256, 0, st>>>(m->f64a.as<d4>(), nf, bpart);
        TP_LAUNCH_CHECK();
        k_bbox_final<<<1, 32, 0, st>>>(bpart, nblk);
        TP_LAUNCH_CHECK();
        k_morton<<<(nf + 255) / 256, 256, 0, st>>>(m->f64a.as<d4>(), nf, bpart + 6 * 1024, kin);
        TP_LAUNCH_CHECK();
        TP_CUDA(cub::DeviceRadixSort::SortKeys(m->bvh_sortws.ptr, sort_bytes, kin, kout, nf, 0, 62, st));
    }
    k_sorted_faces<<<(nf + 255) / 256, 256, 0, st>>>(kout, nf, m->pos.as<double>(), m->faces.as<int>(),
                                                     m->center.as<double>(), m->f64a.as<d4>(),
                                                     m->f32a.as<float4>(), m->f32b.as<float4>(),
                                                     m->f32c.as<float4>(), perm, m->bvh_f32a.as<float4>(),
                                                     m->bvh_f32b.as<float4>(), m->bvh_f32c.as<float4>(), fbox);
    TP_LAUNCH_CHECK();
    for (int d = h.maxdepth; d >= 0; --d) {
        int n0 = h.level_off[d], n1 = h.level_off[d + 1];
        k_nodes_level<<<(n1 - n0 + 127) / 128, 128, 0, st>>>(shape, right, order, n0, n1, perm,
                                                             m->pos.as<double>(), m->faces.as<int>(),
                                                             m->center.as<double>(), m->f64a.as<d4>(), fbox,
                                                             node, node64, noder, nodelo);
        TP_LAUNCH_CHECK();
    }
    // exact radii (the per-level pass above used the child bound for inner nodes)
    {
        unsigned long long* rbits = reinterpret_cast<unsigned long long*>(kin);   // keys no longer needed
        TP_CUDA(cudaMemsetAsync(rbits, 0, sizeof(unsigned long long) * (size_t)h.nnodes, st));
        k_node_radius_exact<<<(nf + 255) / 256, 256, 0, st>>>(perm, nf, h.leaf, shape, right, node64,
                                                              m->pos.as<double>(), m->faces.as<int>(),
                                                              m->center.as<double>(), rbits);
        TP_LAUNCH_CHECK();
        k_node_radius_apply<<<(h.nnodes + 255) / 256, 256, 0, st>>>(rbits, h.nnodes, noder, node);
        TP_LAUNCH_CHECK();
    }
    m->bvh_valid = true;
    m->bvh_ordered = true;
    m->bvh_version++;
    return TP_OK;
}

int bvh_view(tp_mesh* m, const tp_params* p, cudaStream_t st, BvhView* v) {
    TP_TRY(bvh_build(m, p, st));
    const NodeArrays na = node_arrays(m);
    const NodeShape* shape = m->bvh_tmp.as<NodeShape>();
    const int* right = (const int*)(shape + m->bvh_nodes);
    v->nnodes = m->bvh_nodes;
    v->maxdepth = m->bvh_maxdepth;
    v->node = na.node;
    v->nodelo = na.nodelo;
    v->sa = m->bvh_f32a.as<float4>();
    v->sb = m->bvh_f32b.as<float4>();
    v->sl = m->bvh_f32c.as<float4>();
    v->perm = m->bvh_perm.as<int>();
    v->fbox = (const FaceBox*)(v->perm + m->nf);
    v->right = right;
    v->level_order = right + m->bvh_nodes;
    v->level_off = m->bvh_level_off.data();
    return TP_OK;
}

// ---------------------------------------------------------------------------
// traversal
// ---------------------------------------------------------------------------

__device__ __forceinline__ float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fpow(float x, float y) {
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y * l));
    return r;
}

struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Warp-cooperative traversal. Each lane owns one target (sorted position
// i); the warp walks the pre-order node sequence together, and lane L is
// active at node id only when id >= skip_L. When a lane finishes a node (an
// admissible node, or an inadmissible leaf summed exactly) it sets skip_L to
// the node's escape index; the warp descends (id + 1) if any active lane needs
// to, else jumps to the escape index. Every jump target lies at or before
// the escape index of each lane's finished nodes, so each lane sees exactly
// the nodes of its own stackless traversal: the admissible sets are those of
// the per-target definition, while node loads and leaf-face loads are the
// same address across the warp.
template <bool P6>
__global__ void __launch_bounds__(128)
k_bh_energy(const BvhNode* __restrict__ node, const float4* __restrict__ nodelo, int nnodes,
            const float4* __restrict__ sa, const float4* __restrict__ sb, const float4* __restrict__ sl,
            const FaceBox* __restrict__ fbox, const int* __restrict__ perm,
            const int* __restrict__ inv_targets /* sorted positions of a target list, or null */, int nt,
            float theta2, float halfp, const d4* __restrict__ f64a, double* __restrict__ rows,
            unsigned long long* __restrict__ count) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = t < nt;
    const int i = has ? (inv_targets ? inv_targets[t] : t) : 0;
    const float4 A = sa[i], B = sb[i], Al = sl[i];
    const FaceBox fb = fbox[i];
    int skip = has ? 0 : nnodes;
    float acc = 0.f;
    KahanF sum;
    int nint = 0, run = 0;
    int id = 0;
    while (id < nnodes) {
        const BvhNode n = node[id];
        bool desc = false;
        if (id >= skip) {
            float d2 = box_dist2(fb.lox, fb.loy, fb.loz, fb.hix, fb.hiy, fb.hiz, n);
            float mr2 = fmaxf(fb.r2, n.r2);
            if (mr2 < __fmul_rn(theta2, d2)) {
                float4 nl = nodelo[id];
                float dx = (A.x - n.cx) + (Al.x - nl.x), dy = (A.y - n.cy) + (Al.y - nl.y),
                      dz = (A.z - n.cz) + (Al.z - nl.z);
                float r2 = dx * dx + dy * dy + dz * dz;
                float u = B.x * dx + B.y * dy + B.z * dz;
                float ir2 = frcp(fmaxf(r2, 1e-18f));
                float q = u * u * (ir2 * ir2);
                float K = P6 ? q * q * q : fpow(q, halfp);
                acc = fmaf(K, n.a, acc);
                ++nint;
                if (++run == 32) { sum.add(acc); acc = 0.f; run = 0; }
                skip = n.skip;
            } else if (n.leaf) {
                for (int j = n.first; j < n.first + n.count; ++j) {
                    if (j == i) continue;
                    float4 s = sa[j], l = sl[j];
                    float dx = (A.x - s.x) + (Al.x - l.x), dy = (A.y - s.y) + (Al.y - l.y),
                          dz = (A.z - s.z) + (Al.z - l.z);
                    float r2 = dx * dx + dy * dy + dz * dz;
                    float u = B.x * dx + B.y * dy + B.z * dz;
                    float ir2 = frcp(fmaxf(r2, 1e-18f));
                    float q = u * u * (ir2 * ir2);
                    float K = P6 ? q * q * q : fpow(q, halfp);
                    acc = fmaf(K, s.w, acc);
                    ++nint;
                }
                sum.add(acc);
                acc = 0.f;
                run = 0;
                skip = n.skip;
            } else {
                desc = true;
            }
        }
        id = __any_sync(0xffffffffu, desc) ? id + 1 : n.skip;
    }
    sum.add(acc);
    if (has) rows[t] = f64a[perm[i]].w * sum.value();
    if (count && nint) atomicAdd(count, (unsigned long long)nint);
}

// ---------------------------------------------------------------------------
// interaction lists
// ---------------------------------------------------------------------------
//
// The per-target admissible sets of §4.1 are kept exactly, but found for a
// whole group of 32 consecutive sorted targets (one warp) at a time. Every
// candidate node is first tested against the group: against the bounding box
// of the group's target boxes with the largest target radius (if admissible
// there, it is admissible for every target: the box gap only shrinks and the
// radius only grows) and against the farthest-gap box with the smallest
// radius (if inadmissible there, it is inadmissible for every target). The
// FP32 operations are monotone, so both implications hold for the FP32
// decisions too. Only the nodes that are neither get the exact per-target
// test of the walk kernels, lane by lane. A candidate carries the mask of the
// group's targets for which none of its ancestors was admissible; the 32
// lanes test 32 candidates at once, from a stack in shared memory. The output
// per group: far entries (node, mask) and near entries (first face of an
// inadmissible leaf, mask; the leaf holds min(leaf size, nf - first) faces).
// The lists depend only on the tree and theta: they are built once per
// tree and serve the energy, the differential and every operator apply of
// the tree, whose evaluation kernels then stream the lists without a walk.

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ float wmin(float x) {
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ float wmax(float x) {
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// WRITE = false: counts per group; WRITE = true: the entries at the offsets
template <bool WRITE>
__global__ void __launch_bounds__(128)
k_bh_list(const BvhNode* __restrict__ node, const int* __restrict__ right, const FaceBox* __restrict__ fbox,
          int nf, float theta2, int cap, long long* __restrict__ cnt, const long long* __restrict__ far_off,
          const long long* __restrict__ near_off, int2* __restrict__ far_out, int2* __restrict__ near_out,
          int* __restrict__ err, unsigned long long* __restrict__ inter) {
    extern __shared__ int2 lstack[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ngroups = (nf + BHL_GROUP - 1) / BHL_GROUP;
    const int g = blockIdx.x * (blockDim.x >> 5) + w;
    if (g >= ngroups) return;                       // the whole warp
    int2* stk = lstack + (size_t)w * cap;
    const int i = g * BHL_GROUP + lane;
    const bool has = i < nf;
    const FaceBox fb = fbox[has ? i : 0];
    const float glx = wmin(has ? fb.lox : 3e38f), gly = wmin(has ? fb.loy : 3e38f), glz = wmin(has ? fb.loz : 3e38f);
    const float ghx = wmax(has ? fb.hix : -3e38f), ghy = wmax(has ? fb.hiy : -3e38f), ghz = wmax(has ? fb.hiz : -3e38f);
    const float gr2max = wmax(has ? fb.r2 : 0.f), gr2min = wmin(has ? fb.r2 : 3e38f);
    const unsigned full = __ballot_sync(0xffffffffu, has);
    const unsigned lt = lanemask_lt();
    int sp = 1;
    if (lane == 0) stk[0] = make_int2(0, (int)full);
    __syncwarp();
    long long nfar = 0, nnear = 0;
    const long long fo = WRITE ? far_off[g] : 0, no = WRITE ? near_off[g] : 0;
    // writes stay inside the group's range whatever happens (the second pass
    // must reproduce the first pass's counts; a mismatch is reported)
    const long long flim = WRITE ? far_off[g + 1] : 0, nlim = WRITE ? near_off[g + 1] : 0;
    bool over = false;
    // interactions the lists give (WRITE pass): popc(mask) per far entry,
    // and per near leaf popc(mask) x its faces minus the self pairs
    unsigned long long ninter = 0;
    const int g0 = g * BHL_GROUP;
    auto near_terms = [&](const BvhNode& nd, unsigned msk) -> unsigned long long {
        const int lo = max(nd.first, g0) - g0, hi = min(nd.first + nd.count, g0 + BHL_GROUP) - g0;
        const unsigned self = hi > lo ? (((hi - lo) >= 32 ? 0xffffffffu : ((1u << (hi - lo)) - 1u)) << lo) : 0u;
        return (unsigned long long)__popc(msk) * (unsigned)nd.count - (unsigned)__popc(msk & self);
    };
    while (sp > 0 && !over) {
        const int n = min(32, sp);
        const bool act = lane < n;
        int2 e = make_int2(0, 0);
        if (act) e = stk[sp - n + lane];
        __syncwarp();
        sp -= n;
        bool cadm = false, cnot = false, leaf = false;
        BvhNode nd;
        if (act) {
            nd = node[e.x];
            leaf = nd.leaf != 0;
            const float d2lo = box_dist2(glx, gly, glz, ghx, ghy, ghz, nd);
            cadm = fmaxf(gr2max, nd.r2) < __fmul_rn(theta2, d2lo);
            const float ux = fmaxf(fmaxf(__fsub_rn(nd.lox, glx), __fsub_rn(ghx, nd.hix)), 0.f);
            const float uy = fmaxf(fmaxf(__fsub_rn(nd.loy, gly), __fsub_rn(ghy, nd.hiy)), 0.f);
            const float uz = fmaxf(fmaxf(__fsub_rn(nd.loz, glz), __fsub_rn(ghz, nd.hiz)), 0.f);
            const float d2hi = __fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), __fmul_rn(uz, uz));
            cnot = !cadm && !(fmaxf(gr2min, nd.r2) < __fmul_rn(theta2, d2hi));
        }
        // certain for the whole group
        const unsigned bf = __ballot_sync(0xffffffffu, cadm);
        if (WRITE && cadm && fo + nfar + __popc(bf & lt) < flim) far_out[fo + nfar + __popc(bf & lt)] = e;
        nfar += __popc(bf);
        const unsigned bn = __ballot_sync(0xffffffffu, cnot && leaf);
        if (WRITE && cnot && leaf && no + nnear + __popc(bn & lt) < nlim)
            near_out[no + nnear + __popc(bn & lt)] = make_int2(nd.first, e.y);
        nnear += __popc(bn);
        if (WRITE) {
            if (cadm) ninter += (unsigned)__popc((unsigned)e.y);
            if (cnot && leaf) ninter += near_terms(nd, (unsigned)e.y);
        }
        const unsigned bd = __ballot_sync(0xffffffffu, cnot && !leaf);
        if (sp + 2 * __popc(bd) > cap) {
            over = true;
        } else {
            if (cnot && !leaf) {
                const int at = sp + 2 * __popc(bd & lt);
                stk[at] = make_int2(right[e.x], e.y);
                stk[at + 1] = make_int2(e.x + 1, e.y);
            }
            sp += 2 * __popc(bd);
        }
        // the rest: the exact per-target test, one candidate at a time
        unsigned bi = __ballot_sync(0xffffffffu, act && !cadm && !cnot);
        while (bi && !over) {
            const int src = __ffs(bi) - 1;
            bi &= bi - 1;
            const int nid = __shfl_sync(0xffffffffu, e.x, src);
            const unsigned msk = (unsigned)__shfl_sync(0xffffffffu, e.y, src);
            const BvhNode n2 = node[nid];
            bool adm = false;
            if ((msk >> lane) & 1u) {
                const float d2 = box_dist2(fb.lox, fb.loy, fb.loz, fb.hix, fb.hiy, fb.hiz, n2);
                adm = fmaxf(fb.r2, n2.r2) < __fmul_rn(theta2, d2);
            }
            const unsigned am = __ballot_sync(0xffffffffu, adm) & msk;
            const unsigned rest = msk & ~am;
            if (am) {
                if (WRITE && lane == 0 && fo + nfar < flim) far_out[fo + nfar] = make_int2(nid, (int)am);
                if (WRITE && lane == 0) ninter += (unsigned)__popc(am);
                ++nfar;
            }
            if (rest) {
                if (n2.leaf) {
                    if (WRITE && lane == 0 && no + nnear < nlim) near_out[no + nnear] = make_int2(n2.first, (int)rest);
                    if (WRITE && lane == 0) ninter += near_terms(n2, rest);
                    ++nnear;
                } else if (sp + 2 > cap) {
                    over = true;
                } else {
                    if (lane == 0) {
                        stk[sp] = make_int2(right[nid], (int)rest);
                        stk[sp + 1] = make_int2(nid + 1, (int)rest);
                    }
                    sp += 2;
                }
            }
        }
        __syncwarp();
    }
    if (WRITE) {
        for (int o = 16; o > 0; o >>= 1) ninter += __shfl_xor_sync(0xffffffffu, ninter, o);
    }
    if (lane == 0) {
        if (over) atomicExch(err, 1);
        if (WRITE && ninter) atomicAdd(inter, ninter);
        if (!WRITE) {
            cnt[g] = nfar;
            cnt[ngroups + 1 + g] = nnear;
        } else if (nfar != flim - fo || nnear != nlim - no) {
            atomicExch(err, 2);   // the two passes must agree
        }
    }
}

int bh_lists(tp_mesh* m, const tp_params* p, cudaStream_t st, BhLists* out, bool* ok) {
    *ok = false;
    TP_TRY(bvh_build(m, p, st));
    const int nf = m->nf, nn = m->bvh_nodes;
    const int ngroups = (nf + BHL_GROUP - 1) / BHL_GROUP;
    auto fill = [&]() {
        const long long* off = m->bhl_cnt.as<long long>();
        out->ngroups = ngroups;
        out->far_off = off;
        out->near_off = off + ngroups + 1;
        out->far = m->bhl_far.as<int2>();
        out->near = m->bhl_near.as<int2>();
        out->interactions = m->bhl_inter;
        out->leaf = m->bvh_shape_leaf;
    };
    if (m->bhl_version == m->bvh_version && m->bhl_theta == p->theta) {
        if (m->bhl_failed) return TP_OK;
        fill();
        *ok = true;
        return TP_OK;
    }
    m->bhl_version = m->bvh_version;
    m->bhl_theta = p->theta;
    m->bhl_failed = true;
    const NodeArrays na = node_arrays(m);
    const NodeShape* shape = m->bvh_tmp.as<NodeShape>();
    const int* right = (const int*)(shape + nn);
    const FaceBox* fbox = (const FaceBox*)(m->bvh_perm.as<int>() + nf);
    const int cap = 64 * (m->bvh_maxdepth + 2);
    const int warps = 4;
    const size_t smem = sizeof(int2) * (size_t)cap * warps;
    if (smem > 200 * 1024) return TP_OK;            // too deep a tree for the stack: walks serve
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (smem > 48 * 1024 && dev >= 0 && dev < 64 && !attr_set[dev]) {
        TP_CUDA(cudaFuncSetAttribute(k_bh_list<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        TP_CUDA(cudaFuncSetAttribute(k_bh_list<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr_set[dev] = true;
    }
    size_t scan_bytes = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, (long long*)nullptr, (long long*)nullptr, ngroups + 1);
    // offsets [2 (ngroups + 1)], counts [2 (ngroups + 1)], error word, scan workspace
    const size_t head = 4 * ((size_t)ngroups + 1) + 8;
    TP_TRY(ensure(m->bhl_cnt, sizeof(long long) * head + scan_bytes + 256));
    long long* off = m->bhl_cnt.as<long long>();
    long long* counts = off + 2 * (ngroups + 1);
    int* err = reinterpret_cast<int*>(counts + 2 * (ngroups + 1));
    void* scan_ws = reinterpret_cast<char*>(m->bhl_cnt.ptr) + sizeof(long long) * head;
    TP_CUDA(cudaMemsetAsync(off, 0, sizeof(long long) * head, st));
    const float theta2 = (float)(p->theta * p->theta);
    const int blocks = (ngroups + warps - 1) / warps;
    unsigned long long* inter = reinterpret_cast<unsigned long long*>(err + 2);
    k_bh_list<false><<<blocks, 32 * warps, smem, st>>>(na.node, right, fbox, nf, theta2, cap, counts, nullptr,
                                                       nullptr, nullptr, nullptr, err, inter);
    TP_LAUNCH_CHECK();
    // counts -> exclusive offsets (the extra last entry becomes the total)
    TP_CUDA(cub::DeviceScan::ExclusiveSum(scan_ws, scan_bytes, counts, off, ngroups + 1, st));
    TP_CUDA(cub::DeviceScan::ExclusiveSum(scan_ws, scan_bytes, counts + ngroups + 1, off + ngroups + 1, ngroups + 1,
                                          st));
    long long tot[2] = {0, 0};
    int e1 = 0;
    TP_CUDA(cudaMemcpyAsync(&tot[0], off + ngroups, sizeof(long long), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaMemcpyAsync(&tot[1], off + 2 * ngroups + 1, sizeof(long long), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaMemcpyAsync(&e1, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    if (e1 != 0) return TP_OK;                       // a stack overflowed: the walks serve this tree
    // entries are addressed with int offsets inside the kernels' loops
    if (tot[0] >= (1LL << 31) || tot[1] >= (1LL << 31)) return TP_OK;
    if (ensure(m->bhl_far, sizeof(int2) * ((size_t)tot[0] + 1)) != TP_OK ||
        ensure(m->bhl_near, sizeof(int2) * ((size_t)tot[1] + 1)) != TP_OK) {
        set_error("");
        return TP_OK;                                // no room for the lists: the walks serve
    }
    k_bh_list<true><<<blocks, 32 * warps, smem, st>>>(na.node, right, fbox, nf, theta2, cap, nullptr, off,
                                                      off + ngroups + 1, m->bhl_far.as<int2>(),
                                                      m->bhl_near.as<int2>(), err, inter);
    TP_LAUNCH_CHECK();
    unsigned long long ninter = 0;
    TP_CUDA(cudaMemcpyAsync(&e1, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaMemcpyAsync(&ninter, inter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    if (e1 != 0) return TP_OK;
    m->bhl_nfar = tot[0];
    m->bhl_nnear = tot[1];
    m->bhl_inter = ninter;
    m->bhl_failed = false;
    fill();
    *ok = true;
    return TP_OK;
}

// device counters of Barnes-Hut interactions: [0] energy, [1] differential
int bh_counter(tp_mesh* m, cudaStream_t st) {
    if (m->bhcount.ptr) return TP_OK;
    TP_TRY(ensure(m->bhcount, BH_NCOUNT * sizeof(unsigned long long)));
    TP_CUDA(cudaMemsetAsync(m->bhcount.ptr, 0, BH_NCOUNT * sizeof(unsigned long long), st));
    return TP_OK;
}

int bh_counts_read(tp_mesh* m, unsigned long long out[BH_NCOUNT], bool reset, cudaStream_t st) {
    for (int i = 0; i < BH_NCOUNT; ++i) out[i] = 0;
    if (!m->bhcount.ptr) return TP_OK;
    TP_CUDA(cudaMemcpyAsync(out, m->bhcount.ptr, BH_NCOUNT * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    if (reset) TP_CUDA(cudaMemsetAsync(m->bhcount.ptr, 0, BH_NCOUNT * sizeof(unsigned long long), st));
    return TP_OK;
}

// inverse permutation (face -> sorted position) for target lists
__global__ void k_inv_perm(const int* __restrict__ perm, int nf, int* __restrict__ inv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) inv[perm[i]] = i;
}
__global__ void k_map_targets(const int* __restrict__ tl, int nt, const int* __restrict__ inv, int* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) out[t] = inv[tl[t]];
}
// rows in sorted order -> rows in face order
__global__ void k_unsort_rows(const double* __restrict__ rs, const int* __restrict__ perm, int nf,
                              double* __restrict__ rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) rows[perm[i]] = rs[i];
}

// Energy rows from the interaction lists: one warp per group of 32 sorted
// targets, streaming the group's far entries (node terms) and near entries
// (exact sums over the leaf's faces, T != S); lanes whose bit is not set in
// an entry's mask add nothing. FP32 terms in runs of 32 entries, Kahan across
// runs, FP64 result (sorted order).
template <bool P6>
__global__ void __launch_bounds__(128)
k_bh_energy_list(const float4* __restrict__ node4, const float4* __restrict__ nodelo, const float4* __restrict__ sa,
                 const float4* __restrict__ sb, const float4* __restrict__ sl, int nf, BhLists L, float halfp,
                 const d4* __restrict__ f64a, const int* __restrict__ perm, double* __restrict__ rows,
                 unsigned long long* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= L.ngroups) return;
    const int i = g * BHL_GROUP + lane;
    const bool has = i < nf;
    const int ii = has ? i : 0;
    const float4 A = sa[ii], B = sb[ii], Al = sl[ii];
    const unsigned me = 1u << lane;
    KahanF sum;
    float acc = 0.f;
    const int f0 = (int)L.far_off[g], f1 = (int)L.far_off[g + 1];
    int run = 0;
#pragma unroll 4
    for (int e = f0; e < f1; ++e) {
        const int2 en = L.far[e];
        const float4 c = node4[4 * en.x];          // barycenter (hi), area
        const float4 nl = nodelo[en.x];
        const float dx = (A.x - c.x) + (Al.x - nl.x), dy = (A.y - c.y) + (Al.y - nl.y), dz = (A.z - c.z) + (Al.z - nl.z);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-18f)));
        const float u = B.x * dx + B.y * dy + B.z * dz;
        const float ir2 = frcp(r2);
        const float q = u * u * (ir2 * ir2);
        const float K = P6 ? q * q * q : fpow(q, halfp);
        const bool on = (unsigned)en.y & me;
        acc = fmaf(on ? K : 0.f, c.w, acc);
        if (++run == 32) {
            sum.add(acc);
            acc = 0.f;
            run = 0;
        }
    }
    sum.add(acc);
    acc = 0.f;
    const int n0 = (int)L.near_off[g], n1 = (int)L.near_off[g + 1];
    for (int e = n0; e < n1; ++e) {
        const int2 en = L.near[e];
        const int2 fc = make_int2(en.x, min(L.leaf, nf - en.x));   // the leaf's first face, count
        const bool on = (unsigned)en.y & me;
        for (int j = fc.x; j < fc.x + fc.y; ++j) {
            const float4 s = sa[j], l = sl[j];
            const float dx = (A.x - s.x) + (Al.x - l.x), dy = (A.y - s.y) + (Al.y - l.y), dz = (A.z - s.z) + (Al.z - l.z);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-18f)));
            const float u = B.x * dx + B.y * dy + B.z * dz;
            const float ir2 = frcp(r2);
            const float q = u * u * (ir2 * ir2);
            const float K = P6 ? q * q * q : fpow(q, halfp);
            const bool t = on && j != i;
            acc = fmaf(t ? K : 0.f, s.w, acc);
        }
        sum.add(acc);
        acc = 0.f;
    }
    if (has) rows[perm[i]] = f64a[perm[i]].w * sum.value();
    if (count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(count, L.interactions);
}

// packed FP32 pair arithmetic (two IEEE lanes per instruction)
__device__ __forceinline__ unsigned long long bp2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 bu2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}

// ---------------------------------------------------------------------------
// Staged list evaluation (p = 6). A warp streams its group's entries in
// batches of 32 sources: 32 far entries, or the faces of 32 / leaf near
// leaves. Lane k loads the record of source k of the NEXT batch while the
// warp evaluates the current one, so the dependent loads (list entry ->
// record) of 32 sources are in flight together instead of one entry at a
// time. A batch sits in shared memory in source pairs, in the order the
// packed FP32 arithmetic takes them (sources 2q and 2q + 1):
//     H[2q] = {x0, x1, y0, y1}     H[2q+1] = {z0, z1, a0, a1}
//     D[2q] = {lx0, lx1, ly0, ly1} D[2q+1] = {lz0, lz1, mask0, mask1}
// (barycenter hi part and area, low parts, the entry's lane mask). Slots past
// the end of the list hold a source parked far away with zero area and mask.
// ---------------------------------------------------------------------------

struct BhSrc {
    float4 c;        // barycenter (hi), area
    float4 l;        // low parts of the barycenter
    unsigned mask;   // lanes of the group that take this source
    int idx;         // node (far) or face (near)
};

__device__ __forceinline__ BhSrc bh_parked() {
    BhSrc s;
    s.c = make_float4(1e15f, 1e15f, 1e15f, 0.f);
    s.l = make_float4(0.f, 0.f, 0.f, 0.f);
    s.mask = 0u;
    s.idx = -1;
    return s;
}

// a group's batch sequence: far batches first, then near batches
struct BhBatches {
    int f0, f1, n0, n1;   // entry ranges
    int nbf, nb;          // far batches, all batches
    int lb, kl, fi;       // near leaves per batch; this lane's leaf slot and face in it
    __device__ BhBatches(const BhLists& L, int g, int lane) {
        f0 = (int)L.far_off[g];
        f1 = (int)L.far_off[g + 1];
        n0 = (int)L.near_off[g];
        n1 = (int)L.near_off[g + 1];
        lb = 32 / L.leaf;
        kl = lane / L.leaf;
        fi = lane - kl * L.leaf;
        nbf = (f1 - f0 + 31) >> 5;
        nb = nbf + (n1 - n0 + lb - 1) / lb;
    }
    // this lane's list entry in batch b (x < 0: none)
    __device__ __forceinline__ int2 entry(const BhLists& L, int b, int lane) const {
        if (b < nbf) {
            const int e = f0 + 32 * b + lane;
            return e < f1 ? L.far[e] : make_int2(-1, 0);
        }
        const int e = n0 + lb * (b - nbf) + kl;
        return (kl < lb && e < n1) ? L.near[e] : make_int2(-1, 0);
    }
    // sources in batch b (slots 0 .. count - 1 may be taken)
    __device__ __forceinline__ int count(int b, int leaf) const {
        if (b < nbf) return min(32, f1 - f0 - 32 * b);
        return min(lb, n1 - n0 - lb * (b - nbf)) * leaf;
    }
};

// the record of this lane's source in batch b: far node (barycenter, area,
// low part) or near face (the same per face)
__device__ __forceinline__ BhSrc bh_record(const BhBatches& B, int b, int2 en, int leaf, int nf,
                                           const float4* __restrict__ node4, const float4* __restrict__ nodelo,
                                           const float4* __restrict__ sa, const float4* __restrict__ sl) {
    BhSrc s = bh_parked();
    if (en.x >= 0) {
        if (b < B.nbf) {
            s.c = node4[4 * en.x];
            s.l = nodelo[en.x];
            s.mask = (unsigned)en.y;
            s.idx = en.x;
        } else if (B.fi < min(leaf, nf - en.x)) {
            const int j = en.x + B.fi;
            s.c = sa[j];
            s.l = sl[j];
            s.mask = (unsigned)en.y;
            s.idx = j;
        }
    }
    return s;
}

// writes the warp's records into the pair layout (two shuffles per value pair)
__device__ __forceinline__ void bh_stage(float4* H, float4* D, const BhSrc& s, int lane) {
    const bool odd = lane & 1;
    const float mk = __uint_as_float(s.mask);
    const float s0 = odd ? s.c.x : s.c.z, s1 = odd ? s.c.y : s.c.w;
    const float s2 = odd ? s.l.x : s.l.z, s3 = odd ? s.l.y : mk;
    const float r0 = __shfl_xor_sync(0xffffffffu, s0, 1), r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
    const float r2 = __shfl_xor_sync(0xffffffffu, s2, 1), r3 = __shfl_xor_sync(0xffffffffu, s3, 1);
    H[lane] = odd ? make_float4(r0, s.c.z, r1, s.c.w) : make_float4(s.c.x, r0, s.c.y, r1);
    D[lane] = odd ? make_float4(r2, s.l.z, r3, mk) : make_float4(s.l.x, r2, s.l.y, r3);
}

// p = 6 term of one target against a source pair (packed lanes), with
// compensated differences d = (t - s) + (tl - sl), K = ((N.d)^2/|d|^4)^3 and
// |d|^2 + eps in the FMA chain (eps = 1e-18: the self pair gives d = 0 and
// K = 0 exactly). Lanes outside an entry's mask get K = 0 by a bit mask (bit
// `lane` of the mask moved to the sign and spread), so a large K of a source
// this lane does not take never reaches the sum. acc += K a.
__device__ __forceinline__ unsigned long long bh_energy2_p6(
    unsigned long long tx, unsigned long long ty, unsigned long long tz, unsigned long long ux,
    unsigned long long uy, unsigned long long uz, unsigned long long nx, unsigned long long ny,
    unsigned long long nz, unsigned long long sx, unsigned long long sy, unsigned long long sz,
    unsigned long long lx, unsigned long long ly, unsigned long long lz, unsigned long long sa,
    unsigned long long msk, unsigned sh, unsigned long long acc, unsigned long long eps) {
    unsigned long long out;
    asm("{\n\t.reg .b64 dx, dy, dz, ex, ey, ez, r2, u, ir2, q, mm;\n\t.reg .f32 lo, hi;\n\t.reg .b32 m0, m1;\n\t"
        "sub.rn.f32x2 dx, %1, %10;\n\t"
        "sub.rn.f32x2 dy, %2, %11;\n\t"
        "sub.rn.f32x2 dz, %3, %12;\n\t"
        "sub.rn.f32x2 ex, %4, %13;\n\t"
        "sub.rn.f32x2 ey, %5, %14;\n\t"
        "sub.rn.f32x2 ez, %6, %15;\n\t"
        "add.rn.f32x2 dx, dx, ex;\n\t"
        "add.rn.f32x2 dy, dy, ey;\n\t"
        "add.rn.f32x2 dz, dz, ez;\n\t"
        "fma.rn.f32x2 r2, dz, dz, %20;\n\t"
        "fma.rn.f32x2 r2, dy, dy, r2;\n\t"
        "fma.rn.f32x2 r2, dx, dx, r2;\n\t"
        "mul.rn.f32x2 u, %7, dx;\n\t"
        "fma.rn.f32x2 u, %8, dy, u;\n\t"
        "fma.rn.f32x2 u, %9, dz, u;\n\t"
        "mov.b64 {lo, hi}, r2;\n\t"
        "rcp.approx.ftz.f32 lo, lo;\n\t"
        "rcp.approx.ftz.f32 hi, hi;\n\t"
        "mov.b64 ir2, {lo, hi};\n\t"
        "mul.rn.f32x2 u, u, ir2;\n\t"
        "mul.rn.f32x2 q, u, u;\n\t"
        "mul.rn.f32x2 u, q, q;\n\t"
        "mul.rn.f32x2 q, u, q;\n\t"
        "mov.b64 {m0, m1}, %17;\n\t"
        "shl.b32 m0, m0, %18;\n\t"
        "shl.b32 m1, m1, %18;\n\t"
        "shr.s32 m0, m0, 31;\n\t"
        "shr.s32 m1, m1, 31;\n\t"
        "mov.b64 mm, {m0, m1};\n\t"
        "and.b64 q, q, mm;\n\t"
        "fma.rn.f32x2 %0, q, %16, %19;\n\t}"
        : "=l"(out)
        : "l"(tx), "l"(ty), "l"(tz), "l"(ux), "l"(uy), "l"(uz), "l"(nx), "l"(ny), "l"(nz), "l"(sx), "l"(sy),
          "l"(sz), "l"(lx), "l"(ly), "l"(lz), "l"(sa), "l"(msk), "r"(sh), "l"(acc), "l"(eps));
    return out;
}

// Energy rows from the interaction lists for p = 6, staged batches of
// source pairs (see above); FP32 terms per batch, Kahan across batches.
__global__ void __launch_bounds__(128)
k_bh_energy_list2(const float4* __restrict__ node4, const float4* __restrict__ nodelo, const float4* __restrict__ sa,
                  const float4* __restrict__ sb, const float4* __restrict__ sl, int nf, BhLists L,
                  const d4* __restrict__ f64a, const int* __restrict__ perm, double* __restrict__ rows,
                  unsigned long long* __restrict__ count) {
    __shared__ float4 sH[4][32], sD[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = blockIdx.x * 4 + w;
    if (g >= L.ngroups) return;
    const int i = g * BHL_GROUP + lane;
    const bool has = i < nf;
    const int ii = has ? i : 0;
    const float4 A = sa[ii], N = sb[ii], Al = sl[ii];
    const unsigned long long TX = bp2(A.x, A.x), TY = bp2(A.y, A.y), TZ = bp2(A.z, A.z);
    const unsigned long long UX = bp2(Al.x, Al.x), UY = bp2(Al.y, Al.y), UZ = bp2(Al.z, Al.z);
    const unsigned long long NX = bp2(N.x, N.x), NY = bp2(N.y, N.y), NZ = bp2(N.z, N.z);
    const unsigned long long EPS = bp2(1e-18f, 1e-18f);
    const unsigned sh = 31u - (unsigned)lane;
    float4* H = sH[w];
    float4* D = sD[w];
    const ulonglong2* H2 = reinterpret_cast<const ulonglong2*>(H);
    const ulonglong2* D2 = reinterpret_cast<const ulonglong2*>(D);
    const BhBatches Bt(L, g, lane);
    KahanF sum;
    int2 en = Bt.entry(L, 0, lane);
    BhSrc rec = bh_record(Bt, 0, en, L.leaf, nf, node4, nodelo, sa, sl);
    bh_stage(H, D, rec, lane);
    en = Bt.entry(L, 1, lane);
    for (int b = 0; b < Bt.nb; ++b) {
        const bool more = b + 1 < Bt.nb;
        if (more) rec = bh_record(Bt, b + 1, en, L.leaf, nf, node4, nodelo, sa, sl);
        const int2 en2 = Bt.entry(L, b + 2, lane);
        __syncwarp();
        const int np = (Bt.count(b, L.leaf) + 1) >> 1;
        unsigned long long acc = 0ull;
#pragma unroll 8
        for (int q = 0; q < np; ++q) {
            const ulonglong2 h0 = H2[2 * q], h1 = H2[2 * q + 1], d0 = D2[2 * q], d1 = D2[2 * q + 1];
            acc = bh_energy2_p6(TX, TY, TZ, UX, UY, UZ, NX, NY, NZ, h0.x, h0.y, h1.x, d0.x, d0.y, d1.x, h1.y, d1.y,
                                sh, acc, EPS);
        }
        const float2 a = bu2(acc);
        sum.add(a.x + a.y);
        __syncwarp();
        if (more) bh_stage(H, D, rec, lane);
        en = en2;
    }
    if (has) rows[perm[i]] = f64a[perm[i]].w * sum.value();
    if (count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(count, L.interactions);
}

int energy_rows_bh(tp_mesh* m, const tp_params* p, const int32_t* tl, int nt, double* rows, cudaStream_t st) {
    TP_TRY(bvh_build(m, p, st));
    const int nf = m->nf;
    if (!tl) {
        // every face a target: the interaction lists of the tree
        BhLists L;
        bool ok = false;
        TP_TRY(bh_lists(m, p, st, &L, &ok));
        if (ok) {
            TP_TRY(bh_counter(m, st));
            const NodeArrays na = node_arrays(m);
            ProfScope ps(m, PK_BH_ENERGY, 0.0, st);
            unsigned long long* cnt = m->bhcount.as<unsigned long long>();
            const float4* n4 = reinterpret_cast<const float4*>(na.node);
            const int blocks = (L.ngroups + 3) / 4;
            if (p->p == 6.0)
                k_bh_energy_list2<<<blocks, 128, 0, st>>>(n4, na.nodelo, m->bvh_f32a.as<float4>(),
                                                          m->bvh_f32b.as<float4>(), m->bvh_f32c.as<float4>(), nf, L,
                                                          m->f64a.as<d4>(), m->bvh_perm.as<int>(), rows, cnt);
            else
                k_bh_energy_list<false><<<blocks, 128, 0, st>>>(n4, na.nodelo, m->bvh_f32a.as<float4>(),
                                                                m->bvh_f32b.as<float4>(), m->bvh_f32c.as<float4>(),
                                                                nf, L, (float)(0.5 * p->p), m->f64a.as<d4>(),
                                                                m->bvh_perm.as<int>(), rows, cnt);
            TP_LAUNCH_CHECK();
            return TP_OK;
        }
    }
    int* perm = m->bvh_perm.as<int>();
    FaceBox* fbox = (FaceBox*)(perm + nf);
    float theta2 = (float)(p->theta * p->theta);
    float halfp = (float)(0.5 * p->p);
    const int* map = nullptr;
    double* out = rows;
    TP_TRY(ensure(m->tmpv[6], sizeof(double) * 64 + sizeof(int) * 2 * (size_t)nf + sizeof(double) * nf));
    char* base = m->tmpv[6].as<char>() + sizeof(double) * 64;
    int* inv = (int*)base;
    int* mapped = inv + nf;
    double* rs = (double*)(mapped + nf);
    if (tl) {
        k_inv_perm<<<(nf + 255) / 256, 256, 0, st>>>(perm, nf, inv);
        k_map_targets<<<(nt + 255) / 256, 256, 0, st>>>(tl, nt, inv, mapped);
        TP_LAUNCH_CHECK();
        map = mapped;
    } else {
        out = rs;  // sorted order, unsorted afterwards
    }
    TP_TRY(bh_counter(m, st));
    const NodeArrays na = node_arrays(m);
    const BvhNode* node = na.node;
    const float4* nodelo = na.nodelo;
    const float4* sa = m->bvh_f32a.as<float4>();
    const float4* sb = m->bvh_f32b.as<float4>();
    const float4* sl = m->bvh_f32c.as<float4>();
    {
        ProfScope ps(m, PK_BH_ENERGY, 0.0, st);
        unsigned long long* cnt = m->bhcount.as<unsigned long long>();
        if (p->p == 6.0)
            k_bh_energy<true><<<(nt + 127) / 128, 128, 0, st>>>(node, nodelo, m->bvh_nodes, sa, sb, sl,
                                                               fbox, perm, map, nt, theta2, halfp,
                                                               m->f64a.as<d4>(), out, cnt);
        else
            k_bh_energy<false><<<(nt + 127) / 128, 128, 0, st>>>(node, nodelo, m->bvh_nodes, sa, sb, sl,
                                                                fbox, perm, map, nt, theta2, halfp,
                                                                m->f64a.as<d4>(), out, cnt);
        TP_LAUNCH_CHECK();
    }
    if (!tl) {
        k_unsort_rows<<<(nf + 255) / 256, 256, 0, st>>>(rs, perm, nf, rows);
        TP_LAUNCH_CHECK();
    }
    return TP_OK;
}

// ---------------------------------------------------------------------------
// differential
// ---------------------------------------------------------------------------

// warp sum of a float over all 32 lanes (inactive lanes pass 0)
__device__ __forceinline__ float warp_sum(float x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Differential, same warp-cooperative traversal as the energy.
// target-side accumulators: 0 sum a c | 1-3 sum a c d | 4-6 sum a K d/|d|^2 | 7 sum a K
// source side (FULL): G = -a_S w dK/dd and Q = a_S K of the lanes that interact
// with the same node or leaf face are summed across the warp first, then added
// with one FP64 atomic per warp: node accumulators nacc[id*4 + 0..2] = G,
// [3] = Q; near faces facc[j*4 + ...]
template <bool P6, bool FULL>
__global__ void __launch_bounds__(128)
k_bh_diff(const BvhNode* __restrict__ node, const float4* __restrict__ nodelo, int nnodes,
          const float4* __restrict__ sa, const float4* __restrict__ sb, const float4* __restrict__ sl,
          const FaceBox* __restrict__ fbox, int nf, float theta2, float hm1,
          float p, double* __restrict__ tacc /* [nf][8] sorted */, double* __restrict__ nacc,
          double* __restrict__ facc, unsigned long long* __restrict__ count) {
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = i0 < nf;
    const int i = has ? i0 : 0;
    const float4 A = sa[i], B = sb[i], Al = sl[i];
    const FaceBox fb = fbox[i];
    const float aS = A.w;
    const int lane = threadIdx.x & 31;
    KahanF acc[8];
    float pt[8];
    for (int k = 0; k < 8; ++k) pt[k] = 0.f;
    int run = 0, nint = 0;
    auto flush = [&]() {
        for (int k = 0; k < 8; ++k) {
            acc[k].add(pt[k]);
            pt[k] = 0.f;
        }
        run = 0;
    };
    // one interaction with a source of barycenter src (+ low part lo) and
    // weight w; returns the source-side derivative G, Q
    auto interact = [&](float4 src, float4 lo, float w, float* G, float& Q) {
        float dx = (A.x - src.x) + (Al.x - lo.x), dy = (A.y - src.y) + (Al.y - lo.y),
              dz = (A.z - src.z) + (Al.z - lo.z);
        float r2 = dx * dx + dy * dy + dz * dz;
        float u = B.x * dx + B.y * dy + B.z * dz;
        float ir2 = frcp(fmaxf(r2, 1e-18f));
        float ir4 = ir2 * ir2;
        float q = u * u * ir4;
        float mq = P6 ? q * q : fpow(q, hm1);
        float K = mq * q;
        float c = mq * u * ir4;  // |u|^{p-2} u / |d|^{2p}
        float wc = w * c, wK = w * K, wKd = wK * ir2;
        pt[0] += wc;
        pt[1] = fmaf(wc, dx, pt[1]);
        pt[2] = fmaf(wc, dy, pt[2]);
        pt[3] = fmaf(wc, dz, pt[3]);
        pt[4] = fmaf(wKd, dx, pt[4]);
        pt[5] = fmaf(wKd, dy, pt[5]);
        pt[6] = fmaf(wKd, dz, pt[6]);
        pt[7] += wK;
        // dK/dd = p c N - 2p K d/|d|^2 ; source side gets -a_S w dK/dd
        float s1 = -aS * p * wc, s2 = 2.f * aS * p * wKd;
        G[0] = s1 * B.x + s2 * dx;
        G[1] = s1 * B.y + s2 * dy;
        G[2] = s1 * B.z + s2 * dz;
        Q = aS * K;
    };
    int skip = has ? 0 : nnodes;
    int id = 0;
    while (id < nnodes) {
        const BvhNode n = node[id];
        const bool act = id >= skip;
        bool adm = false;
        if (act) {
            float d2 = box_dist2(fb.lox, fb.loy, fb.loz, fb.hix, fb.hiy, fb.hiz, n);
            float mr2 = fmaxf(fb.r2, n.r2);
            adm = mr2 < __fmul_rn(theta2, d2);
        }
        const bool near = act && !adm && n.leaf;
        const bool desc = act && !adm && !n.leaf;
        if (__any_sync(0xffffffffu, adm)) {
            float G[3] = {0.f, 0.f, 0.f}, Q = 0.f;
            if (adm) {
                interact(make_float4(n.cx, n.cy, n.cz, 0.f), nodelo[id], n.a, G, Q);
                ++nint;
                if (++run == 32) flush();
            }
            if (FULL) {
                G[0] = warp_sum(G[0]);
                G[1] = warp_sum(G[1]);
                G[2] = warp_sum(G[2]);
                Q = warp_sum(Q);
                if (lane == 0) {
                    atomicAdd(nacc + 4 * id + 0, (double)G[0]);
                    atomicAdd(nacc + 4 * id + 1, (double)G[1]);
                    atomicAdd(nacc + 4 * id + 2, (double)G[2]);
                    atomicAdd(nacc + 4 * id + 3, (double)Q);
                }
            }
        }
        if (__any_sync(0xffffffffu, near)) {
            for (int j = n.first; j < n.first + n.count; ++j) {
                float G[3] = {0.f, 0.f, 0.f}, Q = 0.f;
                if (near && j != i) {
                    interact(sa[j], sl[j], sa[j].w, G, Q);
                    ++nint;
                }
                if (FULL) {
                    G[0] = warp_sum(G[0]);
                    G[1] = warp_sum(G[1]);
                    G[2] = warp_sum(G[2]);
                    Q = warp_sum(Q);
                    if (lane == 0) {
                        atomicAdd(facc + 4 * j + 0, (double)G[0]);
                        atomicAdd(facc + 4 * j + 1, (double)G[1]);
                        atomicAdd(facc + 4 * j + 2, (double)G[2]);
                        atomicAdd(facc + 4 * j + 3, (double)Q);
                    }
                }
            }
            if (near) flush();
        }
        if (adm || near) skip = n.skip;
        id = __any_sync(0xffffffffu, desc) ? id + 1 : n.skip;
    }
    flush();
    if (has) {
        for (int k = 0; k < 8; ++k) tacc[(size_t)i * 8 + k] = acc[k].value();
    }
    if (nint) atomicAdd(count, (unsigned long long)nint);
}

// FP32 -> FP64 by rebiasing the exponent with integer operations (exact for
// normal numbers, zero for FP32 subnormals): a float-to-double conversion
// instruction runs on the FP64 pipe, which this GPU has little of
__device__ __forceinline__ double f2d_int(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
    if (e == 0) return __longlong_as_double((long long)sgn);
    const unsigned long long de = e == 0xffu ? 0x7ffull : (unsigned long long)(e + (1023 - 127));
    return __longlong_as_double((long long)(sgn | (de << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// sums of four values over the warp: lanes 0, 8, 16 and 24 end with the sums
// of v0, v1, v2 and v3 (the lanes of an octet share their value); 6 shuffles
// instead of 4 x 5
__device__ __forceinline__ float warp_sum4(float v0, float v1, float v2, float v3) {
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8;
    float k0 = b4 ? v2 : v0, k1 = b4 ? v3 : v1;
    const float s0 = b4 ? v0 : v2, s1 = b4 ? v1 : v3;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    float keep = b3 ? k1 : k0;
    const float send = b3 ? k0 : k1;
    keep += __shfl_xor_sync(0xffffffffu, send, 8);
    keep += __shfl_xor_sync(0xffffffffu, keep, 4);
    keep += __shfl_xor_sync(0xffffffffu, keep, 2);
    keep += __shfl_xor_sync(0xffffffffu, keep, 1);
    return keep;
}

// Differential from the interaction lists: the target side as in k_bh_diff;
// the source side (FULL) of an entry is summed over the lanes in its mask and
// added with one FP64 atomic per entry (node accumulators for far entries,
// face accumulators for the faces of near leaves).
template <bool P6, bool FULL>
__global__ void __launch_bounds__(128)
k_bh_diff_list(const float4* __restrict__ node4, const float4* __restrict__ nodelo, const float4* __restrict__ sa,
               const float4* __restrict__ sb, const float4* __restrict__ sl, int nf, BhLists L, float hm1, float p,
               double* __restrict__ tacc, double* __restrict__ nacc, double* __restrict__ facc,
               unsigned long long* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= L.ngroups) return;
    const int i0 = g * BHL_GROUP + lane;
    const bool has = i0 < nf;
    const int i = has ? i0 : 0;
    const float4 A = sa[i], B = sb[i], Al = sl[i];
    const float aS = A.w;
    const unsigned me = 1u << lane;
    KahanF acc[8];
    float pt[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) pt[k] = 0.f;
    auto flush = [&]() {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            acc[k].add(pt[k]);
            pt[k] = 0.f;
        }
    };
    // one interaction (source barycenter src + low part lo, weight w), masked
    // by on; returns the source-side G, Q of this lane
    auto interact = [&](float4 src, float4 lo, float w, bool on, float* G, float& Q) {
        const float dx = (A.x - src.x) + (Al.x - lo.x), dy = (A.y - src.y) + (Al.y - lo.y),
                    dz = (A.z - src.z) + (Al.z - lo.z);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-18f)));
        const float u = B.x * dx + B.y * dy + B.z * dz;
        const float ir2 = frcp(r2);
        const float ir4 = ir2 * ir2;
        const float q = u * u * ir4;
        const float mq = P6 ? q * q : fpow(q, hm1);
        const float K = mq * q;
        const float c = mq * u * ir4;
        const float ww = on ? w : 0.f;
        const float wc = ww * c, wK = ww * K, wKd = wK * ir2;
        pt[0] += wc;
        pt[1] = fmaf(wc, dx, pt[1]);
        pt[2] = fmaf(wc, dy, pt[2]);
        pt[3] = fmaf(wc, dz, pt[3]);
        pt[4] = fmaf(wKd, dx, pt[4]);
        pt[5] = fmaf(wKd, dy, pt[5]);
        pt[6] = fmaf(wKd, dz, pt[6]);
        pt[7] += wK;
        const float s1 = -aS * p * wc, s2 = 2.f * aS * p * wKd;
        G[0] = s1 * B.x + s2 * dx;
        G[1] = s1 * B.y + s2 * dy;
        G[2] = s1 * B.z + s2 * dz;
        Q = on ? aS * K : 0.f;   // a_S K (the source's area derivative carries no a_T)
    };
    const int f0 = (int)L.far_off[g], f1 = (int)L.far_off[g + 1];
    int run = 0;
    for (int e = f0; e < f1; ++e) {
        const int2 en = L.far[e];
        const float4 c = node4[4 * en.x];
        float G[3], Q;
        interact(c, nodelo[en.x], c.w, (unsigned)en.y & me, G, Q);
        if (FULL) {
            const float r = warp_sum4(G[0], G[1], G[2], Q);
            if ((lane & 7) == 0) atomicAdd(nacc + 4 * en.x + (lane >> 3), f2d_int(r));
        }
        if (++run == 32) {
            flush();
            run = 0;
        }
    }
    flush();
    const int n0 = (int)L.near_off[g], n1 = (int)L.near_off[g + 1];
    for (int e = n0; e < n1; ++e) {
        const int2 en = L.near[e];
        const int2 fc = make_int2(en.x, min(L.leaf, nf - en.x));   // the leaf's first face, count
        const bool on = (unsigned)en.y & me;
        for (int j = fc.x; j < fc.x + fc.y; ++j) {
            const float4 s = sa[j];
            float G[3], Q;
            interact(s, sl[j], s.w, on && j != i0, G, Q);
            if (FULL) {
                const float r = warp_sum4(G[0], G[1], G[2], Q);
                if ((lane & 7) == 0) atomicAdd(facc + 4 * j + (lane >> 3), f2d_int(r));
            }
        }
        flush();
    }
    if (has)
        for (int k = 0; k < 8; ++k) tacc[(size_t)i0 * 8 + k] = acc[k].value();
    if (count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(count, L.interactions);
}


// bit `lane` of each half of a packed mask pair, spread over the half
// (all ones where set, zero where not): sh = 31 - lane
__device__ __forceinline__ unsigned long long lane_bits2(float2 m, unsigned sh) {
    unsigned long long r;
    asm("{\n\t.reg .b32 m0, m1;\n\t"
        "mov.b32 m0, %1;\n\tmov.b32 m1, %2;\n\t"
        "shl.b32 m0, m0, %3;\n\tshl.b32 m1, m1, %3;\n\t"
        "shr.s32 m0, m0, 31;\n\tshr.s32 m1, m1, 31;\n\t"
        "mov.b64 %0, {m0, m1};\n\t}"
        : "=l"(r) : "f"(m.x), "f"(m.y), "r"(sh));
    return r;
}
__device__ __forceinline__ float2 q2and(float2 a, unsigned long long m) {
    float2 d;
    asm("{\n\t.reg .b64 ra;\n\tmov.b64 ra, {%2, %3};\n\tand.b64 ra, ra, %4;\n\tmov.b64 {%0, %1}, ra;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "l"(m));
    return d;
}

// k_bh_diff_list for p = 6 over staged batches of source pairs (as the
// energy): the target side as in k_bh_diff_list, two sources per packed
// instruction; lanes outside an entry's mask get c = K = 0 by a bit mask.
// FULL: every lane stores the source sides (G, Q) of both sources of a pair
// in its own row of a per-warp table; after 8 pairs (16 sources) lane l sums
// rows 2l and 2l + 1 of the table's columns over the 32 targets and adds them
// with two FP64 atomics (node accumulators in far batches, face accumulators
// in near batches): a transpose through shared memory instead of a shuffle
// reduction per pair and one atomic per source and component.
constexpr int BHD_CHUNK = 8;                     // source pairs per table flush
constexpr int BHD_RS = 8 * BHD_CHUNK + 4;        // row stride in floats (16-byte rows, no bank conflicts)
template <bool FULL>
__global__ void __launch_bounds__(128, 5)
k_bh_diff_list2(const float4* __restrict__ node4, const float4* __restrict__ nodelo, const float4* __restrict__ sa,
                const float4* __restrict__ sb, const float4* __restrict__ sl, int nf, BhLists L, float p,
                double* __restrict__ tacc, double* __restrict__ nacc, double* __restrict__ facc,
                unsigned long long* __restrict__ count) {
    __shared__ float4 sH[4][32], sD[4][32];
    __shared__ int sI[4][32];
    __shared__ __align__(16) float sR[FULL ? 4 * 32 * BHD_RS : 4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = blockIdx.x * 4 + w;
    if (g >= L.ngroups) return;
    const int i0 = g * BHL_GROUP + lane;
    const bool has = i0 < nf;
    const int i = has ? i0 : 0;
    const float4 A = sa[i], B = sb[i], Al = sl[i];
    const float aS = A.w;
    const float2 TX = q2(A.x), TY = q2(A.y), TZ = q2(A.z), UX = q2(Al.x), UY = q2(Al.y), UZ = q2(Al.z);
    const float2 NX = q2(B.x), NY = q2(B.y), NZ = q2(B.z), EPS2 = q2(1e-18f);
    const float2 S1 = q2(-aS * p), S2 = q2(2.f * aS * p), AS = q2(aS);
    float* R = sR + (FULL ? w * 32 * BHD_RS : 0);
    const unsigned sh = 31u - (unsigned)lane;
    float4* H = sH[w];
    float4* D = sD[w];
    int* I = sI[w];
    KahanF acc[8];
    float2 pt[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) pt[k] = make_float2(0.f, 0.f);
    const BhBatches Bt(L, g, lane);
    int2 en = Bt.entry(L, 0, lane);
    BhSrc rec = bh_record(Bt, 0, en, L.leaf, nf, node4, nodelo, sa, sl);
    bh_stage(H, D, rec, lane);
    I[lane] = rec.idx;
    en = Bt.entry(L, 1, lane);
    for (int b = 0; b < Bt.nb; ++b) {
        const bool more = b + 1 < Bt.nb;
        if (more) rec = bh_record(Bt, b + 1, en, L.leaf, nf, node4, nodelo, sa, sl);
        const int2 en2 = Bt.entry(L, b + 2, lane);
        double* sacc = b < Bt.nbf ? nacc : facc;
        __syncwarp();
        const int np = (Bt.count(b, L.leaf) + 1) >> 1;
        for (int q0 = 0; q0 < np; q0 += BHD_CHUNK) {
            const int nq = min(BHD_CHUNK, np - q0);
            for (int t = 0; t < nq; ++t) {
                const int q = q0 + t;
                const float4 h0 = H[2 * q], h1 = H[2 * q + 1], d0 = D[2 * q], d1 = D[2 * q + 1];
                const unsigned long long mm = lane_bits2(make_float2(d1.z, d1.w), sh);
                const float2 dx = q2add(q2sub(TX, make_float2(h0.x, h0.y)), q2sub(UX, make_float2(d0.x, d0.y)));
                const float2 dy = q2add(q2sub(TY, make_float2(h0.z, h0.w)), q2sub(UY, make_float2(d0.z, d0.w)));
                const float2 dz = q2add(q2sub(TZ, make_float2(h1.x, h1.y)), q2sub(UZ, make_float2(d1.x, d1.y)));
                const float2 W = make_float2(h1.z, h1.w);
                const float2 r2 = q2fma(dx, dx, q2fma(dy, dy, q2fma(dz, dz, EPS2)));
                const float2 u = q2fma(NX, dx, q2fma(NY, dy, q2mul(NZ, dz)));
                const float2 ir2 = make_float2(frcp(r2.x), frcp(r2.y));
                const float2 ir4 = q2mul(ir2, ir2);
                const float2 qq = q2mul(q2mul(u, u), ir4);
                const float2 mq = q2mul(qq, qq);
                const float2 K = q2and(q2mul(mq, qq), mm);
                const float2 c = q2and(q2mul(q2mul(mq, u), ir4), mm);
                const float2 wc = q2mul(W, c), wK = q2mul(W, K), wKd = q2mul(wK, ir2);
                pt[0] = q2add(pt[0], wc);
                pt[1] = q2fma(wc, dx, pt[1]);
                pt[2] = q2fma(wc, dy, pt[2]);
                pt[3] = q2fma(wc, dz, pt[3]);
                pt[4] = q2fma(wKd, dx, pt[4]);
                pt[5] = q2fma(wKd, dy, pt[5]);
                pt[6] = q2fma(wKd, dz, pt[6]);
                pt[7] = q2add(pt[7], wK);
                if (FULL) {
                    const float2 s1 = q2mul(S1, wc), s2 = q2mul(S2, wKd);
                    const float2 G0 = q2fma(s2, dx, q2mul(s1, NX)), G1 = q2fma(s2, dy, q2mul(s1, NY)),
                                 G2 = q2fma(s2, dz, q2mul(s1, NZ));
                    const float2 Q = q2mul(AS, K);
                    // row `lane`, columns 8 t .. 8 t + 7: (G, Q) of sources 2 q and 2 q + 1
                    float4* row = reinterpret_cast<float4*>(R + lane * BHD_RS + 8 * t);
                    row[0] = make_float4(G0.x, G1.x, G2.x, Q.x);
                    row[1] = make_float4(G0.y, G1.y, G2.y, Q.y);
                }
            }
            if (FULL) {
                // column pair (2 lane, 2 lane + 1) = source 2 q0 + (lane >> 1),
                // components 2 (lane & 1) and 2 (lane & 1) + 1, summed over the rows
                __syncwarp();
                const float2* col = reinterpret_cast<const float2*>(R) + lane;
                float2 c0 = col[0], c1 = col[BHD_RS / 2], c2 = col[BHD_RS], c3 = col[3 * BHD_RS / 2];
#pragma unroll
                for (int k = 4; k < 32; k += 4) {
                    const float2* ck = col + k * (BHD_RS / 2);
                    c0 = q2add(c0, ck[0]);
                    c1 = q2add(c1, ck[BHD_RS / 2]);
                    c2 = q2add(c2, ck[BHD_RS]);
                    c3 = q2add(c3, ck[3 * BHD_RS / 2]);
                }
                const float2 sum = q2add(q2add(c0, c1), q2add(c2, c3));
                const int src = lane >> 1;
                const int idx = src < 2 * nq ? I[2 * q0 + src] : -1;
                if (idx >= 0) {
                    double* dst = sacc + 4 * idx + 2 * (lane & 1);
                    atomicAdd(dst, f2d_int(sum.x));
                    atomicAdd(dst + 1, f2d_int(sum.y));
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            acc[k].add(pt[k].x + pt[k].y);
            pt[k] = make_float2(0.f, 0.f);
        }
        __syncwarp();
        if (more) {
            bh_stage(H, D, rec, lane);
            I[lane] = rec.idx;
        }
        en = en2;
    }
    if (has)
        for (int k = 0; k < 8; ++k) tacc[(size_t)i0 * 8 + k] = acc[k].value();
    if (count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(count, L.interactions);
}

// per node: g1 = G/a_I, q = Q - G.X_I/a_I (FP64 node data)
__global__ void k_node_push_terms(double* __restrict__ nacc, const d4* __restrict__ node64, int nnodes) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nnodes) return;
    d4 X = node64[id];
    double G[3] = {nacc[4 * id], nacc[4 * id + 1], nacc[4 * id + 2]};
    double Q = nacc[4 * id + 3];
    nacc[4 * id + 0] = G[0] / X.w;
    nacc[4 * id + 1] = G[1] / X.w;
    nacc[4 * id + 2] = G[2] / X.w;
    nacc[4 * id + 3] = Q - (G[0] * X.x + G[1] * X.y + G[2] * X.z) / X.w;
}

// per sorted face i: walk root -> leaf of i summing the node terms, then
// assemble the FP64 face adjoints (face order) from target and source sides
__global__ void k_bh_diff_combine(const NodeShape* __restrict__ shape, const int* __restrict__ right, int nnodes,
                                  int leaf, const int* __restrict__ perm, int nf, const double* __restrict__ tacc,
                                  const double* __restrict__ nacc, const double* __restrict__ facc,
                                  const d4* __restrict__ f64a, const d4* __restrict__ f64b, double p, int full,
                                  double* __restrict__ adj, double* __restrict__ erow) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int S = perm[i];
    d4 X = f64a[S], N = f64b[S];
    double a = X.w;
    const double* t = tacc + (size_t)i * 8;
    double gX[3], gN[3], ga;
    double NS[3] = {N.x, N.y, N.z};
    for (int c = 0; c < 3; ++c) {
        gX[c] = a * (p * t[0] * NS[c] - 2.0 * p * t[4 + c]);
        gN[c] = a * p * t[1 + c];
    }
    ga = t[7];
    if (erow) erow[S] = a * t[7];
    if (full) {
        double g1[3] = {0, 0, 0}, q = 0.0;
        int lf = i / leaf;
        int id = 0;
        for (;;) {
            for (int c = 0; c < 3; ++c) g1[c] += nacc[4 * id + c];
            q += nacc[4 * id + 3];
            NodeShape s = shape[id];
            if (s.leaf) break;
            int L = id + 1;
            NodeShape sl = shape[L];
            int lfirst = sl.first / leaf, lcount = (sl.skip - L + 1) / 2;
            id = (lf >= lfirst && lf < lfirst + lcount) ? L : right[id];
        }
        double Xv[3] = {X.x, X.y, X.z};
        for (int c = 0; c < 3; ++c) gX[c] += a * g1[c] + facc[4 * i + c];
        ga += q + g1[0] * Xv[0] + g1[1] * Xv[1] + g1[2] * Xv[2] + facc[4 * i + 3];
    }
    for (int c = 0; c < 3; ++c) {
        adj[7 * S + c] = gX[c];
        adj[7 * S + 3 + c] = gN[c];
    }
    adj[7 * S + 6] = ga;
}

int diff_adjoints_bh(tp_mesh* m, const tp_params* p, double* adj, double* erow, cudaStream_t st) {
    TP_TRY(bvh_build(m, p, st));
    const int nf = m->nf, nn = m->bvh_nodes;
    int* perm = m->bvh_perm.as<int>();
    FaceBox* fbox = (FaceBox*)(perm + nf);
    const NodeArrays na = node_arrays(m);
    BvhNode* node = na.node;
    d4* node64 = na.node64;
    const float4* nodelo = na.nodelo;
    TP_TRY(ensure(m->part, sizeof(double) * ((size_t)8 * nf + 4 * (size_t)nn + 4 * (size_t)nf)));
    double* tacc = m->part.as<double>();
    double* nacc = tacc + (size_t)8 * nf;
    double* facc = nacc + (size_t)4 * nn;
    TP_CUDA(cudaMemsetAsync(nacc, 0, sizeof(double) * (4 * (size_t)nn + 4 * (size_t)nf), st));
    const bool full = p->bh_diff_mode == TP_BH_DIFF_FULL;
    float theta2 = (float)(p->theta * p->theta);
    float hm1 = (float)(0.5 * p->p - 1.0);
    const float4* sa = m->bvh_f32a.as<float4>();
    const float4* sb = m->bvh_f32b.as<float4>();
    const float4* sl = m->bvh_f32c.as<float4>();
    dim3 g((nf + 127) / 128);
    TP_TRY(bh_counter(m, st));
    BhLists L;
    bool lists = false;
    TP_TRY(bh_lists(m, p, st, &L, &lists));
    if (lists) {
        ProfScope ps(m, PK_BH_DIFF, 0.0, st);
        unsigned long long* cnt = m->bhcount.as<unsigned long long>() + 1;
        const float pf = (float)p->p;
        const float4* n4 = reinterpret_cast<const float4*>(node);
        const int blocks = (L.ngroups + 3) / 4;
        static bool carveout_set[64] = {false};
        int dev = 0;
        cudaGetDevice(&dev);
        if (full && dev >= 0 && dev < 64 && !carveout_set[dev]) {
            // five blocks of 39 KB (the source-side tables) per SM
            TP_CUDA(cudaFuncSetAttribute((const void*)k_bh_diff_list2<true>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            carveout_set[dev] = true;
        }
        if (p->p == 6.0) {
            if (full) k_bh_diff_list2<true><<<blocks, 128, 0, st>>>(n4, nodelo, sa, sb, sl, nf, L, pf, tacc, nacc, facc, cnt);
            else k_bh_diff_list2<false><<<blocks, 128, 0, st>>>(n4, nodelo, sa, sb, sl, nf, L, pf, tacc, nacc, facc, cnt);
        } else {
            if (full) k_bh_diff_list<false, true><<<blocks, 128, 0, st>>>(n4, nodelo, sa, sb, sl, nf, L, hm1, pf, tacc, nacc, facc, cnt);
            else k_bh_diff_list<false, false><<<blocks, 128, 0, st>>>(n4, nodelo, sa, sb, sl, nf, L, hm1, pf, tacc, nacc, facc, cnt);
        }
        TP_LAUNCH_CHECK();
    } else {
        ProfScope ps(m, PK_BH_DIFF, 0.0, st);
        unsigned long long* cnt = m->bhcount.as<unsigned long long>() + 1;
        const float pf = (float)p->p;
        if (p->p == 6.0) {
            if (full) k_bh_diff<true, true><<<g, 128, 0, st>>>(node, nodelo, nn, sa, sb, sl, fbox, nf, theta2, hm1, pf, tacc, nacc, facc, cnt);
            else k_bh_diff<true, false><<<g, 128, 0, st>>>(node, nodelo, nn, sa, sb, sl, fbox, nf, theta2, hm1, pf, tacc, nacc, facc, cnt);
        } else {
            if (full) k_bh_diff<false, true><<<g, 128, 0, st>>>(node, nodelo, nn, sa, sb, sl, fbox, nf, theta2, hm1, pf, tacc, nacc, facc, cnt);
            else k_bh_diff<false, false><<<g, 128, 0, st>>>(node, nodelo, nn, sa, sb, sl, fbox, nf, theta2, hm1, pf, tacc, nacc, facc, cnt);
        }
        TP_LAUNCH_CHECK();
    }
    if (full) {
        k_node_push_terms<<<(nn + 255) / 256, 256, 0, st>>>(nacc, node64, nn);
        TP_LAUNCH_CHECK();
    }
    const NodeShape* shape = m->bvh_tmp.as<NodeShape>();
    const int* right = (const int*)(shape + nn);
    k_bh_diff_combine<<<(nf + 255) / 256, 256, 0, st>>>(shape, right, nn, m->bvh_leaf, perm, nf, tacc, nacc, facc,
                                                        m->f64a.as<d4>(), m->f64b.as<d4>(), p->p, full ? 1 : 0,
                                                        adj, erow);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

}  // namespace tp
