// Internal declarations shared by the translation units of libtpsurf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "tp.h"

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------

namespace tp {

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define TP_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return ::tp::fail(e_ == cudaErrorMemoryAllocation ? TP_ERR_OOM         \
                                                              : TP_ERR_CUDA,       \
                              std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TP_TRY(call)                 \
    do {                             \
        int s_ = (call);             \
        if (s_ != TP_OK) return s_;  \
    } while (0)

// every launch site of the library calls TP_LAUNCH_CHECK once per launch
void count_launches(unsigned long long n);
#define TP_LAUNCH_CHECK()            \
    do {                             \
        ::tp::count_launches(1);     \
        TP_CUDA(cudaGetLastError()); \
    } while (0)

// ---------------------------------------------------------------------------
// device buffers (grow-only)
// ---------------------------------------------------------------------------

struct Buf {
    void* ptr = nullptr;
    size_t bytes = 0;
    tp_ctx* ctx = nullptr;   // the context whose allocator holds ptr (freed through it)
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// grows b to at least `bytes` through the calling thread's current context
// (its allocator, or cudaMalloc); release() frees through b.ctx
int ensure(Buf& b, size_t bytes);
void release(Buf& b);
// the context of the current library call on this thread (set by the entry
// points for the mesh they serve; the per-device default context otherwise)
tp_ctx*& current_ctx();
tp_ctx* default_ctx(int device);

// 32-byte FP64 quadruple used for face tables of the FP64 path
struct alignas(32) d4 {
    double x, y, z, w;
};

// number of SMs of the current device (cached per device)
int sm_count();

// ---------------------------------------------------------------------------
// Barnes-Hut tree (implicit, Morton-ordered; built on the device)
// ---------------------------------------------------------------------------

struct BvhNode {          // 64 bytes, FP32 (pair path)
    float cx, cy, cz, a;  // area-weighted barycenter (relative frame), total area
    float lox, loy, loz, r2;   // AABB of the barycenters' faces (lower), squared radius
    float hix, hiy, hiz, pad;  // AABB (upper)
    int first, count, skip, leaf;  // face range in Morton order, escape index, leaf flag
};

// sorted (Morton order) target face: bounding box of its vertices, squared
// radius from its barycenter, area
struct FaceBox {
    float lox, loy, loz, r2;
    float hix, hiy, hiz, a;
};

// squared distance between a face box and a node box; max(0, ...) per axis,
// fixed operation order (the admissibility test of §4.1 is decided in FP32
// identically by every kernel)
__device__ __forceinline__ float box_dist2(float alx, float aly, float alz, float ahx, float ahy, float ahz,
                                           const BvhNode& n) {
    float gx = fmaxf(fmaxf(__fsub_rn(n.lox, ahx), __fsub_rn(alx, n.hix)), 0.f);
    float gy = fmaxf(fmaxf(__fsub_rn(n.loy, ahy), __fsub_rn(aly, n.hiy)), 0.f);
    float gz = fmaxf(fmaxf(__fsub_rn(n.loz, ahz), __fsub_rn(alz, n.hiz)), 0.f);
    return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
}

// Barnes-Hut interaction lists (per group of 32 consecutive sorted targets):
// far entries (node, mask): node admissible for the targets of the group whose
// lane bit is set in mask, and none of its ancestors admissible for them;
// near entries (leaf, mask): an inadmissible leaf of those targets
constexpr int BHL_GROUP = 32;
struct BhLists {
    int ngroups = 0;
    const long long* far_off = nullptr;    // [ngroups + 1]
    const long long* near_off = nullptr;   // [ngroups + 1]
    const int2* far = nullptr;
    const int2* near = nullptr;    // near entries: (first face of the leaf, lane mask)
    int leaf = 0;                  // leaf size: a near leaf holds min(leaf, nf - first) faces
    unsigned long long interactions = 0;   // (target, node) plus (target, face) terms of one evaluation
};

// read-only view of a built tree for kernels outside bvh.cu
struct BvhView {
    int nnodes = 0, maxdepth = 0;
    const BvhNode* node = nullptr;
    const float4* nodelo = nullptr;      // low parts of the node barycenters
    const float4* sa = nullptr;          // sorted faces: X - c, a
    const float4* sb = nullptr;          // sorted faces: N
    const float4* sl = nullptr;          // sorted faces: low parts of X - c
    const FaceBox* fbox = nullptr;
    const int* perm = nullptr;           // sorted position -> face
    const int* right = nullptr;          // right child of an inner node
    const int* level_order = nullptr;    // nodes grouped by depth
    const int* level_off = nullptr;      // host: offsets of the depths in level_order
};

// packed float2 arithmetic (two IEEE lanes per instruction)
__device__ __forceinline__ float2 q2add(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 q2sub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 q2mul(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 q2fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 q2(float a) { return make_float2(a, a); }

// ---------------------------------------------------------------------------
// per-mesh kernel statistics (CUDA events on the launching stream)
// ---------------------------------------------------------------------------

enum ProfKey { PK_ENERGY = 0, PK_DIFF, PK_APPLY_A, PK_APPLY_B, PK_APPLY_B0, PK_APPLY_L, PK_BH_ENERGY,
               PK_BH_DIFF, PK_BVH_BUILD, PK_CG, PK_CHOL_FACTOR, PK_CHOL_SOLVE, PK_BH_APPLY,
               PK_OBSTACLE, PK_BH_OBSTACLE, PK_COUNT };

struct Profiler {
    bool on = false;
    long long launches[PK_COUNT] = {};
    double ms[PK_COUNT] = {};
    double units[PK_COUNT] = {};
    double cols[PK_COUNT] = {};    // operator columns processed (apply kernels)
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
};

}  // namespace tp

namespace tp {
struct CholState;   // sparse Cholesky factor of the cotan Laplacian (chol.cu)
}

// a device and the allocator of the device memory of its meshes
struct tp_ctx {
    int device = 0;
    bool is_default = false;      // the per-device context of tp_mesh_create (never destroyed)
    bool custom = false;          // al set by tp_ctx_set_allocator
    tp_allocator al{};
    std::atomic<long long> in_use{0}, peak{0};
    std::atomic<int> meshes{0};
};

struct tp_mesh {
    tp_ctx* ctx = nullptr;
    int device = 0;
    int nv = 0, nf = 0;
    // topology (fixed for the life of the mesh)
    tp::Buf faces;      // int32 [nf*3]
    tp::Buf vf_ptr;     // int32 [nv+1]  vertex -> incident (face*3+corner)
    tp::Buf vf_idx;     // int32 [3*nf]
    // connected components (through the face edges): one barycenter each (§7.1.1)
    int ncomp = 1;
    std::vector<int> comp_host;   // component of each vertex
    tp::Buf vcomp;      // int32 [nv]        component of each vertex
    tp::Buf comp_ptr;   // int32 [ncomp+1]   vertices of component c: comp_verts[comp_ptr[c] .. comp_ptr[c+1])
    tp::Buf comp_verts; // int32 [nv]
    // positions
    tp::Buf pos;        // double [nv*3]
    tp::Buf center;     // double [4]    reference frame of the FP32 face table; [3] = near-pair distance^2
    tp::Buf errflag;    // int [4]
    // face tables
    tp::Buf f32a;       // float4 [nf]   X - c, a
    tp::Buf f32b;       // float4 [nf]   N, 0
    tp::Buf f32c;       // float4 [nf]   (X - c) - hi: the low parts of the FP32 barycenters
    tp::Buf tilebox;    // float4 [2*ntiles] bounding box of the FP32 barycenters of each 128-face tile
    tp::Buf f64a;       // d4 [nf]       X - c, a
    tp::Buf f64b;       // d4 [nf]       N, 0
    tp::Buf fgrad;      // double [nf*9] gradients of the three hat functions
    // cotan Laplacian (pattern fixed, values per positions)
    int nnz = 0;
    tp::Buf rowptr, col, cotsrc, diagpos, val, dinv, val32;
    bool lap_valid = false;
    // within-face term of the preconditioner's L^{2-s} (values on the CSR
    // pattern of C, for the weight and order it was built with)
    tp::Buf gval;
    bool gself_valid = false;
    // Willmore term (§7.3.5): weight in the step, workspace, lumped mass valid for the positions
    double willmore_w = 0.0;
    tp::Buf wm;
    bool wm_valid = false;
    double gself_kappa = 0.0, gself_sigma = 0.0;
    tp::CholState* chol = nullptr;   // created on the first factorised solve
    // Barnes-Hut tree (rebuilt per positions on demand)
    int bvh_nodes = 0, bvh_leaf = 0;
    int bvh_shape_leaf = 0, bvh_maxdepth = 0;
    std::vector<int> bvh_level_off;
    bool bvh_valid = false;
    bool bvh_ordered = false;     // perm holds a face order for the current leaf size (refit keeps it)
    tp::Buf bvh_node, bvh_perm, bvh_keys, bvh_tmp, bvh_sortws;
    tp::Buf bvh_f32a, bvh_f32b, bvh_f32c;   // face tables (and low parts) permuted to Morton order
    tp::Buf bh_apply_ws;          // Barnes-Hut applies: sorted X vectors, node sums, node projectors
    // Barnes-Hut interaction lists of the current tree (bhlist.cu): per group
    // of 32 sorted targets, (node, lane mask) entries of the admissible nodes
    // and of the inadmissible leaves
    unsigned long long bvh_version = 0;   // incremented by every tree build or refit
    unsigned long long bhl_version = 0;   // tree version the lists were built for (0: none)
    double bhl_theta = -1.0;
    long long bhl_nfar = 0, bhl_nnear = 0;
    unsigned long long bhl_inter = 0;     // interactions of one evaluation over the lists
    bool bhl_failed = false;              // the lists could not be built for this tree (walk kernels serve)
    tp::Buf bhl_cnt, bhl_far, bhl_near;
    // workspaces
    tp::Buf part, part2, scal, corner, wv64, wv32, tmpv[8];
    tp::Buf io_in, io_out, adj, erow, tlist, rowsum;
    tp::Buf kry;        // FGMRES bases V and Z
    tp::Buf gsdev;      // FGMRES: first-pass Gram-Schmidt coefficients on the device
    tp::Buf tickets;    // completion tickets of the fused reductions (tp::TICKET_*)
    tp::Buf tcbuf;      // tensor-core A apply: packed source tiles
    tp::Buf tcerr;      // tensor-core A apply: a wait gave up (device int)
    tp::Buf stepv[8];   // vectors of the constrained step
    tp::Buf prec[3];    // preconditioner temporaries
    tp::Buf bhcount;    // device counter of Barnes-Hut interactions
    // static obstacle (§7.3.2): a mesh of its own (positions, face tables,
    // BVH), and its faces re-expressed in this mesh's frame for the direct sums
    tp_mesh* obs = nullptr;
    double obs_weight = 0.0;
    tp::Buf obs_perm, obs_f64a, obs_f32a, obs_f32c, obs_tilebox, obs_thr, obs_part;
    // vertex pins (§7.1.2, §7.2): indices, component of each vertex and
    // pinned flags, W = C^+ S^T and the inverse of the pins' small system
    int npins = 0, pin_ncomp = 0;
    bool pin_valid = false;          // W and the small system match the positions
    std::vector<int> pin_host, pin_comp_host;
    tp::Buf pin_idx, pin_vcomp, pin_W, pin_Minv, pin_tmp;
    tp::Profiler prof;
    double pairs = 0.0; // pair interactions evaluated (host-known part)
};

namespace tp {

// -------- mesh.cu ----------------------------------------------------------
int refresh_geometry(tp_mesh* m, cudaStream_t st);   // face tables from m->pos
int components_setup(tp_mesh* m, const std::vector<int>& faces_host);   // at creation
// remove the mean of each connected component from each column of x [nv][k]
int project_components(tp_mesh* m, double* x_dev, int k, cudaStream_t st);
int corners_to_vertices(tp_mesh* m, const double* corner, int k, double* y, cudaStream_t st);
int copy_in(void* dst, const void* src, size_t bytes, int ptr_kind, cudaStream_t st);
int copy_out(void* dst, const void* src, size_t bytes, int ptr_kind, cudaStream_t st);
int sum_f64(const double* x, int n, double* out_dev, tp_mesh* m, cudaStream_t st);
int colsum(tp_mesh* m, const double* x, long n, int k, double scale, double* out_dev, cudaStream_t st);
// completion tickets of the fused (single-launch) reductions: one slot per
// reduction kind, zero between launches
enum { TICKET_COLSUM = 0, TICKET_DOTS = 1, TICKET_COMP = 2, TICKET_CHOL = 3, TICKET_COUNT = 8 };
int mesh_tickets(tp_mesh* m, unsigned** out, cudaStream_t st);
const char* last_error();
// profiling: wrap a launch (or a group of launches) of kernel class `key`
// processing `units` of algorithmic work
struct ProfScope {
    tp_mesh* m;
    int key;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st;
    ProfScope(tp_mesh* m, int key, double units, cudaStream_t st);
    ~ProfScope();
};
void prof_release(tp_mesh* m);
unsigned long long launch_count();

// -------- pairs.cu ---------------------------------------------------------
// per-target rows of Eq. 10 (targets == nullptr: all faces), written to rows_dev [nt]
int energy_rows_direct(tp_mesh* m, const tp_params* p, const int32_t* targets_dev, int nt,
                       double* rows_dev, cudaStream_t st);
// face adjoints gX,gN,ga (FP64 [nf*7]) and energy rows
int diff_adjoints_direct(tp_mesh* m, const tp_params* p, double* adj_dev, double* erow_dev,
                         cudaStream_t st);
// adjoints -> per-face corner gradients [nf*3*3] -> dE [nv*3]
int adjoints_to_dE(tp_mesh* m, const double* adj_dev, double* dE_dev, cudaStream_t st);
// y = O v (device, [nv*k]); direct all pairs
int apply_direct(tp_mesh* m, const tp_params* p, int op, const double* v_dev, int k,
                 double* y_dev, cudaStream_t st);
// y = O v over the Barnes-Hut interaction lists (theta > 0, FP32)
int apply_bh(tp_mesh* m, const tp_params* p, int op, const double* v_dev, int k, double* y_dev,
             cudaStream_t st);
// whether a bounded wait of the tensor-core A apply gave up since the last
// call (reads a device flag: synchronises the stream)
int apply_tc_error(tp_mesh* m, int* gave_up, cudaStream_t st);
// direct for theta = 0, Barnes-Hut otherwise
int apply_op(tp_mesh* m, const tp_params* p, int op, const double* v_dev, int k, double* y_dev,
             cudaStream_t st);

// -------- bvh.cu -----------------------------------------------------------
int bvh_build(tp_mesh* m, const tp_params* p, cudaStream_t st);
int energy_rows_bh(tp_mesh* m, const tp_params* p, const int32_t* targets_dev, int nt,
                   double* rows_dev, cudaStream_t st);
int diff_adjoints_bh(tp_mesh* m, const tp_params* p, double* adj_dev, double* erow_dev,
                     cudaStream_t st);
int bh_counter(tp_mesh* m, cudaStream_t st);
// device counters of Barnes-Hut interactions: [0] energy, [1] differential, [2] operator applies,
// [3] obstacle potential
constexpr int BH_NCOUNT = 4;
int bh_counts_read(tp_mesh* m, unsigned long long out[BH_NCOUNT], bool reset, cudaStream_t st);
int bvh_view(tp_mesh* m, const tp_params* p, cudaStream_t st, BvhView* out);   // builds the tree if needed
// interaction lists of the tree for p->theta (built on first use per tree and
// theta); *ok = false when they cannot be built (the walk kernels then serve)
int bh_lists(tp_mesh* m, const tp_params* p, cudaStream_t st, BhLists* out, bool* ok);

// -------- cg.cu ------------------------------------------------------------
int laplacian_setup(tp_mesh* m);                        // CSR pattern (host, once)
int laplacian_values(tp_mesh* m, cudaStream_t st);      // cotan values for current positions
int cg_solve(tp_mesh* m, const tp_params* p, const double* b_dev, int k, double* z_dev,
             cudaStream_t st, int* iters, bool deferred = false);
// y += G x (k columns), G the within-face term of the preconditioner's
// L^{2-s} with weight p->prec_self_weight (nothing when the weight is 0)
int self_term_add(tp_mesh* m, const tp_params* p, const double* x_dev, int k, double* y_dev,
                  cudaStream_t st);
// -------- chol.cu ----------------------------------------------------------
// z = C^+ b through the sparse Cholesky factor; *used = false when the
// factor cannot serve the mesh (panel too large) or refinement stalled
int chol_solve(tp_mesh* m, const tp_params* p, const double* b_dev, int k, double* z_dev,
               cudaStream_t st, int* iters, bool* used, bool deferred = false);
// deferred solves (deferred = true: no host read per solve, the sweeps cg_tol
// needs, flags accumulated on the device): read (unless reset) and clear the
// accumulated wait error and unconverged-solve flags
int chol_deferred_flags(tp_mesh* m, cudaStream_t st, int* err, int* unconverged, bool reset);
int chol_info(tp_mesh* m, tp_chol_info* out);
// waits in one kernel on a word nothing sets: TP_ERR_TIMEOUT and *timed_out = 1
// once the bounded wait gives up (current device)
int wait_selftest(int* timed_out);
void chol_invalidate(tp_mesh* m);   // positions changed: refactor before the next solve
void chol_release(tp_mesh* m);
// vector helpers (device, FP64, deterministic)
int project_mean_zero(tp_mesh* m, double* x_dev, int k, cudaStream_t st);
int dots(tp_mesh* m, const double* const* xs, const double* y, int nvec, size_t n,
         double* out_host, cudaStream_t st);
int dot_pairs(tp_mesh* m, const double* const* xs, const double* const* ys, int nvec, size_t n,
              double* out_host, cudaStream_t st);   // out_host[j] = xs[j] . ys[j], nvec <= 512
int axpy(double* y, const double* x, double a, size_t n, cudaStream_t st);
// device-resident variant (no host synchronisation): dot products into
// device memory (lincomb_sys reads them as coefficients)
int dot_pairs_dev(tp_mesh* m, const double* const* xs, const double* const* ys, int nvec, size_t n,
                  double* out_dev, cudaStream_t st);
int lincomb(double* y, const double* const* xs, const double* coef_host, int nvec, size_t n,
            double beta, cudaStream_t st);
// one launch for ns <= 4 systems with nvec vectors each: out[s] = scale[s] *
// (beta y[s] + sum_l c[s * nvec + l] xs[s * nvec + l]), with c = coef_host, or
// c = -coef_dev read from device memory (the Gram-Schmidt update w -= V h);
// ns * nvec <= 128
int lincomb_sys(int ns, double* const* out, const double* const* y, const double* const* xs, int nvec,
                const double* coef_dev, const double* coef_host, const double* scale, double beta, size_t n,
                cudaStream_t st);

// -------- obstacle.cu ------------------------------------------------------
int obstacle_attach(tp_mesh* m, tp_mesh* obstacle, double weight, cudaStream_t st);  // m owns it
int obstacle_frame(tp_mesh* m, cudaStream_t st);   // obstacle faces in m's current frame
// obstacle rows w a_T E_obs(X_T) into erow_dev (and with diff its face
// adjoints into adj_dev [nf*7]); accumulate: add to what is there
int obstacle_terms(tp_mesh* m, const tp_params* p, bool diff, bool accumulate, double* erow_dev,
                   double* adj_dev, cudaStream_t st);
void obstacle_release(tp_mesh* m);

// -------- pins.cu ----------------------------------------------------------
int pins_set(tp_mesh* m, int n, const int* idx_host, cudaStream_t st);   // n = 0 removes the pins
void pins_release(tp_mesh* m);
// z = first block of [C S^T; S 0]^{-1} [b; 0] (k <= 9 columns); TP_ERR_NOT_CONVERGED
// from the inner solve is passed on with z filled
int pinned_solve(tp_mesh* m, const tp_params* p, const double* b_dev, int k, double* z_dev,
                 cudaStream_t st, int* iters);
// zero the pinned rows (pins set) or remove the mean of each component (no pins)
int project_space(tp_mesh* m, double* x_dev, int k, cudaStream_t st);

// -------- willmore.cu -------------------------------------------------------
// E_W = f^T C M^-1 C f into E_dev (device scalar, may be null); with dE_dev, dE += w dE_W
int willmore_eval(tp_mesh* m, double* E_dev, double* dE_dev, double w, cudaStream_t st);
// y += w C M^-1 C v (k <= 9 columns)
int willmore_operator_add(tp_mesh* m, const double* v_dev, int k, double* y_dev, double w, cudaStream_t st);

// -------- solver.cu --------------------------------------------------------
// E (host) of Eq. 10 or 16; with aux = true plus the terms the step adds (static
// obstacle, weighted Willmore energy), as is the differential
int energy_value(tp_mesh* m, const tp_params* p, double* E_host, cudaStream_t st, bool aux = false);
int differential_dev(tp_mesh* m, const tp_params* p, double* dE_dev, double* E_host,
                     cudaStream_t st, bool aux = false);
int precond_apply_dev(tp_mesh* m, const tp_params* p, const double* b, int k, double* z,
                      cudaStream_t st, int* cg_iters, bool strict = true);
int precond_step_dev(tp_mesh* m, const tp_params* p, const tp_constraints* c, tp_step_report* rep,
                     cudaStream_t st);
// total area (§7.1.3) and enclosed signed volume (§7.1.4) of the current positions (host)
int area_volume(tp_mesh* m, double out[2], cudaStream_t st);

}  // namespace tp
