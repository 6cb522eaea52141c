/*
 * tp.h -- C ABI of the GB300 tangent-point surface-flow library (libtpsurf).
 *
 * The library evaluates the hot path of "Repulsive Surfaces" (Yu,
 * Brakensiek, Schumacher, Crane 2021) on one GPU:
 *   - the discrete tangent-point energy E (§3.1, Eq. 9-10) and its
 *     differential dE (§3.1, chain rule),
 *   - the forward application of the fractional operators B, B0, A = B + B0
 *     (§3.2, §5.1.2-5.1.3, Appendix A) and L^{2-s} (§5.1.1, §5.2),
 *   - Barnes-Hut approximations of E and dE over a GPU-built BVH (§4),
 *   - the cotan-Laplacian Poisson solves of the preconditioner (§5.2):
 *     a pre-factorised sparse Cholesky (default) or Jacobi CG,
 *   - the constrained preconditioned descent step (§3.3, §5.3, §5.4).
 *
 * Conventions shared by every call:
 *   - Return value: TP_OK (0) or one of the TP_ERR_* codes. On error the
 *     outputs are unspecified and tp_last_error() (thread-local) describes it.
 *   - Positions are float64 [nv][3] row-major (x,y,z per vertex); faces are
 *     int32 [nf][3], counter-clockwise, 0-based, every face non-degenerate.
 *   - Vertex vectors v, y, b, z with k columns are float64 [nv][k] row-major.
 *   - ptr_kind says whether the array arguments of a call are host memory
 *     (TP_PTR_HOST; copied synchronously on `stream`) or device memory of
 *     the mesh's GPU (TP_PTR_DEVICE; must stay valid until `stream` has
 *     passed the call).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls that
 *     return host scalars synchronise `stream` before returning.
 *   - The caller owns every array it passes; the library owns the state of a
 *     tp_mesh (positions, face tables, BVH, CSR Laplacian, workspaces) and
 *     frees it in tp_mesh_destroy. A tp_mesh must be used by one host thread
 *     at a time.
 */
#ifndef TP_H
#define TP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TP_OK                 0
#define TP_ERR_INVALID_ARG    1  /* null pointer, bad size, index out of range, bad enum */
#define TP_ERR_DEGENERATE     2  /* zero-area face or non-finite position */
#define TP_ERR_OOM            3  /* device allocation failed */
#define TP_ERR_NOT_CONVERGED  4  /* CG or Krylov solver hit its iteration cap */
#define TP_ERR_TIMEOUT        5  /* a bounded device-side wait gave up */
#define TP_ERR_CUDA           6  /* any other CUDA runtime error */

/* ptr_kind */
#define TP_PTR_HOST   0
#define TP_PTR_DEVICE 1

/* precision of the pair terms */
#define TP_PREC_FP32  0  /* FP32 pair terms, compensated FP32 sums, FP64 final reduction */
#define TP_PREC_FP64  1  /* plain FP64 pair terms */

/* operators of fractional_apply */
#define TP_OP_A   0  /* A = B + B0, the H^s inner product (§2.4, §5.1.2-5.1.3) */
#define TP_OP_B   1  /* high-order term B, kernel |d|^{-2s} (§5.1.2)            */
#define TP_OP_B0  2  /* low-order term B0, kernel (k2(S;T)+k2(T;S))/(2|d|^{2s}) (§5.1.3) */
#define TP_OP_L   3  /* L^{2-s} of the preconditioner, kernel |d|^{-(6-2s)} (§5.1.1, §5.2) */

/* Barnes-Hut differential modes (§4.2) */
#define TP_BH_DIFF_FULL     0  /* forward terms plus node-level reverse terms pushed to faces */
#define TP_BH_DIFF_LITERAL  1  /* only the terms in which the face is the target S */

/* Poisson solver of the preconditioner (§5.2) */
#define TP_POISSON_CHOLESKY 0  /* pre-factorised C (sparse Cholesky, FP32 factor, FP64 refinement) */
#define TP_POISSON_CG       1  /* Jacobi-preconditioned CG, FP64 */

/* largest number of vertex pins of a mesh (tp_pins_set) */
#define TP_MAX_PINS 64

/* constraint flags (the barycenter constraint of §7.1.1 is on unless pins are set) */
#define TP_CONSTRAINT_AREA    1  /* total area, §7.1.3 */
#define TP_CONSTRAINT_VOLUME  2  /* total signed volume, §7.1.4 */
#define TP_CONSTRAINT_FREE_BARYCENTER 4  /* let each component's barycenter float (§7.1.1, barycenter
                                            motions): the direction gains minus the area-weighted mean of
                                            dE per component; not with pins */

typedef struct tp_params {
    double p;             /* tangent-point exponent p (numerator |P d|^p, denominator |d|^{2p}); paper default 6 (§2.1) */
    double theta;         /* Barnes-Hut separation theta; 0 = exact all-pairs sums (§4.1) */
    int    leaf_size;     /* BVH leaf size l, 1..32; paper default 8 (§4.1) */
    int    precision;     /* TP_PREC_FP32 or TP_PREC_FP64 */
    int    bh_diff_mode;  /* TP_BH_DIFF_FULL or TP_BH_DIFF_LITERAL */
    double krylov_tol;    /* relative residual of the outer GMRES solves */
    int    krylov_max;    /* iteration cap of one GMRES solve (all restarts) */
    int    gmres_restart; /* restart length m */
    double cg_tol;        /* relative residual of the Poisson solves (FP64 residual, both solvers) */
    int    cg_max;        /* iteration cap of one CG solve (refinement sweeps: min(cg_max, 40)) */
    double armijo_c;      /* sufficient-decrease constant of the line search */
    double armijo_shrink; /* step shrink factor */
    double tau0;          /* initial step */
    int    ls_max;        /* maximum line-search trials */
    int    fixed_tau;     /* 1 = take tau0 without line search */
    int    proj_iters;    /* corrective projections per step (§3.3.2: one suffices; repeats allowed) */
    int    poisson_solver; /* TP_POISSON_CHOLESKY (default) or TP_POISSON_CG */
    int    bvh_refit;     /* 1 = after the positions change, keep the tree's face order and
                             recompute only the node data (refit); 0 = rebuild (new Morton order) */
    double prec_self_weight; /* kappa >= 0 of the within-face term added to L^{2-s} in the
                                preconditioner (see precond_apply); 0 = L^{2-s} of §5.1.1 alone */
    double tau0_disp;     /* > 0: the line search starts from min(tau0, tau0_disp h / max_v |x_v|),
                             h = sqrt(total area / nf), so that the first trial moves no vertex by
                             more than tau0_disp face sizes; 0 (default) = start from tau0 */
    int    tensor_cores;  /* direct FP32 A applies on 4-9 columns: 1 = the accumulation of the kernel
                             values times the source vectors on tcgen05 tensor cores (split TF32
                             products, FP32 accumulators drained into compensated sums every 128
                             sources); 0 (default) = CUDA cores (packed FP32) */
} tp_params;

typedef struct tp_constraints {
    int    flags;   /* TP_CONSTRAINT_AREA | TP_CONSTRAINT_VOLUME */
    double A0;      /* target total area   */
    double V0;      /* target total volume */
} tp_constraints;

typedef struct tp_step_report {
    double E_before;       /* E(f) */
    double E_after;        /* E(f_new) */
    double tau;            /* accepted step */
    double slope;          /* dE . x (negative for a descent direction) */
    double phi_before[2];  /* constraint values at f + tau x (area, volume) */
    double phi_after[2];   /* constraint values at f_new */
    int    krylov_iters;   /* total GMRES iterations of the step */
    int    cg_iters;       /* total Poisson-solver iterations of the step (CG iterations or refinement sweeps) */
    int    ls_trials;      /* energy evaluations of the line search */
    int    status;         /* TP_OK or the first non-fatal solver status */
    double pair_interactions; /* (target, source) terms evaluated during the step */
} tp_step_report;

/* Per-kernel statistics of a mesh (tp_profile_read). `units` is the
 * algorithmic work of the launches: pair interactions for the pair and
 * Barnes-Hut kernels, bytes of matrix and vector traffic for CG. */
typedef struct tp_kernel_stat {
    char      name[32];
    long long launches;
    double    ms;        /* summed CUDA-event durations (0 unless profiling is on) */
    double    units;
    double    columns;   /* operator columns summed over the launches (apply kernels; else 0) */
} tp_kernel_stat;

typedef struct tp_mesh tp_mesh;

/* A library context: one CUDA device and the allocator that supplies the
 * device memory of the meshes created in it (their positions, face tables,
 * BVH, Laplacian, factor and workspaces). The paper's problem statement (a
 * mesh, its energy and the step, §3, §5.4) does not involve one; it is the
 * ownership boundary of the library's memory. */
typedef struct tp_ctx tp_ctx;

/* Caller-set allocator of a context. alloc returns `bytes` of device memory
 * on `device`, aligned to 256 bytes, or NULL (the library call then fails
 * with TP_ERR_OOM); free returns a block obtained from alloc with the size it
 * was asked for. The library synchronises the device before each free, so a
 * freed block may be handed to other work at once. Both are called on the
 * thread of the library call that needs the memory; `user` is passed
 * through. Buffers grow and are freed rarely: when a mesh first needs a
 * workspace, when a larger one is needed, and in tp_mesh_destroy. */
typedef struct tp_allocator {
    void* (*alloc)(size_t bytes, int device, void* user);
    void (*free)(void* ptr, size_t bytes, int device, void* user);
    void* user;
} tp_allocator;

/* Create a context on CUDA device `device` with the default allocator
 * (cudaMalloc / cudaFree). TP_ERR_INVALID_ARG for a device that does not
 * exist. */
int tp_create(int device, tp_ctx** out);

/* Destroy a context. TP_ERR_INVALID_ARG while meshes created in it are
 * alive (destroy them first). Accepts NULL. */
int tp_destroy(tp_ctx* ctx);

/* Set the allocator of a context (alloc = free = NULL restores cudaMalloc /
 * cudaFree). TP_ERR_INVALID_ARG while meshes created in it are alive, or for
 * a half-set pair. */
int tp_ctx_set_allocator(tp_ctx* ctx, const tp_allocator* a);

/* Device bytes a context's meshes hold now and at most so far (host
 * integers; either pointer may be NULL). */
int tp_ctx_memory(const tp_ctx* ctx, size_t* in_use, size_t* peak);

/* tp_mesh_create in a context: the mesh's device memory comes from the
 * context's allocator, on the context's device. */
int tp_mesh_create_ctx(tp_ctx* ctx, int nv, int nf, const double* pos,
                       const int32_t* faces, int ptr_kind, void* stream,
                       tp_mesh** out);

/* Fill *p with the defaults: p=6, theta=0, leaf_size=8, FP32 pairs,
 * full BH differential, krylov_tol=1e-6, krylov_max=200, restart 30,
 * cg_tol=1e-6, cg_max=20000, Armijo c=1e-4, shrink 0.5, tau0=1, ls_max=30,
 * proj_iters=1, Cholesky Poisson solver, prec_self_weight=24, tau0_disp=0. */
void tp_params_default(tp_params* p);

/* Create a mesh on CUDA device `device` from nv positions and nf faces
 * (the mesh M = (V, E, F) and embedding f of §3.1), in the device's default
 * context (cudaMalloc). Validates the face indices (TP_ERR_INVALID_ARG) and
 * the geometry (TP_ERR_DEGENERATE). Allocates the device state of the mesh;
 * workspaces are added on first use. */
int tp_mesh_create(int device, int nv, int nf, const double* pos,
                   const int32_t* faces, int ptr_kind, void* stream,
                   tp_mesh** out);

/* Replace the positions (same topology) and refresh the face tables. */
int tp_mesh_set_positions(tp_mesh* m, const double* pos, int ptr_kind, void* stream);

/* Copy the current positions (float64 [nv][3]) out. */
int tp_mesh_get_positions(tp_mesh* m, double* pos, int ptr_kind, void* stream);

/* Total area sum_T a_T (§7.1.3) and enclosed signed volume
 * (1/6) sum_{ijk} f_i . (f_j x f_k) (§7.1.4) of the current positions: the
 * quantities the constraints A0 and V0 of precond_step refer to. Either
 * output (host doubles) may be NULL, not both. Synchronises `stream`. */
int tp_mesh_area_volume(tp_mesh* m, double* area, double* volume, void* stream);

/* Free every device resource of the mesh. Accepts NULL. */
int tp_mesh_destroy(tp_mesh* m);

/* Device bytes a mesh of this size holds, for admission control. Not
 * included: a static obstacle (a mesh of its own), vertex pins (8 nv bytes
 * per pin) and the Willmore workspace (192 nv bytes), which exist only once
 * set. */
size_t tp_mesh_footprint_bytes(int nv, int nf, const tp_params* p);

/* Discrete tangent-point energy E (§3.1, Eq. 10; ordered pairs S != T),
 * or its Barnes-Hut approximation (§4.1, Eq. 16) when theta > 0.
 * *E_out is a host double. */
int tp_energy(tp_mesh* m, const tp_params* p, double* E_out, void* stream);

/* Row sums E_S = sum_{T != S} K(S,T) a_S a_T of Eq. 10 (or of Eq. 16 when
 * theta > 0) for n target faces `targets` (int32); rows is float64 [n]. */
int tp_energy_rows(tp_mesh* m, const tp_params* p, const int32_t* targets, int n,
                   double* rows, int ptr_kind, void* stream);

/* Differential dE/df (float64 [nv][3]) of Eq. 10 by the chain rule through
 * the face barycenters, normals and areas (§3.1); with theta > 0 the
 * Barnes-Hut derivative of §4.2 (mode bh_diff_mode). E_out (host, may be
 * NULL) receives the energy of the same pass. */
int tp_differential(tp_mesh* m, const tp_params* p, double* dE, int ptr_kind,
                    double* E_out, void* stream);

/* y = O v for op in TP_OP_* and k columns (1 <= k <= 9), each column
 * separately (the vector operator O_3 of §3.2.1 for k = 3), through the
 * kernel-matrix form of §5.1.1-5.1.3 and Appendix A:
 *   O v = 2 W^T [diag(diag(a)^-1 H a) - H] W v,
 * W = diag(a) D (op B) or the area-weighted face average (ops B0, L).
 * theta = 0: H by the direct all-pairs sums. theta > 0 (FP32 only): H by
 * Barnes-Hut over the tree and admissibility test of the energy (§4.1):
 * an admissible node I contributes h(X_S, P_S; X_I, P_I) times the node
 * sums of a and W, P_I the node-average projector of §5.1.4 (in the
 * low-order kernel); inadmissible leaves are summed exactly. The row sums
 * H a use the same approximation, so constants stay in the nullspace.
 * precond_apply and precond_step use the same choice for their applies. */
int fractional_apply(tp_mesh* m, const tp_params* p, int op, const double* v,
                     int k, double* y, int ptr_kind, void* stream);

/* z = C^+ b for the cotan stiffness matrix C of the current positions
 * (§5.2), k columns (1 <= k <= 9), b and z FP64 [nv][k].
 * TP_POISSON_CHOLESKY: the pre-factorisation of §5.2. One vertex per
 * connected component is pinned, the rest is factored by a supernodal sparse
 * Cholesky (nested-dissection order, FP32 factor on the device, recomputed
 * when the positions change); b is projected to zero mean per component and
 * FP64 iterative refinement runs until every column has
 * |b - C z| <= cg_tol |b|; z has zero mean per component. A mesh whose
 * largest supernode panel does not fit in shared memory, or a solve whose
 * refinement stops converging, is handed to the CG solver.
 * TP_POISSON_CG: Jacobi-preconditioned CG (FP64) with b and z projected to
 * zero mean over the whole mesh (connected meshes).
 * With vertex pins set (tp_pins_set) the pin rows are appended to C (§7.2):
 * z solves [C S^T; S 0] [z; mu] = [b; 0] (z = 0 at the pins, C z = b on the
 * free vertices, b's pinned rows ignored), computed from the unpinned solver
 * above by a correction with one solve per pin (once per positions).
 * *iters_out (host, may be NULL) receives the CG iterations or refinement
 * sweeps. TP_ERR_NOT_CONVERGED if cg_max is hit; TP_ERR_TIMEOUT if a
 * device-side wait gave up. */
int cotan_solve(tp_mesh* m, const tp_params* p, const double* b, int k, double* z,
                int ptr_kind, void* stream, int* iters_out);

/* Structure of the sparse Cholesky factor of C (§5.2) of a mesh: computed
 * on the first call (host analysis of the topology), no device work. */
typedef struct tp_chol_info {
    int    available;      /* 1 if the factorised solver serves this mesh */
    int    components;     /* connected components (one pinned vertex each) */
    int    unknowns;       /* factored unknowns: nv - components */
    int    supernodes;     /* supernodes of the elimination tree */
    int    levels;         /* tree height + 1 (sequential launches per substitution) */
    int    max_front;      /* largest front (own + structure rows) */
    double factor_floats;  /* stored factor entries (L11^-1 and L21 blocks) */
    double update_floats;  /* update-matrix entries */
} tp_chol_info;

int cotan_factor_info(tp_mesh* m, tp_chol_info* out);

/* z = C^+ (L^{2-s} + G) C^+ b, the preconditioner of §5.2, k columns.
 * G is the within-face part of the L^{2-s} double integral that the pair
 * sums of §5.1.1 leave out (pairs of points inside one face): for
 * piecewise-linear functions it is the P1 stiffness matrix with face
 * weights kappa a_S^{1-(2-s)}, kappa = prec_self_weight (default 24; 0 gives
 * the paper's C^+ L^{2-s} C^+). It makes the preconditioned operator's
 * spectrum mesh-independent and narrow; it does not change the solutions
 * of the Krylov solves. With pins set, both Laplacian solves are pinned. */
int precond_apply(tp_mesh* m, const tp_params* p, const double* b, int k,
                  double* z, int ptr_kind, void* stream);

/* Vertex pins (§7.1.2) of a mesh, handled as fast positional constraints
 * (§7.2): n vertex indices (int32, 0 <= n <= TP_MAX_PINS; n = 0 removes the
 * pins and `vertices` may be NULL). A pin keeps its vertex where it is:
 * precond_step solves the saddle system with the pin rows inside A (the
 * Krylov vectors are zero at the pins) and appends them to the Laplacians
 * of the preconditioner (cotan_solve and precond_apply then solve the pinned
 * systems), so the step and its projection leave pinned vertices in place.
 * Pins replace the barycenter constraint of §7.1.1 (they remove the
 * nullspace). TP_ERR_INVALID_ARG for an index out of range, a repeated
 * vertex, or a connected component without a pin. Synchronises `stream`. */
int tp_pins_set(tp_mesh* m, int n, const int32_t* vertices, int ptr_kind, void* stream);

/* Willmore term of a mesh (§7.3.5): with weight w > 0, precond_step
 * minimises E + w E_W, E_W = f^T C M^{-1} C f (C the cotan stiffness
 * matrix, M the lumped mass: a third of the area of each face around a
 * vertex, summed over the three coordinate columns of f), and adds the H^2
 * term w C M^{-1} C to the operator it inverts (its report's energies are
 * E + w E_W). w = 0 (the default) removes the term. TP_ERR_INVALID_ARG for a
 * negative or non-finite weight. */
int tp_willmore_set(tp_mesh* m, double weight);

/* E_W (host, may be NULL) and dE_W/df (float64 [nv][3], may be NULL; not
 * both NULL) of the current positions, whatever weight is set: FP64 sparse
 * products on the pattern of C and per-face corner terms (derivatives of
 * the cotangents and of the lumped mass). */
int tp_willmore_energy(tp_mesh* m, double* E_out, double* dE, int ptr_kind, void* stream);

/* One constrained descent step (§5.4): dE, the Schur-complement solution
 * of the saddle problem (Eq. 14, 17, 18) with GMRES on A_3 preconditioned
 * by precond_apply, Armijo line search, and proj_iters corrective
 * projections (Eq. 15, 19) with the constraint Jacobian of the start of the
 * step. Updates the mesh positions in place. rep may be NULL. */
int precond_step(tp_mesh* m, const tp_params* p, const tp_constraints* c,
                 tp_step_report* rep, void* stream);

/* Static mesh obstacle of a mesh (§7.3.2). The obstacle is a fixed triangle
 * mesh O (nv positions float64 [nv][3], nf faces int32 [nf][3], validated
 * like tp_mesh_create); every point x of the surface feels the potential
 *   E_obs(x) = sum_{S in F_O} |f_O(S) - x|^{-p} a_O(S)
 * (f_O(S), a_O(S): barycenter and area of obstacle face S; p of tp_params).
 * Reading of the paper: the potential is a density over the surface,
 * integrated with the one-point rule of Eq. 10 and scaled by `weight`:
 *   E_O = weight * sum_T a_T E_obs(X_T).
 * Once set, precond_step minimises E + E_O (its report's energies are the
 * sum); tp_energy and tp_differential stay Eq. 10 / Eq. 16 alone.
 * The library copies the obstacle (the caller keeps its arrays) and keeps
 * it until it is replaced, removed (nf = 0; pos and faces may then be
 * NULL) or the mesh is destroyed. weight >= 0. Synchronises `stream`. */
int tp_obstacle_set(tp_mesh* m, int nv, int nf, const double* pos, const int32_t* faces,
                    double weight, int ptr_kind, void* stream);

/* E_O (host, may be NULL) and dE_O/df (float64 [nv][3], may be NULL) of
 * the obstacle set on the mesh: theta = 0 by direct sums over all
 * (surface face, obstacle face) pairs in the precision of tp_params;
 * theta > 0 (FP32) by Barnes-Hut over a BVH of the obstacle (leaf_size),
 * an admissible node I adding a_I |X_I - x|^{-p}, X_I its area-weighted
 * barycenter. The differential goes through the face barycenters and
 * areas (§3.1 chain rule). TP_ERR_INVALID_ARG if no obstacle is set. */
int tp_obstacle_energy(tp_mesh* m, const tp_params* p, double* E_out, double* dE, int ptr_kind,
                       void* stream);

/* Turn per-launch CUDA-event timing of the pair, Barnes-Hut and CG kernels
 * of this mesh on (1) or off (0). Events are recorded on the launching
 * stream; launches and units are counted whether or not timing is on. */
int tp_profile_enable(tp_mesh* m, int on);

/* Copy up to `max` per-kernel statistics (accumulated since the last read)
 * into out, set *n to the number written, and reset them. Synchronises
 * with the recorded events. */
int tp_profile_read(tp_mesh* m, tp_kernel_stat* out, int max, int* n);

/* Number of CUDA kernels this library has launched in this process. */
unsigned long long tp_launch_count(void);

/* The direct energy E (FP32 pair terms, compensated sums, FP64 reduction;
 * the same quantity as tp_energy with theta = 0) for callers that are not
 * allowed to allocate device memory: plug-ins inside a host program that
 * owns the device allocator and forbids side allocations, and real-time
 * loops that must not block on allocator locks or meet an out-of-memory
 * failure mid-run. The paper has no counterpart of this entry point.
 *   pos   device float64 [nv][3], faces device int32 [nf][3], E device
 *         float64 [1] (output), all on the calling thread's current CUDA
 *         device; p > 2. A face naming a vertex outside 0..nv-1 makes *E a
 *         quiet NaN (the call still returns TP_OK: the check runs on the GPU).
 * Allocates nothing: every intermediate lives in one static device array of
 * 5,767,232 bytes (5.5 MiB) that each GPU loading the library holds until the
 * process exits. At most 32768 faces (larger meshes: TP_ERR_INVALID_ARG
 * before anything is launched; use tp_mesh_create + tp_energy). The first
 * call on a device (and context) looks up that array's device address; make
 * it before any stream capture. Calls share the array: calls whose kernels
 * overlap on the GPU (other streams, other threads) race, so the caller must
 * serialise them. Asynchronous on `stream`; *E is valid once the stream has
 * passed the call. */
int tp_energy_noalloc(const double* pos, int nv, const int32_t* faces, int nf,
                      double p, double* E, void* stream);

/* Self-test of failure detection (the paper has no counterpart): one
 * kernel on `device` waits for a device word that nothing sets, with the
 * bounded wait that the sparse Cholesky sweep uses for its cross-block
 * signals. The wait gives up after about one second, records the timeout
 * and returns, so the context stays usable. Returns TP_ERR_TIMEOUT with
 * *timed_out = 1 when that happened as designed (TP_OK with *timed_out = 0
 * would mean the wait saw a value it should not have). Synchronous. */
int tp_selftest_wait(int device, int* timed_out);

/* Thread-local description of the last error of this thread ("" if none). */
const char* tp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TP_H */
