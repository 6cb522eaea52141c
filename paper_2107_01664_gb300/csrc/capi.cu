// The extern "C" entry points declared in include/tp.h: argument checks,
// device selection, staging of host arrays, and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tp_internal.cuh"

using namespace tp;

namespace {

// selects the mesh's device (and the mesh's context, whose allocator serves
// the buffers the call grows) for the duration of a call and restores the
// caller's current device afterwards
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    tp_ctx* prev_ctx = nullptr;
    explicit DeviceGuard(int dev, tp_ctx* ctx = nullptr) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
        prev_ctx = current_ctx();
        current_ctx() = ctx ? ctx : default_ctx(dev);
    }
    explicit DeviceGuard(const tp_mesh* m) : DeviceGuard(m->device, m->ctx) {}
    ~DeviceGuard() {
        current_ctx() = prev_ctx;
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int check_params(const tp_params* p) {
    if (!p) return fail(TP_ERR_INVALID_ARG, "params is NULL");
    if (!(p->p > 2.0) || !std::isfinite(p->p)) return fail(TP_ERR_INVALID_ARG, "p must be > 2");
    if (!(p->theta >= 0.0) || !std::isfinite(p->theta))
        return fail(TP_ERR_INVALID_ARG, "theta must be finite and >= 0");
    if (p->leaf_size < 1 || p->leaf_size > 32) return fail(TP_ERR_INVALID_ARG, "leaf_size must be in 1..32");
    if (p->precision != TP_PREC_FP32 && p->precision != TP_PREC_FP64)
        return fail(TP_ERR_INVALID_ARG, "unknown precision");
    if (p->theta > 0.0 && p->precision != TP_PREC_FP32)
        return fail(TP_ERR_INVALID_ARG, "Barnes-Hut (theta > 0) runs in TP_PREC_FP32 only");
    if (p->poisson_solver != TP_POISSON_CHOLESKY && p->poisson_solver != TP_POISSON_CG)
        return fail(TP_ERR_INVALID_ARG, "unknown Poisson solver");
    if (p->bvh_refit != 0 && p->bvh_refit != 1) return fail(TP_ERR_INVALID_ARG, "bvh_refit must be 0 or 1");
    if (!(p->prec_self_weight >= 0.0) || !std::isfinite(p->prec_self_weight))
        return fail(TP_ERR_INVALID_ARG, "prec_self_weight must be finite and >= 0");
    if (!(p->tau0_disp >= 0.0) || !std::isfinite(p->tau0_disp))
        return fail(TP_ERR_INVALID_ARG, "tau0_disp must be finite and >= 0");
    if (p->tensor_cores != 0 && p->tensor_cores != 1) return fail(TP_ERR_INVALID_ARG, "tensor_cores must be 0 or 1");
    return TP_OK;
}

int check_mesh(const tp_mesh* m) {
    if (!m) return fail(TP_ERR_INVALID_ARG, "mesh is NULL");
    return TP_OK;
}

int check_kind(int ptr_kind) {
    if (ptr_kind != TP_PTR_HOST && ptr_kind != TP_PTR_DEVICE)
        return fail(TP_ERR_INVALID_ARG, "ptr_kind must be TP_PTR_HOST or TP_PTR_DEVICE");
    return TP_OK;
}

// returns a device pointer holding `bytes` of `src` (staged through `buf`
// when src is host memory)
int stage_in(Buf& buf, const void* src, size_t bytes, int ptr_kind, cudaStream_t st, const void** out) {
    if (ptr_kind == TP_PTR_DEVICE) {
        *out = src;
        return TP_OK;
    }
    TP_TRY(ensure(buf, bytes));
    TP_TRY(copy_in(buf.ptr, src, bytes, TP_PTR_HOST, st));
    *out = buf.ptr;
    return TP_OK;
}

}  // namespace

extern "C" {

void tp_params_default(tp_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->p = 6.0;
    p->theta = 0.0;
    p->leaf_size = 8;
    p->precision = TP_PREC_FP32;
    p->bh_diff_mode = TP_BH_DIFF_FULL;
    p->krylov_tol = 1e-6;
    p->krylov_max = 200;
    p->gmres_restart = 30;
    p->cg_tol = 1e-6;
    p->cg_max = 20000;
    p->armijo_c = 1e-4;
    p->armijo_shrink = 0.5;
    p->tau0 = 1.0;
    p->ls_max = 30;
    p->fixed_tau = 0;
    p->proj_iters = 1;
    p->poisson_solver = TP_POISSON_CHOLESKY;
    p->bvh_refit = 0;
    p->prec_self_weight = 24.0;
    p->tau0_disp = 0.0;
    p->tensor_cores = 0;
}

const char* tp_last_error(void) { return tp::last_error(); }

static int device_exists(int device) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= 64)
        return fail(TP_ERR_INVALID_ARG, "no such CUDA device");
    return TP_OK;
}

int tp_create(int device, tp_ctx** out) {
    set_error("");
    if (!out) return fail(TP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    TP_TRY(device_exists(device));
    tp_ctx* c = new tp_ctx();
    c->device = device;
    *out = c;
    return TP_OK;
}

int tp_destroy(tp_ctx* ctx) {
    set_error("");
    if (!ctx) return TP_OK;
    if (ctx->is_default) return fail(TP_ERR_INVALID_ARG, "the default context of a device is not destroyed");
    if (ctx->meshes.load() != 0)
        return fail(TP_ERR_INVALID_ARG, std::to_string(ctx->meshes.load()) + " mesh(es) of the context are alive");
    delete ctx;
    return TP_OK;
}

int tp_ctx_set_allocator(tp_ctx* ctx, const tp_allocator* a) {
    set_error("");
    if (!ctx) return fail(TP_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->is_default) return fail(TP_ERR_INVALID_ARG, "the default context keeps cudaMalloc; use tp_create");
    if (ctx->meshes.load() != 0)
        return fail(TP_ERR_INVALID_ARG, "the allocator cannot change while meshes of the context are alive");
    if (a && ((a->alloc == nullptr) != (a->free == nullptr)))
        return fail(TP_ERR_INVALID_ARG, "alloc and free must both be set or both be NULL");
    if (!a || !a->alloc) {
        ctx->custom = false;
        ctx->al = tp_allocator{};
    } else {
        ctx->custom = true;
        ctx->al = *a;
    }
    return TP_OK;
}

int tp_ctx_memory(const tp_ctx* ctx, size_t* in_use, size_t* peak) {
    set_error("");
    if (!ctx) return fail(TP_ERR_INVALID_ARG, "ctx is NULL");
    if (in_use) *in_use = (size_t)std::max(0LL, ctx->in_use.load());
    if (peak) *peak = (size_t)std::max(0LL, ctx->peak.load());
    return TP_OK;
}

int tp_mesh_create(int device, int nv, int nf, const double* pos, const int32_t* faces, int ptr_kind,
                   void* stream, tp_mesh** out) {
    set_error("");
    if (!out) return fail(TP_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    TP_TRY(device_exists(device));
    return tp_mesh_create_ctx(default_ctx(device), nv, nf, pos, faces, ptr_kind, stream, out);
}

int tp_mesh_create_ctx(tp_ctx* ctx, int nv, int nf, const double* pos, const int32_t* faces, int ptr_kind,
                       void* stream, tp_mesh** out) {
    set_error("");
    if (!ctx || !out || !pos || !faces) return fail(TP_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    TP_TRY(check_kind(ptr_kind));
    if (nv < 3 || nf < 1) return fail(TP_ERR_INVALID_ARG, "need nv >= 3 and nf >= 1");
    if ((long long)nf * 3 > (1LL << 30)) return fail(TP_ERR_INVALID_ARG, "too many faces");
    const int device = ctx->device;
    TP_TRY(device_exists(device));
    DeviceGuard g(device, ctx);
    if (!g.ok) return fail(TP_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    // faces on the host for validation and the incidence structures
    std::vector<int> F(3 * (size_t)nf);
    if (ptr_kind == TP_PTR_HOST)
        std::memcpy(F.data(), faces, sizeof(int) * 3 * (size_t)nf);
    else {
        TP_CUDA(cudaMemcpyAsync(F.data(), faces, sizeof(int) * 3 * (size_t)nf, cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
    }
    for (int S = 0; S < nf; ++S) {
        int a = F[3 * S], b = F[3 * S + 1], c = F[3 * S + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv)
            return fail(TP_ERR_INVALID_ARG, "face " + std::to_string(S) + " has a vertex index out of range");
        if (a == b || b == c || a == c)
            return fail(TP_ERR_INVALID_ARG, "face " + std::to_string(S) + " repeats a vertex");
    }
    // vertex -> (face*3+corner) incidence, sorted by face
    std::vector<int> vptr(nv + 1, 0), vidx(3 * (size_t)nf);
    for (int e = 0; e < 3 * nf; ++e) vptr[F[e] + 1]++;
    for (int v = 0; v < nv; ++v) vptr[v + 1] += vptr[v];
    {
        std::vector<int> fill(vptr.begin(), vptr.end() - 1);
        for (int e = 0; e < 3 * nf; ++e) vidx[fill[F[e]]++] = e;
    }
    tp_mesh* m = new tp_mesh();
    m->ctx = ctx;
    ctx->meshes++;
    m->device = device;
    m->nv = nv;
    m->nf = nf;
    auto bail = [&](int code) {
        tp_mesh_destroy(m);
        return code;
    };
    int s = TP_OK;
    if ((s = ensure(m->faces, sizeof(int) * 3 * (size_t)nf)) ||
        (s = ensure(m->vf_ptr, sizeof(int) * (nv + 1))) || (s = ensure(m->vf_idx, sizeof(int) * 3 * (size_t)nf)) ||
        (s = ensure(m->pos, sizeof(double) * 3 * (size_t)nv)) || (s = ensure(m->center, sizeof(double) * 4)) ||
        (s = ensure(m->errflag, sizeof(int) * 4)) || (s = ensure(m->f32a, sizeof(float4) * (size_t)nf)) ||
        (s = ensure(m->f32b, sizeof(float4) * (size_t)nf)) || (s = ensure(m->f32c, sizeof(float4) * (size_t)nf)) ||
        (s = ensure(m->f64a, sizeof(d4) * (size_t)nf)) ||
        (s = ensure(m->f64b, sizeof(d4) * (size_t)nf)) || (s = ensure(m->fgrad, sizeof(double) * 9 * (size_t)nf)))
        return bail(s);
    if (cudaMemcpy(m->faces.ptr, F.data(), sizeof(int) * 3 * (size_t)nf, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->vf_ptr.ptr, vptr.data(), sizeof(int) * (nv + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->vf_idx.ptr, vidx.data(), sizeof(int) * 3 * (size_t)nf, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(TP_ERR_CUDA, "copying the topology failed"));
    if ((s = components_setup(m, F))) return bail(s);
    if ((s = laplacian_setup(m))) return bail(s);
    if ((s = copy_in(m->pos.ptr, pos, sizeof(double) * 3 * (size_t)nv, ptr_kind, st))) return bail(s);
    if ((s = refresh_geometry(m, st))) return bail(s);
    *out = m;
    return TP_OK;
}

int tp_mesh_set_positions(tp_mesh* m, const double* pos, int ptr_kind, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_kind(ptr_kind));
    if (!pos) return fail(TP_ERR_INVALID_ARG, "pos is NULL");
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    TP_TRY(copy_in(m->pos.ptr, pos, sizeof(double) * 3 * (size_t)m->nv, ptr_kind, st));
    return refresh_geometry(m, st);
}

int tp_mesh_get_positions(tp_mesh* m, double* pos, int ptr_kind, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_kind(ptr_kind));
    if (!pos) return fail(TP_ERR_INVALID_ARG, "pos is NULL");
    DeviceGuard g(m);
    return copy_out(pos, m->pos.ptr, sizeof(double) * 3 * (size_t)m->nv, ptr_kind, (cudaStream_t)stream);
}

int tp_mesh_destroy(tp_mesh* m) {
    if (!m) return TP_OK;
    DeviceGuard g(m);
    Buf* all[] = {&m->faces, &m->vf_ptr, &m->vf_idx, &m->vcomp, &m->comp_ptr, &m->comp_verts, &m->pos, &m->center, &m->errflag, &m->f32a, &m->f32b,
                  &m->f32c, &m->tilebox,
                  &m->f64a, &m->f64b, &m->fgrad, &m->rowptr, &m->col, &m->cotsrc, &m->diagpos, &m->val,
                  &m->dinv, &m->val32, &m->gval, &m->wm, &m->bvh_node, &m->bvh_perm, &m->bvh_keys, &m->bvh_tmp, &m->bvh_sortws,
                  &m->bvh_f32a, &m->bvh_f32b, &m->bvh_f32c, &m->bh_apply_ws, &m->part, &m->part2, &m->tickets, &m->tcbuf, &m->tcerr, &m->scal, &m->corner,
                  &m->wv64, &m->wv32, &m->io_in, &m->io_out, &m->adj, &m->erow, &m->tlist, &m->rowsum,
                  &m->kry, &m->gsdev};
    for (Buf* b : all) release(*b);
    obstacle_release(m);
    pins_release(m);
    chol_release(m);
    release(m->bhcount);
    release(m->bhl_cnt);
    release(m->bhl_far);
    release(m->bhl_near);
    prof_release(m);
    for (auto& b : m->tmpv) release(b);
    for (auto& b : m->stepv) release(b);
    for (auto& b : m->prec) release(b);
    if (m->ctx) m->ctx->meshes--;
    delete m;
    return TP_OK;
}

size_t tp_mesh_footprint_bytes(int nv, int nf, const tp_params* p) {
    if (nv < 0 || nf < 0) return 0;
    const int restart = p ? std::max(1, std::min(60, p->gmres_restart)) : 30;
    size_t F = (size_t)nf, V = (size_t)nv;
    size_t geom = F * (12 + 4 + 16 + 16 + 32 + 32 + 72) + V * (24 + 4);
    // cotan CSR (pattern, values, FP32 copy), the preconditioner's within-face
    // term on the same pattern, and the connected-component tables
    size_t lap = (7 * V + F) * (4 + 8 + 8) + V * 16 + (7 * V) * 8 + V * 12;
    size_t bvh = F * (4 + 8 + 16 + 16 + 16) + F * 64;
    size_t nsplit = 16;
    size_t pairs = nsplit * F * 14 * 8 + F * (96 + 72 + 72 + 56 + 8);
    size_t krylov = (size_t)(2 * restart + 1) * 3 * V * 8;
    size_t vecs = 24 * 3 * V * 8;
    // sparse Cholesky (nested dissection on a surface: factor and update
    // matrices grow like V log V; about 190 floats per vertex at 10^4
    // vertices) plus its FP32 and FP64 solve vectors
    size_t chol = 0;
    if (!p || p->poisson_solver == TP_POISSON_CHOLESKY)
        chol = (size_t)(V * 4.0 * 24.0 * std::log2((double)V + 2.0)) + V * 9 * (4 * 3 + 8 * 3) + V * 64;
    return geom + lap + bvh + pairs + krylov + vecs + chol;
}

int tp_energy(tp_mesh* m, const tp_params* p, double* E_out, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_params(p));
    if (!E_out) return fail(TP_ERR_INVALID_ARG, "E_out is NULL");
    DeviceGuard g(m);
    return energy_value(m, p, E_out, (cudaStream_t)stream);
}

int tp_energy_rows(tp_mesh* m, const tp_params* p, const int32_t* targets, int n, double* rows, int ptr_kind,
                   void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_params(p));
    TP_TRY(check_kind(ptr_kind));
    if (n < 0 || (n > 0 && (!targets || !rows))) return fail(TP_ERR_INVALID_ARG, "bad targets/rows");
    if (n == 0) return TP_OK;
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    if (ptr_kind == TP_PTR_HOST)
        for (int i = 0; i < n; ++i)
            if (targets[i] < 0 || targets[i] >= m->nf) return fail(TP_ERR_INVALID_ARG, "target index out of range");
    const void* tl = nullptr;
    TP_TRY(stage_in(m->tlist, targets, sizeof(int) * (size_t)n, ptr_kind, st, &tl));
    TP_TRY(ensure(m->io_out, sizeof(double) * (size_t)n));
    double* out = ptr_kind == TP_PTR_DEVICE ? rows : m->io_out.as<double>();
    if (p->theta > 0.0)
        TP_TRY(energy_rows_bh(m, p, (const int32_t*)tl, n, out, st));
    else
        TP_TRY(energy_rows_direct(m, p, (const int32_t*)tl, n, out, st));
    if (ptr_kind == TP_PTR_HOST) TP_TRY(copy_out(rows, out, sizeof(double) * (size_t)n, TP_PTR_HOST, st));
    return TP_OK;
}

int tp_differential(tp_mesh* m, const tp_params* p, double* dE, int ptr_kind, double* E_out, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_params(p));
    TP_TRY(check_kind(ptr_kind));
    if (!dE) return fail(TP_ERR_INVALID_ARG, "dE is NULL");
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = sizeof(double) * 3 * (size_t)m->nv;
    TP_TRY(ensure(m->io_out, bytes));
    double* out = ptr_kind == TP_PTR_DEVICE ? dE : m->io_out.as<double>();
    TP_TRY(differential_dev(m, p, out, E_out, st));
    if (ptr_kind == TP_PTR_HOST) TP_TRY(copy_out(dE, out, bytes, TP_PTR_HOST, st));
    return TP_OK;
}

int fractional_apply(tp_mesh* m, const tp_params* p, int op, const double* v, int k, double* y, int ptr_kind,
                     void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_params(p));
    TP_TRY(check_kind(ptr_kind));
    if (op < TP_OP_A || op > TP_OP_L) return fail(TP_ERR_INVALID_ARG, "unknown operator");
    if (k < 1 || k > 9) return fail(TP_ERR_INVALID_ARG, "k must be in 1..9");
    if (!v || !y) return fail(TP_ERR_INVALID_ARG, "NULL vector");
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = sizeof(double) * (size_t)m->nv * k;
    const void* vin = nullptr;
    TP_TRY(stage_in(m->io_in, v, bytes, ptr_kind, st, &vin));
    TP_TRY(ensure(m->io_out, bytes));
    double* out = ptr_kind == TP_PTR_DEVICE ? y : m->io_out.as<double>();
    TP_TRY(apply_op(m, p, op, (const double*)vin, k, out, st));
    if (ptr_kind == TP_PTR_HOST) TP_TRY(copy_out(y, out, bytes, TP_PTR_HOST, st));
    return TP_OK;
}

int cotan_solve(tp_mesh* m, const tp_params* p, const double* b, int k, double* z, int ptr_kind, void* stream,
                int* iters_out) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_params(p));
    TP_TRY(check_kind(ptr_kind));
    if (k < 1 || k > 9) return fail(TP_ERR_INVALID_ARG, "k must be in 1..9");
    if (!b || !z) return fail(TP_ERR_INVALID_ARG, "NULL vector");
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = sizeof(double) * (size_t)m->nv * k;
    const void* bin = nullptr;
    TP_TRY(stage_in(m->io_in, b, bytes, ptr_kind, st, &bin));
    TP_TRY(ensure(m->io_out, bytes));
    double* out = ptr_kind == TP_PTR_DEVICE ? z : m->io_out.as<double>();
    int it = 0;
    int s = m->npins ? pinned_solve(m, p, (const double*)bin, k, out, st, &it)
                     : cg_solve(m, p, (const double*)bin, k, out, st, &it);
    if (iters_out) *iters_out = it;
    if (s != TP_OK) return s;
    if (ptr_kind == TP_PTR_HOST) TP_TRY(copy_out(z, out, bytes, TP_PTR_HOST, st));
    return TP_OK;
}

int cotan_factor_info(tp_mesh* m, tp_chol_info* out) {
    set_error("");
    TP_TRY(check_mesh(m));
    if (!out) return fail(TP_ERR_INVALID_ARG, "out is NULL");
    DeviceGuard g(m);
    return chol_info(m, out);
}

int precond_apply(tp_mesh* m, const tp_params* p, const double* b, int k, double* z, int ptr_kind, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_params(p));
    TP_TRY(check_kind(ptr_kind));
    if (k < 1 || k > 9) return fail(TP_ERR_INVALID_ARG, "k must be in 1..9");
    if (!b || !z) return fail(TP_ERR_INVALID_ARG, "NULL vector");
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = sizeof(double) * (size_t)m->nv * k;
    const void* bin = nullptr;
    TP_TRY(stage_in(m->io_in, b, bytes, ptr_kind, st, &bin));
    TP_TRY(ensure(m->io_out, bytes));
    double* out = ptr_kind == TP_PTR_DEVICE ? z : m->io_out.as<double>();
    TP_TRY(precond_apply_dev(m, p, (const double*)bin, k, out, st, nullptr));
    if (ptr_kind == TP_PTR_HOST) TP_TRY(copy_out(z, out, bytes, TP_PTR_HOST, st));
    return TP_OK;
}

int precond_step(tp_mesh* m, const tp_params* p, const tp_constraints* c, tp_step_report* rep, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_params(p));
    if (!c) return fail(TP_ERR_INVALID_ARG, "constraints is NULL");
    if (c->flags & ~(TP_CONSTRAINT_AREA | TP_CONSTRAINT_VOLUME | TP_CONSTRAINT_FREE_BARYCENTER))
        return fail(TP_ERR_INVALID_ARG, "unknown constraint flag");
    if ((c->flags & TP_CONSTRAINT_FREE_BARYCENTER) && m->npins)
        return fail(TP_ERR_INVALID_ARG, "a free barycenter cannot be combined with pins");
    if (p->krylov_max < 1 || p->cg_max < 1 || p->ls_max < 1 || p->proj_iters < 0 || p->proj_iters > 100 ||
        !(p->armijo_shrink > 0.0 && p->armijo_shrink < 1.0))
        return fail(TP_ERR_INVALID_ARG, "bad solver parameters");
    DeviceGuard g(m);
    return precond_step_dev(m, p, c, rep, (cudaStream_t)stream);
}

int tp_mesh_area_volume(tp_mesh* m, double* area, double* volume, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    if (!area && !volume) return fail(TP_ERR_INVALID_ARG, "area and volume are both NULL");
    DeviceGuard g(m);
    double v[2] = {0.0, 0.0};
    TP_TRY(area_volume(m, v, (cudaStream_t)stream));
    if (area) *area = v[0];
    if (volume) *volume = v[1];
    return TP_OK;
}

int tp_obstacle_set(tp_mesh* m, int nv, int nf, const double* pos, const int32_t* faces, double weight,
                    int ptr_kind, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_kind(ptr_kind));
    if (nf < 0 || nv < 0) return fail(TP_ERR_INVALID_ARG, "negative obstacle size");
    if (!std::isfinite(weight) || weight < 0.0) return fail(TP_ERR_INVALID_ARG, "weight must be finite and >= 0");
    DeviceGuard g(m);
    if (!g.ok) return fail(TP_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    if (nf == 0) {
        TP_CUDA(cudaStreamSynchronize(st));
        obstacle_release(m);
        return TP_OK;
    }
    tp_mesh* o = nullptr;
    TP_TRY(tp_mesh_create_ctx(m->ctx, nv, nf, pos, faces, ptr_kind, stream, &o));
    TP_CUDA(cudaStreamSynchronize(st));
    TP_TRY(obstacle_attach(m, o, weight, st));
    TP_CUDA(cudaStreamSynchronize(st));
    return TP_OK;
}

int tp_willmore_set(tp_mesh* m, double weight) {
    set_error("");
    TP_TRY(check_mesh(m));
    if (!std::isfinite(weight) || weight < 0.0) return fail(TP_ERR_INVALID_ARG, "weight must be finite and >= 0");
    m->willmore_w = weight;
    return TP_OK;
}

int tp_willmore_energy(tp_mesh* m, double* E_out, double* dE, int ptr_kind, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_kind(ptr_kind));
    if (!E_out && !dE) return fail(TP_ERR_INVALID_ARG, "E_out and dE are both NULL");
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    TP_TRY(ensure(m->rowsum, sizeof(double) * 8));
    const size_t bytes = sizeof(double) * 3 * (size_t)m->nv;
    double* out = nullptr;
    if (dE) {
        TP_TRY(ensure(m->io_out, bytes));
        out = ptr_kind == TP_PTR_DEVICE ? dE : m->io_out.as<double>();
        TP_CUDA(cudaMemsetAsync(out, 0, bytes, st));
    }
    TP_TRY(willmore_eval(m, E_out ? m->rowsum.as<double>() + 1 : nullptr, out, 1.0, st));
    if (dE && ptr_kind == TP_PTR_HOST) TP_TRY(copy_out(dE, out, bytes, TP_PTR_HOST, st));
    if (E_out) {
        TP_CUDA(cudaMemcpyAsync(E_out, m->rowsum.as<double>() + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
    }
    return TP_OK;
}

int tp_pins_set(tp_mesh* m, int n, const int32_t* vertices, int ptr_kind, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_kind(ptr_kind));
    if (n < 0 || n > TP_MAX_PINS) return fail(TP_ERR_INVALID_ARG, "n must be in 0..TP_MAX_PINS");
    if (n > 0 && !vertices) return fail(TP_ERR_INVALID_ARG, "vertices is NULL");
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> idx(n);
    if (n > 0) {
        if (ptr_kind == TP_PTR_HOST) {
            std::memcpy(idx.data(), vertices, sizeof(int) * (size_t)n);
        } else {
            TP_CUDA(cudaMemcpyAsync(idx.data(), vertices, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, st));
            TP_CUDA(cudaStreamSynchronize(st));
        }
    }
    return pins_set(m, n, idx.data(), st);
}

int tp_obstacle_energy(tp_mesh* m, const tp_params* p, double* E_out, double* dE, int ptr_kind, void* stream) {
    set_error("");
    TP_TRY(check_mesh(m));
    TP_TRY(check_params(p));
    TP_TRY(check_kind(ptr_kind));
    if (!m->obs) return fail(TP_ERR_INVALID_ARG, "no obstacle is set on this mesh");
    DeviceGuard g(m);
    cudaStream_t st = (cudaStream_t)stream;
    TP_TRY(ensure(m->erow, sizeof(double) * m->nf));
    TP_TRY(ensure(m->rowsum, sizeof(double) * 8));
    if (dE) {
        TP_TRY(ensure(m->adj, sizeof(double) * 7 * (size_t)m->nf));
        TP_TRY(obstacle_terms(m, p, true, false, m->erow.as<double>(), m->adj.as<double>(), st));
        const size_t bytes = sizeof(double) * 3 * (size_t)m->nv;
        TP_TRY(ensure(m->io_out, bytes));
        double* out = ptr_kind == TP_PTR_DEVICE ? dE : m->io_out.as<double>();
        TP_TRY(adjoints_to_dE(m, m->adj.as<double>(), out, st));
        if (ptr_kind == TP_PTR_HOST) TP_TRY(copy_out(dE, out, bytes, TP_PTR_HOST, st));
    } else {
        TP_TRY(obstacle_terms(m, p, false, false, m->erow.as<double>(), nullptr, st));
    }
    if (E_out) {
        TP_TRY(sum_f64(m->erow.as<double>(), m->nf, m->rowsum.as<double>(), m, st));
        TP_CUDA(cudaMemcpyAsync(E_out, m->rowsum.ptr, sizeof(double), cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
    }
    return TP_OK;
}

int tp_profile_enable(tp_mesh* m, int on) {
    set_error("");
    TP_TRY(check_mesh(m));
    m->prof.on = on != 0;
    return TP_OK;
}

int tp_profile_read(tp_mesh* m, tp_kernel_stat* out, int max, int* n) {
    set_error("");
    TP_TRY(check_mesh(m));
    if (!n || (max > 0 && !out)) return fail(TP_ERR_INVALID_ARG, "NULL output");
    DeviceGuard g(m);
    static const char* names[PK_COUNT] = {"energy_direct", "diff_direct", "apply_A", "apply_B", "apply_B0",
                                          "apply_L", "bh_energy", "bh_diff", "bvh_build", "cg",
                                          "chol_factor", "chol_solve", "bh_apply", "obstacle_direct",
                                          "bh_obstacle"};
    Profiler& P = m->prof;
    for (auto& pe : P.pending) {
        float ms = 0.f;
        TP_CUDA(cudaEventSynchronize(pe.second.second));
        TP_CUDA(cudaEventElapsedTime(&ms, pe.second.first, pe.second.second));
        P.ms[pe.first] += ms;
        P.pool.push_back(pe.second.first);
        P.pool.push_back(pe.second.second);
    }
    P.pending.clear();
    unsigned long long bh[BH_NCOUNT];
    TP_TRY(bh_counts_read(m, bh, true, nullptr));
    P.units[PK_BH_ENERGY] += (double)bh[0];
    P.units[PK_BH_DIFF] += (double)bh[1];
    P.units[PK_BH_APPLY] += (double)bh[2];
    P.units[PK_BH_OBSTACLE] += (double)bh[3];
    int k = 0;
    for (int i = 0; i < PK_COUNT && k < max; ++i) {
        if (P.launches[i] == 0) continue;
        std::memset(out[k].name, 0, sizeof(out[k].name));
        std::strncpy(out[k].name, names[i], sizeof(out[k].name) - 1);
        out[k].launches = P.launches[i];
        out[k].ms = P.ms[i];
        out[k].units = P.units[i];
        out[k].columns = P.cols[i];
        ++k;
    }
    *n = k;
    for (int i = 0; i < PK_COUNT; ++i) {
        P.launches[i] = 0;
        P.ms[i] = 0.0;
        P.units[i] = 0.0;
        P.cols[i] = 0.0;
    }
    return TP_OK;
}

unsigned long long tp_launch_count(void) { return tp::launch_count(); }

int tp_selftest_wait(int device, int* timed_out) {
    set_error("");
    if (!timed_out) return fail(TP_ERR_INVALID_ARG, "timed_out is NULL");
    *timed_out = 0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(TP_ERR_INVALID_ARG, "no such CUDA device");
    DeviceGuard g(device);
    if (!g.ok) return fail(TP_ERR_CUDA, "cudaSetDevice failed");
    return wait_selftest(timed_out);
}

}  // extern "C"
