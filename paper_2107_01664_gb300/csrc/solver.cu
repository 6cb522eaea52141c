// Device-resident orchestration of the descent step (§5.4):
//   energy and differential (direct or Barnes-Hut),
//   the preconditioner C^+ L^{2-s} C^+ (§5.2),
//   flexible GMRES on A_3 in the mean-zero subspace (§5, §5.4 step 3a),
//   the Schur-complement direction and correction (§5.3, Eq. 17-19),
//   Armijo line search and the corrective projection (§3.3.2).
// All solver vectors are FP64 [nv][3] on the device; only the small
// Hessenberg / Schur systems live on the host.
#include <cmath>
#include <vector>

#include "tp_internal.cuh"

namespace tp {

// ---------------------------------------------------------------------------
// energy / differential dispatch
// ---------------------------------------------------------------------------

int energy_value(tp_mesh* m, const tp_params* p, double* E_host, cudaStream_t st, bool aux) {
    TP_TRY(ensure(m->erow, sizeof(double) * m->nf));
    TP_TRY(ensure(m->rowsum, sizeof(double) * 8));
    if (p->theta > 0.0)
        TP_TRY(energy_rows_bh(m, p, nullptr, m->nf, m->erow.as<double>(), st));
    else
        TP_TRY(energy_rows_direct(m, p, nullptr, m->nf, m->erow.as<double>(), st));
    if (aux) TP_TRY(obstacle_terms(m, p, false, true, m->erow.as<double>(), nullptr, st));
    TP_TRY(sum_f64(m->erow.as<double>(), m->nf, m->rowsum.as<double>(), m, st));
    const bool wm = aux && m->willmore_w > 0.0;
    if (wm) TP_TRY(willmore_eval(m, m->rowsum.as<double>() + 1, nullptr, 0.0, st));
    double r[2] = {0.0, 0.0};
    TP_CUDA(cudaMemcpyAsync(r, m->rowsum.ptr, sizeof(double) * (wm ? 2 : 1), cudaMemcpyDeviceToHost, st));
    TP_CUDA(cudaStreamSynchronize(st));
    *E_host = r[0] + (wm ? m->willmore_w * r[1] : 0.0);
    return TP_OK;
}

int differential_dev(tp_mesh* m, const tp_params* p, double* dE, double* E_host, cudaStream_t st,
                     bool aux) {
    TP_TRY(ensure(m->adj, sizeof(double) * 7 * (size_t)m->nf));
    TP_TRY(ensure(m->erow, sizeof(double) * m->nf));
    if (p->theta > 0.0)
        TP_TRY(diff_adjoints_bh(m, p, m->adj.as<double>(), m->erow.as<double>(), st));
    else
        TP_TRY(diff_adjoints_direct(m, p, m->adj.as<double>(), m->erow.as<double>(), st));
    if (aux)
        TP_TRY(obstacle_terms(m, p, true, true, m->erow.as<double>(), m->adj.as<double>(), st));
    TP_TRY(adjoints_to_dE(m, m->adj.as<double>(), dE, st));
    TP_TRY(ensure(m->rowsum, sizeof(double) * 8));
    const bool wm = aux && m->willmore_w > 0.0;
    if (wm) TP_TRY(willmore_eval(m, m->rowsum.as<double>() + 1, dE, m->willmore_w, st));
    if (E_host) {
        TP_TRY(sum_f64(m->erow.as<double>(), m->nf, m->rowsum.as<double>(), m, st));
        double r[2] = {0.0, 0.0};
        TP_CUDA(cudaMemcpyAsync(r, m->rowsum.ptr, sizeof(double) * (wm ? 2 : 1), cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
        *E_host = r[0] + (wm ? m->willmore_w * r[1] : 0.0);
    }
    return TP_OK;
}

// z = C^+ L^{2-s} C^+ b (§5.2); b, z [nv][k] device
// With strict = false (inside flexible GMRES) an inner CG solve that stops at
// its iteration cap still returns its iterate: the outer method only needs
// some fixed-quality approximation of the preconditioner.
int precond_apply_dev(tp_mesh* m, const tp_params* p, const double* b, int k, double* z,
                      cudaStream_t st, int* cg_iters, bool strict) {
    const size_t n = (size_t)m->nv * k;
    TP_TRY(ensure(m->prec[0], sizeof(double) * n));
    TP_TRY(ensure(m->prec[1], sizeof(double) * n));
    int it1 = 0, it2 = 0;
    // with pins the pin rows are appended to both Laplacians (§7.2)
    // inside flexible GMRES (strict = false) the factorised solves run
    // deferred: no host read per solve; the step reads their flags once
    auto solve = [&](const double* rhs, double* out, int* it) {
        return m->npins ? pinned_solve(m, p, rhs, k, out, st, it) : cg_solve(m, p, rhs, k, out, st, it, !strict);
    };
    int s1 = solve(b, m->prec[0].as<double>(), &it1);
    if (s1 != TP_OK && (strict || s1 != TP_ERR_NOT_CONVERGED)) return s1;
    // (the second solve projects its right-hand side itself, or ignores its pinned rows)
    TP_TRY(apply_op(m, p, TP_OP_L, m->prec[0].as<double>(), k, m->prec[1].as<double>(), st));
    TP_TRY(self_term_add(m, p, m->prec[0].as<double>(), k, m->prec[1].as<double>(), st));
    int s2 = solve(m->prec[1].as<double>(), z, &it2);
    if (s2 != TP_OK && (strict || s2 != TP_ERR_NOT_CONVERGED)) return s2;
    if (cg_iters) *cg_iters += it1 + it2;
    return TP_OK;
}

// ---------------------------------------------------------------------------
// flexible GMRES(m), right preconditioning, on the mean-zero subspace, for up
// to three right-hand sides in lockstep
// ---------------------------------------------------------------------------
//
// The Schur step needs A_3 solves with g and with the rows of dPhi (Eq. 17,
// 18). The systems keep separate Krylov spaces, Hessenberg matrices and
// restarts, but every preconditioner application (two CG solves and one
// L^{2-s} product) and every A product is done once for all active systems,
// on their vectors packed side by side as [nv][3 * nsys] columns.

struct KrylovStats {
    int iters = 0, cg_iters = 0;
};

constexpr int MAXSYS = 3;

struct SysPtrs {
    double* p[MAXSYS];
};

// dst[v][3*s + c] = src_s[v][c] for the ns systems listed
__global__ void k_pack(SysPtrs src, int ns, int nv, double* __restrict__ dst) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)nv * 3 * ns;
    if (i >= n) return;
    int w = 3 * ns;
    size_t v = i / w;
    int r = (int)(i % w), sI = r / 3, c = r % 3;
    dst[i] = src.p[sI][v * 3 + c];
}

__global__ void k_unpack(const double* __restrict__ srcp, int ns, int nv, SysPtrs dst) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)nv * 3 * ns;
    if (i >= n) return;
    int w = 3 * ns;
    size_t v = i / w;
    int r = (int)(i % w), sI = r / 3, c = r % 3;
    dst.p[sI][v * 3 + c] = srcp[i];
}

static int pack(const std::vector<double*>& src, int nv, double* dst, cudaStream_t st) {
    SysPtrs sp{};
    for (size_t i = 0; i < src.size(); ++i) sp.p[i] = src[i];
    size_t n = (size_t)nv * 3 * src.size();
    k_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sp, (int)src.size(), nv, dst);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

static int unpack(const double* srcp, int nv, const std::vector<double*>& dst, cudaStream_t st) {
    SysPtrs sp{};
    for (size_t i = 0; i < dst.size(); ++i) sp.p[i] = dst[i];
    size_t n = (size_t)nv * 3 * dst.size();
    k_unpack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(srcp, (int)dst.size(), nv, sp);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

// y = A v on packed columns (plus w C M^-1 C v with a Willmore weight w, the
// H^2 term of §7.3.5), projected to the step's subspace
static int apply_A_packed(tp_mesh* m, const tp_params* p, const double* v, int k, double* y, cudaStream_t st) {
    TP_TRY(apply_op(m, p, TP_OP_A, v, k, y, st));
    if (m->willmore_w > 0.0) TP_TRY(willmore_operator_add(m, v, k, y, m->willmore_w, st));
    return project_space(m, y, k, st);
}

// dst_s[v][c] = y[v][3 s + c] - mean[3 s + c] (the mean-zero projection of a
// one-component mesh fused with the unpacking of the lockstep systems)
__global__ void k_sub_mean_unpack(const double* __restrict__ y, const double* __restrict__ mean, int ns, int nv,
                                  SysPtrs dst) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int w = 3 * ns;
    if (i >= (size_t)nv * w) return;
    const size_t v = i / w;
    const int r = (int)(i % w), sI = r / 3, c = r % 3;
    dst.p[sI][v * 3 + c] = y[i] - mean[r];
}

// apply_A_packed, its result unpacked into the systems' vectors (y is scratch)
static int apply_A_unpacked(tp_mesh* m, const tp_params* p, const double* v, int ns, double* y,
                            const std::vector<double*>& dst, cudaStream_t st) {
    const int k = 3 * ns;
    if (m->npins != 0 || m->ncomp != 1) {
        TP_TRY(apply_A_packed(m, p, v, k, y, st));
        return unpack(y, m->nv, dst, st);
    }
    TP_TRY(apply_op(m, p, TP_OP_A, v, k, y, st));
    if (m->willmore_w > 0.0) TP_TRY(willmore_operator_add(m, v, k, y, m->willmore_w, st));
    TP_TRY(ensure(m->tmpv[6], sizeof(double) * 64));
    double* mean = m->tmpv[6].as<double>();
    TP_TRY(colsum(m, y, m->nv, k, 1.0 / m->nv, mean, st));
    SysPtrs sp{};
    for (size_t i = 0; i < dst.size(); ++i) sp.p[i] = dst[i];
    const size_t n = (size_t)m->nv * k;
    k_sub_mean_unpack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, mean, ns, m->nv, sp);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

struct GmSys {
    double* b;
    double* x;
    double* V;   // (mr+1) basis vectors
    double* Z;   // mr preconditioned vectors
    double* w;
    double bnorm = 0.0, beta = 0.0;
    bool active = true, converged = false;
    int iters = 0;
    std::vector<double> H, cs, sn, g;
};

static int fgmres_multi(tp_mesh* m, const tp_params* p, int ns, const double* const* b, double* const* x,
                        cudaStream_t st, KrylovStats* ks, int* status) {
    const int mr = p->gmres_restart < 1 ? 1 : (p->gmres_restart > 60 ? 60 : p->gmres_restart);
    const int nv = m->nv;
    const size_t n = (size_t)nv * 3;
    // per system: V (mr+1), Z (mr), w; shared: three packed [nv][3*ns] buffers
    const size_t per = (size_t)(2 * mr + 2) * n;
    TP_TRY(ensure(m->kry, sizeof(double) * (per * ns + 3 * n * ns)));
    double* base = m->kry.as<double>();
    double* P0 = base + per * ns;
    double* P1 = P0 + n * ns;
    double* P2 = P1 + n * ns;
    std::vector<GmSys> S(ns);
    for (int i = 0; i < ns; ++i) {
        GmSys& q = S[i];
        q.b = const_cast<double*>(b[i]);
        q.x = x[i];
        q.V = base + per * i;
        q.Z = q.V + (size_t)(mr + 1) * n;
        q.w = q.Z + (size_t)mr * n;
        q.H.assign((mr + 1) * mr, 0.0);
        q.cs.assign(mr, 0.0);
        q.sn.assign(mr, 0.0);
        q.g.assign(mr + 1, 0.0);
        status[i] = TP_OK;
        TP_CUDA(cudaMemsetAsync(q.x, 0, sizeof(double) * n, st));
        TP_CUDA(cudaMemcpyAsync(q.V, q.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        TP_TRY(project_space(m, q.V, 3, st));
        double bn2;
        const double* xs[1] = {q.V};
        TP_TRY(dots(m, xs, q.V, 1, n, &bn2, st));
        q.bnorm = q.beta = std::sqrt(bn2);
        if (q.bnorm == 0.0) {
            q.active = false;
            q.converged = true;
        }
    }
    auto Vj = [&](GmSys& q, int j) { return q.V + (size_t)j * n; };
    auto Zj = [&](GmSys& q, int j) { return q.Z + (size_t)j * n; };
    int total = 0;
    for (;;) {
        std::vector<int> act;
        for (int i = 0; i < ns; ++i)
            if (S[i].active) act.push_back(i);
        if (act.empty() || total >= p->krylov_max) break;
        // start of a cycle: normalise r into V_0
        for (int i : act) {
            GmSys& q = S[i];
            double sc = 1.0 / q.beta;
            const double* xs[1] = {q.V};
            TP_TRY(lincomb(q.V, xs, &sc, 1, n, 0.0, st));
            std::fill(q.g.begin(), q.g.end(), 0.0);
            q.g[0] = q.beta;
        }
        std::vector<int> jlen(ns, 0);
        std::vector<int> cyc = act;
        for (int j = 0; j < mr && !cyc.empty() && total < p->krylov_max; ++j) {
            const int na = (int)cyc.size();
            std::vector<double*> vin, zout, wout;
            for (int i : cyc) {
                vin.push_back(Vj(S[i], j));
                zout.push_back(Zj(S[i], j));
                wout.push_back(S[i].w);
            }
            TP_TRY(pack(vin, nv, P0, st));
            TP_TRY(precond_apply_dev(m, p, P0, 3 * na, P1, st, &ks->cg_iters, false));
            TP_TRY(unpack(P1, nv, zout, st));
            TP_TRY(apply_A_unpacked(m, p, P1, na, P2, wout, st));
            ++total;
            std::vector<int> still;
            // classical Gram-Schmidt, twice, for all systems of the cycle at
            // once: pass 1 h = V^T w; pass 2 h2 = V^T w' together with |w'|^2,
            // so |w''|^2 = |w'|^2 - |h2|^2 (V orthonormal); two host syncs
            std::vector<const double*> dx, dy;
            for (int i : cyc)
                for (int l = 0; l <= j; ++l) {
                    dx.push_back(Vj(S[i], l));
                    dy.push_back(S[i].w);
                }
            std::vector<double> h1(dx.size()), h2(dx.size() + cyc.size());
            // pass 1 stays on the device (coefficients read by the kernel);
            // its dots reach the host with pass 2's, one synchronisation
            TP_TRY(ensure(m->gsdev, sizeof(double) * 1024));
            double* h1dev = m->gsdev.as<double>();
            TP_TRY(dot_pairs_dev(m, dx.data(), dy.data(), (int)dx.size(), n, h1dev, st));
            std::vector<double*> ws;
            std::vector<const double*> wc, basis_all;
            for (int i : cyc) {
                ws.push_back(S[i].w);
                wc.push_back(S[i].w);
                for (int l = 0; l <= j; ++l) basis_all.push_back(Vj(S[i], l));
            }
            // w -= V h1 for every system of the cycle, one launch
            TP_TRY(lincomb_sys(na, ws.data(), wc.data(), basis_all.data(), j + 1, h1dev, nullptr, nullptr, 1.0, n,
                               st));
            TP_CUDA(cudaMemcpyAsync(h1.data(), h1dev, sizeof(double) * h1.size(), cudaMemcpyDeviceToHost, st));
            for (int i : cyc) {
                dx.push_back(S[i].w);
                dy.push_back(S[i].w);
            }
            TP_TRY(dot_pairs(m, dx.data(), dy.data(), (int)dx.size(), n, h2.data(), st));
            // pass 2 and the normalisation V_{j+1} = (w - V h2) / |w - V h2| of every system in
            // one launch, |w''|^2 from the dots; a system near breakdown measures |w''| directly
            std::vector<double> hn_of(na, 0.0), neg_all((size_t)na * (j + 1)), sc_all(na, 1.0);
            std::vector<char> near_bd(na, 0);
            bool direct = false;
            for (int ii = 0; ii < na; ++ii) {
                const double* hh = h2.data() + ii * (j + 1);
                double hh2 = 0.0;
                for (int l = 0; l <= j; ++l) {
                    neg_all[(size_t)ii * (j + 1) + l] = -hh[l];
                    hh2 += hh[l] * hh[l];
                }
                const double ww = h2[(size_t)na * (j + 1) + ii];
                hn_of[ii] = ww - hh2;
                if (!(hn_of[ii] > 1e-6 * ww)) near_bd[ii] = 1, direct = true;
            }
            std::vector<double*> vnext;
            for (int i : cyc) vnext.push_back(Vj(S[i], j + 1));
            if (direct) {
                // w'' stored first, then |w''|^2 measured for the systems near breakdown
                TP_TRY(lincomb_sys(na, ws.data(), wc.data(), basis_all.data(), j + 1, nullptr, neg_all.data(),
                                   nullptr, 1.0, n, st));
                for (int ii = 0; ii < na; ++ii)
                    if (near_bd[ii]) {
                        const double* xs[1] = {S[cyc[ii]].w};
                        TP_TRY(dots(m, xs, S[cyc[ii]].w, 1, n, &hn_of[ii], st));
                    }
            }
            for (int ii = 0; ii < na; ++ii) {
                const double hn = std::sqrt(std::max(0.0, hn_of[ii]));
                hn_of[ii] = hn;
                sc_all[ii] = hn > 0.0 ? 1.0 / hn : 0.0;
            }
            if (direct)
                TP_TRY(lincomb_sys(na, vnext.data(), wc.data(), basis_all.data(), 0, nullptr, nullptr, sc_all.data(),
                                   1.0, n, st));
            else
                TP_TRY(lincomb_sys(na, vnext.data(), wc.data(), basis_all.data(), j + 1, nullptr, neg_all.data(),
                                   sc_all.data(), 1.0, n, st));
            for (size_t ii = 0; ii < cyc.size(); ++ii) {
                const int i = cyc[ii];
                GmSys& q = S[i];
                const double* hh = h2.data() + ii * (j + 1);
                for (int l = 0; l <= j; ++l) q.H[l * mr + j] = h1[ii * (j + 1) + l] + hh[l];
                const double hn = hn_of[ii];
                q.H[(j + 1) * mr + j] = hn;
                for (int l = 0; l < j; ++l) {  // Givens rotations
                    double a = q.H[l * mr + j], c = q.H[(l + 1) * mr + j];
                    q.H[l * mr + j] = q.cs[l] * a + q.sn[l] * c;
                    q.H[(l + 1) * mr + j] = -q.sn[l] * a + q.cs[l] * c;
                }
                double a = q.H[j * mr + j], c = q.H[(j + 1) * mr + j];
                double r = std::hypot(a, c);
                q.cs[j] = r > 0.0 ? a / r : 1.0;
                q.sn[j] = r > 0.0 ? c / r : 0.0;
                q.H[j * mr + j] = r;
                q.H[(j + 1) * mr + j] = 0.0;
                q.g[j + 1] = -q.sn[j] * q.g[j];
                q.g[j] = q.cs[j] * q.g[j];
                q.iters++;
                jlen[i] = j + 1;
                double rel = std::fabs(q.g[j + 1]) / q.bnorm;
                if (rel <= p->krylov_tol || hn == 0.0) {
                    q.converged = true;
                    q.active = false;
                } else {
                    still.push_back(i);
                }
            }
            cyc = still;
        }
        // x += Z y with H y = g (upper triangular, size jlen)
        for (int i : act) {
            GmSys& q = S[i];
            int J = jlen[i];
            std::vector<double> y(J);
            for (int l = J - 1; l >= 0; --l) {
                double sum = q.g[l];
                for (int t = l + 1; t < J; ++t) sum -= q.H[l * mr + t] * y[t];
                y[l] = q.H[l * mr + l] != 0.0 ? sum / q.H[l * mr + l] : 0.0;
            }
            std::vector<const double*> zs(J);
            for (int l = 0; l < J; ++l) zs[l] = Zj(q, l);
            if (J > 0) TP_TRY(lincomb(q.x, zs.data(), y.data(), J, n, 1.0, st));
        }
        // restart the unconverged systems from their true residuals r = b - A x
        std::vector<int> rest;
        for (int i : act)
            if (S[i].active) rest.push_back(i);
        if (rest.empty() || total >= p->krylov_max) break;
        std::vector<double*> xin, rout;
        for (int i : rest) {
            xin.push_back(S[i].x);
            rout.push_back(S[i].w);
        }
        TP_TRY(pack(xin, nv, P0, st));
        TP_TRY(apply_A_unpacked(m, p, P0, (int)rest.size(), P2, rout, st));
        for (int i : rest) {
            GmSys& q = S[i];
            const double* xs[2] = {q.b, q.w};
            double cf[2] = {1.0, -1.0};
            TP_TRY(lincomb(q.V, xs, cf, 2, n, 0.0, st));
            TP_TRY(project_space(m, q.V, 3, st));
            double rn2;
            const double* x1[1] = {q.V};
            TP_TRY(dots(m, x1, q.V, 1, n, &rn2, st));
            q.beta = std::sqrt(rn2);
            if (q.beta / q.bnorm <= p->krylov_tol) {
                q.active = false;
                q.converged = true;
            }
        }
    }
    ks->iters += total;
    for (int i = 0; i < ns; ++i) {
        TP_TRY(project_space(m, S[i].x, 3, st));
        if (!S[i].converged) status[i] = TP_ERR_NOT_CONVERGED;
    }
    return TP_OK;
}

// ---------------------------------------------------------------------------
// constraints (§7.1.3 area, §7.1.4 volume): values and gradients
// ---------------------------------------------------------------------------

// per face: area, volume term; per corner: area and volume gradients
__global__ void k_constraint_terms(const double* __restrict__ pos, const int* __restrict__ faces, int nf,
                                   double* __restrict__ fterm /* [nf][2] */,
                                   double* __restrict__ cga /* [nf*3][3] */,
                                   double* __restrict__ cgv /* [nf*3][3] */) {
    int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S >= nf) return;
    int id[3] = {faces[3 * S], faces[3 * S + 1], faces[3 * S + 2]};
    double P[3][3];
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 3; ++q) P[c][q] = pos[3 * id[c] + q];
    double e1[3], e2[3];
    for (int q = 0; q < 3; ++q) {
        e1[q] = P[1][q] - P[0][q];
        e2[q] = P[2][q] - P[0][q];
    }
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double N[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
    const double* a = P[0];
    const double* b = P[1];
    const double* c = P[2];
    double bxc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    fterm[2 * S] = 0.5 * nn;
    fterm[2 * S + 1] = (a[0] * bxc[0] + a[1] * bxc[1] + a[2] * bxc[2]) / 6.0;
    for (int cr = 0; cr < 3; ++cr) {
        const double* pj = P[(cr + 1) % 3];
        const double* pk = P[(cr + 2) % 3];
        double e[3] = {pk[0] - pj[0], pk[1] - pj[1], pk[2] - pj[2]};
        double ga[3] = {N[1] * e[2] - N[2] * e[1], N[2] * e[0] - N[0] * e[2], N[0] * e[1] - N[1] * e[0]};
        double gv[3] = {pj[1] * pk[2] - pj[2] * pk[1], pj[2] * pk[0] - pj[0] * pk[2],
                        pj[0] * pk[1] - pj[1] * pk[0]};
        for (int q = 0; q < 3; ++q) {
            cga[(3 * S + cr) * 3 + q] = 0.5 * ga[q];
            cgv[(3 * S + cr) * 3 + q] = gv[q] / 6.0;
        }
    }
}

// values [area, volume] to host; gradients (if gA/gV non-null) to device [nv][3]
static int constraints_eval(tp_mesh* m, const double* pos, double vals[2], double* gA, double* gV,
                            cudaStream_t st) {
    const int nf = m->nf;
    TP_TRY(ensure(m->tmpv[7], sizeof(double) * 2 * (size_t)nf));
    TP_TRY(ensure(m->corner, sizeof(double) * 18 * (size_t)nf));
    TP_TRY(ensure(m->rowsum, sizeof(double) * 8));
    double* ft = m->tmpv[7].as<double>();
    double* cga = m->corner.as<double>();
    double* cgv = cga + 9 * (size_t)nf;
    k_constraint_terms<<<(nf + 255) / 256, 256, 0, st>>>(pos, m->faces.as<int>(), nf, ft, cga, cgv);
    TP_LAUNCH_CHECK();
    TP_TRY(colsum(m, ft, nf, 2, 1.0, m->rowsum.as<double>(), st));
    TP_CUDA(cudaMemcpyAsync(vals, m->rowsum.ptr, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (gA) TP_TRY(corners_to_vertices(m, cga, 3, gA, st));
    if (gV) TP_TRY(corners_to_vertices(m, cgv, 3, gV, st));
    TP_CUDA(cudaStreamSynchronize(st));
    return TP_OK;
}

int area_volume(tp_mesh* m, double out[2], cudaStream_t st) {
    return constraints_eval(m, m->pos.as<double>(), out, nullptr, nullptr, st);
}

// ---------------------------------------------------------------------------
// one constrained descent step
// ---------------------------------------------------------------------------

static int set_positions_dev(tp_mesh* m, const double* src, cudaStream_t st) {
    if (src != m->pos.as<double>())
        TP_CUDA(cudaMemcpyAsync(m->pos.ptr, src, sizeof(double) * 3 * (size_t)m->nv,
                                cudaMemcpyDeviceToDevice, st));
    return refresh_geometry(m, st);
}

// Barycenter motion (§7.1.1): per connected component, t_c = -(sum m_i g_i) /
// (sum m_i) with m_i the lumped mass (a third of the area of each face around
// vertex i); one block per (component, coordinate), fixed summation order
__global__ void k_bary_motion(const int* __restrict__ comp_ptr, const int* __restrict__ comp_verts,
                              const int* __restrict__ vf_ptr, const int* __restrict__ vf_idx,
                              const d4* __restrict__ f64a, const double* __restrict__ g, double* __restrict__ t) {
    const int c = blockIdx.x, j = blockIdx.y;
    __shared__ double rs[256], rw[256];
    double s = 0.0, w = 0.0;
    for (int e = comp_ptr[c] + threadIdx.x; e < comp_ptr[c + 1]; e += blockDim.x) {
        const int v = comp_verts[e];
        double mv = 0.0;
        for (int q = vf_ptr[v]; q < vf_ptr[v + 1]; ++q) mv += f64a[vf_idx[q] / 3].w;
        mv /= 3.0;
        s += mv * g[3 * (size_t)v + j];
        w += mv;
    }
    rs[threadIdx.x] = s;
    rw[threadIdx.x] = w;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            rs[threadIdx.x] += rs[threadIdx.x + k];
            rw[threadIdx.x] += rw[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) t[3 * c + j] = -rs[0] / rw[0];
}

__global__ void k_bary_add(const int* __restrict__ vcomp, int nv, const double* __restrict__ t,
                           double* __restrict__ x) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nv * 3) return;
    x[i] += t[3 * (size_t)vcomp[i / 3] + (i % 3)];
}

// max over vertices of |x_v|^2 (one block, fixed order of the final
// reduction: deterministic)
__global__ void k_max_norm2(const double* __restrict__ x, int nv, double* __restrict__ out) {
    __shared__ double red[256];
    double mx = 0.0;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const double a = x[3 * (size_t)v], b = x[3 * (size_t)v + 1], c = x[3 * (size_t)v + 2];
        mx = fmax(mx, a * a + b * b + c * c);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// x += the translation of each component by minus the area-weighted mean of g
static int barycenter_motion(tp_mesh* m, const double* g, double* x, cudaStream_t st) {
    TP_TRY(ensure(m->part2, sizeof(double) * 3 * (size_t)m->ncomp));
    double* t = m->part2.as<double>();
    k_bary_motion<<<dim3(m->ncomp, 3), 256, 0, st>>>(m->comp_ptr.as<int>(), m->comp_verts.as<int>(),
                                                    m->vf_ptr.as<int>(), m->vf_idx.as<int>(), m->f64a.as<d4>(), g, t);
    TP_LAUNCH_CHECK();
    const size_t n = (size_t)m->nv * 3;
    k_bary_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->vcomp.as<int>(), m->nv, t, x);
    TP_LAUNCH_CHECK();
    return TP_OK;
}

int precond_step_dev(tp_mesh* m, const tp_params* p, const tp_constraints* c, tp_step_report* rep,
                     cudaStream_t st) {
    const size_t n = (size_t)m->nv * 3;
    for (int i = 0; i < 8; ++i) TP_TRY(ensure(m->stepv[i], sizeof(double) * n));
    double* f0 = m->stepv[0].as<double>();   // positions at the start
    double* g = m->stepv[1].as<double>();    // dE
    double* Ag = m->stepv[2].as<double>();   // A^-1 g
    double* J[2] = {m->stepv[3].as<double>(), m->stepv[4].as<double>()};   // dPhi rows
    double* Z[2] = {m->stepv[5].as<double>(), m->stepv[6].as<double>()};   // A^-1 dPhi^T
    double* x = m->stepv[7].as<double>();    // direction
    tp_step_report r{};
    r.status = TP_OK;
    const double pairs0 = m->pairs;
    unsigned long long bh0[BH_NCOUNT];
    TP_TRY(bh_counts_read(m, bh0, false, st));
    TP_CUDA(cudaMemcpyAsync(f0, m->pos.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    {
        int e0 = 0, u0 = 0;
        TP_TRY(chol_deferred_flags(m, st, &e0, &u0, true));
    }

    // 1. differential
    double E0 = 0.0;
    TP_TRY(differential_dev(m, p, g, &E0, st, true));
    r.E_before = E0;
    // 2. constraint Jacobian rows at f
    int use[2] = {(c->flags & TP_CONSTRAINT_AREA) ? 1 : 0, (c->flags & TP_CONSTRAINT_VOLUME) ? 1 : 0};
    double phi0[2];
    TP_TRY(constraints_eval(m, f0, phi0, J[0], J[1], st));
    int nc = 0;
    double* Jr[2];
    double* Zr[2];
    for (int i = 0; i < 2; ++i)
        if (use[i]) {
            Jr[nc] = J[i];
            Zr[nc] = Z[i];
            ++nc;
        }
    // 3. k+1 solves with A_3 (Eq. 17, 18), in lockstep
    KrylovStats ks;
    {
        const double* rhs[MAXSYS] = {g, nullptr, nullptr};
        double* sol[MAXSYS] = {Ag, nullptr, nullptr};
        for (int i = 0; i < nc; ++i) {
            rhs[1 + i] = Jr[i];
            sol[1 + i] = Zr[i];
        }
        int sts[MAXSYS] = {TP_OK, TP_OK, TP_OK};
        TP_TRY(fgmres_multi(m, p, 1 + nc, rhs, sol, st, &ks, sts));
        for (int i = 0; i < 1 + nc; ++i)
            if (sts[i] != TP_OK) r.status = sts[i];
    }
    // 4. Schur complement S = dPhi Z (= -(M/A)), x = -(Ag - Z S^-1 dPhi Ag)
    double Sm[2][2] = {{0, 0}, {0, 0}}, JAg[2] = {0, 0};
    for (int i = 0; i < nc; ++i) {
        std::vector<const double*> zs(Zr, Zr + nc);
        double out[2];
        TP_TRY(dots(m, zs.data(), Jr[i], nc, n, out, st));
        for (int j = 0; j < nc; ++j) Sm[i][j] = out[j];
        const double* a1[1] = {Ag};
        TP_TRY(dots(m, a1, Jr[i], 1, n, &JAg[i], st));
    }
    double lam[2] = {0, 0};
    auto solve_small = [&](const double rhs[2], double out[2]) {
        if (nc == 1) {
            out[0] = rhs[0] / Sm[0][0];
        } else if (nc == 2) {
            double det = Sm[0][0] * Sm[1][1] - Sm[0][1] * Sm[1][0];
            out[0] = (Sm[1][1] * rhs[0] - Sm[0][1] * rhs[1]) / det;
            out[1] = (-Sm[1][0] * rhs[0] + Sm[0][0] * rhs[1]) / det;
        }
    };
    solve_small(JAg, lam);
    {
        std::vector<const double*> xs;
        std::vector<double> cf;
        xs.push_back(Ag);
        cf.push_back(-1.0);
        for (int i = 0; i < nc; ++i) {
            xs.push_back(Zr[i]);
            cf.push_back(lam[i]);
        }
        TP_TRY(lincomb(x, xs.data(), cf.data(), (int)xs.size(), n, 0.0, st));
    }
    if (c->flags & TP_CONSTRAINT_FREE_BARYCENTER) TP_TRY(barycenter_motion(m, g, x, st));
    {
        const double* a1[1] = {g};
        TP_TRY(dots(m, a1, x, 1, n, &r.slope, st));
    }
    // 5. Armijo line search on E(f + tau x); with tau0_disp the first trial
    //    moves no vertex by more than tau0_disp face sizes
    double tau = p->tau0;
    if (p->tau0_disp > 0.0) {
        TP_TRY(ensure(m->rowsum, sizeof(double) * 8));
        k_max_norm2<<<1, 256, 0, st>>>(x, m->nv, m->rowsum.as<double>() + 4);
        TP_LAUNCH_CHECK();
        double mx2 = 0.0;
        TP_CUDA(cudaMemcpyAsync(&mx2, m->rowsum.as<double>() + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
        TP_CUDA(cudaStreamSynchronize(st));
        const double h = std::sqrt(std::max(phi0[0], 0.0) / m->nf);
        if (mx2 > 0.0 && h > 0.0) tau = std::min(tau, p->tau0_disp * h / std::sqrt(mx2));
    }
    double* ftrial = m->pos.as<double>();
    int trials = 0;
    double E1 = E0;
    for (;;) {
        const double* xs[2] = {f0, x};
        double cf[2] = {1.0, tau};
        TP_TRY(lincomb(ftrial, xs, cf, 2, n, 0.0, st));
        int gs = refresh_geometry(m, st);
        ++trials;
        if (gs == TP_OK) {
            TP_TRY(energy_value(m, p, &E1, st, true));
            if (p->fixed_tau || E1 <= E0 + p->armijo_c * tau * r.slope) break;
        } else if (gs != TP_ERR_DEGENERATE) {
            return gs;
        }
        if (trials >= p->ls_max) break;
        tau *= p->armijo_shrink;
    }
    r.tau = tau;
    r.ls_trials = trials;
    // 6. corrective projection (Eq. 15 / 19): h = -Z S^-1 Phi(f_k), Z and S
    //    of the start of the step, repeated proj_iters times
    double phi1[2];
    TP_TRY(constraints_eval(m, m->pos.as<double>(), phi1, nullptr, nullptr, st));
    r.phi_before[0] = use[0] ? phi1[0] - c->A0 : 0.0;
    r.phi_before[1] = use[1] ? phi1[1] - c->V0 : 0.0;
    for (int it = 0; it < p->proj_iters && nc > 0; ++it) {
        if (it > 0) {
            TP_TRY(refresh_geometry(m, st));
            TP_TRY(constraints_eval(m, m->pos.as<double>(), phi1, nullptr, nullptr, st));
        }
        double res[2] = {0, 0};
        int ci = 0;
        if (use[0]) res[ci++] = phi1[0] - c->A0;
        if (use[1]) res[ci++] = phi1[1] - c->V0;
        double mu[2] = {0, 0};
        solve_small(res, mu);
        std::vector<double> cf(nc);
        for (int i = 0; i < nc; ++i) cf[i] = -mu[i];
        TP_TRY(lincomb(m->pos.as<double>(), (const double* const*)Zr, cf.data(), nc, n, 1.0, st));
    }
    TP_TRY(set_positions_dev(m, m->pos.as<double>(), st));
    double phi2[2];
    TP_TRY(constraints_eval(m, m->pos.as<double>(), phi2, nullptr, nullptr, st));
    r.phi_after[0] = use[0] ? phi2[0] - c->A0 : 0.0;
    r.phi_after[1] = use[1] ? phi2[1] - c->V0 : 0.0;
    TP_TRY(energy_value(m, p, &r.E_after, st, true));
    r.krylov_iters = ks.iters;
    r.cg_iters = ks.cg_iters;
    {
        // the deferred Poisson solves of the Krylov loop: a wait that gave up
        // is an error; solves that stopped short of cg_tol only made the
        // (flexible) preconditioner less exact
        int derr = 0, dunc = 0;
        TP_TRY(chol_deferred_flags(m, st, &derr, &dunc, false));
        if (derr) return fail(TP_ERR_TIMEOUT, "precond_step: a wait of the factorised sweep gave up");
        int tcerr = 0;
        if (p->tensor_cores) TP_TRY(apply_tc_error(m, &tcerr, st));
        if (tcerr) return fail(TP_ERR_TIMEOUT, "precond_step: a wait of the tensor-core A apply gave up");
    }
    unsigned long long bh1[BH_NCOUNT];
    TP_TRY(bh_counts_read(m, bh1, false, st));
    r.pair_interactions = m->pairs - pairs0;
    for (int i = 0; i < BH_NCOUNT; ++i) r.pair_interactions += (double)(bh1[i] - bh0[i]);
    if (rep) *rep = r;
    return TP_OK;
}

}  // namespace tp
