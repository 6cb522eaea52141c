// Test driver for the host analysis of the sparse Cholesky factor
// (chol_symbolic.h): runs the multifrontal factorisation and the two
// substitutions in FP64 on the host through the analysis' index maps and
// checks the structural invariants of the supernodal tree.
//
//   in  file: int32 nv, nnz, k, leaf; int32 rowptr[nv+1], col[nnz];
//             float64 val[nnz], b[nv*k]   (symmetric C, diagonal included)
//   out file: int32 n, ncomp, nnode, levels, max_front; float64 z[nv*k]
//             (pinned rows zero; no mean projection)
// Exit status 0 on success; a violated invariant prints a message and exits 3.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "chol_symbolic.h"

using tp::CholSymbolic;

static int die(const char* msg, int a = 0, int b = 0) {
    std::fprintf(stderr, "invariant: %s (%d %d)\n", msg, a, b);
    return 3;
}

template <class T>
static bool rd(FILE* f, T* p, size_t n) { return std::fread(p, sizeof(T), n, f) == n; }

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int hdr[4];
    if (!rd(f, hdr, 4)) return 2;
    const int nv = hdr[0], nnz = hdr[1], K = hdr[2], leaf = hdr[3];
    std::vector<int> rowptr(nv + 1), col(nnz);
    std::vector<double> val(nnz), b((size_t)nv * K);
    if (!rd(f, rowptr.data(), nv + 1) || !rd(f, col.data(), nnz) || !rd(f, val.data(), nnz) ||
        !rd(f, b.data(), b.size()))
        return 2;
    std::fclose(f);

    CholSymbolic S;
    if (!tp::chol_analyze(nv, rowptr.data(), col.data(), leaf, S)) return die("analysis failed");
    // --- invariants
    std::vector<int> seen(nv, 0);
    for (int q = 0; q < S.n; ++q) {
        int v = S.perm[q];
        if (v < 0 || v >= nv || seen[v]++) return die("perm is not injective", q, v);
        if (S.pos[v] != q) return die("pos is not the inverse of perm", q, v);
    }
    for (int c = 0; c < S.ncomp; ++c) {
        int p = S.pinned[c];
        if (seen[p] || S.pos[p] != -1) return die("pinned vertex ordered", c, p);
        for (int v = 0; v < p; ++v)
            if (S.comp[v] == c) return die("pinned vertex is not the lowest of its component", c, v);
    }
    if (S.n + S.ncomp != nv) return die("unknowns + components != vertices", S.n, S.ncomp);
    int covered = 0;
    for (int J = 0; J < S.nnode; ++J) {
        if (S.p0[J] != covered) return die("supernodes not contiguous", J, S.p0[J]);
        covered += S.nJ[J];
        const int P = S.parent[J];
        if (P >= 0 && P <= J) return die("parent not after child", J, P);
        if (P < 0 && S.mJ[J] != 0) return die("root with a structure", J, S.mJ[J]);
        // every structure entry belongs to an ancestor
        for (int x = S.struct_ptr[J]; x < S.struct_ptr[J + 1]; ++x) {
            int q = S.struct_pos[x], A = P;
            while (A >= 0 && !(q >= S.p0[A] && q < S.p0[A] + S.nJ[A])) A = S.parent[A];
            if (A < 0) return die("structure entry outside the ancestors", J, q);
            if (x > S.struct_ptr[J] && q <= S.struct_pos[x - 1]) return die("structure not increasing", J, q);
        }
        for (int c = S.child_ptr[J]; c < S.child_ptr[J + 1]; ++c)
            if (S.parent[S.child_idx[c]] != J) return die("child list and parent disagree", J, S.child_idx[c]);
    }
    if (covered != S.n) return die("supernodes do not cover the unknowns", covered, S.n);
    const int H = (int)S.level_ptr.size() - 1;
    for (int J = 0; J < S.nnode; ++J)
        if (S.parent[J] >= 0 && S.height[S.parent[J]] <= S.height[J]) return die("height order", J, S.parent[J]);

    // --- multifrontal factorisation (FP64), level by level
    std::vector<double> L(S.lsize), U(S.usize);
    for (int h = 0; h < H; ++h)
        for (int ii = S.level_ptr[h]; ii < S.level_ptr[h + 1]; ++ii) {
            const int J = S.level_nodes[ii], n = S.nJ[J], m = S.mJ[J], t = n + m;
            std::vector<double> P((size_t)t * n, 0.0);
            double* UJ = U.data() + S.uoff[J];
            for (int i = 0; i < m * m; ++i) UJ[i] = 0.0;
            for (int e = S.asm_ptr[J]; e < S.asm_ptr[J + 1]; ++e) P[S.asm_dst[e]] += val[S.asm_src[e]];
            for (int cc = S.child_ptr[J]; cc < S.child_ptr[J + 1]; ++cc) {
                const int c = S.child_idx[cc], mc = S.mJ[c];
                const int* rel = S.rel.data() + S.struct_ptr[c];
                const double* Uc = U.data() + S.uoff[c];
                for (int y = 0; y < mc; ++y)
                    for (int x = y; x < mc; ++x) {
                        const int R = rel[x], C = rel[y];
                        if (R < C || R >= t) return die("relative index order", R, C);
                        if (C < n)
                            P[R + (size_t)C * t] += Uc[x + y * mc];
                        else
                            UJ[(R - n) + (C - n) * m] += Uc[x + y * mc];
                    }
            }
            for (int k = 0; k < n; ++k) {
                double d = P[k + (size_t)k * t];
                if (!(d > 0.0)) return die("non-positive pivot", J, k);
                d = std::sqrt(d);
                P[k + (size_t)k * t] = d;
                for (int i = k + 1; i < t; ++i) P[i + (size_t)k * t] /= d;
                for (int j = k + 1; j < n; ++j)
                    for (int i = j; i < t; ++i) P[i + (size_t)j * t] -= P[i + (size_t)k * t] * P[j + (size_t)k * t];
            }
            for (int y = 0; y < m; ++y)
                for (int x = y; x < m; ++x) {
                    double s = 0.0;
                    for (int k = 0; k < n; ++k) s += P[n + x + (size_t)k * t] * P[n + y + (size_t)k * t];
                    UJ[x + y * m] -= s;
                }
            double* Li = L.data() + S.loff[J];
            double* L21 = Li + (size_t)n * n;
            for (int i = 0; i < n * n; ++i) Li[i] = 0.0;
            for (int c = 0; c < n; ++c)
                for (int i = c; i < n; ++i) {
                    double s = i == c ? 1.0 : 0.0;
                    for (int k = c; k < i; ++k) s -= P[i + (size_t)k * t] * Li[k + c * n];
                    Li[i + c * n] = s / P[i + (size_t)i * t];
                }
            for (int k = 0; k < n; ++k)
                for (int x = 0; x < m; ++x) L21[x + k * m] = P[n + x + (size_t)k * t];
        }
    // --- substitutions
    std::vector<double> y((size_t)S.n * K), xs((size_t)S.n * K), uv((size_t)S.vsize * K), z((size_t)nv * K, 0.0);
    for (int h = 0; h < H; ++h)
        for (int ii = S.level_ptr[h]; ii < S.level_ptr[h + 1]; ++ii) {
            const int J = S.level_nodes[ii], n = S.nJ[J], m = S.mJ[J], t = n + m;
            std::vector<double> w((size_t)t * K, 0.0);
            for (int a = 0; a < n; ++a)
                for (int c = 0; c < K; ++c) w[a * K + c] = b[(size_t)S.perm[S.p0[J] + a] * K + c];
            for (int cc = S.child_ptr[J]; cc < S.child_ptr[J + 1]; ++cc) {
                const int ch = S.child_idx[cc];
                const int* rel = S.rel.data() + S.struct_ptr[ch];
                for (int x = 0; x < S.mJ[ch]; ++x)
                    for (int c = 0; c < K; ++c) w[rel[x] * K + c] += uv[((size_t)S.voff[ch] + x) * K + c];
            }
            const double* Li = L.data() + S.loff[J];
            const double* L21 = Li + (size_t)n * n;
            for (int a = 0; a < n; ++a)
                for (int c = 0; c < K; ++c) {
                    double s = 0.0;
                    for (int k = 0; k <= a; ++k) s += Li[a + k * n] * w[k * K + c];
                    y[(size_t)(S.p0[J] + a) * K + c] = s;
                }
            for (int x = 0; x < m; ++x)
                for (int c = 0; c < K; ++c) {
                    double s = w[(n + x) * K + c];
                    for (int k = 0; k < n; ++k) s -= L21[x + k * m] * y[(size_t)(S.p0[J] + k) * K + c];
                    uv[((size_t)S.voff[J] + x) * K + c] = s;
                }
        }
    for (int h = H - 1; h >= 0; --h)
        for (int ii = S.level_ptr[h]; ii < S.level_ptr[h + 1]; ++ii) {
            const int J = S.level_nodes[ii], n = S.nJ[J], m = S.mJ[J];
            const double* Li = L.data() + S.loff[J];
            const double* L21 = Li + (size_t)n * n;
            std::vector<double> zz((size_t)n * K);
            for (int a = 0; a < n; ++a)
                for (int c = 0; c < K; ++c) {
                    double s = y[(size_t)(S.p0[J] + a) * K + c];
                    for (int x = 0; x < m; ++x)
                        s -= L21[x + a * m] * xs[(size_t)S.struct_pos[S.struct_ptr[J] + x] * K + c];
                    zz[a * K + c] = s;
                }
            for (int a = 0; a < n; ++a)
                for (int c = 0; c < K; ++c) {
                    double s = 0.0;
                    for (int k = a; k < n; ++k) s += Li[k + a * n] * zz[k * K + c];
                    xs[(size_t)(S.p0[J] + a) * K + c] = s;
                    z[(size_t)S.perm[S.p0[J] + a] * K + c] = s;
                }
        }
    FILE* o = std::fopen(argv[2], "wb");
    if (!o) return 2;
    int oh[5] = {S.n, S.ncomp, S.nnode, H, S.max_t};
    std::fwrite(oh, sizeof(int), 5, o);
    std::fwrite(z.data(), sizeof(double), z.size(), o);
    std::fclose(o);
    return 0;
}
