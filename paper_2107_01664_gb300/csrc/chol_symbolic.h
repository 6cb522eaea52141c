// Symbolic analysis of the sparse Cholesky factorisation of the cotan
// Laplacian (host code, once per mesh topology).
//
// §5.2 applies the preconditioner through a pre-factorised integer Laplacian.
// C is singular (the constants of every connected component span its
// nullspace), so one vertex per component is pinned: its row and column are
// removed, which leaves a symmetric positive definite matrix whose solution,
// shifted to zero mean per component, is C^+ b for b of zero mean per
// component.
//
// Ordering: nested dissection with BFS level-set separators. A connected
// vertex set larger than the leaf size is cut at the BFS level (from a
// pseudo-peripheral vertex) where half of its vertices are reached; only the
// vertices of that level with a neighbour in the next level are kept in the
// separator. Every vertex set outside the separator is bounded by separators
// of its ancestors only, so the factor's column structure is that of a
// supernodal tree: one supernode per leaf or separator, eliminated in
// postorder (children before parents).
//
// Supernode J owns the contiguous positions [p0, p0 + nJ) and its dense
// front has t = nJ + mJ rows: its own positions, then struct(J), the sorted
// positions of later (ancestor) vertices that its column block touches:
//   struct(J) = (neighbours of J's vertices after J) U (struct(children) after J).
// The diagonal block is kept dense, so the front may hold explicit zeros;
// it always contains the true fill.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace tp {

struct CholSymbolic {
    int nv = 0;                       // vertices
    int n = 0;                        // unknowns (vertices minus one pinned vertex per component)
    int ncomp = 0;
    std::vector<int> comp;            // component of each vertex
    std::vector<int> pinned;          // pinned vertex of each component (its lowest index)
    std::vector<int> perm;            // position -> vertex (n)
    std::vector<int> pos;             // vertex -> position, -1 for pinned vertices (nv)
    // supernodes in postorder
    int nnode = 0;
    std::vector<int> p0, nJ, mJ, parent, height;
    std::vector<int> child_ptr, child_idx;      // children of each node
    std::vector<int> struct_ptr, struct_pos;    // struct(J) (mJ positions, increasing)
    std::vector<int> rel;                       // per struct entry: local row in the parent's front
    std::vector<int64_t> loff, uoff;            // float offsets of [Linv | L21] (multiples of 4) and of U
    std::vector<int> voff;                      // row offsets of the update vectors (mJ rows each)
    int64_t lsize = 0, usize = 0;
    int vsize = 0;
    // original entries: for node J, entries asm_ptr[J]..asm_ptr[J+1] put CSR
    // value asm_src[e] at panel index asm_dst[e] (row + col * t)
    std::vector<int> asm_ptr, asm_dst, asm_src;
    // nodes grouped by height (0 = leaves), each group in postorder
    std::vector<int> level_ptr, level_nodes;
    int max_t = 0;                    // largest front
    int64_t max_panel = 0;            // largest t * nJ
    int max_nJ = 0;
};

// leading dimension of a stored factor block with r rows (odd, 0 for no rows)
inline int64_t chol_ld(int64_t r) { return r == 0 ? 0 : (r | 1); }

namespace chol_detail {

// A separator whose front would hold more than SEP_PANEL entries (its
// vertices times the rows of its front: its own vertices plus the ancestor
// separator vertices next to the set it cuts, an upper bound of the front)
// is split into a chain of supernodes of at most SEP_PANEL / rows vertices
// each (at least SEP_MIN_CHUNK).
constexpr long long SEP_PANEL = 24576;
constexpr int SEP_MIN_CHUNK = 8;

struct NestedDissection {
    int nv;
    const int* rowptr;
    const int* col;
    int leaf;
    std::vector<int> mark;    // vertex -> current vertex-set id, -1 once in a separator or pinned
    std::vector<int> seen;    // BFS stamp
    std::vector<int> lev;     // BFS level (valid where seen == stamp)
    std::vector<char> in_sep; // vertex placed in a separator
    std::vector<int> bstamp;  // stamps of the boundary count
    int stamp = 0, bst = 0;
    int next_id = 1;
    struct Node {
        std::vector<int> verts;
        std::vector<int> kids;
    };
    std::vector<Node> nodes;

    // BFS over vertices with mark == id from s; order holds the visit order,
    // lstart the first index of each level (plus the end)
    void bfs(int s, int id, std::vector<int>& order, std::vector<int>& lstart) {
        ++stamp;
        order.clear();
        lstart.clear();
        order.push_back(s);
        seen[s] = stamp;
        lev[s] = 0;
        lstart.push_back(0);
        size_t head = 0;
        int cur = 0;
        while (head < order.size()) {
            int v = order[head];
            if (lev[v] != cur) {
                cur = lev[v];
                lstart.push_back((int)head);
            }
            ++head;
            for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                int u = col[e];
                if (u == v || mark[u] != id || seen[u] == stamp) continue;
                seen[u] = stamp;
                lev[u] = lev[v] + 1;
                order.push_back(u);
            }
        }
        lstart.push_back((int)order.size());
    }

    int degree_in(int v, int id) const {
        int d = 0;
        for (int e = rowptr[v]; e < rowptr[v + 1]; ++e)
            if (col[e] != v && mark[col[e]] == id) ++d;
        return d;
    }

    // vertex set S (all marked id) -> roots of its elimination forest
    void build(const std::vector<int>& S, int id, std::vector<int>& roots) {
        // connected components of S, each gets its own id
        std::vector<int> order, lstart;
        std::vector<int> sorted(S);
        std::sort(sorted.begin(), sorted.end());
        std::vector<std::vector<int>> comps;
        for (int s : sorted) {
            if (mark[s] != id) continue;
            bfs(s, id, order, lstart);
            int cid = next_id++;
            for (int v : order) mark[v] = cid;
            comps.push_back(order);
        }
        for (auto& C : comps) component(C, mark[C[0]], roots);
    }

    void component(std::vector<int>& C, int id, std::vector<int>& roots) {
        const int N = (int)C.size();
        if (N <= leaf) {
            leaf_node(C, roots);
            return;
        }
        // pseudo-peripheral root: repeat BFS from a minimum-degree vertex of
        // the last level while the eccentricity grows
        std::vector<int> order, lstart;
        int s = *std::min_element(C.begin(), C.end());
        bfs(s, id, order, lstart);
        int ecc = (int)lstart.size() - 2;
        for (int sweep = 0; sweep < 6; ++sweep) {
            int best = -1, bd = 1 << 30;
            for (int i = lstart[lstart.size() - 2]; i < lstart.back(); ++i) {
                int v = order[i], d = degree_in(v, id);
                if (d < bd || (d == bd && v < best)) {
                    bd = d;
                    best = v;
                }
            }
            std::vector<int> o2, l2;
            bfs(best, id, o2, l2);
            int e2 = (int)l2.size() - 2;
            if (e2 <= ecc) {
                bfs(s, id, order, lstart);   // restore the levels of the kept root
                break;
            }
            s = best;
            ecc = e2;
            order.swap(o2);
            lstart.swap(l2);
        }
        const int h = (int)lstart.size() - 2;   // levels 0..h
        // separator level: the first level by which half of the set is reached
        int l = 0;
        while (l < h && lstart[l + 1] < (N + 1) / 2) ++l;
        if (l == 0) l = 1;
        if (l > h) l = h;
        if (h < 2) {   // no level splits the set in two: keep it whole
            leaf_node(C, roots);
            return;
        }
        if (l == h) l = h - 1;
        std::vector<int> sep, A, B;
        for (int i = 0; i < lstart[l]; ++i) A.push_back(order[i]);
        for (int i = lstart[l + 1]; i < lstart[h + 1]; ++i) B.push_back(order[i]);
        for (int i = lstart[l]; i < lstart[l + 1]; ++i) {
            int v = order[i];
            bool touches_next = false;
            for (int e = rowptr[v]; e < rowptr[v + 1] && !touches_next; ++e) {
                int u = col[e];
                touches_next = u != v && mark[u] == id && seen[u] == stamp && lev[u] == l + 1;
            }
            (touches_next ? sep : A).push_back(v);
        }
        if (2 * (int)sep.size() > N) {   // degenerate graph: no useful separator
            leaf_node(C, roots);
            return;
        }
        // rows of the separator's front: its vertices plus the separator
        // vertices of ancestors next to C (counted before the recursion marks
        // the separators inside C)
        ++bst;
        long long bnd = 0;
        for (int v : C)
            for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                const int u = col[e];
                if (u != v && in_sep[u] && bstamp[u] != bst) {
                    bstamp[u] = bst;
                    ++bnd;
                }
            }
        for (int v : sep) in_sep[v] = 1;
        const long long rows = (long long)sep.size() + bnd;
        int chunk = (int)sep.size();
        if ((long long)sep.size() * rows > SEP_PANEL)
            chunk = (int)std::max<long long>(SEP_MIN_CHUNK, SEP_PANEL / rows);
        int ia = next_id++, ib = next_id++;
        for (int v : sep) mark[v] = -1;
        for (int v : A) mark[v] = ia;
        for (int v : B) mark[v] = ib;
        std::vector<int> kids;
        build(A, ia, kids);
        build(B, ib, kids);
        std::sort(sep.begin(), sep.end());
        // a separator with a wide front becomes a chain of supernodes of at
        // most `chunk` vertices (same elimination order, same fill): every
        // panel then stays narrow enough for shared memory
        for (size_t c0 = 0; c0 < sep.size(); c0 += chunk) {
            Node nd;
            nd.verts.assign(sep.begin() + c0, sep.begin() + std::min(sep.size(), c0 + (size_t)chunk));
            nd.kids = kids;
            nodes.push_back(nd);
            kids.assign(1, (int)nodes.size() - 1);
        }
        roots.push_back(kids[0]);
    }

    void leaf_node(std::vector<int>& C, std::vector<int>& roots) {
        for (int v : C) mark[v] = -1;
        Node nd;
        nd.verts = C;
        std::sort(nd.verts.begin(), nd.verts.end());
        nodes.push_back(nd);
        roots.push_back((int)nodes.size() - 1);
    }
};

}  // namespace chol_detail

// Builds the ordering, supernodal tree, structures and index maps. rowptr /
// col: the symmetric CSR pattern of C (diagonal included). Returns false if
// the pattern is empty.
inline bool chol_analyze(int nv, const int* rowptr, const int* col, int leaf, CholSymbolic& S) {
    S = CholSymbolic();
    S.nv = nv;
    if (nv <= 0) return false;
    // components and pinned vertices (the lowest index of each component)
    S.comp.assign(nv, -1);
    std::vector<int> stack;
    for (int v = 0; v < nv; ++v) {
        if (S.comp[v] >= 0) continue;
        int c = S.ncomp++;
        S.pinned.push_back(v);
        S.comp[v] = c;
        stack.push_back(v);
        while (!stack.empty()) {
            int a = stack.back();
            stack.pop_back();
            for (int e = rowptr[a]; e < rowptr[a + 1]; ++e)
                if (S.comp[col[e]] < 0) {
                    S.comp[col[e]] = c;
                    stack.push_back(col[e]);
                }
        }
    }
    chol_detail::NestedDissection nd;
    nd.nv = nv;
    nd.rowptr = rowptr;
    nd.col = col;
    nd.leaf = leaf < 1 ? 1 : leaf;
    nd.mark.assign(nv, 0);
    nd.seen.assign(nv, 0);
    nd.lev.assign(nv, 0);
    nd.in_sep.assign(nv, 0);
    nd.bstamp.assign(nv, 0);
    for (int p : S.pinned) nd.mark[p] = -1;
    std::vector<int> all;
    for (int v = 0; v < nv; ++v)
        if (nd.mark[v] == 0) all.push_back(v);
    std::vector<int> roots;
    if (!all.empty()) nd.build(all, 0, roots);
    // postorder (children before parents) by an explicit stack
    std::vector<int> post;
    {
        std::vector<std::pair<int, int>> st;
        for (int r : roots) {
            st.push_back({r, 0});
            while (!st.empty()) {
                auto& top = st.back();
                auto& kids = nd.nodes[top.first].kids;
                if (top.second < (int)kids.size()) {
                    int k = kids[top.second++];
                    st.push_back({k, 0});
                } else {
                    post.push_back(top.first);
                    st.pop_back();
                }
            }
        }
    }
    const int nn = (int)post.size();
    S.nnode = nn;
    std::vector<int> newid(nd.nodes.size(), -1);
    for (int i = 0; i < nn; ++i) newid[post[i]] = i;
    S.pos.assign(nv, -1);
    S.p0.resize(nn);
    S.nJ.resize(nn);
    S.parent.assign(nn, -1);
    for (int i = 0; i < nn; ++i) {
        auto& N = nd.nodes[post[i]];
        S.p0[i] = (int)S.perm.size();
        S.nJ[i] = (int)N.verts.size();
        for (int v : N.verts) {
            S.pos[v] = (int)S.perm.size();
            S.perm.push_back(v);
        }
    }
    S.n = (int)S.perm.size();
    S.child_ptr.assign(nn + 1, 0);
    for (int i = 0; i < nn; ++i) {
        for (int k : nd.nodes[post[i]].kids) {
            S.parent[newid[k]] = i;
            S.child_idx.push_back(newid[k]);
        }
        S.child_ptr[i + 1] = (int)S.child_idx.size();
    }
    // structures, in postorder
    std::vector<std::vector<int>> st(nn);
    std::vector<int> seen(S.n, -1);
    for (int J = 0; J < nn; ++J) {
        const int end = S.p0[J] + S.nJ[J];
        auto& s = st[J];
        for (int a = 0; a < S.nJ[J]; ++a) {
            int v = S.perm[S.p0[J] + a];
            for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                int q = S.pos[col[e]];
                if (q >= end && seen[q] != J) {
                    seen[q] = J;
                    s.push_back(q);
                }
            }
        }
        for (int c = S.child_ptr[J]; c < S.child_ptr[J + 1]; ++c)
            for (int q : st[S.child_idx[c]])
                if (q >= end && seen[q] != J) {
                    seen[q] = J;
                    s.push_back(q);
                }
        std::sort(s.begin(), s.end());
    }
    S.mJ.resize(nn);
    S.struct_ptr.assign(nn + 1, 0);
    for (int J = 0; J < nn; ++J) {
        S.mJ[J] = (int)st[J].size();
        S.struct_pos.insert(S.struct_pos.end(), st[J].begin(), st[J].end());
        S.struct_ptr[J + 1] = (int)S.struct_pos.size();
    }
    // relative indices into the parent's front
    S.rel.assign(S.struct_pos.size(), -1);
    for (int J = 0; J < nn; ++J) {
        int P = S.parent[J];
        if (P < 0) continue;   // a root has an empty structure
        const int pp0 = S.p0[P], pn = S.nJ[P];
        const int* ps = S.struct_pos.data() + S.struct_ptr[P];
        for (int x = 0; x < S.mJ[J]; ++x) {
            int q = S.struct_pos[S.struct_ptr[J] + x];
            int r;
            if (q >= pp0 && q < pp0 + pn)
                r = q - pp0;
            else
                r = pn + (int)(std::lower_bound(ps, ps + S.mJ[P], q) - ps);
            S.rel[S.struct_ptr[J] + x] = r;
        }
    }
    // heights and level groups
    S.height.assign(nn, 0);
    int H = 0;
    for (int J = 0; J < nn; ++J) {
        int h = 0;
        for (int c = S.child_ptr[J]; c < S.child_ptr[J + 1]; ++c) h = std::max(h, S.height[S.child_idx[c]] + 1);
        S.height[J] = h;
        H = std::max(H, h);
    }
    S.level_ptr.assign(H + 2, 0);
    for (int J = 0; J < nn; ++J) S.level_ptr[S.height[J] + 1]++;
    for (int h = 0; h <= H; ++h) S.level_ptr[h + 1] += S.level_ptr[h];
    S.level_nodes.assign(nn, 0);
    {
        std::vector<int> fill(S.level_ptr.begin(), S.level_ptr.end() - 1);
        for (int J = 0; J < nn; ++J) S.level_nodes[fill[S.height[J]]++] = J;
    }
    // storage offsets
    S.loff.resize(nn);
    S.uoff.resize(nn);
    S.voff.resize(nn);
    for (int J = 0; J < nn; ++J) {
        const int64_t n_ = S.nJ[J], m_ = S.mJ[J];
        // L11^-1 (n x n) and L21 (m x n) are stored column-major with odd
        // leading dimensions (n | 1, m | 1): rows and columns are then both
        // read without shared-memory bank conflicts; blocks start on 16-byte
        // boundaries
        S.loff[J] = S.lsize;
        S.lsize += (n_ * chol_ld(n_) + n_ * chol_ld(m_) + 3) & ~int64_t(3);
        S.uoff[J] = S.usize;
        S.usize += m_ * m_;
        S.voff[J] = S.vsize;
        S.vsize += (int)m_;
        const int t = (int)(n_ + m_);
        S.max_t = std::max(S.max_t, t);
        S.max_panel = std::max(S.max_panel, (int64_t)t * n_);
        S.max_nJ = std::max(S.max_nJ, (int)n_);
    }
    // original entries of each column block (lower part: rows at or after the column)
    S.asm_ptr.assign(nn + 1, 0);
    for (int J = 0; J < nn; ++J) {
        const int p0 = S.p0[J], n_ = S.nJ[J], t = n_ + S.mJ[J], end = p0 + n_;
        const int* ps = S.struct_pos.data() + S.struct_ptr[J];
        for (int a = 0; a < n_; ++a) {
            int v = S.perm[p0 + a];
            for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                int q = S.pos[col[e]];
                if (q < p0 + a) continue;   // pinned (-1) or an earlier column's entry
                int r = q < end ? q - p0 : n_ + (int)(std::lower_bound(ps, ps + S.mJ[J], q) - ps);
                S.asm_dst.push_back(r + a * t);
                S.asm_src.push_back(e);
            }
        }
        S.asm_ptr[J + 1] = (int)S.asm_dst.size();
    }
    return true;
}

}  // namespace tp
