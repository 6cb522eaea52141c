// Host helpers of the mesh and pin code (plain C++, no CUDA, so that they
// are also exercised on the CPU by a test driver):
//   - connected components of a triangle mesh through its face edges
//     (union-find), labelled in the order of their smallest vertex;
//   - the inverse of a small dense matrix (Gauss-Jordan with partial
//     pivoting), used for the pins' (pins + components) system.
#pragma once

#include <cmath>
#include <utility>
#include <vector>

namespace tp {

// comp[v] = component of vertex v; returns the number of components.
// faces: 3 vertex indices per face, all in 0..nv-1.
inline int label_components(int nv, const std::vector<int>& faces, std::vector<int>& comp) {
    std::vector<int> parent(nv);
    for (int v = 0; v < nv; ++v) parent[v] = v;
    auto find = [&](int x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    for (size_t e = 0; e + 2 < faces.size(); e += 3)
        for (int c = 0; c < 3; ++c) {
            const int a = find(faces[e + c]), b = find(faces[e + (c + 1) % 3]);
            if (a != b) parent[a > b ? a : b] = a < b ? a : b;
        }
    std::vector<int> label(nv, -1);
    comp.assign(nv, 0);
    int nc = 0;
    for (int v = 0; v < nv; ++v) {
        const int r = find(v);
        if (label[r] < 0) label[r] = nc++;
        comp[v] = label[r];
    }
    return nc;
}

// inv = a^-1 for a row-major n x n matrix; false if a pivot is exactly 0
inline bool invert_dense(std::vector<double> a, int n, std::vector<double>& inv) {
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = r;
        if (!(std::fabs(a[(size_t)piv * n + c]) > 0.0)) return false;
        if (piv != c)
            for (int q = 0; q < n; ++q) {
                std::swap(a[(size_t)c * n + q], a[(size_t)piv * n + q]);
                std::swap(inv[(size_t)c * n + q], inv[(size_t)piv * n + q]);
            }
        const double d = 1.0 / a[(size_t)c * n + c];
        for (int q = 0; q < n; ++q) {
            a[(size_t)c * n + q] *= d;
            inv[(size_t)c * n + q] *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = a[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int q = 0; q < n; ++q) {
                a[(size_t)r * n + q] -= f * a[(size_t)c * n + q];
                inv[(size_t)r * n + q] -= f * inv[(size_t)c * n + q];
            }
        }
    }
    return true;
}

}  // namespace tp
