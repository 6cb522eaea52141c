// Test driver for the host helpers of host_util.h. Reads a request on stdin
// and prints the result on stdout:
//   components <nv> <nf> <3*nf face indices>   ->  <ncomp> <nv labels>
//   invert <n> <n*n row-major entries>          ->  ok <n*n entries> | singular
#include <cstdio>
#include <cstring>
#include <vector>

#include "host_util.h"

int main() {
    char cmd[32];
    if (std::scanf("%31s", cmd) != 1) return 2;
    if (std::strcmp(cmd, "components") == 0) {
        int nv, nf;
        if (std::scanf("%d %d", &nv, &nf) != 2) return 2;
        std::vector<int> F(3 * (size_t)nf);
        for (auto& x : F)
            if (std::scanf("%d", &x) != 1) return 2;
        std::vector<int> comp;
        const int nc = tp::label_components(nv, F, comp);
        std::printf("%d", nc);
        for (int c : comp) std::printf(" %d", c);
        std::printf("\n");
        return 0;
    }
    if (std::strcmp(cmd, "invert") == 0) {
        int n;
        if (std::scanf("%d", &n) != 1) return 2;
        std::vector<double> a((size_t)n * n), inv;
        for (auto& x : a)
            if (std::scanf("%lf", &x) != 1) return 2;
        if (!tp::invert_dense(a, n, inv)) {
            std::printf("singular\n");
            return 0;
        }
        std::printf("ok");
        for (double x : inv) std::printf(" %.17g", x);
        std::printf("\n");
        return 0;
    }
    return 2;
}
