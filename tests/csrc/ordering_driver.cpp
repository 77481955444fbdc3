// Test driver for paper_2206_11009_gb300/csrc/ordering.h (host C++ only).
// stdin:  mode n nnz  then nnz pairs "r c" (symmetric pattern, both triangles)
//   mode 0: minimum degree (large budget); mode 1: nested dissection; mode 2: reverse MCS
// stdout: perm (n ints), then Lp (n+1 ints), then Li
#include <cstdio>
#include <vector>

#include "ordering.h"

int main() {
    int mode, n;
    long long nnz;
    if (scanf("%d %d %lld", &mode, &n, &nnz) != 3) return 1;
    std::vector<std::vector<int>> rows(n);
    for (long long e = 0; e < nnz; ++e) {
        int r, c;
        if (scanf("%d %d", &r, &c) != 2) return 1;
        rows[r].push_back(c);
    }
    ot::ordering::Graph g;
    g.n = n;
    g.ptr.assign(n + 1, 0);
    for (int r = 0; r < n; ++r) {
        std::sort(rows[r].begin(), rows[r].end());
        rows[r].erase(std::unique(rows[r].begin(), rows[r].end()), rows[r].end());
        g.adj.insert(g.adj.end(), rows[r].begin(), rows[r].end());
        g.ptr[r + 1] = (int)g.adj.size();
    }
    std::vector<int32_t> perm, Lp, Li;
    if (mode == 0) {
        if (!ot::ordering::minimum_degree(g, 1LL << 40, perm)) return 2;
    } else if (mode == 1) {
        ot::ordering::nested_dissection(g, perm, 8);
    } else {
        ot::ordering::mcs_order(g, perm);
    }
    if (!ot::ordering::symbolic_factor(g, perm, 1LL << 40, Lp, Li)) return 3;
    for (int q = 0; q < n; ++q) printf("%d ", perm[q]);
    printf("\n");
    for (int q = 0; q <= n; ++q) printf("%d ", Lp[q]);
    printf("\n");
    for (size_t t = 0; t < Li.size(); ++t) printf("%d ", Li[t]);
    printf("\n");
    return 0;
}
