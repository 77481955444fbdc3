// Host-side symbolic analysis for the LDL^T of S_M: fill-reducing orderings and the pattern
// of L for a given ordering.  Plain C++ (no CUDA), so it can also be exercised on the CPU.
//
//  * minimum_degree: explicit elimination graph, ties broken by the smallest index; gives up
//    (returns false) once the fill exceeds a budget.  Near optimality S_M is chordal (the
//    corollary of Theorem 2) and minimum degree then eliminates with little or no fill.
//  * mcs_order: maximum cardinality search (Tarjan & Yannakakis, SIAM J. Comput. 13, 1984); its
//    reverse is a perfect elimination ordering exactly when the graph is chordal, so with it a
//    chordal S_M factors with zero fill (Theorem 1 of the paper).
//  * nested_dissection: automatic nested dissection by level structures (George & Liu,
//    "Computer Solution of Large Sparse Positive Definite Systems", 1981): on each connected
//    part, BFS from a pseudo-peripheral node, the middle level is a separator (edges only join
//    adjacent levels), both sides are ordered recursively, the separator last.
//  * symbolic_factor: elimination tree (Liu's algorithm with path compression) and the row
//    structure of L by walking the tree from each entry of the permuted lower triangle up to
//    the row; column patterns come out sorted.  O(nnz(L)).
#pragma once

#include <algorithm>
#include <cstdint>
#include <queue>
#include <set>
#include <vector>

namespace ot {
namespace ordering {

struct Graph {
    int n = 0;
    std::vector<int32_t> ptr, adj;  // symmetric, no self loops, sorted rows
};

inline bool minimum_degree(const Graph &g, int64_t max_fill, std::vector<int32_t> &perm) {
    const int n = g.n;
    std::vector<std::vector<int32_t>> adj(n);
    for (int r = 0; r < n; ++r) adj[r].assign(g.adj.begin() + g.ptr[r], g.adj.begin() + g.ptr[r + 1]);
    std::set<std::pair<int32_t, int32_t>> pq;
    std::vector<int32_t> deg(n);
    for (int r = 0; r < n; ++r) { deg[r] = (int32_t)adj[r].size(); pq.insert({deg[r], r}); }
    perm.assign(n, 0);
    int64_t fill = 0;
    std::vector<int32_t> tmp;
    for (int q = 0; q < n; ++q) {
        const int v = pq.begin()->second;
        pq.erase(pq.begin());
        perm[q] = v;
        std::vector<int32_t> nb;
        nb.swap(adj[v]);
        fill += (int64_t)nb.size();
        if (fill > max_fill) return false;
        for (int a : nb) {
            auto &la = adj[a];
            tmp.clear();
            std::set_union(la.begin(), la.end(), nb.begin(), nb.end(), std::back_inserter(tmp));
            la.clear();
            for (int x : tmp)
                if (x != a && x != v) la.push_back(x);
            pq.erase({deg[a], a});
            deg[a] = (int32_t)la.size();
            pq.insert({deg[a], a});
        }
    }
    return true;
}

// Reverse maximum-cardinality-search order (perm[q] = vertex eliminated q-th).
inline void mcs_order(const Graph &g, std::vector<int32_t> &perm) {
    const int n = g.n;
    std::vector<int32_t> weight(n, 0), order(n);
    std::vector<char> done(n, 0);
    // bucket lists by weight (doubly linked), pick the largest weight, ties: smallest index
    std::vector<std::set<int32_t>> bucket(n + 1);
    for (int v = 0; v < n; ++v) bucket[0].insert(v);
    int top = 0;
    for (int step = n - 1; step >= 0; --step) {
        while (top > 0 && bucket[top].empty()) --top;
        const int v = *bucket[top].begin();
        bucket[top].erase(bucket[top].begin());
        done[v] = 1;
        order[step] = v;  // visited first -> eliminated last
        for (int e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
            const int w = g.adj[e];
            if (done[w]) continue;
            bucket[weight[w]].erase(w);
            ++weight[w];
            bucket[weight[w]].insert(w);
            if (weight[w] > top) top = weight[w];
        }
    }
    perm = order;
}

namespace detail {

// BFS over the vertices with mark == tag; fills levels (vertex lists) from `start`
inline void bfs_levels(const Graph &g, int start, const std::vector<int32_t> &mark, int tag,
                       std::vector<int32_t> &level_of, std::vector<std::vector<int32_t>> &levels) {
    levels.clear();
    std::vector<int32_t> cur{start};
    level_of[start] = 0;
    while (!cur.empty()) {
        levels.push_back(cur);
        std::vector<int32_t> nxt;
        for (int v : cur)
            for (int e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
                const int w = g.adj[e];
                if (mark[w] == tag && level_of[w] < 0) {
                    level_of[w] = (int32_t)levels.size();
                    nxt.push_back(w);
                }
            }
        cur.swap(nxt);
    }
}

}  // namespace detail

inline void nested_dissection(const Graph &g, std::vector<int32_t> &perm, int leaf = 64) {
    const int n = g.n;
    perm.clear();
    perm.reserve(n);
    std::vector<int32_t> mark(n, -1), level_of(n, -1);
    std::vector<std::vector<int32_t>> levels;
    // work stack of (vertex set, state); a set is pushed as: separator-after marker, then parts
    struct Item { std::vector<int32_t> verts; bool emit; };
    std::vector<Item> stack;
    std::vector<int32_t> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    stack.push_back({all, false});
    int tag = 0;
    while (!stack.empty()) {
        Item it = std::move(stack.back());
        stack.pop_back();
        if (it.emit) {
            perm.insert(perm.end(), it.verts.begin(), it.verts.end());
            continue;
        }
        auto &vs = it.verts;
        if ((int)vs.size() <= leaf) {
            std::sort(vs.begin(), vs.end());
            perm.insert(perm.end(), vs.begin(), vs.end());
            continue;
        }
        ++tag;
        for (int v : vs) { mark[v] = tag; level_of[v] = -1; }
        // split into connected parts first
        std::vector<std::vector<int32_t>> parts;
        for (int v : vs) {
            if (level_of[v] >= 0) continue;
            detail::bfs_levels(g, v, mark, tag, level_of, levels);
            std::vector<int32_t> comp;
            for (auto &l : levels) comp.insert(comp.end(), l.begin(), l.end());
            parts.push_back(std::move(comp));
        }
        if (parts.size() > 1) {
            for (auto &p : parts) stack.push_back({std::move(p), false});
            continue;
        }
        // one connected part: pseudo-peripheral start (repeat BFS from the farthest vertex)
        auto &comp = parts[0];
        int start = comp[0];
        int depth = 0;
        for (int rep = 0; rep < 4; ++rep) {
            for (int v : comp) level_of[v] = -1;
            detail::bfs_levels(g, start, mark, tag, level_of, levels);
            if ((int)levels.size() <= depth) break;
            depth = (int)levels.size();
            const auto &last = levels.back();
            int best = last[0], bd = 1 << 30;
            for (int v : last) {
                int d = 0;
                for (int e = g.ptr[v]; e < g.ptr[v + 1]; ++e) d += mark[g.adj[e]] == tag;
                if (d < bd) { bd = d; best = v; }
            }
            start = best;
        }
        for (int v : comp) level_of[v] = -1;
        detail::bfs_levels(g, start, mark, tag, level_of, levels);
        if (levels.size() < 3) {  // no separating level: order the part as it is
            std::sort(comp.begin(), comp.end());
            perm.insert(perm.end(), comp.begin(), comp.end());
            continue;
        }
        // separator: the level that splits the vertices most evenly
        const int64_t total = (int64_t)comp.size();
        int64_t acc = 0;
        int sep = 1;
        for (int l = 0; l < (int)levels.size(); ++l) {
            if (acc + (int64_t)levels[l].size() / 2 >= total / 2) { sep = std::max(1, std::min(l, (int)levels.size() - 2)); break; }
            acc += (int64_t)levels[l].size();
        }
        std::vector<int32_t> a, b;
        for (int l = 0; l < sep; ++l) a.insert(a.end(), levels[l].begin(), levels[l].end());
        for (int l = sep + 1; l < (int)levels.size(); ++l) b.insert(b.end(), levels[l].begin(), levels[l].end());
        std::vector<int32_t> s = levels[sep];
        std::sort(s.begin(), s.end());
        stack.push_back({std::move(s), true});   // separator emitted after both sides
        stack.push_back({std::move(b), false});
        stack.push_back({std::move(a), false});
    }
}

// Pattern of the strictly lower L of P A P^T (perm[q] = original index of position q).
// Returns false when nnz(L) would exceed max_nnz.
inline bool symbolic_factor(const Graph &g, const std::vector<int32_t> &perm, int64_t max_nnz,
                            std::vector<int32_t> &Lp, std::vector<int32_t> &Li) {
    const int n = g.n;
    std::vector<int32_t> iperm(n);
    for (int q = 0; q < n; ++q) iperm[perm[q]] = q;
    // lower-triangular entries of the permuted matrix by row: for row i, columns k < i
    std::vector<int32_t> parent(n, -1), anc(n, -1);
    for (int i = 0; i < n; ++i) {
        const int v = perm[i];
        for (int e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
            int k = iperm[g.adj[e]];
            if (k >= i) continue;
            while (k != -1 && k != i) {  // climb with path compression to the current root
                const int nk = anc[k];
                anc[k] = i;
                if (nk == -1) parent[k] = i;
                k = nk;
            }
        }
    }
    // row structures by walking up the tree; columns receive rows in increasing order
    std::vector<int32_t> cnt(n, 0), flag(n, -1);
    std::vector<int32_t> rows;  // (row, col) pairs appended per row
    std::vector<std::vector<int32_t>> colrows(n);
    int64_t nnz = 0;
    for (int i = 0; i < n; ++i) {
        flag[i] = i;
        const int v = perm[i];
        for (int e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
            int k = iperm[g.adj[e]];
            if (k >= i) continue;
            while (k != -1 && flag[k] != i) {
                colrows[k].push_back(i);
                flag[k] = i;
                if (++nnz > max_nnz) return false;
                k = parent[k];
            }
        }
    }
    Lp.assign(n + 1, 0);
    Li.clear();
    Li.reserve(nnz);
    for (int q = 0; q < n; ++q) {
        Li.insert(Li.end(), colrows[q].begin(), colrows[q].end());
        Lp[q + 1] = (int32_t)Li.size();
    }
    return true;
}

}  // namespace ordering
}  // namespace ot
