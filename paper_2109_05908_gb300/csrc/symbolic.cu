// Symbolic phase of a sparse local Cholesky factorisation (the local solver of
// Sec. 4.1 is an exact Cholesky factorisation of A_ii; a sparse factor in a
// fill-reducing order has the same solution and far fewer entries than the
// dense one).  Host code only, no GPU involved:
//   * nested dissection (George 1973): a set larger than the leaf size is cut
//     by a level set of a breadth-first search from a pseudo-peripheral
//     vertex, the two sides are ordered first (recursively) and the
//     separator last; disconnected sets are ordered component by component;
//   * the elimination tree of the permuted pattern (Liu 1986, with path
//     compression) and the column counts of the factor from the row subtrees
//     (row i of L is the union of the tree paths from its below-diagonal
//     entries up to i).
#include "amdd_internal.h"
#include "amdd.h"

#include <algorithm>
#include <vector>

namespace {

struct Graph {
    int n;
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
};

// symmetric adjacency without the diagonal, each list ascending and unique
Graph symmetrise(int n, const int64_t* rowptr, const int32_t* colind) {
    std::vector<std::vector<int32_t>> lists(n);
    for (int r = 0; r < n; ++r)
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            const int32_t c = colind[k];
            if (c == r) continue;
            lists[r].push_back(c);
            lists[c].push_back(r);
        }
    Graph g;
    g.n = n;
    g.ptr.assign(n + 1, 0);
    for (int r = 0; r < n; ++r) {
        auto& l = lists[r];
        std::sort(l.begin(), l.end());
        l.erase(std::unique(l.begin(), l.end()), l.end());
        g.ptr[r + 1] = g.ptr[r] + (int64_t)l.size();
    }
    g.adj.reserve(g.ptr[n]);
    for (int r = 0; r < n; ++r) g.adj.insert(g.adj.end(), lists[r].begin(), lists[r].end());
    return g;
}

struct Dissect {
    const Graph& g;
    int leaf;
    std::vector<int> tag;    // set id of each vertex (a vertex is in the set being split iff tag == cur)
    std::vector<int> level;  // BFS level scratch
    std::vector<int32_t> order;
    int next_tag = 1;

    Dissect(const Graph& gg, int lf) : g(gg), leaf(lf), tag(gg.n, 0), level(gg.n, -1) {}

    // BFS inside the set `t` from s: visit order, levels in `level`
    std::vector<int32_t> bfs(int32_t s, int t) {
        std::vector<int32_t> q{s};
        level[s] = 0;
        for (size_t h = 0; h < q.size(); ++h) {
            const int32_t v = q[h];
            for (int64_t k = g.ptr[v]; k < g.ptr[v + 1]; ++k) {
                const int32_t w = g.adj[k];
                if (tag[w] == t && level[w] < 0) {
                    level[w] = level[v] + 1;
                    q.push_back(w);
                }
            }
        }
        return q;
    }
    void clear_levels(const std::vector<int32_t>& vs) {
        for (int32_t v : vs) level[v] = -1;
    }
    int degree_in(int32_t v, int t) const {
        int d = 0;
        for (int64_t k = g.ptr[v]; k < g.ptr[v + 1]; ++k) d += tag[g.adj[k]] == t;
        return d;
    }

    // order the vertices of `set` (all tagged t) and append them to `order`
    void run(std::vector<int32_t> set, int t) {
        if (set.empty()) return;
        // connected components first
        std::vector<int32_t> comp = bfs(set[0], t);
        if (comp.size() < set.size()) {
            std::vector<std::vector<int32_t>> comps;
            for (int32_t v : set)
                if (level[v] < 0) {
                    std::vector<int32_t> c = bfs(v, t);
                    comps.push_back(c);
                }
            clear_levels(set);
            comps.insert(comps.begin(), comp);
            for (auto& c : comps) {
                const int tc = next_tag++;
                for (int32_t v : c) tag[v] = tc;
                run(c, tc);
            }
            return;
        }
        if ((int)set.size() <= leaf) {
            order.insert(order.end(), comp.begin(), comp.end());  // BFS order inside a leaf
            clear_levels(comp);
            return;
        }
        // pseudo-peripheral start: a farthest vertex of least degree, while the
        // eccentricity grows (at most a few sweeps)
        int ecc = level[comp.back()];
        int32_t start = comp[0];
        for (int sweep = 0; sweep < 4; ++sweep) {
            int32_t best = comp.back();
            int bd = degree_in(best, t);
            for (auto it = comp.rbegin(); it != comp.rend() && level[*it] == ecc; ++it) {
                const int d = degree_in(*it, t);
                if (d < bd) {
                    bd = d;
                    best = *it;
                }
            }
            clear_levels(comp);
            std::vector<int32_t> c2 = bfs(best, t);
            const int e2 = level[c2.back()];
            if (e2 <= ecc && sweep > 0) {
                clear_levels(c2);
                comp = bfs(start, t);
                break;
            }
            start = best;
            ecc = e2;
            comp.swap(c2);
        }
        const int nlev = ecc + 1;
        if (nlev < 3) {  // no level set separates it: a leaf
            order.insert(order.end(), comp.begin(), comp.end());
            clear_levels(comp);
            return;
        }
        // the middle level by count, kept off the ends so both sides are non-empty
        std::vector<int64_t> cnt(nlev, 0);
        for (int32_t v : comp) ++cnt[level[v]];
        int mid = 1;
        int64_t acc = cnt[0];
        while (mid < nlev - 2 && acc + cnt[mid] < (int64_t)comp.size() / 2) acc += cnt[mid++];
        // separator: the vertices of the middle level with a neighbour beyond it
        // (the others join the near side)
        std::vector<int32_t> A, B, S;
        for (int32_t v : comp) {
            const int l = level[v];
            if (l < mid) {
                A.push_back(v);
            } else if (l > mid) {
                B.push_back(v);
            } else {
                bool far = false;
                for (int64_t k = g.ptr[v]; k < g.ptr[v + 1] && !far; ++k) {
                    const int32_t w = g.adj[k];
                    far = tag[w] == t && level[w] == mid + 1;
                }
                (far ? S : A).push_back(v);
            }
        }
        clear_levels(comp);
        const int ta = next_tag++, tb = next_tag++, ts = next_tag++;
        for (int32_t v : A) tag[v] = ta;
        for (int32_t v : B) tag[v] = tb;
        for (int32_t v : S) tag[v] = ts;
        run(A, ta);
        run(B, tb);
        order.insert(order.end(), S.begin(), S.end());
    }
};

}  // namespace

namespace amdd {

bool nd_factor_pattern(int n, const int64_t* rowptr, const int32_t* colind, int leaf, std::vector<int32_t>& perm,
                       std::vector<int32_t>& colptr, std::vector<int32_t>& rows) {
    if (n < 0 || leaf < 1 || (n > 0 && (!rowptr || !colind)) || (n > 0 && rowptr[0] != 0)) return false;
    for (int r = 0; r < n; ++r)
        if (rowptr[r + 1] < rowptr[r]) return false;
    for (int64_t k = 0; n > 0 && k < rowptr[n]; ++k)
        if (colind[k] < 0 || colind[k] >= n) return false;
    perm.assign(n, 0);
    colptr.assign(n + 1, 0);
    rows.clear();
    if (n == 0) return true;
    const Graph g = symmetrise(n, rowptr, colind);
    Dissect d(g, leaf);
    std::vector<int32_t> all(n);
    for (int v = 0; v < n; ++v) all[v] = v;
    d.run(all, 0);
    if ((int)d.order.size() != n) return false;
    std::vector<int32_t> iperm(n);
    for (int k = 0; k < n; ++k) {
        perm[k] = d.order[k];
        iperm[d.order[k]] = k;
    }
    // elimination tree of P A P^T (ancestor path compression)
    std::vector<int32_t> par(n, -1), anc(n, -1);
    for (int k = 0; k < n; ++k) {
        const int32_t v = perm[k];
        for (int64_t q = g.ptr[v]; q < g.ptr[v + 1]; ++q) {
            int32_t j = iperm[g.adj[q]];
            if (j >= k) continue;
            while (anc[j] != -1 && anc[j] != k) {
                const int32_t nx = anc[j];
                anc[j] = k;
                j = nx;
            }
            if (anc[j] == -1) {
                anc[j] = k;
                par[j] = k;
            }
        }
    }
    // row i of the factor holds the columns of its row subtree: the paths from
    // each j < i with a_ij != 0 up the tree to i; collected column by column,
    // so each column lists its rows in ascending order after the diagonal
    std::vector<std::vector<int32_t>> col(n);
    for (int j = 0; j < n; ++j) col[j].push_back(j);
    std::vector<int32_t> mark(n, -1);
    for (int i = 0; i < n; ++i) {
        mark[i] = i;
        const int32_t v = perm[i];
        for (int64_t q = g.ptr[v]; q < g.ptr[v + 1]; ++q) {
            int32_t j = iperm[g.adj[q]];
            if (j >= i) continue;
            while (mark[j] != i) {
                col[j].push_back(i);
                mark[j] = i;
                j = par[j];
            }
        }
    }
    for (int j = 0; j < n; ++j) colptr[j + 1] = colptr[j] + (int32_t)col[j].size();
    rows.reserve(colptr[n]);
    for (int j = 0; j < n; ++j) rows.insert(rows.end(), col[j].begin(), col[j].end());
    return true;
}

}  // namespace amdd

extern "C" amdd_status amdd_nd_order(int64_t n, const int64_t* rowptr, const int32_t* colind, int32_t leaf,
                                     int32_t* perm, int32_t* parent, int64_t* colcount, int64_t* nnzL) {
    if (n < 0 || n > INT32_MAX || leaf < 1 || (n > 0 && (!rowptr || !colind || !perm))) return AMDD_ERR_INVALID;
    if (n == 0) {
        if (nnzL) *nnzL = 0;
        return AMDD_OK;
    }
    if (rowptr[0] != 0) return AMDD_ERR_INVALID;
    for (int64_t r = 0; r < n; ++r)
        if (rowptr[r + 1] < rowptr[r]) return AMDD_ERR_INVALID;
    for (int64_t k = 0; k < rowptr[n]; ++k)
        if (colind[k] < 0 || colind[k] >= n) return AMDD_ERR_INVALID;
    try {
        const int N = (int)n;
        const Graph g = symmetrise(N, rowptr, colind);
        Dissect d(g, leaf);
        std::vector<int32_t> all(N);
        for (int v = 0; v < N; ++v) all[v] = v;
        std::fill(d.tag.begin(), d.tag.end(), 0);
        d.run(all, 0);
        if ((int)d.order.size() != N) return AMDD_ERR_INVALID;
        std::vector<int32_t> iperm(N);
        for (int k = 0; k < N; ++k) {
            perm[k] = d.order[k];
            iperm[d.order[k]] = k;
        }
        // elimination tree of P A P^T
        std::vector<int32_t> par(N, -1), anc(N, -1);
        for (int k = 0; k < N; ++k) {
            const int32_t v = perm[k];
            for (int64_t q = g.ptr[v]; q < g.ptr[v + 1]; ++q) {
                int32_t j = iperm[g.adj[q]];
                if (j >= k) continue;
                while (anc[j] != -1 && anc[j] != k) {
                    const int32_t nx = anc[j];
                    anc[j] = k;  // path compression
                    j = nx;
                }
                if (anc[j] == -1) {
                    anc[j] = k;
                    par[j] = k;
                }
            }
        }
        // column counts from the row subtrees
        std::vector<int64_t> cc(N, 1);
        std::vector<int32_t> mark(N, -1);
        for (int i = 0; i < N; ++i) {
            mark[i] = i;
            const int32_t v = perm[i];
            for (int64_t q = g.ptr[v]; q < g.ptr[v + 1]; ++q) {
                int32_t j = iperm[g.adj[q]];
                if (j >= i) continue;
                while (mark[j] != i) {
                    ++cc[j];
                    mark[j] = i;
                    j = par[j];
                }
            }
        }
        int64_t tot = 0;
        for (int k = 0; k < N; ++k) tot += cc[k];
        if (parent) std::copy(par.begin(), par.end(), parent);
        if (colcount) std::copy(cc.begin(), cc.end(), colcount);
        if (nnzL) *nnzL = tot;
    } catch (const std::bad_alloc&) {
        return AMDD_ERR_OOM;
    }
    return AMDD_OK;
}
