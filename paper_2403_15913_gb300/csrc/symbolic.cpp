// Host symbolic analysis of the condensed KKT matrix K = W + J^T D J + diag
// (Sec. V-B: computed once for the fixed pattern, reused by every numeric
// refactorisation).
//
// The ordering is fully specified so that results are reproducible:
//  1. graph G = pattern(W + J^T J) without self loops;
//  2. level-structure nested dissection (George & Liu 1981): components in
//     increasing order of their smallest node; components of at most
//     leaf_size nodes (or with fewer than three BFS levels) are ordered by
//     exact minimum degree (ties to the smallest index); otherwise a
//     pseudo-peripheral node is found from the smallest node (repeat: BFS,
//     take the minimum-degree node of the last level, ties to the smallest
//     index, keep it while the number of levels grows); with levels
//     L_0..L_e the separator is { v in L_{e/2} adjacent to L_{e/2+1} };
//     the rest is ordered recursively, then the separator by index;
//  3. elimination tree (Liu, path compression), depth-first postorder with
//     children and roots in increasing index;
//  4. column counts by structure union over etree children;
//  5. fundamental supernodes, then one backward relaxation pass
//     (merge s into the following supernode when parent(last(s)) lies in
//     it, the merged width is <= relax_cols and the merged panel holds
//     <= relax_zeros explicit zeros), then cuts at max_width columns;
//  6. supernode rows: cols(s) u lower neighbours u rows of child supernodes,
//     restricted to rows beyond last(s).
#include "symbolic.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <future>
#include <numeric>
#include <set>
#include <thread>

namespace kktgb {

namespace {
// body(lo, hi) over [0, n): on threads in contiguous ranges when n is large
// (every range independent), else in one call
constexpr int kParallelGraphNodes = 100000;
template <typename F>
void for_ranges(int n, F&& body) {
    const int hw = (int)std::min(16u, std::max(1u, std::thread::hardware_concurrency()));
    if (n < kParallelGraphNodes || hw < 2) { body(0, n); return; }
    std::vector<std::future<void>> running;
    for (int t = 1; t < hw; ++t) {
        const int lo = (int)((long long)n * t / hw), hi = (int)((long long)n * (t + 1) / hw);
        running.push_back(std::async(std::launch::async | std::launch::deferred, [&body, lo, hi] { body(lo, hi); }));
    }
    body(0, (int)((long long)n / hw));
    for (auto& f : running) f.get();
}
}  // namespace

std::string build_graph(int n, int m, const int* W_colptr, const int* W_rowind,
                        const int* J_rowptr, const int* J_colind, Graph& g) {
    if (n <= 0 || m < 0) return "n must be positive and m non-negative";
    if (!W_colptr || !J_rowptr || (m > 0 && !J_colind)) return "NULL pattern array";
    if (W_colptr[0] != 0) return "W_colptr[0] must be 0";
    for (int j = 0; j < n; ++j)
        if (W_colptr[j + 1] < W_colptr[j]) return "W_colptr not monotone";
    if (W_colptr[n] > 0 && !W_rowind) return "NULL W_rowind";
    for (int j = 0; j < n; ++j)
        for (int p = W_colptr[j]; p < W_colptr[j + 1]; ++p) {
            int i = W_rowind[p];
            if (i < j || i >= n) return "W pattern entry outside the lower triangle";
        }
    if (J_rowptr[0] != 0) return "J_rowptr[0] must be 0";
    // a row of J may not name a column twice: every pair of entries of a row
    // becomes one product J_ra J_rb of J^T D J, which a repeated column would
    // get wrong (and the counts below assume distinct columns)
    std::vector<int> seen(n, -1);
    for (int r = 0; r < m; ++r) {
        if (J_rowptr[r + 1] < J_rowptr[r]) return "J_rowptr not monotone";
        for (int p = J_rowptr[r]; p < J_rowptr[r + 1]; ++p) {
            const int c = J_colind[p];
            if (c < 0 || c >= n) return "J column index out of range";
            if (seen[c] == r) return "a row of J repeats a column index";
            seen[c] = r;
        }
    }
    std::vector<int64_t> cnt(n + 1, 0);
    for (int j = 0; j < n; ++j)
        for (int p = W_colptr[j]; p < W_colptr[j + 1]; ++p)
            if (W_rowind[p] != j) { cnt[W_rowind[p]]++; cnt[j]++; }
    for (int r = 0; r < m; ++r) {
        int q = J_rowptr[r + 1] - J_rowptr[r];
        for (int p = J_rowptr[r]; p < J_rowptr[r + 1]; ++p) cnt[J_colind[p]] += q - 1;
    }
    std::vector<int64_t> ptr(n + 1, 0);
    for (int i = 0; i < n; ++i) ptr[i + 1] = ptr[i] + cnt[i];
    std::vector<int> tmp(ptr[n]);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int j = 0; j < n; ++j)
        for (int p = W_colptr[j]; p < W_colptr[j + 1]; ++p) {
            int i = W_rowind[p];
            if (i != j) { tmp[fill[i]++] = j; tmp[fill[j]++] = i; }
        }
    for (int r = 0; r < m; ++r)
        for (int p = J_rowptr[r]; p < J_rowptr[r + 1]; ++p)
            for (int q = J_rowptr[r]; q < J_rowptr[r + 1]; ++q)
                if (J_colind[p] != J_colind[q]) tmp[fill[J_colind[p]]++] = J_colind[q];
    // every node's list: sorted, duplicates and the node itself dropped (in
    // place, independent per node), then compacted; large graphs split the
    // nodes into ranges on threads, which changes nothing in the result
    g.n = n;
    std::vector<int64_t> len(n);
    auto dedup = [&](int lo, int hi) {
        for (int i = lo; i < hi; ++i) {
            auto b = tmp.begin() + ptr[i], e = tmp.begin() + ptr[i + 1];
            std::sort(b, e);
            auto u = std::remove(b, std::unique(b, e), i);
            len[i] = u - b;
        }
    };
    g.xadj.assign(n + 1, 0);
    for_ranges(n, dedup);
    for (int i = 0; i < n; ++i) g.xadj[i + 1] = g.xadj[i] + len[i];
    g.adj.resize(g.xadj[n]);
    for_ranges(n, [&](int lo, int hi) {
        for (int i = lo; i < hi; ++i)
            std::copy(tmp.begin() + ptr[i], tmp.begin() + ptr[i] + len[i], g.adj.begin() + g.xadj[i]);
    });
    return "";
}

namespace {

// ----------------------------------------------------------- nested dissection
//
// The components left by a separator are disconnected from one another, and
// every node adjacent to one of them is already numbered (tag 0, never
// written again), so the recursion on sibling components touches disjoint
// entries of tag / stamp / level.  The top levels of the recursion therefore
// run sibling components on their own threads, each writing its ordering into
// its own vector; the vectors are concatenated in component order, so the
// result is the one of the sequential recursion.  Tags and stamps only encode
// membership and visits: any unique value works, so both come from atomic
// counters.
constexpr int kParallelDepth = 4;         // recursion levels that fork
constexpr int kParallelMinNodes = 4096;   // smaller components stay sequential

struct NestedDissection {
    const Graph& g;
    int leaf;
    bool parallel;
    std::vector<int> tag;     // set membership: nodes of the component being
                              // processed carry its tag; numbered nodes carry 0
    std::atomic<int> next_tag{1};
    std::vector<int> stamp;   // BFS visit stamps
    std::vector<int> level;   // BFS level of stamped nodes
    std::atomic<int> next_stamp{0};
    std::vector<int> order;

    NestedDissection(const Graph& g_, int leaf_, bool parallel_)
        : g(g_), leaf(leaf_), parallel(parallel_) {
        tag.assign(g.n, 0);
        stamp.assign(g.n, 0);
        level.assign(g.n, -1);
        order.reserve(g.n);
    }

    // BFS level structure of root inside the nodes tagged t; returns the
    // flat node list and level pointers, and the stamp its visits carry.
    int bfs(int root, int t, std::vector<int>& nodes, std::vector<int>& lptr) {
        const int cur_stamp = ++next_stamp;
        nodes.clear();
        lptr.clear();
        nodes.push_back(root);
        stamp[root] = cur_stamp;
        level[root] = 0;
        lptr.push_back(0);
        size_t head = 0;
        int lv = 0;
        while (head < nodes.size()) {
            size_t end = nodes.size();
            lptr.push_back((int)end);   // provisional end of level lv
            for (size_t q = head; q < end; ++q) {
                int v = nodes[q];
                for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
                    int w = g.adj[p];
                    if (tag[w] == t && stamp[w] != cur_stamp) {
                        stamp[w] = cur_stamp;
                        level[w] = lv + 1;
                        nodes.push_back(w);
                    }
                }
            }
            head = end;
            ++lv;
        }
        // lptr has one entry per level start plus the final end
        lptr.back() = (int)nodes.size();
        return cur_stamp;
    }

    int degree_in(int v, int t) const {
        int d = 0;
        for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p)
            if (tag[g.adj[p]] == t) ++d;
        return d;
    }

    // components of the nodes tagged t among `nodes` (sorted ascending);
    // every component receives a fresh tag; returned in order of their
    // smallest node, each sorted ascending.
    void components(const std::vector<int>& nodes, int t,
                    std::vector<std::vector<int>>& comps, std::vector<int>& tags) {
        std::vector<int> stack;
        for (int s : nodes) {
            if (tag[s] != t) continue;
            int nt = next_tag++;
            std::vector<int> comp;
            tag[s] = nt;
            stack.push_back(s);
            while (!stack.empty()) {
                int v = stack.back();
                stack.pop_back();
                comp.push_back(v);
                for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
                    int w = g.adj[p];
                    if (tag[w] == t) { tag[w] = nt; stack.push_back(w); }
                }
            }
            std::sort(comp.begin(), comp.end());
            comps.push_back(std::move(comp));
            tags.push_back(nt);
        }
    }

    void minimum_degree(const std::vector<int>& comp, int t, std::vector<int>& order) {
        const int c = (int)comp.size();
        if (c == 0) return;
        // local index = rank in the sorted component (so ties to the
        // smallest local index are ties to the smallest original index)
        std::vector<int> loc_of;  // only for neighbours: binary search
        auto local = [&](int v) -> int {
            auto it = std::lower_bound(comp.begin(), comp.end(), v);
            return (it != comp.end() && *it == v) ? (int)(it - comp.begin()) : -1;
        };
        const int words = (c + 63) / 64;
        if ((int64_t)words * c <= (int64_t)1 << 26) {
            std::vector<uint64_t> bits((size_t)words * c, 0);
            auto row = [&](int a) { return bits.data() + (size_t)a * words; };
            for (int a = 0; a < c; ++a) {
                int v = comp[a];
                for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
                    int w = g.adj[p];
                    if (tag[w] != t) continue;
                    int b = local(w);
                    if (b >= 0) row(a)[b >> 6] |= 1ull << (b & 63);
                }
            }
            std::vector<char> alive(c, 1);
            std::vector<int> deg(c);
            for (int a = 0; a < c; ++a) {
                int d = 0;
                for (int w = 0; w < words; ++w) d += __builtin_popcountll(row(a)[w]);
                deg[a] = d;
            }
            std::vector<int> nb;
            for (int step = 0; step < c; ++step) {
                int best = -1;
                for (int a = 0; a < c; ++a)
                    if (alive[a] && (best < 0 || deg[a] < deg[best])) best = a;
                alive[best] = 0;
                order.push_back(comp[best]);
                uint64_t* rb = row(best);
                nb.clear();
                for (int w = 0; w < words; ++w) {
                    uint64_t x = rb[w];
                    while (x) {
                        int b = __builtin_ctzll(x);
                        nb.push_back(w * 64 + b);
                        x &= x - 1;
                    }
                }
                for (int a : nb) {
                    uint64_t* ra = row(a);
                    ra[best >> 6] &= ~(1ull << (best & 63));
                    int d = 0;
                    for (int w = 0; w < words; ++w) {
                        ra[w] |= rb[w];
                        if (w == (a >> 6)) ra[w] &= ~(1ull << (a & 63));
                        if (w == (best >> 6)) ra[w] &= ~(1ull << (best & 63));
                        d += __builtin_popcountll(ra[w]);
                    }
                    deg[a] = d;
                }
            }
        } else {
            std::vector<std::set<int>> gs(c);
            for (int a = 0; a < c; ++a) {
                int v = comp[a];
                for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
                    int w = g.adj[p];
                    if (tag[w] != t) continue;
                    int b = local(w);
                    if (b >= 0) gs[a].insert(b);
                }
            }
            std::vector<char> alive(c, 1);
            for (int step = 0; step < c; ++step) {
                int best = -1;
                for (int a = 0; a < c; ++a)
                    if (alive[a] && (best < 0 || gs[a].size() < gs[best].size())) best = a;
                alive[best] = 0;
                order.push_back(comp[best]);
                std::set<int> nbs = std::move(gs[best]);
                for (int a : nbs) {
                    gs[a].erase(best);
                    for (int b : nbs)
                        if (b != a) gs[a].insert(b);
                }
            }
        }
    }

    void component(const std::vector<int>& comp, int t, std::vector<int>& order, int depth) {
        if ((int)comp.size() <= leaf) { minimum_degree(comp, t, order); return; }
        std::vector<int> nodes, lptr, nodes2, lptr2;
        int r = comp[0];
        bfs(r, t, nodes, lptr);
        while (true) {
            int nlev = (int)lptr.size() - 1;
            int best = -1, bestd = 0;
            for (int q = lptr[nlev - 1]; q < lptr[nlev]; ++q) {
                int w = nodes[q];
                int d = degree_in(w, t);
                if (best < 0 || d < bestd || (d == bestd && w < best)) { best = w; bestd = d; }
            }
            bfs(best, t, nodes2, lptr2);
            if ((int)lptr2.size() > (int)lptr.size()) {
                r = best;
                nodes.swap(nodes2);
                lptr.swap(lptr2);
            } else {
                break;
            }
        }
        // `nodes`/`lptr` hold the level structure of r; re-run it so that the
        // stamps/levels correspond to r (the last BFS was of the candidate)
        const int cur_stamp = bfs(r, t, nodes, lptr);
        int e = (int)lptr.size() - 2;   // levels 0..e
        if (e < 2) { minimum_degree(comp, t, order); return; }
        int lv = e / 2;
        std::vector<int> sep;
        for (int q = lptr[lv]; q < lptr[lv + 1]; ++q) {
            int v = nodes[q];
            for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
                int w = g.adj[p];
                if (tag[w] == t && stamp[w] == cur_stamp && level[w] == lv + 1) {
                    sep.push_back(v);
                    break;
                }
            }
        }
        std::sort(sep.begin(), sep.end());
        for (int v : sep) tag[v] = 0;
        std::vector<int> rest;
        rest.reserve(comp.size() - sep.size());
        for (int v : comp)
            if (tag[v] == t) rest.push_back(v);
        std::vector<std::vector<int>> comps;
        std::vector<int> tags;
        components(rest, t, comps, tags);
        if (parallel && depth < kParallelDepth && comps.size() > 1 &&
            (int)comp.size() >= kParallelMinNodes) {
            // async | deferred: without a free thread the task runs here at get()
            std::vector<std::vector<int>> parts(comps.size());
            std::vector<std::future<void>> running;
            for (size_t i = 1; i < comps.size(); ++i)
                running.push_back(std::async(std::launch::async | std::launch::deferred,
                                             [this, &comps, &tags, &parts, i, depth] {
                    sub(comps[i], tags[i], parts[i], depth + 1);
                }));
            sub(comps[0], tags[0], parts[0], depth + 1);
            for (auto& f : running) f.get();
            for (auto& part : parts) order.insert(order.end(), part.begin(), part.end());
        } else {
            for (size_t i = 0; i < comps.size(); ++i) sub(comps[i], tags[i], order, depth + 1);
        }
        for (int v : sep) order.push_back(v);
    }

    // one component of a split: order it, then mark its nodes numbered
    void sub(std::vector<int>& c, int t, std::vector<int>& order, int depth) {
        component(c, t, order, depth);
        for (int v : c) tag[v] = 0;
    }

    void run() {
        std::vector<int> all(g.n);
        std::iota(all.begin(), all.end(), 0);
        int t0 = next_tag++;
        for (int v = 0; v < g.n; ++v) tag[v] = t0;
        std::vector<std::vector<int>> comps;
        std::vector<int> tags;
        components(all, t0, comps, tags);
        for (size_t i = 0; i < comps.size(); ++i) sub(comps[i], tags[i], order, 0);
    }
};

void etree_of(const Graph& g, const std::vector<int>& perm, const std::vector<int>& iperm,
              std::vector<int>& parent) {
    int n = g.n;
    parent.assign(n, -1);
    std::vector<int> ancestor(n, -1);
    for (int j = 0; j < n; ++j) {
        int v = perm[j];
        for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
            int i = iperm[g.adj[p]];
            if (i >= j) continue;
            int r = i;
            while (ancestor[r] != -1 && ancestor[r] != j) {
                int nxt = ancestor[r];
                ancestor[r] = j;
                r = nxt;
            }
            if (ancestor[r] == -1) { ancestor[r] = j; parent[r] = j; }
        }
    }
}

void postorder_of(const std::vector<int>& parent, std::vector<int>& post) {
    int n = (int)parent.size();
    std::vector<int> head(n, -1), next(n, -1), tail(n, -1);
    std::vector<int> roots;
    for (int j = 0; j < n; ++j) {
        int p = parent[j];
        if (p < 0) { roots.push_back(j); continue; }
        if (head[p] < 0) head[p] = j; else next[tail[p]] = j;
        tail[p] = j;
    }
    post.clear();
    post.reserve(n);
    std::vector<std::pair<int, int>> stack;   // (node, next child to visit)
    for (int r : roots) {
        stack.push_back({r, head[r]});
        while (!stack.empty()) {
            auto& top = stack.back();
            if (top.second >= 0) {
                int c = top.second;
                top.second = next[c];
                stack.push_back({c, head[c]});
            } else {
                post.push_back(top.first);
                stack.pop_back();
            }
        }
    }
}

// supernode rows by the supernodal recursion
void supernode_rows(const Graph& g, const std::vector<int>& perm, const std::vector<int>& iperm,
                    const std::vector<int>& ptr, std::vector<int>& rowptr,
                    std::vector<int>& rows, std::vector<int>& sparent) {
    int ns = (int)ptr.size() - 1;
    int n = g.n;
    std::vector<int> snode(n);
    for (int s = 0; s < ns; ++s)
        for (int j = ptr[s]; j < ptr[s + 1]; ++j) snode[j] = s;
    std::vector<int> mark(n, -1);
    std::vector<std::vector<int>> kids(ns);
    rowptr.assign(ns + 1, 0);
    rows.clear();
    sparent.assign(ns, -1);
    std::vector<int> buf;
    for (int s = 0; s < ns; ++s) {
        int f = ptr[s], l = ptr[s + 1] - 1;
        buf.clear();
        for (int j = f; j <= l; ++j) { buf.push_back(j); mark[j] = s; }
        for (int j = f; j <= l; ++j) {
            int v = perm[j];
            for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
                int i = iperm[g.adj[p]];
                if (i > l && mark[i] != s) { mark[i] = s; buf.push_back(i); }
            }
        }
        for (int c : kids[s])
            for (int q = rowptr[c]; q < rowptr[c + 1]; ++q) {
                int i = rows[q];
                if (i > l && mark[i] != s) { mark[i] = s; buf.push_back(i); }
            }
        std::sort(buf.begin(), buf.end());
        rows.insert(rows.end(), buf.begin(), buf.end());
        rowptr[s + 1] = (int)rows.size();
        int nc = l - f + 1;
        if ((int)buf.size() > nc) {
            sparent[s] = snode[buf[nc]];
            kids[sparent[s]].push_back(s);
        }
    }
}

}  // namespace

std::string analyse(const Graph& g, const SymbolicOptions& opt, Symbolic& out) {
    const int n = g.n;
    if (opt.leaf_size < 1) return "leaf_size must be >= 1";
    NestedDissection nd(g, opt.leaf_size, opt.parallel);
    nd.run();
    if ((int)nd.order.size() != n) return "internal error: ordering is not a permutation";
    std::vector<int> perm0 = nd.order, iperm0(n);
    for (int k = 0; k < n; ++k) iperm0[perm0[k]] = k;
    std::vector<int> parent0, post;
    etree_of(g, perm0, iperm0, parent0);
    postorder_of(parent0, post);
    out.n = n;
    out.perm.resize(n);
    out.iperm.resize(n);
    for (int k = 0; k < n; ++k) out.perm[k] = perm0[post[k]];
    for (int k = 0; k < n; ++k) out.iperm[out.perm[k]] = k;
    etree_of(g, out.perm, out.iperm, out.parent);
    const std::vector<int>& perm = out.perm;
    const std::vector<int>& iperm = out.iperm;
    const std::vector<int>& parent = out.parent;

    // column counts by structure union over etree children
    out.colcount.assign(n, 0);
    {
        std::vector<int> head(n, -1), next(n, -1);
        for (int j = n - 1; j >= 0; --j)
            if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = j; }
        std::vector<std::vector<int>> live(n);
        std::vector<int> mark(n, -1), buf;
        for (int j = 0; j < n; ++j) {
            buf.clear();
            buf.push_back(j);
            mark[j] = j;
            int v = perm[j];
            for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
                int i = iperm[g.adj[p]];
                if (i > j && mark[i] != j) { mark[i] = j; buf.push_back(i); }
            }
            for (int c = head[j]; c >= 0; c = next[c]) {
                for (int i : live[c])
                    if (i != c && mark[i] != j) { mark[i] = j; buf.push_back(i); }
                std::vector<int>().swap(live[c]);
            }
            out.colcount[j] = (int)buf.size();
            if (parent[j] >= 0) live[j] = buf;
        }
    }
    out.nnz_L = 0;
    int64_t fl = 0;
    for (int j = 0; j < n; ++j) {
        out.nnz_L += out.colcount[j];
        fl += (int64_t)out.colcount[j] * out.colcount[j];
    }
    out.flops = (double)fl;

    // fundamental supernodes
    std::vector<int> nchild(n, 0);
    for (int j = 0; j < n; ++j)
        if (parent[j] >= 0) nchild[parent[j]]++;
    std::vector<int> ptr{0};
    for (int j = 0; j + 1 < n; ++j) {
        bool joins = parent[j] == j + 1 && out.colcount[j] == out.colcount[j + 1] + 1 &&
                     nchild[j + 1] == 1;
        if (!joins) ptr.push_back(j + 1);
    }
    ptr.push_back(n);

    // relaxation: one backward pass
    if (opt.relax_cols > 0 && ptr.size() > 2) {
        std::vector<int> frowptr, frows, fsp;
        supernode_rows(g, perm, iperm, ptr, frowptr, frows, fsp);
        std::vector<int64_t> ccsum(n + 1, 0);
        for (int j = 0; j < n; ++j) ccsum[j + 1] = ccsum[j] + out.colcount[j];
        int ns = (int)ptr.size() - 1;
        std::vector<int> starts;
        int cur_f = ptr[ns - 1], cur_l = ptr[ns] - 1;
        int64_t cur_rows = frowptr[ns] - frowptr[ns - 1];
        for (int s = ns - 2; s >= 0; --s) {
            int f = ptr[s], l = ptr[s + 1] - 1;
            bool ok = parent[l] >= cur_f && parent[l] <= cur_l;
            if (ok) {
                int64_t ncol = cur_l - f + 1;
                int64_t nrow = (l - f + 1) + cur_rows;
                int64_t slots = ncol * nrow - ncol * (ncol - 1) / 2;
                int64_t truenz = ccsum[cur_l + 1] - ccsum[f];
                ok = ncol <= opt.relax_cols && slots - truenz <= opt.relax_zeros;
            }
            if (ok) {
                cur_f = f;
                cur_rows += l - f + 1;
            } else {
                starts.push_back(cur_f);
                cur_f = f;
                cur_l = l;
                cur_rows = frowptr[s + 1] - frowptr[s];
            }
        }
        starts.push_back(cur_f);
        std::sort(starts.begin(), starts.end());
        starts.push_back(n);
        ptr.swap(starts);
    }
    if (opt.max_width > 0) {
        std::vector<int> cut{0};
        for (size_t s = 0; s + 1 < ptr.size(); ++s) {
            int f = ptr[s], e = ptr[s + 1];
            for (int c = f + opt.max_width; c < e; c += opt.max_width) cut.push_back(c);
            cut.push_back(e);
        }
        ptr.swap(cut);
    }
    out.sn_ptr = ptr;
    supernode_rows(g, perm, iperm, out.sn_ptr, out.sn_rowptr, out.sn_rows, out.sn_parent);

    // structural row masks (recompute the exact column structures)
    out.sn_rowmask.clear();
    int maxw = 0;
    for (size_t s = 0; s + 1 < out.sn_ptr.size(); ++s) maxw = std::max(maxw, out.sn_ptr[s + 1] - out.sn_ptr[s]);
    if (maxw <= 64) {
        const int ns = out.ns();
        out.sn_rowmask.assign(out.sn_rows.size(), 0ull);
        std::vector<int> head(n, -1), next(n, -1);
        for (int j = n - 1; j >= 0; --j)
            if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = j; }
        std::vector<std::vector<int>> live(n);
        std::vector<int> mark(n, -1), pos(n, -1), buf;
        int s = 0;
        for (int j = 0; j < n; ++j) {
            if (j == out.sn_ptr[s + 1] || j == 0) {
                if (j != 0) {
                    for (int q = out.sn_rowptr[s]; q < out.sn_rowptr[s + 1]; ++q) pos[out.sn_rows[q]] = -1;
                    ++s;
                }
                for (int q = out.sn_rowptr[s]; q < out.sn_rowptr[s + 1]; ++q)
                    pos[out.sn_rows[q]] = q;
            }
            buf.clear();
            buf.push_back(j);
            mark[j] = j;
            int v = perm[j];
            for (int64_t p = g.xadj[v]; p < g.xadj[v + 1]; ++p) {
                int i = iperm[g.adj[p]];
                if (i > j && mark[i] != j) { mark[i] = j; buf.push_back(i); }
            }
            for (int c = head[j]; c >= 0; c = next[c]) {
                for (int i : live[c])
                    if (i != c && mark[i] != j) { mark[i] = j; buf.push_back(i); }
                std::vector<int>().swap(live[c]);
            }
            const int bit = j - out.sn_ptr[s];
            for (int i : buf) {
                if (pos[i] < 0) return "internal error: column structure outside its supernode panel";
                out.sn_rowmask[pos[i]] |= 1ull << bit;
            }
            if (parent[j] >= 0) live[j] = buf;
        }
        (void)ns;
    }
    return "";
}

void concat(const std::vector<Symbolic>& parts, Symbolic& out) {
    out = Symbolic();
    int64_t n = 0, ns = 0, nrows = 0;
    bool masks = true;
    for (const Symbolic& p : parts) {
        n += p.n;
        ns += p.ns();
        nrows += (int64_t)p.sn_rows.size();
        masks = masks && p.sn_rowmask.size() == p.sn_rows.size();
    }
    out.n = (int)n;
    out.perm.reserve(n);
    out.iperm.reserve(n);
    out.parent.reserve(n);
    out.colcount.reserve(n);
    out.sn_ptr.reserve(ns + 1);
    out.sn_rowptr.reserve(ns + 1);
    out.sn_rows.reserve(nrows);
    out.sn_parent.reserve(ns);
    if (masks) out.sn_rowmask.reserve(nrows);
    out.sn_ptr.push_back(0);
    out.sn_rowptr.push_back(0);
    int col0 = 0, sn0 = 0, row0 = 0;
    for (const Symbolic& p : parts) {
        for (int k = 0; k < p.n; ++k) {
            out.perm.push_back(p.perm[k] + col0);
            out.iperm.push_back(p.iperm[k] + col0);
            out.parent.push_back(p.parent[k] < 0 ? -1 : p.parent[k] + col0);
            out.colcount.push_back(p.colcount[k]);
        }
        for (int s = 0; s < p.ns(); ++s) {
            out.sn_ptr.push_back(p.sn_ptr[s + 1] + col0);
            out.sn_rowptr.push_back(p.sn_rowptr[s + 1] + row0);
            out.sn_parent.push_back(p.sn_parent[s] < 0 ? -1 : p.sn_parent[s] + sn0);
        }
        for (int r : p.sn_rows) out.sn_rows.push_back(r + col0);
        if (masks) out.sn_rowmask.insert(out.sn_rowmask.end(), p.sn_rowmask.begin(), p.sn_rowmask.end());
        out.flops += p.flops;
        out.nnz_L += p.nnz_L;
        col0 += p.n;
        sn0 += p.ns();
        row0 += (int)p.sn_rows.size();
    }
}

}  // namespace kktgb
