// Host-side sparse pattern algebra, nested-dissection ordering and the
// supernodal (multifrontal) symbolic analysis of each level's matrix.
//
// The paper factors the shifted matrix S - mu M once per level with a sparse
// symmetric indefinite LDL^T (Sec. 3.2, "Direct solver"; Alg. 1).  Ordering
// and symbolic analysis are host work; the numeric factorisation and the
// multi-right-hand-side solves run on the GPU over the fronts built here.
//
// Ordering: recursive bisection by breadth-first level structures.  From a
// pseudo-peripheral vertex, BFS levels L_0..L_h are built; the level L_m
// where half of the vertices is reached becomes the separator, trimmed to
// the vertices that touch L_{m+1}.  Disconnected pieces are ordered
// independently.  Every separator and every leaf domain is one dense front.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <exception>
#include <numeric>
#include <thread>

#include "host.h"
#include "parallel.h"

namespace hsim {

Csr mesh_pattern(const MeshGraph &g) {
    Csr A;
    A.n_rows = A.n_cols = g.n;
    A.ptr.assign(g.n + 1, 0);
    A.col.reserve(g.idx.size() + g.n);
    for (int i = 0; i < g.n; ++i) {
        bool diag = false;
        for (int e = g.ptr[i]; e < g.ptr[i + 1]; ++e) {
            int j = g.idx[e];
            if (!diag && j > i) { A.col.push_back(i); diag = true; }
            A.col.push_back(j);
        }
        if (!diag) A.col.push_back(i);
        A.ptr[i + 1] = (int)A.col.size();
    }
    return A;
}

Csr transpose_pattern(const Csr &A) {
    Csr T;
    T.n_rows = A.n_cols;
    T.n_cols = A.n_rows;
    T.ptr.assign(T.n_rows + 1, 0);
    const int64_t nnz = A.nnz();
    T.col.resize(nnz);
    bool vals = !A.val.empty();
    if (vals) T.val.resize(nnz);
    for (int64_t e = 0; e < nnz; ++e) T.ptr[A.col[e] + 1]++;
    for (int i = 0; i < T.n_rows; ++i) T.ptr[i + 1] += T.ptr[i];
    std::vector<int> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int i = 0; i < A.n_rows; ++i)
        for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
            int d = fill[A.col[e]]++;
            T.col[d] = i;
            if (vals) T.val[d] = A.val[e];
        }
    return T;
}

Csr pattern_product(const Csr &A, const Csr &B) {
    HSIM_CHECK_ARG(A.n_cols == B.n_rows, "pattern_product: shape mismatch");
    Csr C;
    C.n_rows = A.n_rows;
    C.n_cols = B.n_cols;
    C.ptr.assign(A.n_rows + 1, 0);
    // row chunks concurrently, each with its own marker array; the chunks'
    // column lists are concatenated in row order
    const int nch = chunk_count(A.n_rows, 2048);
    std::vector<std::vector<int>> part(nch);
    parallel_chunks(A.n_rows, 2048, [&](int ch, int64_t i0, int64_t i1) {
        std::vector<int> mark(B.n_cols, -1);
        std::vector<int> row;
        std::vector<int> &out = part[ch];
        for (int i = (int)i0; i < (int)i1; ++i) {
            row.clear();
            for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
                int k = A.col[e];
                for (int f = B.ptr[k]; f < B.ptr[k + 1]; ++f) {
                    int j = B.col[f];
                    if (mark[j] != i) { mark[j] = i; row.push_back(j); }
                }
            }
            std::sort(row.begin(), row.end());
            out.insert(out.end(), row.begin(), row.end());
            C.ptr[i + 1] = (int)row.size();  // row length; prefix-summed below
        }
    });
    int64_t total = 0;
    for (int i = 0; i < A.n_rows; ++i) {
        total += C.ptr[i + 1];
        if (total > (int64_t)INT32_MAX) fail(HSIM_E_INVALID_ARG, "pattern too large for int32 CSR");
        C.ptr[i + 1] = (int)total;
    }
    C.col.reserve(total);
    for (const auto &p : part) C.col.insert(C.col.end(), p.begin(), p.end());
    return C;
}

Csr permute_symmetric(const Csr &A, const std::vector<int> &iperm, std::vector<int64_t> *value_map) {
    const int n = A.n_rows;
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[iperm[i]] = i;
    Csr B;
    B.n_rows = B.n_cols = n;
    B.ptr.assign(n + 1, 0);
    for (int p = 0; p < n; ++p) B.ptr[p + 1] = B.ptr[p] + (A.ptr[perm[p] + 1] - A.ptr[perm[p]]);
    B.col.resize(A.nnz());
    if (value_map) value_map->resize(A.nnz());
    parallel_chunks(n, 4096, [&](int, int64_t p0, int64_t p1) {
        std::vector<std::pair<int, int>> row;
        for (int p = (int)p0; p < (int)p1; ++p) {
            int i = perm[p];
            row.clear();
            for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) row.push_back({iperm[A.col[e]], e});
            std::sort(row.begin(), row.end());
            int base = B.ptr[p];
            for (size_t k = 0; k < row.size(); ++k) {
                B.col[base + k] = row[k].first;
                if (value_map) (*value_map)[base + k] = row[k].second;
            }
        }
    });
    return B;
}

Csr restrict_pattern(const Csr &A, const std::vector<int> &keep, std::vector<int64_t> *value_map) {
    std::vector<int> id(A.n_rows, -1);
    for (size_t k = 0; k < keep.size(); ++k) {
        HSIM_CHECK_ARG(keep[k] >= 0 && keep[k] < A.n_rows && (k == 0 || keep[k] > keep[k - 1]),
                       "restriction indices must ascend within the matrix");
        id[keep[k]] = (int)k;
    }
    Csr B;
    B.n_rows = B.n_cols = (int)keep.size();
    B.ptr.assign(keep.size() + 1, 0);
    if (value_map) value_map->clear();
    for (size_t k = 0; k < keep.size(); ++k) {
        const int i = keep[k];
        for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
            const int j = id[A.col[e]];
            if (j < 0) continue;
            B.col.push_back(j);  // ascending: keep ascends and A's columns are sorted
            if (value_map) value_map->push_back(e);
        }
        B.ptr[k + 1] = (int)B.col.size();
    }
    return B;
}

Csr permute_rows_cols(const Csr &A, const std::vector<int> &row_iperm, const std::vector<int> &col_iperm) {
    const int n = A.n_rows;
    std::vector<int> rperm(n);
    for (int i = 0; i < n; ++i) rperm[row_iperm[i]] = i;
    Csr B;
    B.n_rows = A.n_rows;
    B.n_cols = A.n_cols;
    B.ptr.assign(n + 1, 0);
    for (int p = 0; p < n; ++p) B.ptr[p + 1] = B.ptr[p] + (A.ptr[rperm[p] + 1] - A.ptr[rperm[p]]);
    B.col.resize(A.nnz());
    B.val.resize(A.nnz());
    parallel_chunks(n, 4096, [&](int, int64_t p0, int64_t p1) {
        std::vector<std::pair<int, double>> row;
        for (int p = (int)p0; p < (int)p1; ++p) {
            int i = rperm[p];
            row.clear();
            for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) row.push_back({col_iperm[A.col[e]], A.val[e]});
            std::sort(row.begin(), row.end());
            int base = B.ptr[p];
            for (size_t k = 0; k < row.size(); ++k) {
                B.col[base + k] = row[k].first;
                B.val[base + k] = row[k].second;
            }
        }
    });
    return B;
}

// ---------------------------------------------------------------------------
// nested dissection
// ---------------------------------------------------------------------------
namespace {

struct NdNode {
    std::vector<int> verts;
    std::vector<int> children;
};

// Nodes of a subtree in creation order (children before parents); ids are
// positions in this list.
using NdList = std::vector<NdNode>;

// Append `part` to `out`, shifting its node ids; returns the shift.
int append_nodes(NdList &out, NdList &&part) {
    const int off = (int)out.size();
    for (NdNode &nn : part) {
        for (int &c : nn.children) c += off;
        out.push_back(std::move(nn));
    }
    return off;
}

struct Nd {
    const Csr &A;
    int leaf;
    // vertex -> id of the set being split (relaxed atomics: sets ordered
    // concurrently are disjoint, but a search reads its neighbours' ids)
    std::vector<std::atomic<int>> stamp;
    std::vector<int> level;   // BFS level scratch (written only for members of the set)
    std::atomic<int> next_stamp{1};
    int spawn_depth = 0;      // subtrees of this depth or less run on their own threads

    Nd(const Csr &a, int l) : A(a), leaf(l), stamp(a.n_rows), level(a.n_rows, -1) {
        for (auto &x : stamp) x.store(0, std::memory_order_relaxed);
        int t = host_threads(), d = 0;
        while ((1 << d) < t) ++d;
        spawn_depth = d;
    }
    int st_of(int v) const { return stamp[v].load(std::memory_order_relaxed); }

    // BFS within the set marked `st` from r; fills order and returns levels
    // via level[] (relative to this search); returns number of levels.
    int bfs(int r, int st, std::vector<int> &order) {
        order.clear();
        order.push_back(r);
        level[r] = 0;
        int nl = 1;
        for (size_t h = 0; h < order.size(); ++h) {
            int v = order[h];
            for (int e = A.ptr[v]; e < A.ptr[v + 1]; ++e) {
                int u = A.col[e];
                if (u == v || st_of(u) != st || level[u] >= 0) continue;
                level[u] = level[v] + 1;
                nl = std::max(nl, level[u] + 1);
                order.push_back(u);
            }
        }
        return nl;
    }
    void clear_levels(const std::vector<int> &order) {
        for (int v : order) level[v] = -1;
    }
    int degree(int v) const { return A.ptr[v + 1] - A.ptr[v]; }

    // Orders W: appends the nodes of its subtrees to `nodes` (children before
    // parents) and returns the ids of their roots.  The node list does not
    // depend on which subtrees ran concurrently.
    std::vector<int> run(std::vector<int> W, NdList &nodes, int depth) {
        if (W.empty()) return {};
        const int st = next_stamp.fetch_add(1, std::memory_order_relaxed);
        for (int v : W) stamp[v].store(st, std::memory_order_relaxed);
        std::vector<int> order;
        // connected components
        {
            std::vector<std::vector<int>> comps;
            for (int v : W) {
                if (level[v] >= 0) continue;
                bfs(v, st, order);
                comps.push_back(order);
            }
            for (auto &c : comps) clear_levels(c);
            if (comps.size() > 1) {
                std::vector<int> roots;
                for (auto &c : comps) {
                    auto r = run(std::move(c), nodes, depth);
                    roots.insert(roots.end(), r.begin(), r.end());
                }
                return roots;
            }
        }
        auto make_leaf = [&](std::vector<int> verts) {
            nodes.push_back(NdNode{std::move(verts), {}});
            return std::vector<int>{(int)nodes.size() - 1};
        };
        if ((int)W.size() <= leaf) return make_leaf(std::move(W));
        // pseudo-peripheral vertex
        int r = W[0];
        int nl = bfs(r, st, order);
        for (int it = 0; it < 4; ++it) {
            int best = -1;
            for (int v : order)
                if (level[v] == nl - 1 && (best < 0 || degree(v) < degree(best))) best = v;
            clear_levels(order);
            int nl2 = bfs(best, st, order);
            if (nl2 <= nl) {
                clear_levels(order);
                nl = bfs(r, st, order);
                break;
            }
            r = best;
            nl = nl2;
        }
        if (nl < 3) {
            clear_levels(order);
            return make_leaf(std::move(W));
        }
        std::vector<int> cnt(nl, 0);
        for (int v : order) cnt[level[v]]++;
        int half = (int)W.size() / 2, acc = 0, m = 0;
        for (m = 0; m < nl; ++m) {
            acc += cnt[m];
            if (acc >= half) break;
        }
        m = std::max(1, std::min(m, nl - 2));
        std::vector<int> sep, Apart, Bpart;
        for (int v : order) {
            int lv = level[v];
            if (lv < m) Apart.push_back(v);
            else if (lv > m) Bpart.push_back(v);
            else {
                bool touches = false;
                for (int e = A.ptr[v]; e < A.ptr[v + 1] && !touches; ++e) {
                    int u = A.col[e];
                    touches = (st_of(u) == st && level[u] == m + 1);
                }
                (touches ? sep : Apart).push_back(v);
            }
        }
        clear_levels(order);
        std::vector<int> kids;
        if (depth < spawn_depth && std::min(Apart.size(), Bpart.size()) >= 4096) {
            // the two halves are disjoint: order the first on another thread
            NdList la, lb;
            std::vector<int> ka, kb;
            std::exception_ptr err;
            std::thread th([&] {
                try {
                    ka = run(std::move(Apart), la, depth + 1);
                } catch (...) {
                    err = std::current_exception();
                }
            });
            try {
                kb = run(std::move(Bpart), lb, depth + 1);
            } catch (...) {
                th.join();
                throw;
            }
            th.join();
            if (err) std::rethrow_exception(err);
            const int oa = append_nodes(nodes, std::move(la));
            const int ob = append_nodes(nodes, std::move(lb));
            for (int k : ka) kids.push_back(k + oa);
            for (int k : kb) kids.push_back(k + ob);
        } else {
            kids = run(std::move(Apart), nodes, depth + 1);
            std::vector<int> kb = run(std::move(Bpart), nodes, depth + 1);
            kids.insert(kids.end(), kb.begin(), kb.end());
        }
        nodes.push_back(NdNode{std::move(sep), std::move(kids)});
        return {(int)nodes.size() - 1};
    }
};

}  // namespace

FrontSymbolic analyse(const Csr &A, int leaf_size) {
    const int n = A.n_rows;
    HSIM_CHECK_ARG(n > 0 && A.n_cols == n, "analyse: square pattern expected");
    leaf_size = std::max(leaf_size, 4);
    Nd nd(A, leaf_size);
    std::vector<int> all(n);
    std::iota(all.begin(), all.end(), 0);
    NdList nd_nodes;
    const auto t_nd = std::chrono::steady_clock::now();
    std::vector<int> roots = nd.run(all, nd_nodes, 0);
    const auto t_st = std::chrono::steady_clock::now();

    FrontSymbolic fs;
    fs.n = n;
    // postorder: children first, then the node's own vertices
    std::vector<int> post;  // nd node ids in postorder
    {
        std::vector<std::pair<int, int>> stack;
        for (int ri = (int)roots.size() - 1; ri >= 0; --ri) stack.push_back({roots[ri], 0});
        while (!stack.empty()) {
            auto &top = stack.back();
            const NdNode &nn = nd_nodes[top.first];
            if (top.second < (int)nn.children.size()) {
                int c = nn.children[top.second++];
                stack.push_back({c, 0});
            } else {
                post.push_back(top.first);
                stack.pop_back();
            }
        }
    }
    const int N = (int)post.size();
    fs.n_nodes = N;
    std::vector<int> newid(nd_nodes.size(), -1);
    for (int k = 0; k < N; ++k) newid[post[k]] = k;
    fs.perm.resize(n);
    fs.iperm.assign(n, -1);
    fs.pstart.resize(N);
    fs.ns.resize(N);
    fs.parent.assign(N, -1);
    fs.height.assign(N, 0);
    int pos = 0;
    for (int k = 0; k < N; ++k) {
        const NdNode &nn = nd_nodes[post[k]];
        fs.pstart[k] = pos;
        fs.ns[k] = (int)nn.verts.size();
        for (int v : nn.verts) {
            fs.perm[pos] = v;
            fs.iperm[v] = pos;
            ++pos;
        }
        for (int c : nn.children) {
            fs.parent[newid[c]] = k;
            fs.height[k] = std::max(fs.height[k], fs.height[newid[c]] + 1);
        }
    }
    if (pos != n) fail(HSIM_E_INTERNAL, "nested dissection lost vertices");
    fs.pos_node.resize(n);
    for (int k = 0; k < N; ++k)
        for (int i = 0; i < fs.ns[k]; ++i) fs.pos_node[fs.pstart[k] + i] = k;

    // struct(t): positions beyond t's pivots adjacent to t's pivots or in a
    // child's struct
    std::vector<std::vector<int>> st(N);
    std::vector<std::vector<int>> kids(N);
    for (int k = 0; k < N; ++k)
        if (fs.parent[k] >= 0) kids[fs.parent[k]].push_back(k);
    for (int k = 0; k < N; ++k) {
        int pe = fs.pstart[k] + fs.ns[k];
        std::vector<int> s;
        for (int i = 0; i < fs.ns[k]; ++i) {
            int v = fs.perm[fs.pstart[k] + i];
            for (int e = A.ptr[v]; e < A.ptr[v + 1]; ++e) {
                int pu = fs.iperm[A.col[e]];
                if (pu >= pe) s.push_back(pu);
            }
        }
        for (int c : kids[k])
            for (int x : st[c]) {
                if (x < fs.pstart[k]) fail(HSIM_E_INTERNAL, "child struct below parent pivots");
                if (x >= pe) s.push_back(x);
            }
        std::sort(s.begin(), s.end());
        s.erase(std::unique(s.begin(), s.end()), s.end());
        st[k] = std::move(s);
        if (fs.parent[k] < 0 && !st[k].empty()) fail(HSIM_E_INTERNAL, "root front with a non-empty struct");
    }
    // fronts, arena, relmaps
    fs.nf.resize(N);
    fs.rows_off.resize(N + 1);
    fs.foff.resize(N + 1);
    fs.relmap_off.resize(N + 1);
    fs.nsteps.resize(N);
    int64_t roff = 0, aoff = 0, moff = 0;
    for (int k = 0; k < N; ++k) {
        fs.nf[k] = fs.ns[k] + (int)st[k].size();
        fs.rows_off[k] = roff;
        fs.foff[k] = aoff;
        fs.relmap_off[k] = moff;
        roff += fs.nf[k];
        aoff += ((int64_t)fs.nf[k] * fs.nf[k] + 1) & ~(int64_t)1;
        moff += (int64_t)st[k].size();
        fs.nsteps[k] = (fs.ns[k] + kPanel - 1) / kPanel;
        fs.max_front = std::max(fs.max_front, fs.nf[k]);
        for (int j = 0; j < fs.ns[k]; ++j) {
            fs.nnz_L += fs.nf[k] - j;
            double t = (double)(fs.nf[k] - j - 1);
            fs.flops += t * t + 2.0 * t;  // rank-1 update of the trailing lower part + scaling
        }
    }
    fs.rows_off[N] = roff;
    fs.foff[N] = aoff;
    fs.relmap_off[N] = moff;
    if (const char *e = std::getenv("HSIM_TRACE"); e && std::atoi(e) >= 2) {
        const auto t1 = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[hsim] analyse n=%d: nested dissection %.1f ms, fronts %.1f ms\n", n,
                     std::chrono::duration<double, std::milli>(t_st - t_nd).count(),
                     std::chrono::duration<double, std::milli>(t1 - t_st).count());
    }
    fs.arena = aoff;
    fs.rows.resize(roff);
    fs.relmap.resize(moff);
    for (int k = 0; k < N; ++k) {
        int64_t o = fs.rows_off[k];
        for (int i = 0; i < fs.ns[k]; ++i) fs.rows[o + i] = fs.pstart[k] + i;
        for (size_t i = 0; i < st[k].size(); ++i) fs.rows[o + fs.ns[k] + i] = st[k][i];
    }
    for (int k = 0; k < N; ++k) {
        int p = fs.parent[k];
        if (p < 0) continue;
        int ppe = fs.pstart[p] + fs.ns[p];
        for (size_t i = 0; i < st[k].size(); ++i) {
            int x = st[k][i], loc;
            if (x < ppe) {
                loc = x - fs.pstart[p];
            } else {
                auto it = std::lower_bound(st[p].begin(), st[p].end(), x);
                if (it == st[p].end() || *it != x) fail(HSIM_E_INTERNAL, "struct row missing in parent front");
                loc = fs.ns[p] + (int)(it - st[p].begin());
            }
            if (loc < 0 || loc >= fs.nf[p]) fail(HSIM_E_INTERNAL, "relmap out of range");
            fs.relmap[fs.relmap_off[k] + i] = loc;
        }
    }
    // schedules
    fs.max_height = 0;
    for (int k = 0; k < N; ++k) fs.max_height = std::max(fs.max_height, fs.height[k]);
    fs.by_height.assign(fs.max_height + 1, {});
    fs.ea_children.assign(fs.max_height + 1, {});
    for (int k = 0; k < N; ++k) {
        fs.by_height[fs.height[k]].push_back(k);
        if (fs.parent[k] >= 0 && fs.nf[k] > fs.ns[k]) fs.ea_children[fs.height[fs.parent[k]]].push_back(k);
    }
    for (auto &v : fs.by_height)
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return fs.nsteps[a] > fs.nsteps[b]; });
    for (auto &v : fs.ea_children)
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return fs.nf[a] - fs.ns[a] > fs.nf[b] - fs.ns[b]; });
    return fs;
}

std::vector<int64_t> assembly_map(const FrontSymbolic &fs, const Csr &A) {
    std::vector<int64_t> dst(A.nnz(), -1);
    for (int pi = 0; pi < fs.n; ++pi) {
        for (int e = A.ptr[pi]; e < A.ptr[pi + 1]; ++e) {
            int pj = A.col[e];
            if (pi < pj) continue;
            int t = fs.pos_node[pj];
            int ps = fs.pstart[t], pe = ps + fs.ns[t];
            int lc = pj - ps, lr;
            if (pi < pe) {
                lr = pi - ps;
            } else {
                const int *b = fs.rows.data() + fs.rows_off[t] + fs.ns[t];
                const int *en = fs.rows.data() + fs.rows_off[t] + fs.nf[t];
                const int *it = std::lower_bound(b, en, pi);
                if (it == en || *it != pi) fail(HSIM_E_INTERNAL, "matrix entry outside its front");
                lr = fs.ns[t] + (int)(it - b);
            }
            dst[e] = fs.foff[t] + (int64_t)lc * fs.nf[t] + lr;
        }
    }
    return dst;
}

}  // namespace hsim
