// Host-side mesh graph, farthest-point sampling and prolongation operators.
//
// Sec. 4.1 of the paper: vertex hierarchy by farthest-point sampling (Alg. 2)
// with Dijkstra distances on the weighted edge graph, and prolongations
// U^tau whose entries are (1 - d/rho) inside the support radius rho
// (eq. basis), rows normalised to one.  Compiled with -ffp-contract=off so
// every distance, weight and area is the plain IEEE result of the same
// expression in the same order, independent of the host architecture.
#include <algorithm>
#include <cmath>
#include <queue>
#include <utility>

#include "host.h"
#include "parallel.h"

namespace hsim {

MeshGraph build_mesh_graph(int n, int m, const double *V, const int *F, const double *L2) {
    HSIM_CHECK_ARG(n > 0 && m > 0, "empty mesh");
    HSIM_CHECK_ARG(F != nullptr, "F is NULL");
    HSIM_CHECK_ARG((V != nullptr) != (L2 != nullptr), "exactly one of V and L2 must be given");
    MeshGraph g;
    g.n = n;
    g.m = m;
    g.l2.resize((size_t)m * 3);
    // per triangle, in parallel; an error names the first bad triangle (the
    // first failing chunk's first failure)
    parallel_chunks(m, 16384, [&](int, int64_t t0, int64_t t1) {
        for (int64_t t = t0; t < t1; ++t) {
            for (int k = 0; k < 3; ++k) {
                int v = F[3 * t + k];
                HSIM_CHECK_ARG(v >= 0 && v < n, "triangle index out of range");
            }
            for (int k = 0; k < 3; ++k) {
                double l2;
                if (V) {
                    const double *a = V + 3 * (size_t)F[3 * t + (k + 1) % 3];
                    const double *b = V + 3 * (size_t)F[3 * t + (k + 2) % 3];
                    double e0 = b[0] - a[0], e1 = b[1] - a[1], e2 = b[2] - a[2];
                    l2 = e0 * e0 + e1 * e1 + e2 * e2;
                } else {
                    l2 = L2[3 * (size_t)t + k];
                }
                HSIM_CHECK_ARG(l2 > 0.0 && std::isfinite(l2), "degenerate or non-finite edge");
                g.l2[3 * (size_t)t + k] = l2;
            }
        }
    });
    // area: plain sequential sum of the Heron areas
    double area = 0.0;
    for (int t = 0; t < m; ++t) {
        double a = g.l2[3 * t], b = g.l2[3 * t + 1], c = g.l2[3 * t + 2];
        double s16 = 2.0 * (a * b + b * c + c * a) - (a * a + b * b + c * c);
        area += 0.25 * std::sqrt(std::max(s16, 0.0));
    }
    g.area = area;
    // undirected edges with the smallest squared length among their
    // triangles: both directions of every triangle edge bucketed by the
    // source vertex, each bucket sorted by (target, squared length) and the
    // first entry per target kept
    std::vector<int64_t> bstart(n + 1, 0);
    for (int t = 0; t < m; ++t)
        for (int k = 0; k < 3; ++k) {
            bstart[F[3 * t + (k + 1) % 3] + 1]++;
            bstart[F[3 * t + (k + 2) % 3] + 1]++;
        }
    for (int i = 0; i < n; ++i) bstart[i + 1] += bstart[i];
    std::vector<std::pair<int, double>> bucket(bstart[n]);
    {
        std::vector<int64_t> fill(bstart.begin(), bstart.end() - 1);
        for (int t = 0; t < m; ++t)
            for (int k = 0; k < 3; ++k) {
                int a = F[3 * t + (k + 1) % 3], b = F[3 * t + (k + 2) % 3];
                double l2 = g.l2[3 * (size_t)t + k];
                bucket[fill[a]++] = {b, l2};
                bucket[fill[b]++] = {a, l2};
            }
    }
    const int nch = chunk_count(n, 4096);
    std::vector<std::vector<int>> cidx(nch);
    std::vector<std::vector<double>> cw(nch);
    std::vector<int> deg(n, 0);
    parallel_chunks(n, 4096, [&](int ch, int64_t u0, int64_t u1) {
        for (int64_t u = u0; u < u1; ++u) {
            auto b = bucket.begin() + bstart[u], e = bucket.begin() + bstart[u + 1];
            std::sort(b, e);
            for (auto it = b; it != e; ++it) {
                if (it != b && it->first == (it - 1)->first) continue;
                HSIM_CHECK_ARG(it->first != u, "triangle with repeated vertex");
                cidx[ch].push_back(it->first);
                cw[ch].push_back(std::sqrt(it->second));
                deg[u]++;
            }
        }
    });
    g.ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) g.ptr[i + 1] = g.ptr[i] + deg[i];
    g.idx.reserve(g.ptr[n]);
    g.w.reserve(g.ptr[n]);
    for (int ch = 0; ch < nch; ++ch) {
        g.idx.insert(g.idx.end(), cidx[ch].begin(), cidx[ch].end());
        g.w.insert(g.w.end(), cw[ch].begin(), cw[ch].end());
    }
    return g;
}

std::vector<int> level_sizes(int n, int p, int levels) {
    int nc = std::max((int)std::ceil(1.5 * p), 1000);
    if (levels <= 1 || n <= nc) return {n};
    double mu = std::pow((double)n / nc, 1.0 / (levels - 1));
    std::vector<int> s{n};
    for (int tau = 1; tau < levels - 1; ++tau)
        s.push_back((int)std::floor(nc * std::pow(mu, (double)(levels - 1 - tau)) + 0.5));
    s.push_back(nc);
    return s;
}

namespace {
struct MinItem {
    double d;
    int v;
    bool operator>(const MinItem &o) const { return d > o.d || (d == o.d && v > o.v); }
};
using MinHeap = std::priority_queue<MinItem, std::vector<MinItem>, std::greater<MinItem>>;

}  // namespace

std::vector<int> boundary_vertices(int n, int m, const int *F) {
    std::vector<int64_t> key;
    key.reserve((size_t)m * 3);
    for (int t = 0; t < m; ++t)
        for (int k = 0; k < 3; ++k) {
            int64_t a = F[3 * t + k], b = F[3 * t + (k + 1) % 3];
            key.push_back(std::min(a, b) * n + std::max(a, b));
        }
    std::sort(key.begin(), key.end());
    std::vector<char> on(n, 0);
    for (size_t i = 0; i < key.size();) {
        size_t j = i;
        while (j < key.size() && key[j] == key[i]) ++j;
        if (j - i == 1) {
            on[key[i] / n] = 1;
            on[key[i] % n] = 1;
        }
        i = j;
    }
    std::vector<int> b;
    for (int v = 0; v < n; ++v)
        if (on[v]) b.push_back(v);
    return b;
}

std::vector<int> farthest_point_order(const MeshGraph &g, int start, int count, const std::vector<char> *cand) {
    HSIM_CHECK_ARG(start >= 0 && start < g.n, "start vertex out of range");
    HSIM_CHECK_ARG(!cand || (*cand)[start], "start vertex is not a degree of freedom");
    int ncand = g.n;
    if (cand) ncand = (int)std::count_if(cand->begin(), cand->end(), [](char c) { return c != 0; });
    HSIM_CHECK_ARG(count >= 1 && count <= ncand, "bad sample count");
    const int n = g.n;
    std::vector<double> dist(n, INFINITY);
    std::vector<int> order;
    order.reserve(count);
    // The farthest candidate is kept in a tournament tree over blocks of kB
    // consecutive vertices; a block whose distances changed is rescanned
    // before the next choice (the lowered region of one sample is small and
    // local, so few blocks change per sample; 64 measured fastest among
    // 32..512 on the 10^6-vertex torus, whose rows of 1000 vertices put each
    // lowered row segment in about one block).
    constexpr int kB = 64;
    const int nb = (n + kB - 1) / kB;
    std::vector<char> dirty(nb, 1);
    std::vector<int> dirty_list(nb);
    for (int b = 0; b < nb; ++b) dirty_list[b] = b;
    auto mark = [&](int v) {
        const int b = v / kB;
        if (!dirty[b]) {
            dirty[b] = 1;
            dirty_list.push_back(b);
        }
    };
    // Lower the field by the distances from src, following only improving
    // edges.  Any order of relaxations that ends with no improving edge gives
    // the same field (the least rounded path sum to every vertex, as the
    // rounded sum is monotone in its first operand), so the search may use a
    // bucket queue of width delta = half the shortest edge: relaxing a vertex
    // of bucket k lands beyond bucket k, every vertex is final when its bucket
    // is reached and is expanded once.  Buckets live in a ring of
    // ceil(longest edge / delta) + 3; a mesh whose edge lengths differ by a
    // factor above 2^15 uses a binary heap instead.
    double wmin = INFINITY, wmax = 0.0;
    for (double w : g.w) {
        wmin = std::min(wmin, w);
        wmax = std::max(wmax, w);
    }
    const bool buckets = !g.w.empty() && wmax <= 32768.0 * wmin;
    const double delta = buckets ? 0.5 * wmin : 1.0;
    const int nring = buckets ? (int)std::ceil(wmax / delta) + 3 : 0;
    std::vector<std::vector<int>> ring(nring);
    std::vector<int> stamp(buckets ? n : 0, -1);
    MinHeap heap;
    auto insert = [&](int src) {
        const int id = (int)order.size();
        order.push_back(src);
        dist[src] = 0.0;
        mark(src);
        if (buckets) {
            int64_t live = 1;
            ring[0].push_back(src);
            for (int64_t k = 0; live > 0; ++k) {
                std::vector<int> &cur = ring[k % nring];
                for (size_t i = 0; i < cur.size(); ++i) {
                    const int v = cur[i];
                    --live;
                    if (stamp[v] == id) continue;  // expanded already (pushed more than once)
                    stamp[v] = id;
                    const double dv = dist[v];
                    for (int e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
                        int u = g.idx[e];
                        double nd = dv + g.w[e];
                        if (nd < dist[u]) {
                            dist[u] = nd;
                            mark(u);
                            ring[(int64_t)(nd / delta) % nring].push_back(u);
                            ++live;
                        }
                    }
                }
                cur.clear();
            }
            return;
        }
        heap.push({0.0, src});
        while (!heap.empty()) {
            MinItem it = heap.top();
            heap.pop();
            if (it.d > dist[it.v]) continue;
            for (int e = g.ptr[it.v]; e < g.ptr[it.v + 1]; ++e) {
                int u = g.idx[e];
                double nd = it.d + g.w[e];
                if (nd < dist[u]) {
                    dist[u] = nd;
                    mark(u);
                    heap.push({nd, u});
                }
            }
        }
    };
    // a is farther than b: larger distance, the lower vertex id on ties (-1: none)
    auto farther = [&](int a, int b) {
        return b < 0 || (a >= 0 && (dist[a] > dist[b] || (dist[a] == dist[b] && a < b)));
    };
    int leaves = 1;
    while (leaves < nb) leaves *= 2;
    std::vector<int> tree(2 * (size_t)leaves, -1);
    insert(start);
    while ((int)order.size() < count) {
        for (int b : dirty_list) {
            int best = -1;
            for (int v = b * kB, e = std::min(n, (b + 1) * kB); v < e; ++v)
                if ((!cand || (*cand)[v]) && farther(v, best)) best = v;
            dirty[b] = 0;
            int i = leaves + b;
            tree[i] = best;
            for (i >>= 1; i >= 1; i >>= 1) tree[i] = farther(tree[2 * i], tree[2 * i + 1]) ? tree[2 * i] : tree[2 * i + 1];
        }
        dirty_list.clear();
        insert(tree[1]);
    }
    return order;
}

Csr prolongation(const MeshGraph &g, const std::vector<int> &order, int nf, int nc, bool fine_is_mesh,
                 double sigma, double *rho_out, int *fallback_rows, const std::vector<int> *dofs) {
    const double rho = std::sqrt(sigma * g.area / ((double)nc * M_PI));
    *rho_out = rho;
    std::vector<int> rank(g.n, -1);
    for (int k = 0; k < (int)order.size(); ++k) rank[order[k]] = k;
    // row of each fine vertex: mesh id, position among the listed degrees of
    // freedom, or position in the sampling order (-1: not on the fine level)
    std::vector<int> row_of;
    if (fine_is_mesh && dofs) {
        row_of.assign(g.n, -1);
        for (int k = 0; k < (int)dofs->size(); ++k) row_of[(*dofs)[k]] = k;
    }
    auto fine_row = [&](int v) { return fine_is_mesh ? (dofs ? row_of[v] : v) : rank[v]; };
    auto fine_vertex = [&](int r) { return fine_is_mesh ? (dofs ? (*dofs)[r] : r) : order[r]; };
    // (row, centre, weight) of every fine vertex within rho of a centre: one
    // truncated Dijkstra per centre, centres split into chunks that run
    // concurrently; each chunk lists its centres' entries in centre order
    struct Trip {
        int row, c;
        double w;
    };
    // The searches use the bucket queue of farthest_point_order when the
    // edge lengths allow it (the distances do not depend on the queue).
    double wmin = INFINITY, wmax = 0.0;
    for (double w : g.w) {
        wmin = std::min(wmin, w);
        wmax = std::max(wmax, w);
    }
    const bool buckets = !g.w.empty() && wmax <= 32768.0 * wmin;
    const double delta = buckets ? 0.5 * wmin : 1.0;
    const int nring = buckets ? (int)std::ceil(wmax / delta) + 3 : 0;
    const int nch = chunk_count(nc, 64);
    std::vector<std::vector<Trip>> part(nch);
    parallel_chunks(nc, 64, [&](int ch, int64_t c0, int64_t c1) {
        std::vector<Trip> &trips = part[ch];
        std::vector<double> dist(g.n, INFINITY);
        std::vector<int> touched;
        MinHeap heap;
        std::vector<std::vector<int>> ring(nring);
        std::vector<int> stamp(buckets ? g.n : 0, -1);
        for (int c = (int)c0; c < (int)c1; ++c) {
            int s = order[c];
            touched.clear();
            dist[s] = 0.0;
            touched.push_back(s);
            int64_t live = 0;  // entries in the bucket ring
            auto relax = [&](int v, double dv) {
                for (int e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
                    int u = g.idx[e];
                    double nd = dv + g.w[e];
                    if (nd < rho && nd < dist[u]) {
                        if (dist[u] == INFINITY) touched.push_back(u);
                        dist[u] = nd;
                        if (buckets) {
                            ring[(int64_t)(nd / delta) % nring].push_back(u);
                            ++live;
                        } else {
                            heap.push({nd, u});
                        }
                    }
                }
            };
            if (buckets) {
                ring[0].push_back(s);
                live = 1;
                for (int64_t k = 0; live > 0; ++k) {
                    std::vector<int> &cur = ring[k % nring];
                    for (size_t i = 0; i < cur.size(); ++i) {
                        const int v = cur[i];
                        --live;
                        if (stamp[v] == c) continue;  // expanded already
                        stamp[v] = c;
                        relax(v, dist[v]);
                    }
                    cur.clear();
                }
            } else {
                heap.push({0.0, s});
                while (!heap.empty()) {
                    MinItem it = heap.top();
                    heap.pop();
                    if (it.d > dist[it.v]) continue;
                    relax(it.v, it.d);
                }
            }
            for (int v : touched) {
                int row = fine_row(v);
                if (row >= 0 && row < nf) trips.push_back({row, c, 1.0 - dist[v] / rho});
                dist[v] = INFINITY;
            }
        }
    });
    // rows without any centre inside the radius: nearest centre, weight one
    std::vector<int> count(nf, 0);
    for (const auto &trips : part)
        for (const Trip &t : trips) count[t.row]++;
    std::vector<int> fallback_centre(nf, -1);
    int missing = 0;
    for (int r = 0; r < nf; ++r) missing += count[r] == 0;
    *fallback_rows = missing;
    if (missing) {
        MinHeap heap;
        std::vector<double> nd(g.n, INFINITY);
        std::vector<int> label(g.n, -1);
        for (int c = 0; c < nc; ++c) {
            nd[order[c]] = 0.0;
            if (label[order[c]] < 0) label[order[c]] = c;
            heap.push({0.0, order[c]});
        }
        while (!heap.empty()) {
            MinItem it = heap.top();
            heap.pop();
            if (it.d > nd[it.v]) continue;
            for (int e = g.ptr[it.v]; e < g.ptr[it.v + 1]; ++e) {
                int u = g.idx[e];
                double d = it.d + g.w[e];
                if (d < nd[u] || (d == nd[u] && label[it.v] < label[u])) {
                    nd[u] = d;
                    label[u] = label[it.v];
                    heap.push({d, u});
                }
            }
        }
        for (int r = 0; r < nf; ++r)
            if (count[r] == 0) {
                int v = fine_vertex(r);
                HSIM_CHECK_ARG(label[v] >= 0, "a connected component of the mesh holds no coarse vertex");
                fallback_centre[r] = label[v];
                count[r] = 1;
            }
    }
    // CSR by rows; within a row the entries arrive in increasing centre
    // order (chunks in order, centres in order inside a chunk)
    Csr U;
    U.n_rows = nf;
    U.n_cols = nc;
    U.ptr.assign(nf + 1, 0);
    for (int r = 0; r < nf; ++r) U.ptr[r + 1] = U.ptr[r] + count[r];
    U.col.resize(U.ptr[nf]);
    U.val.resize(U.ptr[nf]);
    {
        std::vector<int> fill(U.ptr.begin(), U.ptr.end() - 1);
        for (const auto &trips : part)
            for (const Trip &t : trips) {
                U.col[fill[t.row]] = t.c;
                U.val[fill[t.row]++] = t.w;
            }
        for (int r = 0; r < nf; ++r)
            if (fallback_centre[r] >= 0) {
                U.col[fill[r]] = fallback_centre[r];
                U.val[fill[r]++] = 1.0;
            }
    }
    // normalise each row: sum in increasing centre order
    for (int r = 0; r < nf; ++r) {
        double sum = 0.0;
        for (int e = U.ptr[r]; e < U.ptr[r + 1]; ++e) sum += U.val[e];
        for (int e = U.ptr[r]; e < U.ptr[r + 1]; ++e) U.val[e] /= sum;
    }
    return U;
}

void random_column(int n, uint64_t seed, double *out) {
    // SplitMix64 (Steele, Lea and Flood, 2014): state += gamma, then two
    // xor-shift-multiply rounds and a final xor-shift; output i uses state
    // seed + (i + 1) gamma, so entries can be produced in any order
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < n; ++i) {
        uint64_t z = seed + (uint64_t)(i + 1) * gamma;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[i] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
    }
}

void plain_basis(int n, const double *sdiag, const double *mdiag, const int *perm, const int *iperm, int q,
                 uint64_t seed, std::vector<int> *unit_pos, std::vector<double> *rand_int) {
    HSIM_CHECK_ARG(n >= 1 && q >= 2 && q <= n, "plain SIM needs 2 <= q <= n");
    std::vector<double> ratio(n);
    for (int i = 0; i < n; ++i) ratio[i] = sdiag[i] / mdiag[i];
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    const int nu = q - 2;
    std::partial_sort(idx.begin(), idx.begin() + nu, idx.end(),
                      [&](int a, int b) { return ratio[a] < ratio[b] || (ratio[a] == ratio[b] && a < b); });
    unit_pos->resize(nu);
    for (int c = 0; c < nu; ++c) (*unit_pos)[c] = iperm[idx[c]];
    std::vector<double> rc(n);
    random_column(n, seed, rc.data());
    rand_int->resize(n);
    for (int pos = 0; pos < n; ++pos) (*rand_int)[pos] = rc[perm[pos]];
}

HostHierarchy host_levels(int n, int m, const double *V, const int *F, const double *L2, int p, int levels,
                          int start_vertex, double sigma, int q, bool dirichlet) {
    HSIM_CHECK_ARG(p >= 1, "p must be >= 1");
    HSIM_CHECK_ARG(sigma > 0.0, "sigma must be positive");
    HostHierarchy h;
    h.g = build_mesh_graph(n, m, V, F, L2);
    HSIM_CHECK_ARG(start_vertex >= 0 && start_vertex < n, "start_vertex out of range");
    if (dirichlet) {
        std::vector<char> interior(n, 1);
        for (int v : boundary_vertices(n, m, F)) interior[v] = 0;
        for (int v = 0; v < n; ++v)
            if (interior[v]) h.dofs.push_back(v);
        HSIM_CHECK_ARG(!h.dofs.empty(), "a Dirichlet boundary leaves no interior vertex");
        HSIM_CHECK_ARG(interior[start_vertex], "start_vertex lies on the Dirichlet boundary");
    }
    h.A_mesh = mesh_pattern(h.g);
    if (dirichlet) h.A0 = restrict_pattern(h.A_mesh, h.dofs, &h.smap);
    else h.A0 = h.A_mesh;
    const int n0 = dirichlet ? (int)h.dofs.size() : n;
    h.sizes = level_sizes(n0, p, levels > 0 ? levels : (p <= 200 ? 2 : 3));
    const int T = (int)h.sizes.size();
    HSIM_CHECK_ARG(T <= 8, "at most 8 levels");
    HSIM_CHECK_ARG(q <= h.sizes[T - 1], "p too large for the mesh");
    return h;
}

void host_samples(HostHierarchy &h, int start_vertex, double sigma) {
    const int T = (int)h.sizes.size();
    const bool dirichlet = !h.dofs.empty();
    std::vector<char> interior;
    if (dirichlet) {
        interior.assign(h.g.n, 0);
        for (int v : h.dofs) interior[v] = 1;
    }
    if (T > 1) h.order = farthest_point_order(h.g, start_vertex, h.sizes[1], dirichlet ? &interior : nullptr);
    h.U.resize(T - 1);
    h.rho.assign(T - 1, 0.0);
    h.fallback.assign(T - 1, 0);
    for (int tau = 0; tau + 1 < T; ++tau)
        h.U[tau] = prolongation(h.g, h.order, h.sizes[tau], h.sizes[tau + 1], tau == 0, sigma, &h.rho[tau],
                                &h.fallback[tau], dirichlet ? &h.dofs : nullptr);
}

HostHierarchy build_host_hierarchy(int n, int m, const double *V, const int *F, const double *L2, int p,
                                   int levels, int start_vertex, double sigma, int q, bool dirichlet) {
    HostHierarchy h = host_levels(n, m, V, F, L2, p, levels, start_vertex, sigma, q, dirichlet);
    host_samples(h, start_vertex, sigma);
    return h;
}

}  // namespace hsim
