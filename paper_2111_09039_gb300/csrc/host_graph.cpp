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

namespace hsim {

MeshGraph build_mesh_graph(int n, int m, const double *V, const int *F, const double *L2) {
    HSIM_CHECK_ARG(n > 0 && m > 0, "empty mesh");
    HSIM_CHECK_ARG(F != nullptr, "F is NULL");
    HSIM_CHECK_ARG((V != nullptr) != (L2 != nullptr), "exactly one of V and L2 must be given");
    MeshGraph g;
    g.n = n;
    g.m = m;
    g.l2.resize((size_t)m * 3);
    for (int t = 0; t < m; ++t) {
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
    // area: plain sequential sum of the Heron areas
    double area = 0.0;
    for (int t = 0; t < m; ++t) {
        double a = g.l2[3 * t], b = g.l2[3 * t + 1], c = g.l2[3 * t + 2];
        double s16 = 2.0 * (a * b + b * c + c * a) - (a * a + b * b + c * c);
        area += 0.25 * std::sqrt(std::max(s16, 0.0));
    }
    g.area = area;
    // undirected edges with the smallest squared length among their triangles
    std::vector<std::pair<int64_t, double>> e;
    e.reserve((size_t)m * 6);
    for (int t = 0; t < m; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = F[3 * t + (k + 1) % 3], b = F[3 * t + (k + 2) % 3];
            double l2 = g.l2[3 * (size_t)t + k];
            e.push_back({(int64_t)a * n + b, l2});
            e.push_back({(int64_t)b * n + a, l2});
        }
    std::sort(e.begin(), e.end());
    g.ptr.assign(n + 1, 0);
    for (size_t i = 0; i < e.size(); ++i) {
        if (i > 0 && e[i].first == e[i - 1].first) continue;
        int u = (int)(e[i].first / n), v = (int)(e[i].first % n);
        HSIM_CHECK_ARG(u != v, "triangle with repeated vertex");
        g.ptr[u + 1]++;
        g.idx.push_back(v);
        g.w.push_back(std::sqrt(e[i].second));
    }
    for (int i = 0; i < n; ++i) g.ptr[i + 1] += g.ptr[i];
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

struct MaxItem {
    double d;
    int v;
    // larger distance first; among equal distances the lower vertex id first
    bool operator<(const MaxItem &o) const { return d < o.d || (d == o.d && v > o.v); }
};
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
    std::vector<double> dist(g.n, INFINITY);
    std::vector<int> order;
    order.reserve(count);
    MinHeap heap;
    // Lower the field by the distances from src, following only improving edges.
    auto insert = [&](int src) {
        order.push_back(src);
        dist[src] = 0.0;
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
                    heap.push({nd, u});
                }
            }
        }
    };
    insert(start);
    // Lazy max-heap: each vertex keeps one entry whose key is >= its current
    // distance (distances only decrease); a stale top is re-keyed.
    std::priority_queue<MaxItem> far;
    for (int v = 0; v < g.n; ++v)
        if (!cand || (*cand)[v]) far.push({dist[v], v});
    while ((int)order.size() < count) {
        MaxItem top = far.top();
        far.pop();
        if (top.d != dist[top.v]) {
            far.push({dist[top.v], top.v});
            continue;
        }
        insert(top.v);
        far.push({dist[top.v], top.v});
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
    // triplets (row, centre, weight)
    struct Trip {
        int row, c;
        double w;
    };
    std::vector<Trip> trips;
    trips.reserve((size_t)nf * 8);
    std::vector<double> dist(g.n, INFINITY);
    std::vector<int> touched;
    MinHeap heap;
    for (int c = 0; c < nc; ++c) {
        int s = order[c];
        touched.clear();
        dist[s] = 0.0;
        touched.push_back(s);
        heap.push({0.0, s});
        while (!heap.empty()) {
            MinItem it = heap.top();
            heap.pop();
            if (it.d > dist[it.v]) continue;
            for (int e = g.ptr[it.v]; e < g.ptr[it.v + 1]; ++e) {
                int u = g.idx[e];
                double nd = it.d + g.w[e];
                if (nd < rho && nd < dist[u]) {
                    if (dist[u] == INFINITY) touched.push_back(u);
                    dist[u] = nd;
                    heap.push({nd, u});
                }
            }
        }
        for (int v : touched) {
            int row = fine_row(v);
            if (row >= 0 && row < nf) trips.push_back({row, c, 1.0 - dist[v] / rho});
            dist[v] = INFINITY;
        }
    }
    // rows without any centre inside the radius: nearest centre, weight one
    std::vector<char> covered(nf, 0);
    for (const Trip &t : trips) covered[t.row] = 1;
    int missing = 0;
    for (int r = 0; r < nf; ++r) missing += !covered[r];
    *fallback_rows = missing;
    if (missing) {
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
            if (!covered[r]) {
                int v = fine_vertex(r);
                HSIM_CHECK_ARG(label[v] >= 0, "a connected component of the mesh holds no coarse vertex");
                trips.push_back({r, label[v], 1.0});
            }
    }
    std::sort(trips.begin(), trips.end(), [](const Trip &a, const Trip &b) {
        return a.row < b.row || (a.row == b.row && a.c < b.c);
    });
    Csr U;
    U.n_rows = nf;
    U.n_cols = nc;
    U.ptr.assign(nf + 1, 0);
    U.col.resize(trips.size());
    U.val.resize(trips.size());
    for (const Trip &t : trips) U.ptr[t.row + 1]++;
    for (int r = 0; r < nf; ++r) U.ptr[r + 1] += U.ptr[r];
    for (int r = 0; r < nf; ++r) {
        double sum = 0.0;
        for (int e = U.ptr[r]; e < U.ptr[r + 1]; ++e) sum += trips[e].w;
        for (int e = U.ptr[r]; e < U.ptr[r + 1]; ++e) {
            U.col[e] = trips[e].c;
            U.val[e] = trips[e].w / sum;
        }
    }
    return U;
}

HostHierarchy build_host_hierarchy(int n, int m, const double *V, const int *F, const double *L2, int p,
                                   int levels, int start_vertex, double sigma, int q, bool dirichlet) {
    HSIM_CHECK_ARG(p >= 1, "p must be >= 1");
    HSIM_CHECK_ARG(sigma > 0.0, "sigma must be positive");
    HostHierarchy h;
    h.g = build_mesh_graph(n, m, V, F, L2);
    HSIM_CHECK_ARG(start_vertex >= 0 && start_vertex < n, "start_vertex out of range");
    std::vector<char> interior;
    if (dirichlet) {
        interior.assign(n, 1);
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
    if (T > 1) h.order = farthest_point_order(h.g, start_vertex, h.sizes[1], dirichlet ? &interior : nullptr);
    h.U.resize(T - 1);
    h.rho.assign(T - 1, 0.0);
    h.fallback.assign(T - 1, 0);
    for (int tau = 0; tau + 1 < T; ++tau)
        h.U[tau] = prolongation(h.g, h.order, h.sizes[tau], h.sizes[tau + 1], tau == 0, sigma, &h.rho[tau],
                                &h.fallback[tau], dirichlet ? &h.dofs : nullptr);
    return h;
}

}  // namespace hsim
