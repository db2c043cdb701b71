/*
 * Plain C graph routines for the HSIM oracle (test infrastructure only).
 *
 * Distances are Dijkstra distances on the weighted edge graph of the mesh,
 * the geodesic approximation the paper uses for both farthest-point sampling
 * and the prolongation supports (Sec. 4.1, "Vertex hierarchy" and
 * "Prolongation and restriction").  Everything here is deliberately simple:
 * a binary heap, a linear scan for the farthest vertex, one bounded Dijkstra
 * per coarse vertex.  Compiled with -ffp-contract=off so every sum is the
 * plain IEEE addition of its two operands.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double d;
    int v;
} item_t;

typedef struct {
    item_t *a;
    long n, cap;
} heap_t;

static int item_less(item_t x, item_t y) {
    return x.d < y.d || (x.d == y.d && x.v < y.v);
}

static int heap_push(heap_t *h, double d, int v) {
    if (h->n == h->cap) {
        long nc = h->cap ? 2 * h->cap : 1024;
        item_t *na = (item_t *)realloc(h->a, (size_t)nc * sizeof(item_t));
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    long i = h->n++;
    item_t it = {d, v};
    while (i > 0) {
        long p = (i - 1) / 2;
        if (!item_less(it, h->a[p])) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i] = it;
    return 0;
}

static item_t heap_pop(heap_t *h) {
    item_t top = h->a[0];
    item_t last = h->a[--h->n];
    long i = 0;
    for (;;) {
        long l = 2 * i + 1, r = l + 1, m = i;
        item_t best = last;
        if (l < h->n && item_less(h->a[l], best)) { m = l; best = h->a[l]; }
        if (r < h->n && item_less(h->a[r], best)) { m = r; }
        if (m == i) break;
        h->a[i] = h->a[m];
        i = m;
    }
    if (h->n > 0) h->a[i] = last;
    return top;
}

/* Lower the field dist[] by the distances from src (Dijkstra that only
 * follows edges that improve the field). */
static int relax_from(int src, const int *ptr, const int *idx, const double *w,
                      double *dist, heap_t *h) {
    h->n = 0;
    dist[src] = 0.0;
    if (heap_push(h, 0.0, src)) return -1;
    while (h->n > 0) {
        item_t it = heap_pop(h);
        if (it.d > dist[it.v]) continue;
        for (int e = ptr[it.v]; e < ptr[it.v + 1]; ++e) {
            int u = idx[e];
            double nd = it.d + w[e];
            if (nd < dist[u]) {
                dist[u] = nd;
                if (heap_push(h, nd, u)) return -1;
            }
        }
    }
    return 0;
}

/* Farthest-point sampling (Alg. 2): order[0] = start, then repeatedly the
 * candidate vertex with the largest distance to the chosen set (lowest index
 * on ties).  cand == NULL makes every vertex a candidate; otherwise only the
 * vertices with cand[v] != 0 are chosen, while distances still run over the
 * whole graph.  count must not exceed the number of candidates.  Returns 0,
 * or -1 on allocation failure. */
int oracle_fps_among(int n, const int *ptr, const int *idx, const double *w, int start,
                     int count, const unsigned char *cand, int *order, double *field_out) {
    double *dist = (double *)malloc((size_t)n * sizeof(double));
    heap_t h = {0, 0, 0};
    if (!dist) return -1;
    for (int i = 0; i < n; ++i) dist[i] = INFINITY;
    order[0] = start;
    int rc = relax_from(start, ptr, idx, w, dist, &h);
    for (int k = 1; k < count && rc == 0; ++k) {
        int best = -1;
        for (int v = 0; v < n; ++v)
            if ((!cand || cand[v]) && (best < 0 || dist[v] > dist[best])) best = v;
        order[k] = best;
        rc = relax_from(best, ptr, idx, w, dist, &h);
    }
    if (field_out) memcpy(field_out, dist, (size_t)n * sizeof(double));
    free(dist);
    free(h.a);
    return rc;
}

int oracle_fps(int n, const int *ptr, const int *idx, const double *w, int start,
               int count, int *order, double *field_out) {
    return oracle_fps_among(n, ptr, idx, w, start, count, 0, order, field_out);
}

/* For every centre c (mesh vertex ids centres[0..nc)), all mesh vertices v
 * with Dijkstra distance d(c, v) < rho.  Writes triplets (centre position k,
 * vertex v, distance) into the caller's arrays of capacity cap.  Returns the
 * number of triplets, -needed if cap is too small, or a large negative
 * value on allocation failure. */
long oracle_balls(int n, const int *ptr, const int *idx, const double *w, int nc,
                  const int *centres, double rho, long cap, int *out_c, int *out_v,
                  double *out_d) {
    double *dist = (double *)malloc((size_t)n * sizeof(double));
    int *touched = (int *)malloc((size_t)n * sizeof(int));
    heap_t h = {0, 0, 0};
    long cnt = 0;
    if (!dist || !touched) { free(dist); free(touched); return -(1L << 62); }
    for (int i = 0; i < n; ++i) dist[i] = INFINITY;
    for (int k = 0; k < nc; ++k) {
        int nt = 0;
        int s = centres[k];
        h.n = 0;
        dist[s] = 0.0;
        touched[nt++] = s;
        heap_push(&h, 0.0, s);
        while (h.n > 0) {
            item_t it = heap_pop(&h);
            if (it.d > dist[it.v]) continue;
            for (int e = ptr[it.v]; e < ptr[it.v + 1]; ++e) {
                int u = idx[e];
                double nd = it.d + w[e];
                if (nd < rho && nd < dist[u]) {
                    if (dist[u] == INFINITY) touched[nt++] = u;
                    dist[u] = nd;
                    heap_push(&h, nd, u);
                }
            }
        }
        for (int t = 0; t < nt; ++t) {
            int v = touched[t];
            if (cnt < cap) { out_c[cnt] = k; out_v[cnt] = v; out_d[cnt] = dist[v]; }
            ++cnt;
            dist[v] = INFINITY;
        }
    }
    free(dist);
    free(touched);
    free(h.a);
    return cnt <= cap ? cnt : -cnt;
}

/* Multi-source Dijkstra from all centres: label[v] = position k of the
 * nearest centre (lowest k on equal distance), dist_out[v] its distance. */
int oracle_nearest(int n, const int *ptr, const int *idx, const double *w, int nc,
                   const int *centres, int *label, double *dist_out) {
    heap_t h = {0, 0, 0};
    for (int i = 0; i < n; ++i) { dist_out[i] = INFINITY; label[i] = -1; }
    for (int k = 0; k < nc; ++k) {
        dist_out[centres[k]] = 0.0;
        if (label[centres[k]] < 0) label[centres[k]] = k;
        if (heap_push(&h, 0.0, centres[k])) { free(h.a); return -1; }
    }
    while (h.n > 0) {
        item_t it = heap_pop(&h);
        if (it.d > dist_out[it.v]) continue;
        for (int e = ptr[it.v]; e < ptr[it.v + 1]; ++e) {
            int u = idx[e];
            double nd = it.d + w[e];
            /* a label change at equal distance is pushed again so that it
             * reaches everything downstream */
            if (nd < dist_out[u] || (nd == dist_out[u] && label[it.v] < label[u])) {
                dist_out[u] = nd;
                label[u] = label[it.v];
                if (heap_push(&h, nd, u)) { free(h.a); return -1; }
            }
        }
    }
    free(h.a);
    return 0;
}
