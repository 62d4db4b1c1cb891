/*
 * ORACLE — test infrastructure only.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * does, and nothing here is shared with the CUDA side.
 *
 * Betweenness centrality on a graph with positive integer arc weights, in
 * FP64: the ComputeBC program of the paper (Section 2, Fig. 1) with its BFS
 * replaced by shortest distances under the weights, the computation the
 * paper's SSSP program produces (Section 3.5, the Min construct relaxing
 * dist[nbr] > dist[v] + weight).  Per source s:
 *
 *   dist      Dijkstra's algorithm with a binary heap (weights >= 1);
 *   sigma     v in nondecreasing dist: sigma(v) = sum over arcs u -> v with
 *             dist(u) + w(u, v) = dist(v) of sigma(u), pulled in the order of
 *             v's in-arc row (for an undirected graph its row);
 *   delta     v in nonincreasing dist, v != s: delta(v) = sum over arcs
 *             v -> x with dist(v) + w(v, x) = dist(x) of
 *             (sigma(v) / sigma(x)) (1 + delta(x)), in the order of v's row;
 *   BC(v) += delta(v).
 *
 * Every parent u of v has dist(u) < dist(v) (weights are at least 1), so each
 * sum reads final values.  Vertices of equal distance are visited in the
 * heap's settling order, which changes nothing: no vertex's sum reads another
 * vertex of its own distance.  With every weight 1 this is the BFS program:
 * the same sums in the same order, bit for bit.  Path counts are plain
 * doubles; a count that leaves the double range is reported (return 1).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t d;
    int32_t v;
} hent;

static void heap_push(hent* h, int64_t* size, int64_t d, int32_t v) {
    int64_t i = (*size)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= d) break;
        h[i] = h[p];
        i = p;
    }
    h[i].d = d;
    h[i].v = v;
}

static hent heap_pop(hent* h, int64_t* size) {
    hent top = h[0];
    hent last = h[--(*size)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *size) break;
        if (c + 1 < *size && h[c + 1].d < h[c].d) ++c;
        if (h[c].d >= last.d) break;
        h[i] = h[c];
        i = c;
    }
    if (*size > 0) h[i] = last;
    return top;
}

/* Transpose with weights: rows list in-arcs u -> v in increasing u. */
static int transpose_w(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* w, int32_t** trp,
                       int32_t** tci, int32_t** tw) {
    int64_t nnz = n > 0 ? rp[n] : 0;
    *trp = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    *tci = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    *tw = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    int32_t* fill = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!*trp || !*tci || !*tw || !fill) { free(*trp); free(*tci); free(*tw); free(fill); return -2; }
    for (int64_t e = 0; e < nnz; ++e) (*trp)[ci[e] + 1] += 1;
    for (int32_t v = 0; v < n; ++v) (*trp)[v + 1] += (*trp)[v];
    for (int32_t v = 0; v < n; ++v) fill[v] = (*trp)[v];
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t k = fill[ci[e]]++;
            (*tci)[k] = u;
            (*tw)[k] = w[e];
        }
    free(fill);
    return 0;
}

/*
 * bc[n] overwritten.  directed: 0 = (rp, ci, w) lists both directions of
 * every edge with equal weights and the pull reads the rows themselves;
 * 1 = out-arcs, the pull reads the transpose.  dist_out (may be NULL):
 * [nsrc][n] distances, -1 when unreachable.  Returns 0, 1 when a path count
 * left the double range, -1 bad arguments, -2 out of memory.
 */
int oracle_bc_weighted(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* w, int directed,
                       const int32_t* sources, int32_t nsrc, double* bc, int64_t* dist_out) {
    if (n < 0 || nsrc < 0 || (nsrc > 0 && n == 0)) return -1;
    for (int32_t i = 0; i < nsrc; ++i)
        if (sources[i] < 0 || sources[i] >= n) return -1;
    int64_t nnz = n > 0 ? rp[n] : 0;
    for (int64_t e = 0; e < nnz; ++e)
        if (w[e] < 1) return -1;
    for (int32_t v = 0; v < n; ++v) bc[v] = 0.0;
    if (nsrc == 0 || n == 0) return 0;
    const int32_t *prp = rp, *pci = ci, *pw = w;
    int32_t *trp = NULL, *tci = NULL, *tw = NULL;
    if (directed) {
        if (transpose_w(n, rp, ci, w, &trp, &tci, &tw) != 0) return -2;
        prp = trp; pci = tci; pw = tw;
    }
    int64_t* dist = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int32_t* order = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    char* done = (char*)malloc((size_t)n);
    double* sigma = (double*)malloc((size_t)n * sizeof(double));
    double* delta = (double*)malloc((size_t)n * sizeof(double));
    hent* heap = (hent*)malloc((size_t)(nnz + 1) * sizeof(hent));
    int rc = 0;
    if (!dist || !order || !done || !sigma || !delta || !heap) rc = -2;
    for (int32_t i = 0; rc == 0 && i < nsrc; ++i) {
        const int32_t s = sources[i];
        for (int32_t v = 0; v < n; ++v) { dist[v] = -1; done[v] = 0; sigma[v] = 0.0; delta[v] = 0.0; }
        /* Dijkstra: settle in nondecreasing distance */
        int64_t hs = 0, reached = 0;
        dist[s] = 0;
        heap_push(heap, &hs, 0, s);
        while (hs > 0) {
            hent t = heap_pop(heap, &hs);
            if (done[t.v] || t.d != dist[t.v]) continue;
            done[t.v] = 1;
            order[reached++] = t.v;
            for (int32_t e = rp[t.v]; e < rp[t.v + 1]; ++e) {
                int32_t x = ci[e];
                int64_t nd = t.d + w[e];
                if (dist[x] < 0 || nd < dist[x]) {
                    dist[x] = nd;
                    heap_push(heap, &hs, nd, x);
                }
            }
        }
        /* sigma, in settling order */
        sigma[s] = 1.0;
        for (int64_t k = 1; k < reached; ++k) {
            int32_t v = order[k];
            for (int32_t e = prp[v]; e < prp[v + 1]; ++e) {
                int32_t u = pci[e];
                if (dist[u] >= 0 && dist[u] + pw[e] == dist[v]) sigma[v] = sigma[v] + sigma[u];
            }
            if (!(sigma[v] <= 1.7976931348623157e308)) rc = 1;
        }
        if (rc != 0) break;
        /* delta, in reverse settling order */
        for (int64_t k = reached - 1; k >= 1; --k) {
            int32_t v = order[k];
            for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
                int32_t x = ci[e];
                if (dist[x] == dist[v] + w[e]) delta[v] = delta[v] + (sigma[v] / sigma[x]) * (1.0 + delta[x]);
            }
            bc[v] = bc[v] + delta[v];
        }
        if (dist_out)
            for (int32_t v = 0; v < n; ++v) dist_out[(int64_t)i * n + v] = dist[v];
    }
    free(dist); free(order); free(done); free(sigma); free(delta); free(heap);
    free(trp); free(tci); free(tw);
    return rc;
}
