/*
 * ORACLE — test infrastructure only.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * does, and nothing here is shared with the CUDA side.
 *
 * Pull-form PageRank in FP64, written from the paper's generated reduction
 * code for PageRank (Section 3.3, the OpenACC reduction listing): every
 * iteration gives each vertex v
 *
 *     PR'(v) = (1 - delta) / N + delta * sum over in-neighbours u of PR(u) / outdeg(u)
 *
 * (the in-neighbours read from the reverse CSR, the out-degree from the
 * forward CSR) and accumulates the change of the iteration.  Readings taken
 * where the listing is silent or loose: PR starts at 1 / N; the change is
 * the L1 norm sum |PR'(v) - PR(v)| (the listing adds the signed differences,
 * which cancel); the loop stops after the first iteration whose change is at
 * most `tol` (never when tol < 0), or after `max_iter` iterations; a vertex
 * without out-arcs
 * passes nothing on (its share is not redistributed, as in the listing).
 * For an undirected graph both directions of every edge are stored, so the
 * in-neighbours are the neighbours.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The transpose of the out-arc CSR, rows in increasing source id. */
static int in_arcs(int32_t n, const int32_t* rp, const int32_t* ci, int32_t** trp, int32_t** tci) {
    int64_t nnz = n > 0 ? rp[n] : 0;
    *trp = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    *tci = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    int32_t* fill = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!*trp || !*tci || !fill) { free(*trp); free(*tci); free(fill); return -2; }
    for (int64_t e = 0; e < nnz; ++e) (*trp)[ci[e] + 1] += 1;
    for (int32_t v = 0; v < n; ++v) (*trp)[v + 1] += (*trp)[v];
    for (int32_t v = 0; v < n; ++v) fill[v] = (*trp)[v];
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = rp[u]; e < rp[u + 1]; ++e) (*tci)[fill[ci[e]]++] = u;
    free(fill);
    return 0;
}

/*
 * pr[n] receives the ranks; *iters the iterations run; *change the last
 * iteration's L1 change.  Returns 0, -1 on bad arguments, -2 out of memory.
 */
int oracle_pagerank(int32_t n, const int32_t* rp, const int32_t* ci, double damping, double tol, int32_t max_iter,
                    double* pr, int32_t* iters, double* change) {
    if (n <= 0 || max_iter < 0 || !(damping >= 0.0 && damping <= 1.0)) return -1;
    int32_t *trp = NULL, *tci = NULL;
    if (in_arcs(n, rp, ci, &trp, &tci) != 0) return -2;
    double* next = (double*)malloc((size_t)n * sizeof(double));
    if (!next) { free(trp); free(tci); return -2; }
    for (int32_t v = 0; v < n; ++v) pr[v] = 1.0 / (double)n;
    int32_t it = 0;
    double diff = 0.0;
    while (it < max_iter) {
        diff = 0.0;
        for (int32_t v = 0; v < n; ++v) {
            double sum = 0.0;
            for (int32_t e = trp[v]; e < trp[v + 1]; ++e) {
                int32_t u = tci[e];
                sum = sum + pr[u] / (double)(rp[u + 1] - rp[u]);
            }
            double val = (1.0 - damping) / (double)n + damping * sum;
            diff = diff + fabs(val - pr[v]);
            next[v] = val;
        }
        memcpy(pr, next, (size_t)n * sizeof(double));
        ++it;
        if (diff <= tol) break;
    }
    *iters = it;
    *change = diff;
    free(next); free(trp); free(tci);
    return 0;
}
