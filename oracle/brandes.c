/*
 * ORACLE — test infrastructure only.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * does, and nothing here is shared with the CUDA side.
 *
 * Plain single-threaded Brandes betweenness centrality in FP64, written from
 * the method as the paper states it (Section 2, Fig. 1, the ComputeBC program;
 * Brandes' algorithm is cited there):
 *
 *   BC = 0                                            (attachNodeProperty)
 *   for src in sourceSet:
 *       sigma = 0, delta = 0, sigma[src] = 1
 *       iterateInBFS(v from src):                     (forward, BFS order)
 *           for w in neighbours(v): v.sigma += w.sigma
 *       iterateInReverse(v != src):                   (backward, reverse BFS order)
 *           for w in neighbours(v): v.delta += (v.sigma / w.sigma) * (1 + w.delta)
 *           v.BC += v.delta
 *
 * Readings taken where the listing is silent: the forward sum runs over BFS
 * parents only (dist[w] == dist[v] - 1)
 * and the backward sum over BFS children only (dist[w] == dist[v] + 1), as in
 * Brandes' algorithm; graphs are undirected and ordered (s, t) pairs are
 * counted, with no halving; vertices not reached from src have no sigma, no
 * delta and no contribution.  The backward step keeps the per-arc ratio form of
 * the listing, (sigma_v / sigma_w)(1 + delta_w).
 *
 * Path counts grow exponentially with depth on high-diameter graphs and leave
 * the double range.  In XFLOAT mode sigma is held as mantissa * 2^exponent with
 * a 64-bit exponent; every operation on it rescales by exact powers of two (set
 * from the IEEE-754 exponent field), so wherever plain doubles stay finite and
 * normal, XFLOAT gives the plain-double result bit for bit.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORACLE_PLAIN = 0, ORACLE_XFLOAT = 1, ORACLE_AUTO = 2 };

typedef struct {
    int64_t levels;         /* L = 1 + max distance over reached vertices */
    int64_t reached;        /* |R_s| including the source */
    int64_t arcs;           /* A_s = sum of degrees over reached vertices */
    int32_t used_xfloat;    /* 1 if this source needed the extended exponent */
    int32_t pad;
    double max_level_spread_log2; /* max over levels of log2(max sigma / min sigma) in the level */
} oracle_src_stats;

/* ---- exact power-of-two scaling from the IEEE-754 binary64 layout ---- */
static double pow2i(int k) { /* 2^k for -1022 <= k <= 1023 */
    uint64_t bits = (uint64_t)(k + 1023) << 52;
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
}
static double scale2(double x, int64_t k) {
    while (k > 1000) { x *= pow2i(1000); k -= 1000; }
    while (k < -1000) { x *= pow2i(-1000); k += 1000; }
    return x * pow2i((int)k);
}
/* Unbiased exponent of a finite nonzero normal double. */
static int64_t exponent_of(double x) {
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    return (int64_t)((bits >> 52) & 0x7FF) - 1023;
}

/* Extended-range value m * 2^e, m in [1, 2) or m == 0. */
typedef struct { double m; int64_t e; } xf;

static xf xf_norm(double m, int64_t e) {
    xf r;
    if (m == 0.0) { r.m = 0.0; r.e = 0; return r; }
    int64_t k = exponent_of(m);
    r.m = scale2(m, -k);
    r.e = e + k;
    return r;
}
static xf xf_add(xf a, xf b) {
    if (a.m == 0.0) return b;
    if (b.m == 0.0) return a;
    if (a.e < b.e) { xf t = a; a = b; b = t; }
    int64_t d = a.e - b.e;
    double s = d > 1100 ? a.m : a.m + scale2(b.m, -d);
    return xf_norm(s, a.e);
}
/* a / b as a plain double (finite and nonzero inputs). */
static double xf_ratio(xf a, xf b) { return scale2(a.m / b.m, a.e - b.e); }

/* ---- BFS (FIFO), the traversal order of iterateInBFS ---- */
/* order[] receives the vertices in BFS order; returns how many were reached. */
static int64_t bfs_order(int32_t n, const int32_t* rp, const int32_t* ci, int32_t src, int32_t* dist,
                         int32_t* order) {
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    int64_t head = 0, tail = 0;
    dist[src] = 0;
    order[tail++] = src;
    while (head < tail) {
        int32_t u = order[head++];
        for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t v = ci[e];
            if (dist[v] < 0) { dist[v] = dist[u] + 1; order[tail++] = v; }
        }
    }
    return tail;
}

int oracle_bfs(int32_t n, const int32_t* rp, const int32_t* ci, int32_t src, int32_t* dist) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    int32_t* order = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!order) return -2;
    bfs_order(n, rp, ci, src, dist, order);
    free(order);
    return 0;
}

/* One source of ComputeBC.  Adds this source's dependencies into bc.
 * (rp, ci) hold the out-arcs: the BFS and the backward sum run over them.
 * (prp, pci) hold the arcs the forward sum pulls over: the same arrays for an
 * undirected graph, the in-arcs (the transpose) for a directed one. */
static int one_source(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* prp, const int32_t* pci,
                      int32_t src, int use_xf, double* bc,
                      int32_t* dist, int32_t* order, double* sigma, xf* xsigma, double* delta,
                      oracle_src_stats* st, double* mant_out, int64_t* exp_out) {
    int64_t reached = bfs_order(n, rp, ci, src, dist, order);

    /* sigma = 0, delta = 0, src.sigma = 1 */
    for (int64_t i = 0; i < reached; ++i) {
        int32_t v = order[i];
        delta[v] = 0.0;
        if (use_xf) { xsigma[v].m = 0.0; xsigma[v].e = 0; } else sigma[v] = 0.0;
    }
    if (use_xf) xsigma[src] = xf_norm(1.0, 0); else sigma[src] = 1.0;

    /* Forward: v in BFS order, sigma pulled from neighbours one level up. */
    int overflow = 0;
    for (int64_t i = 1; i < reached; ++i) {
        int32_t v = order[i];
        for (int32_t e = prp[v]; e < prp[v + 1]; ++e) {
            int32_t w = pci[e];
            if (dist[w] != dist[v] - 1) continue;
            if (use_xf) xsigma[v] = xf_add(xsigma[v], xsigma[w]);
            else sigma[v] = sigma[v] + sigma[w];
        }
        if (!use_xf && !(sigma[v] <= 1.7976931348623157e308)) overflow = 1;
    }
    if (overflow) return 1; /* caller retries this source in XFLOAT mode */

    /* Backward: v in reverse BFS order, v != src. */
    for (int64_t i = reached - 1; i >= 1; --i) {
        int32_t v = order[i];
        for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
            int32_t w = ci[e];
            if (dist[w] != dist[v] + 1) continue;
            double ratio = use_xf ? xf_ratio(xsigma[v], xsigma[w]) : sigma[v] / sigma[w];
            delta[v] = delta[v] + ratio * (1.0 + delta[w]);
        }
        bc[v] = bc[v] + delta[v];
    }

    if (st) {
        int64_t arcs = 0;
        int32_t maxd = 0;
        for (int64_t i = 0; i < reached; ++i) {
            int32_t v = order[i];
            arcs += rp[v + 1] - rp[v];
            if (dist[v] > maxd) maxd = dist[v];
        }
        st->levels = (int64_t)maxd + 1;
        st->reached = reached;
        st->arcs = arcs;
        st->used_xfloat = use_xf;
        /* Level spread of sigma in log2 units; vertices are contiguous per level in BFS order. */
        double spread = 0.0;
        int64_t i = 0;
        while (i < reached) {
            int32_t d = dist[order[i]];
            double lo = 0, hi = 0;
            int first = 1;
            for (; i < reached && dist[order[i]] == d; ++i) {
                int32_t v = order[i];
                double l2;
                if (use_xf) {
                    /* log2 of m*2^e with m in [1,2): e + log2(m) ~ e + (m - 1) is enough for a spread
                       report; the exact value is not part of any comparison. */
                    l2 = (double)xsigma[v].e + (xsigma[v].m - 1.0);
                } else {
                    l2 = (double)exponent_of(sigma[v]) + (scale2(sigma[v], -exponent_of(sigma[v])) - 1.0);
                }
                if (first || l2 < lo) lo = l2;
                if (first || l2 > hi) hi = l2;
                first = 0;
            }
            if (hi - lo > spread) spread = hi - lo;
        }
        st->max_level_spread_log2 = spread;
    }
    if (mant_out && exp_out) {
        for (int32_t v = 0; v < n; ++v) {
            if (dist[v] < 0) { mant_out[v] = 0.0; exp_out[v] = 0; continue; }
            if (use_xf) { mant_out[v] = xsigma[v].m; exp_out[v] = xsigma[v].e; }
            else {
                int64_t k = exponent_of(sigma[v]);
                mant_out[v] = scale2(sigma[v], -k);
                exp_out[v] = k;
            }
        }
    }
    return 0;
}

/*
 * BC over a multiset of sources (duplicates count once per occurrence).
 * bc[n] is overwritten.  stats may be NULL, else holds nsrc entries.
 * Returns 0, or -1 on bad arguments, -2 when out of memory.
 */
static int bc_over(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* prp, const int32_t* pci,
                   const int32_t* sources, int32_t nsrc, int mode, double* bc, oracle_src_stats* stats) {
    if (n < 0 || nsrc < 0 || (nsrc > 0 && n == 0)) return -1;
    for (int32_t i = 0; i < nsrc; ++i)
        if (sources[i] < 0 || sources[i] >= n) return -1;
    for (int32_t v = 0; v < n; ++v) bc[v] = 0.0;
    if (nsrc == 0 || n == 0) return 0;
    int32_t* dist = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* order = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    double* sigma = (double*)malloc((size_t)n * sizeof(double));
    xf* xsigma = (xf*)malloc((size_t)n * sizeof(xf));
    double* delta = (double*)malloc((size_t)n * sizeof(double));
    if (!dist || !order || !sigma || !xsigma || !delta) {
        free(dist); free(order); free(sigma); free(xsigma); free(delta);
        return -2;
    }
    for (int32_t i = 0; i < nsrc; ++i) {
        oracle_src_stats* st = stats ? &stats[i] : NULL;
        int use_xf = (mode == ORACLE_XFLOAT);
        int rc = one_source(n, rp, ci, prp, pci, sources[i], use_xf, bc, dist, order, sigma, xsigma, delta, st,
                            NULL, NULL);
        if (rc == 1 && mode == ORACLE_AUTO)
            rc = one_source(n, rp, ci, prp, pci, sources[i], 1, bc, dist, order, sigma, xsigma, delta, st, NULL,
                            NULL);
        if (rc == 1) { /* PLAIN mode overflowed: report infinity as the result */
            for (int32_t v = 0; v < n; ++v) bc[v] = 1.0 / 0.0;
            break;
        }
    }
    free(dist); free(order); free(sigma); free(xsigma); free(delta);
    return 0;
}

/*
 * Path counts from one source as mant * 2^exp (mant in [1,2), 0 when not
 * reached).  mode as in oracle_bc.  dist may be NULL.
 */
static int sigma_over(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* prp, const int32_t* pci,
                      int32_t src, int mode, double* mant, int64_t* exp2, int32_t* dist_out, oracle_src_stats* st) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    int32_t* dist = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* order = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    double* sigma = (double*)malloc((size_t)n * sizeof(double));
    xf* xsigma = (xf*)malloc((size_t)n * sizeof(xf));
    double* delta = (double*)malloc((size_t)n * sizeof(double));
    double* bc = (double*)calloc((size_t)n, sizeof(double));
    int rc = -2;
    if (dist && order && sigma && xsigma && delta && bc) {
        int use_xf = (mode == ORACLE_XFLOAT);
        rc = one_source(n, rp, ci, prp, pci, src, use_xf, bc, dist, order, sigma, xsigma, delta, st, mant, exp2);
        if (rc == 1 && mode == ORACLE_AUTO)
            rc = one_source(n, rp, ci, prp, pci, src, 1, bc, dist, order, sigma, xsigma, delta, st, mant, exp2);
        if (rc == 0 && dist_out) memcpy(dist_out, dist, (size_t)n * sizeof(int32_t));
    }
    free(dist); free(order); free(sigma); free(xsigma); free(delta); free(bc);
    return rc;
}

int oracle_bc(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* sources, int32_t nsrc, int mode,
              double* bc, oracle_src_stats* stats) {
    return bc_over(n, rp, ci, rp, ci, sources, nsrc, mode, bc, stats);
}

int oracle_sigma(int32_t n, const int32_t* rp, const int32_t* ci, int32_t src, int mode, double* mant,
                 int64_t* exp2, int32_t* dist_out, oracle_src_stats* st) {
    return sigma_over(n, rp, ci, rp, ci, src, mode, mant, exp2, dist_out, st);
}

/*
 * Directed graphs.  (rp, ci) hold the out-arcs u -> v.  The BFS follows
 * out-arcs; sigma(v) is pulled from the in-neighbours u of v one level up
 * (the BFS parents, u -> v with dist[u] = dist[v] - 1), read from the
 * transpose built here; delta(v) from the out-neighbours w one level down
 * (u -> w with dist[w] = dist[v] + 1), as above.  Transpose rows list their
 * in-neighbours in increasing id.
 */
static int transpose_csr(int32_t n, const int32_t* rp, const int32_t* ci, int32_t** trp, int32_t** tci) {
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

int oracle_bc_directed(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* sources, int32_t nsrc,
                       int mode, double* bc, oracle_src_stats* stats) {
    if (n < 0) return -1;
    int32_t *trp = NULL, *tci = NULL;
    if (transpose_csr(n, rp, ci, &trp, &tci) != 0) return -2;
    int rc = bc_over(n, rp, ci, trp, tci, sources, nsrc, mode, bc, stats);
    free(trp); free(tci);
    return rc;
}

int oracle_sigma_directed(int32_t n, const int32_t* rp, const int32_t* ci, int32_t src, int mode, double* mant,
                          int64_t* exp2, int32_t* dist_out, oracle_src_stats* st) {
    if (n <= 0) return -1;
    int32_t *trp = NULL, *tci = NULL;
    if (transpose_csr(n, rp, ci, &trp, &tci) != 0) return -2;
    int rc = sigma_over(n, rp, ci, trp, tci, src, mode, mant, exp2, dist_out, st);
    free(trp); free(tci);
    return rc;
}

/*
 * Per-source sums of hop distances, for the invariant
 *     sum_v BC(v) = sum over sources s, reached t != s of (d(s, t) - 1):
 * dsum[i] = sum of d(sources[i], t) over reached t, reached[i] = |R_s| with s.
 * Up to 64 sources share one breadth-first search as bits of a 64-bit word
 * per vertex (multi-source BFS: bit i of frontier[v] means d(s_i, v) = the
 * current level), a different method from the FIFO search above, used only
 * for the benchmark-size invariant where one search per source is too slow.
 * Returns 0, -1 on bad arguments, -2 when out of memory.
 */
int oracle_distance_sums(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* sources, int32_t nsrc,
                         int64_t* dsum, int64_t* reached) {
    if (n < 0 || nsrc < 0 || (nsrc > 0 && n == 0)) return -1;
    for (int32_t i = 0; i < nsrc; ++i)
        if (sources[i] < 0 || sources[i] >= n) return -1;
    if (nsrc == 0) return 0;
    uint64_t* seen = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    uint64_t* front = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    uint64_t* next = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    if (!seen || !front || !next) { free(seen); free(front); free(next); return -2; }
    for (int32_t g0 = 0; g0 < nsrc; g0 += 64) {
        int32_t cnt = nsrc - g0 < 64 ? nsrc - g0 : 64;
        memset(seen, 0, (size_t)n * sizeof(uint64_t));
        memset(front, 0, (size_t)n * sizeof(uint64_t));
        for (int32_t i = 0; i < cnt; ++i) {
            uint64_t bit = (uint64_t)1 << i;
            seen[sources[g0 + i]] |= bit;
            front[sources[g0 + i]] |= bit;
            dsum[g0 + i] = 0;
            reached[g0 + i] = 1;
        }
        for (int64_t d = 1;; ++d) {
            memset(next, 0, (size_t)n * sizeof(uint64_t));
            for (int32_t v = 0; v < n; ++v) {
                uint64_t f = front[v];
                if (!f) continue;
                for (int32_t e = rp[v]; e < rp[v + 1]; ++e) next[ci[e]] |= f;
            }
            int any = 0;
            for (int32_t u = 0; u < n; ++u) {
                uint64_t nb = next[u] & ~seen[u];
                front[u] = nb;
                if (!nb) continue;
                any = 1;
                seen[u] |= nb;
                while (nb) {
                    int i = __builtin_ctzll(nb);
                    nb &= nb - 1;
                    dsum[g0 + i] += d;
                    reached[g0 + i] += 1;
                }
            }
            if (!any) break;
        }
    }
    free(seen); free(front); free(next);
    return 0;
}
