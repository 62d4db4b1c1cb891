/*
 * Seeded synthetic graph inputs shared by the oracle side and the CUDA side.
 *
 * This file holds no betweenness-centrality arithmetic: it only draws random
 * numbers, builds undirected int32 CSR graphs and picks source vertices.
 *
 * Random numbers: counter-based SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014).  Draw i of a
 * stream with seed k is the output function applied to k + (i+1)*gamma, which
 * is exactly the (i+1)-th output of a SplitMix64 generator started at state k,
 * so every draw can be computed independently and the result does not depend
 * on how many threads run the loops below.
 *
 * Graph recipes (the paper's graphs of its input table are not available, so
 * these stand in for its uniform-random, RMAT and road-network inputs):
 *   - Erdos-Renyi G(n, m): endpoints uniform, u != v, duplicate undirected
 *     edges rejected until m distinct edges exist.
 *   - RMAT(scale, edge factor, a, b, c, d): 2^scale vertices, ef * 2^scale
 *     draws, pure recursive quadrant choice, seeded random relabelling.
 *   - 2-D k-nearest-neighbour "road-like" graph: n points uniform in the unit
 *     square, Euclidean distance, ties broken by smaller index.
 * Every recipe symmetrises, drops self-loops and duplicate arcs and emits rows
 * sorted by neighbour id.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t draw(uint64_t seed, uint64_t i) { return mix64(seed + (i + 1) * GOLDEN); }
/* 53 random bits -> double in [0, 1). */
static inline double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
/* Multiply-shift map of 64 random bits onto [0, k) (bias below k / 2^64). */
static inline uint64_t below(uint64_t x, uint64_t k) { return (uint64_t)(((__uint128_t)x * k) >> 64); }
/* Independent sub-stream of a seed, one per purpose tag. */
static inline uint64_t substream(uint64_t seed, uint64_t tag) { return mix64(seed ^ mix64(tag + GOLDEN)); }

uint64_t gen_draw(uint64_t seed, uint64_t i) { return draw(seed, i); }
uint64_t gen_substream(uint64_t seed, uint64_t tag) { return substream(seed, tag); }

/* ------------------------------------------------------------------ */
/* LSD radix sort of 64-bit keys, 16-bit digits, only the passes needed. */
static int radix_sort_u64(uint64_t* a, int64_t n, int key_bits) {
    if (n <= 1) return 0;
    uint64_t* tmp = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    int64_t* cnt = (int64_t*)malloc(65536 * sizeof(int64_t));
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    uint64_t* src = a; uint64_t* dst = tmp;
    for (int shift = 0; shift < key_bits; shift += 16) {
        memset(cnt, 0, 65536 * sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> shift) & 0xFFFF]++;
        int64_t s = 0;
        for (int d = 0; d < 65536; ++d) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
    free(tmp); free(cnt);
    return 0;
}

static int bits_for(int64_t n) { int b = 1; while (b < 63 && ((int64_t)1 << b) < n) ++b; return b; }

/*
 * Arc keys (u << 32 | v), both directions already present -> sorted, unique,
 * self-loop-free CSR.  row_ptr has n+1 entries.  col_idx must hold nkeys
 * entries (the unique count is returned through *nnz_out).
 */
static int keys_to_csr(uint64_t* keys, int64_t nkeys, int32_t n, int32_t* row_ptr, int32_t* col_idx,
                       int64_t* nnz_out) {
    int b = bits_for((int64_t)n);
    if (radix_sort_u64(keys, nkeys, 32 + b) != 0) return -1;
    memset(row_ptr, 0, (size_t)(n + 1) * sizeof(int32_t));
    int64_t w = 0;
    uint64_t prev = ~0ULL;
    for (int64_t i = 0; i < nkeys; ++i) {
        uint64_t k = keys[i];
        if (k == prev) continue;
        prev = k;
        uint32_t u = (uint32_t)(k >> 32), v = (uint32_t)(k & 0xFFFFFFFFu);
        if (u == v) continue;
        col_idx[w++] = (int32_t)v;
        row_ptr[u + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    *nnz_out = w;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Erdos-Renyi G(n, m).  Upper bound for col_idx: 2*m. */
int gen_er(int32_t n, int64_t m, uint64_t seed, int32_t* row_ptr, int32_t* col_idx, int64_t* nnz_out) {
    if (n < 2 || m < 0 || (double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
    int64_t cap = 1; while (cap < 2 * m + 2) cap <<= 1;
    uint64_t* table = (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
    uint64_t* keys = (uint64_t*)malloc((size_t)(2 * m + 1) * sizeof(uint64_t));
    if (!table || !keys) { free(table); free(keys); return -2; }
    memset(table, 0xFF, (size_t)cap * sizeof(uint64_t));
    uint64_t s = substream(seed, 1);
    int64_t have = 0;
    uint64_t i = 0;
    while (have < m) {
        uint64_t u = below(draw(s, i), (uint64_t)n), v = below(draw(s, i + 1), (uint64_t)n);
        i += 2;
        if (u == v) continue;
        uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
        uint64_t key = (lo << 32) | hi;
        uint64_t h = mix64(key) & (uint64_t)(cap - 1);
        int dup = 0;
        while (table[h] != ~0ULL) {
            if (table[h] == key) { dup = 1; break; }
            h = (h + 1) & (uint64_t)(cap - 1);
        }
        if (dup) continue;
        table[h] = key;
        keys[2 * have] = (lo << 32) | hi;
        keys[2 * have + 1] = (hi << 32) | lo;
        ++have;
    }
    free(table);
    int rc = keys_to_csr(keys, 2 * m, n, row_ptr, col_idx, nnz_out);
    free(keys);
    return rc;
}

/* ------------------------------------------------------------------ */
/* RMAT.  n = 2^scale; draws = ef * n; upper bound for col_idx: 2 * draws. */
static int rmat_arcs(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed, int both,
                     int32_t* row_ptr, int32_t* col_idx, int64_t* nnz_out) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
    int32_t n = (int32_t)1 << scale;
    int64_t m = (int64_t)edge_factor * (int64_t)n;
    uint64_t* keys = (uint64_t*)malloc((size_t)(2 * m) * sizeof(uint64_t));
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!keys || !perm) { free(keys); free(perm); return -2; }
    uint64_t se = substream(seed, 2), sp = substream(seed, 3);
    double ab = a + b, abc = a + b + c;
    /* Seeded relabelling: Fisher-Yates shuffle of the identity. */
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)below(draw(sp, (uint64_t)i), (uint64_t)i + 1);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t u = 0, v = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double r = u01(draw(se, (uint64_t)e * (uint64_t)scale + (uint64_t)l));
            uint32_t ub, vb;
            if (r < a) { ub = 0; vb = 0; }
            else if (r < ab) { ub = 0; vb = 1; }
            else if (r < abc) { ub = 1; vb = 0; }
            else { ub = 1; vb = 1; }
            u = (u << 1) | ub; v = (v << 1) | vb;
        }
        uint64_t pu = (uint64_t)perm[u], pv = (uint64_t)perm[v];
        if (both) {
            keys[2 * e] = (pu << 32) | pv;
            keys[2 * e + 1] = (pv << 32) | pu;
        } else {
            keys[e] = (pu << 32) | pv;
        }
    }
    free(perm);
    int rc = keys_to_csr(keys, both ? 2 * m : m, n, row_ptr, col_idx, nnz_out);
    free(keys);
    return rc;
}

int gen_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed,
             int32_t* row_ptr, int32_t* col_idx, int64_t* nnz_out) {
    return rmat_arcs(scale, edge_factor, a, b, c, seed, 1, row_ptr, col_idx, nnz_out);
}

/* Directed RMAT: each draw is one arc u -> v (relabelled, deduped, no
   self-loops); upper bound for col_idx: draws. */
int gen_rmat_directed(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed,
                      int32_t* row_ptr, int32_t* col_idx, int64_t* nnz_out) {
    return rmat_arcs(scale, edge_factor, a, b, c, seed, 0, row_ptr, col_idx, nnz_out);
}

/* ------------------------------------------------------------------ */
/* 2-D k-nearest-neighbour graph.  Upper bound for col_idx: 2 * k * n. */
typedef struct { double d2; int32_t j; } nb_t;

static inline int nb_less(double d2, int32_t j, const nb_t* o) {
    return d2 < o->d2 || (d2 == o->d2 && j < o->j);
}

int gen_knn2d(int32_t n, int32_t k, uint64_t seed, double* xy_out, int32_t* row_ptr, int32_t* col_idx,
              int64_t* nnz_out) {
    if (n < 2 || k < 1 || k >= n || k > 16) return -1;
    double* xy = xy_out;
    uint64_t s = substream(seed, 4);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        xy[2 * i] = u01(draw(s, 2 * (uint64_t)i));
        xy[2 * i + 1] = u01(draw(s, 2 * (uint64_t)i + 1));
    }
    int32_t G = (int32_t)ceil(sqrt((double)n / 2.0));
    if (G < 1) G = 1;
    double cs = 1.0 / (double)G;
    int64_t ncell = (int64_t)G * G;
    int32_t* cstart = (int32_t*)calloc((size_t)ncell + 1, sizeof(int32_t));
    int32_t* cpts = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* ccell = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    uint64_t* keys = (uint64_t*)malloc((size_t)2 * k * n * sizeof(uint64_t));
    if (!cstart || !cpts || !ccell || !keys) { free(cstart); free(cpts); free(ccell); free(keys); return -2; }
    for (int32_t i = 0; i < n; ++i) {
        int32_t cx = (int32_t)(xy[2 * i] * G), cy = (int32_t)(xy[2 * i + 1] * G);
        if (cx >= G) cx = G - 1;
        if (cy >= G) cy = G - 1;
        ccell[i] = cy * G + cx;
        cstart[ccell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    {
        int32_t* fill = (int32_t*)malloc((size_t)ncell * sizeof(int32_t));
        if (!fill) { free(cstart); free(cpts); free(ccell); free(keys); return -2; }
        memcpy(fill, cstart, (size_t)ncell * sizeof(int32_t));
        for (int32_t i = 0; i < n; ++i) cpts[fill[ccell[i]]++] = i; /* ascending index within a cell */
        free(fill);
    }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        nb_t best[16];
        int have = 0;
        double px = xy[2 * i], py = xy[2 * i + 1];
        int32_t cx = ccell[i] % G, cy = ccell[i] / G;
        for (int32_t r = 0; r <= G; ++r) {
            for (int32_t y = cy - r; y <= cy + r; ++y) {
                if (y < 0 || y >= G) continue;
                int on_edge_row = (y == cy - r || y == cy + r);
                for (int32_t x = cx - r; x <= cx + r; ++x) {
                    if (x < 0 || x >= G) continue;
                    if (!on_edge_row && x != cx - r && x != cx + r) continue;
                    int64_t c = (int64_t)y * G + x;
                    for (int32_t p = cstart[c]; p < cstart[c + 1]; ++p) {
                        int32_t j = cpts[p];
                        if (j == i) continue;
                        double dx = xy[2 * j] - px, dy = xy[2 * j + 1] - py;
                        double d2 = dx * dx + dy * dy;
                        if (have < k) {
                            int q = have++;
                            while (q > 0 && nb_less(d2, j, &best[q - 1])) { best[q] = best[q - 1]; --q; }
                            best[q].d2 = d2; best[q].j = j;
                        } else if (nb_less(d2, j, &best[k - 1])) {
                            int q = k - 1;
                            while (q > 0 && nb_less(d2, j, &best[q - 1])) { best[q] = best[q - 1]; --q; }
                            best[q].d2 = d2; best[q].j = j;
                        }
                    }
                }
            }
            /* Points outside rings 0..r are at least r*cs away. */
            double reach = (double)r * cs;
            if (have == k && best[k - 1].d2 < reach * reach) break;
        }
        for (int q = 0; q < k; ++q) {
            uint64_t a = (uint64_t)i, b2 = (uint64_t)best[q].j;
            keys[(size_t)2 * (k * i + q)] = (a << 32) | b2;
            keys[(size_t)2 * (k * i + q) + 1] = (b2 << 32) | a;
        }
    }
    free(cstart); free(cpts); free(ccell);
    int rc = keys_to_csr(keys, (int64_t)2 * k * n, n, row_ptr, col_idx, nnz_out);
    free(keys);
    return rc;
}

/* ------------------------------------------------------------------ */
/*
 * k distinct sources drawn uniformly among vertices of degree >= 1, in draw
 * order (partial Fisher-Yates over the eligible ids in increasing order).
 * Returns the number of eligible vertices, or -1 if fewer than k exist.
 */
int64_t gen_sources(int32_t n, const int32_t* row_ptr, int32_t k, uint64_t seed, int32_t* out) {
    int32_t* elig = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!elig) return -2;
    int64_t cnt = 0;
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] > row_ptr[v]) elig[cnt++] = v;
    if (k > cnt) { free(elig); return -1; }
    uint64_t s = substream(seed, 5);
    for (int64_t i = 0; i < k; ++i) {
        int64_t j = i + (int64_t)below(draw(s, (uint64_t)i), (uint64_t)(cnt - i));
        int32_t t = elig[i]; elig[i] = elig[j]; elig[j] = t;
        out[i] = elig[i];
    }
    free(elig);
    return cnt;
}

/* Fill out[i] = draw(seed, first + i) for i < count (exposes the stream to callers). */
void gen_draws(uint64_t seed, uint64_t first, int64_t count, uint64_t* out) {
    for (int64_t i = 0; i < count; ++i) out[i] = draw(seed, first + (uint64_t)i);
}
