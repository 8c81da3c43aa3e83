/*
 * graphgen.c -- seeded synthetic graph inputs for the push/pull sweeps.
 *
 * This file only manufactures inputs: R-MAT and Erdos-Renyi edge lists, their
 * compressed adjacency arrays (CSR = out-edges of each vertex, CSC = in-edges of
 * each vertex), edge weights and random vertex picks.  It holds none of
 * PageRank's or BFS's arithmetic; the CPU oracle and the CUDA library both
 * consume what it produces and nothing else is shared between them.
 *
 * Graph layout follows the paper's Section 2.2: the neighbours of every vertex
 * form one contiguous array, and per-vertex offsets mark where each vertex's
 * neighbours begin (n+1 offsets, m neighbour cells per direction).
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator.  Draw i of the stream with key k is mix(k + (i+1)*gamma) with
 * gamma = 0x9E3779B97F4A7C15 and mix the published 64-bit finaliser, so every
 * draw is addressable and the output does not depend on the thread count.
 *
 * Integer-only except for the R-MAT quadrant test and the weights, which use
 * IEEE double arithmetic that gives identical results on x86-64 and AArch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of the stream for a user seed (the seed itself is hashed once so that
 * small consecutive seeds give unrelated streams). */
uint64_t gg_key(uint64_t seed) { return gg_mix(seed * GG_GAMMA + 0x5851F42D4C957F2DULL); }

/* Draw i of the stream with key k. */
uint64_t gg_draw(uint64_t key, uint64_t i) { return gg_mix(key + (i + 1) * GG_GAMMA); }

/* Uniform double in [0, 1) from the top 53 bits of a draw (exact). */
static inline double gg_u01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

/* Uniform integer in [0, n) by the multiply-high method (Lemire 2019, without
 * the rejection step: the bias is below n / 2^64). */
static inline uint64_t gg_below(uint64_t r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

static void gg_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/*
 * R-MAT edge sampler (Chakrabarti, Zhan and Faloutsos, SDM 2004).  Edge e picks
 * one quadrant per level, most significant bit first: with probability a the
 * (0,0) quadrant, b the (0,1) quadrant (destination bit set), c the (1,0)
 * quadrant (source bit set), otherwise (1,1).  Level l of edge e uses draw
 * e*scale + l.  No noise and no vertex permutation: vertex ids with few set
 * bits are the hubs.
 */
void gg_rmat_edges(int scale, int64_t ne, double a, double b, double c, uint64_t seed,
                   int32_t *src, int32_t *dst, int nthreads) {
    const uint64_t key = gg_key(seed);
    const double ab = a + b, abc = a + b + c;
    gg_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) {
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            const double r = gg_u01(gg_draw(key, (uint64_t)e * (uint64_t)scale + (uint64_t)l));
            const uint32_t bit = 1u << (scale - 1 - l);
            if (r < a) {
            } else if (r < ab) {
                v |= bit;
            } else if (r < abc) {
                u |= bit;
            } else {
                u |= bit;
                v |= bit;
            }
        }
        src[e] = (int32_t)u;
        dst[e] = (int32_t)v;
    }
}

/* Directed Erdos-Renyi G(n, m) sampler: edge e draws its source from draw 2e and
 * its destination from draw 2e+1, both uniform in [0, n). */
void gg_er_edges(int64_t n, int64_t ne, uint64_t seed, int32_t *src, int32_t *dst, int nthreads) {
    const uint64_t key = gg_key(seed);
    gg_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) {
        src[e] = (int32_t)gg_below(gg_draw(key, 2 * (uint64_t)e), (uint64_t)n);
        dst[e] = (int32_t)gg_below(gg_draw(key, 2 * (uint64_t)e + 1), (uint64_t)n);
    }
}

/* The calling OpenMP thread's share [lo, hi) of [0, n) (all of it outside a
 * parallel region). */
static void gg_thread_range(int64_t n, int64_t *lo, int64_t *hi) {
#ifdef _OPENMP
    const int64_t t = omp_get_thread_num(), T = omp_get_num_threads();
#else
    const int64_t t = 0, T = 1;
#endif
    *lo = n * t / T;
    *hi = n * (t + 1) / T;
}

static int gg_cmp_i32(const void *x, const void *y) {
    const int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

static void gg_sort_small(int32_t *p, int64_t len) {
    if (len > 48) {
        qsort(p, (size_t)len, sizeof(int32_t), gg_cmp_i32);
        return;
    }
    for (int64_t i = 1; i < len; ++i) {
        int32_t x = p[i];
        int64_t j = i - 1;
        while (j >= 0 && p[j] > x) {
            p[j + 1] = p[j];
            --j;
        }
        p[j + 1] = x;
    }
}

/*
 * Edge list -> CSR (rows sorted ascending).  symmetrize adds (v,u) for every
 * (u,v); drop_self removes u==v; dedup keeps one copy of repeated (u,v).
 * off has n+1 entries; idx must hold cap >= (symmetrize ? 2 : 1) * ne entries.
 * Returns the number of stored edges m (idx[0..m) is the result), or -1 if an
 * endpoint is outside [0, n) or cap is too small.
 */
int64_t gg_build_csr(int64_t n, int64_t ne, const int32_t *src, const int32_t *dst, int symmetrize,
                     int drop_self, int dedup, int64_t *off, int32_t *idx, int64_t cap, int nthreads) {
    if (cap < (symmetrize ? 2 : 1) * ne) return -1;
    gg_set_threads(nthreads);
    for (int64_t e = 0; e < ne; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    /* Counting sort by row.  Each thread owns a contiguous range of rows and
     * scans the whole edge list in order, touching only its own rows, so a
     * row's entries arrive in edge order whatever the thread count. */
#pragma omp parallel
    {
        int64_t lo = 0, hi = n;
        gg_thread_range(n, &lo, &hi);
        for (int64_t e = 0; e < ne; ++e) {
            const int32_t u = src[e], v = dst[e];
            if (drop_self && u == v) continue;
            if (u >= lo && u < hi) cnt[u]++;
            if (symmetrize && v >= lo && v < hi) cnt[v]++;
        }
    }
    off[0] = 0;
    for (int64_t v = 0; v < n; ++v) off[v + 1] = off[v] + cnt[v];
    for (int64_t v = 0; v < n; ++v) cnt[v] = off[v];
#pragma omp parallel
    {
        int64_t lo = 0, hi = n;
        gg_thread_range(n, &lo, &hi);
        for (int64_t e = 0; e < ne; ++e) {
            const int32_t u = src[e], v = dst[e];
            if (drop_self && u == v) continue;
            if (u >= lo && u < hi) idx[cnt[u]++] = v;
            if (symmetrize && v >= lo && v < hi) idx[cnt[v]++] = u;
        }
    }
    /* sort (and dedup) every row in place; cnt[v] becomes the kept length */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
        int32_t *p = idx + off[v];
        const int64_t len = off[v + 1] - off[v];
        gg_sort_small(p, len);
        int64_t k = len;
        if (dedup && len > 1) {
            k = 1;
            for (int64_t i = 1; i < len; ++i)
                if (p[i] != p[k - 1]) p[k++] = p[i];
        }
        cnt[v] = k;
    }
    /* compact rows towards the front (rows only shrink, so writes never pass reads) */
    int64_t w = 0;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t beg = off[v], k = cnt[v];
        off[v] = w;
        if (w != beg) memmove(idx + w, idx + beg, (size_t)k * sizeof(int32_t));
        w += k;
    }
    off[n] = w;
    free(cnt);
    return w;
}

/*
 * CSR -> CSC by a stable counting sort on the destination, so each column lists
 * its sources in ascending order.  w/tw may be NULL.  perm (nullable) receives,
 * for every CSC slot, the CSR position of the same edge.
 */
void gg_transpose(int64_t n, const int64_t *off, const int32_t *idx, const float *w, int64_t *toff,
                  int32_t *tidx, float *tw, int64_t *perm) {
    const int64_t m = off[n];
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    /* as in gg_build_csr: each thread owns a range of columns and scans all rows in order */
#pragma omp parallel
    {
        int64_t lo = 0, hi = n;
        gg_thread_range(n, &lo, &hi);
        for (int64_t e = 0; e < m; ++e)
            if (idx[e] >= lo && idx[e] < hi) cnt[idx[e]]++;
    }
    toff[0] = 0;
    for (int64_t v = 0; v < n; ++v) toff[v + 1] = toff[v] + cnt[v];
    for (int64_t v = 0; v < n; ++v) cnt[v] = toff[v];
#pragma omp parallel
    {
        int64_t lo = 0, hi = n;
        gg_thread_range(n, &lo, &hi);
        for (int64_t u = 0; u < n; ++u) {
            for (int64_t e = off[u]; e < off[u + 1]; ++e) {
                const int32_t v = idx[e];
                if (v < lo || v >= hi) continue;
                const int64_t slot = cnt[v]++;
                tidx[slot] = (int32_t)u;
                if (w && tw) tw[slot] = w[e];
                if (perm) perm[slot] = e;
            }
        }
    }
    free(cnt);
}

/* Weights uniform in (0, 1]: draw e gives 1 - u01, rounded to float (never 0). */
void gg_uniform_weights(int64_t m, uint64_t seed, float *w, int nthreads) {
    const uint64_t key = gg_key(seed);
    gg_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        float x = (float)(1.0 - gg_u01(gg_draw(key, (uint64_t)e)));
        w[e] = x > 0.0f ? x : 0x1.0p-24f;
    }
}

/* Integer-valued weights uniform in [lo, hi] (one draw per CSR edge), stored as
 * float: path sums stay exact in FP32 while they are below 2^24. */
void gg_int_weights(int64_t m, uint64_t seed, int32_t lo, int32_t hi, float *w, int nthreads) {
    const uint64_t key = gg_key(seed);
    const uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
    gg_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) w[e] = (float)(lo + (int64_t)(gg_draw(key, (uint64_t)e) % span));
}

/* Scale the weights of every CSR row so that they sum to one (in double, then
 * rounded to float): the column-normalised transition matrix of the input
 * recipe.  Rows without edges are left alone. */
void gg_normalize_rows(int64_t n, const int64_t *off, float *w, int nthreads) {
    gg_set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t u = 0; u < n; ++u) {
        double s = 0.0;
        for (int64_t e = off[u]; e < off[u + 1]; ++e) s += (double)w[e];
        if (s > 0.0)
            for (int64_t e = off[u]; e < off[u + 1]; ++e) w[e] = (float)((double)w[e] / s);
    }
}

/*
 * Pick `count` distinct vertices whose degree (off[v+1]-off[v]) is at least
 * min_deg, from draws 0, 1, 2, ... of the stream (rejection sampling).  Returns
 * the number picked (less than count only if too few vertices qualify).
 */
int64_t gg_pick_vertices(int64_t n, const int64_t *off, int64_t count, int64_t min_deg, uint64_t seed,
                         int32_t *out) {
    const uint64_t key = gg_key(seed);
    int64_t eligible = 0;
    for (int64_t v = 0; v < n; ++v) eligible += (off[v + 1] - off[v]) >= min_deg;
    if (count > eligible) count = eligible;
    uint8_t *taken = (uint8_t *)calloc((size_t)n, 1);
    int64_t got = 0;
    for (uint64_t i = 0; got < count; ++i) {
        const int64_t v = (int64_t)gg_below(gg_draw(key, i), (uint64_t)n);
        if (taken[v] || (off[v + 1] - off[v]) < min_deg) continue;
        taken[v] = 1;
        out[got++] = (int32_t)v;
    }
    free(taken);
    return got;
}
