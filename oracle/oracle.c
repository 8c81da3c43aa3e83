/*
 * oracle.c -- plain FP64 CPU oracle for push/pull PageRank and BFS.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file.  The CUDA library never calls it and it
 * never calls the CUDA library; the two share no code, headers or tables.  The
 * only thing both sides consume is the graph produced by the input generator.
 *
 * Everything here is the definition written out, in the order the paper states
 * it, in double precision, with no blocking, fusion or reordering:
 *
 *   - Graph (Section 2.2): the oracle rebuilds its own adjacency arrays (out-
 *     and in-neighbours, n+1 offsets each) from the raw edge list it is given.
 *     Directed graphs (Section 4.8, "Directed Graphs"): pushing walks out-edges,
 *     pulling walks in-edges.
 *   - PageRank (Section 3.1 formula; Algorithm 1, push- and pull-based PR):
 *       y[v] = (1-d) s[v] + d * sum_{(u->v) in E} P_vu x[u]
 *     with P_vu = 1/deg_out(u) (unweighted) or the stored weight w_uv
 *     (weighted), s = 1/n unless a personalization vector is given.  Pull
 *     computes each y[v] from v's in-edges; push zeroes y, lets every u add
 *     d*P_vu*x[u] into y[v] for its out-edges, then adds (1-d)s.
 *   - BFS (Section 3.3; Algorithm 3 with every ready counter equal to one): a
 *     textbook FIFO BFS, and the level-synchronous form whose levels are
 *     explored either top-down (push: frontier vertices scan out-edges) or
 *     bottom-up (pull: unvisited vertices scan in-edges for a frontier vertex).
 *   - Adjoint of the PageRank fixed point (not in the paper): lambda solves
 *     (I - d P^T) lambda = g; dL/ds = (1-d) lambda; dL/dP_vu = d lambda_v x_u.
 *     With raw weights normalised inside (P_vu = W_uv / S_u), the chain rule
 *     through the normalisation gives dL/dW_uv (or_pagerank_adjoint_raw).
 *   - Single-source shortest paths: Dijkstra (the plain definition, min over
 *     paths of the weight sum), and the push- and pull-based Delta-Stepping of
 *     the paper's Section 3 listing, run sequentially with one direction per
 *     relaxation iteration.
 *   - Triangle counting (the NodeIterator listing of Section 3): for every v
 *     and every ordered pair (w1, w2) of v's neighbours with w1 adjacent to
 *     w2, pull adds one to tc[v], push adds one to tc[w1]; both halve.
 *   - Frontier-Exploit PageRank (Section 5's Frontier-Exploit applied to the
 *     PageRank of Section 3.1): only vertices whose pending change exceeds
 *     eps propagate it in an iteration (residual form, below).
 *   - Betweenness centrality (the Brandes scheme of the Section 3 listing):
 *     per source a BFS counting shortest-path multiplicities, then partial
 *     centralities accumulated back over the shortest-path DAG.
 *
 * Readings of the paper where it is silent or ambiguous (each is a choice the
 * CUDA path makes identically):
 *   - x0 = 1/n (Algorithm 1 initialises the ranks to the damping factor; the
 *     fixed point does not depend on x0, fixed-sweep comparisons do).
 *   - `iters` counts the sweeps actually performed (Algorithm 1's loop runs
 *     L-1 sweeps for L steps).
 *   - Jacobi double buffering: every y is computed from the previous x, then
 *     x <- y (Algorithm 1 writes pr[v] inside the parallel loop).
 *   - Dangling vertices (deg_out = 0) contribute nothing; no redistribution.
 *   - Convergence: L1 norm of y - x after each sweep, stop when < tol or after
 *     `iters` sweeps; tol = 0 runs exactly `iters` sweeps.
 *   - Bottom-up BFS stops scanning a vertex's in-edges at the first frontier
 *     neighbour (with ready = 1 the counter reaches zero there).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct or_graph {
    int64_t n, m;
    int64_t *out_off; /* n+1 */
    int32_t *out_idx; /* m: heads of out-edges */
    int64_t *out_eid; /* m: input edge id of each out-edge slot */
    int64_t *in_off;  /* n+1 */
    int32_t *in_idx;  /* m: tails of in-edges */
    int64_t *in_eid;  /* m: input edge id of each in-edge slot */
    double *w;        /* m or NULL: weight of input edge e, P_vu for e = (u->v) */
    int64_t *deg_out; /* n */
} or_graph;

static void or_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Adjacency arrays of Section 2.2 built by a counting sort of the edge list;
 * within a vertex the neighbours keep the order of the input list. */
or_graph *or_graph_new(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const double *w) {
    or_graph *g = (or_graph *)calloc(1, sizeof(or_graph));
    g->n = n;
    g->m = m;
    g->out_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->in_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->out_idx = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    g->in_idx = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    g->out_eid = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    g->in_eid = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    g->deg_out = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    g->w = NULL;
    if (w) {
        g->w = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
        for (int64_t e = 0; e < m; ++e) g->w[e] = w[e];
    }
    for (int64_t e = 0; e < m; ++e) {
        g->out_off[src[e] + 1]++;
        g->in_off[dst[e] + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) {
        g->out_off[v + 1] += g->out_off[v];
        g->in_off[v + 1] += g->in_off[v];
        g->deg_out[v] = 0;
    }
    int64_t *po = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *pi = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) {
        po[v] = g->out_off[v];
        pi[v] = g->in_off[v];
    }
    for (int64_t e = 0; e < m; ++e) {
        const int32_t u = src[e], v = dst[e];
        g->out_idx[po[u]] = v;
        g->out_eid[po[u]++] = e;
        g->in_idx[pi[v]] = u;
        g->in_eid[pi[v]++] = e;
        g->deg_out[u]++;
    }
    free(po);
    free(pi);
    return g;
}

void or_graph_free(or_graph *g) {
    if (!g) return;
    free(g->out_off);
    free(g->in_off);
    free(g->out_idx);
    free(g->in_idx);
    free(g->out_eid);
    free(g->in_eid);
    free(g->w);
    free(g->deg_out);
    free(g);
}

/* Transition entry P_vu of input edge e = (u -> v). */
static inline double or_P(const or_graph *g, int64_t e, int32_t u) {
    if (g->w) return g->w[e];
    return 1.0 / (double)g->deg_out[u];
}

/*
 * PageRank power iteration (Section 3.1; Algorithm 1).
 *   variant 0 = push: y = 0; for u, for (u->v): y[v] += d P_vu x[u]; y += (1-d) s.
 *   variant 1 = pull: for v: y[v] = (1-d) s[v] + d sum_{(u->v)} P_vu x[u].
 * s (nullable) is the personalization vector (uniform 1/n when NULL); x0
 * (nullable) the starting vector (1/n when NULL).  Runs until the L1 norm of
 * y - x is below tol or `iters` sweeps are done; x_out receives the last y.
 * nthreads > 1 parallelises the pull variant over v (each y[v] is still summed
 * in in-edge order by one thread, so the result does not change).
 * Returns 0 if converged (or tol == 0), 1 if the sweep cap was hit.
 */
int or_pagerank(const or_graph *g, int variant, double d, int iters, double tol, const double *s,
                const double *x0, double *x_out, int *iters_done, double *residual, int nthreads) {
    const int64_t n = g->n;
    double *x = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *y = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t v = 0; v < n; ++v) x[v] = x0 ? x0[v] : 1.0 / (double)n;
    or_set_threads(nthreads);
    int k = 0;
    double r = 0.0;
    int converged = 0;
    while (k < iters) {
        if (variant == 0) {
            for (int64_t v = 0; v < n; ++v) y[v] = 0.0;
            for (int64_t u = 0; u < n; ++u)
                for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j)
                    y[g->out_idx[j]] += d * or_P(g, g->out_eid[j], (int32_t)u) * x[u];
            for (int64_t v = 0; v < n; ++v) y[v] += (1.0 - d) * (s ? s[v] : 1.0 / (double)n);
        } else {
#pragma omp parallel for schedule(dynamic, 1024) if (nthreads > 1)
            for (int64_t v = 0; v < n; ++v) {
                double acc = 0.0;
                for (int64_t j = g->in_off[v]; j < g->in_off[v + 1]; ++j) {
                    const int32_t u = g->in_idx[j];
                    acc += or_P(g, g->in_eid[j], u) * x[u];
                }
                y[v] = (1.0 - d) * (s ? s[v] : 1.0 / (double)n) + d * acc;
            }
        }
        r = 0.0;
        for (int64_t v = 0; v < n; ++v) r += fabs(y[v] - x[v]);
        double *t = x;
        x = y;
        y = t;
        ++k;
        if (r < tol) {
            converged = 1;
            break;
        }
    }
    if (iters <= 0) r = 0.0;
    memcpy(x_out, x, (size_t)n * sizeof(double));
    if (iters_done) *iters_done = k;
    if (residual) *residual = r;
    free(x);
    free(y);
    return (converged || tol <= 0.0) ? 0 : 1;
}

/*
 * Textbook FIFO BFS from src over out-edges (Section 3.3): level[src] = 0,
 * parent[src] = src; a vertex is labelled by the first vertex that discovers
 * it in queue order.  Unreached vertices get level -1 and parent -1.
 * Returns the number of vertices reached.
 */
int64_t or_bfs_fifo(const or_graph *g, int32_t src, int32_t *level, int32_t *parent) {
    const int64_t n = g->n;
    for (int64_t v = 0; v < n; ++v) {
        level[v] = -1;
        parent[v] = -1;
    }
    if (src < 0 || src >= n) return 0;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t head = 0, tail = 0;
    queue[tail++] = src;
    level[src] = 0;
    parent[src] = src;
    while (head < tail) {
        const int32_t v = queue[head++];
        for (int64_t j = g->out_off[v]; j < g->out_off[v + 1]; ++j) {
            const int32_t w = g->out_idx[j];
            if (level[w] == -1) {
                level[w] = level[v] + 1;
                parent[w] = v;
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    return tail;
}

/*
 * Level-synchronous BFS of Algorithm 3 with ready = 1 (so the accumulated value
 * R is the level and the vertex it came from), one direction per level:
 *   dir 0, top-down (push): for every v in the frontier F, in frontier order,
 *     for every out-edge (v->w) with w unvisited: w gets level L+1 and parent v
 *     and joins the next frontier.
 *   dir 1, bottom-up (pull): for every unvisited v in vertex order, scan its
 *     in-edges (w->v); at the first w in F, v gets level L+1 and parent w and
 *     joins the next frontier; the scan of v stops there.
 * The direction of level L (the one expanding frontier L into L+1) is
 * dirs[L] if L < ndirs, else dirs[ndirs-1] (0 when ndirs == 0).  dirs_used
 * (nullable, capacity max_levels) receives the direction actually used per
 * level.  Returns the number of levels (depth + 1; 0 if src is invalid).
 */
int or_bfs_levelsync(const or_graph *g, int32_t src, const int8_t *dirs, int ndirs, int32_t *level,
                     int32_t *parent, int8_t *dirs_used, int max_levels) {
    const int64_t n = g->n;
    for (int64_t v = 0; v < n; ++v) {
        level[v] = -1;
        parent[v] = -1;
    }
    if (src < 0 || src >= n) return 0;
    int32_t *F = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *next = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *inF = (uint8_t *)calloc((size_t)n, 1);
    int64_t nf = 0;
    F[nf++] = src;
    level[src] = 0;
    parent[src] = src;
    int L = 0;
    while (nf > 0) {
        const int dir = ndirs == 0 ? 0 : dirs[L < ndirs ? L : ndirs - 1];
        if (dirs_used && L < max_levels) dirs_used[L] = (int8_t)dir;
        int64_t nn = 0;
        if (dir == 0) {
            for (int64_t i = 0; i < nf; ++i) {
                const int32_t v = F[i];
                for (int64_t j = g->out_off[v]; j < g->out_off[v + 1]; ++j) {
                    const int32_t w = g->out_idx[j];
                    if (level[w] == -1) {
                        level[w] = L + 1;
                        parent[w] = v;
                        next[nn++] = w;
                    }
                }
            }
        } else {
            for (int64_t i = 0; i < nf; ++i) inF[F[i]] = 1;
            for (int64_t v = 0; v < n; ++v) {
                if (level[v] != -1) continue;
                for (int64_t j = g->in_off[v]; j < g->in_off[v + 1]; ++j) {
                    const int32_t w = g->in_idx[j];
                    if (inF[w]) {
                        level[v] = L + 1;
                        parent[v] = w;
                        next[nn++] = (int32_t)v;
                        break;
                    }
                }
            }
            for (int64_t i = 0; i < nf; ++i) inF[F[i]] = 0;
        }
        int32_t *t = F;
        F = next;
        next = t;
        nf = nn;
        ++L;
    }
    free(F);
    free(next);
    free(inF);
    return L;
}

/*
 * Adjoint of the PageRank fixed point x = (1-d) s + d P x for the loss
 * L = g^T x (implicit differentiation; not in the paper).
 *   lambda solves (I - d P^T) lambda = g by the Jacobi iteration
 *     lambda_u <- g_u + d sum_{(u->v) in E} P_vu lambda_v
 *   started from lambda = g, until the L1 change is below tol or `iters`.
 *   grad_s[v] = (1-d) lambda_v;  grad_w[e] = d lambda_v x_u for edge e = (u->v),
 *   in input edge order.  x is the fixed point the gradient is taken at.
 * Returns the number of iterations done.
 */
int or_pagerank_adjoint(const or_graph *g, double d, const double *x, const double *gv, int iters,
                        double tol, double *lambda, double *grad_s, double *grad_w, double *residual,
                        int nthreads) {
    const int64_t n = g->n;
    or_set_threads(nthreads);
    double *lam = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *nxt = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t v = 0; v < n; ++v) lam[v] = gv[v];
    int k = 0;
    double r = 0.0;
    while (k < iters) {
        /* each nxt[u] is one in-order sum, so the thread count does not change the result */
#pragma omp parallel for schedule(dynamic, 1024) if (nthreads > 1)
        for (int64_t u = 0; u < n; ++u) {
            double acc = 0.0;
            for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j)
                acc += or_P(g, g->out_eid[j], (int32_t)u) * lam[g->out_idx[j]];
            nxt[u] = gv[u] + d * acc;
        }
        r = 0.0;
        for (int64_t v = 0; v < n; ++v) r += fabs(nxt[v] - lam[v]);
        double *t = lam;
        lam = nxt;
        nxt = t;
        ++k;
        if (r < tol) break;
    }
    for (int64_t v = 0; v < n; ++v) {
        lambda[v] = lam[v];
        grad_s[v] = (1.0 - d) * lam[v];
    }
    if (grad_w)
        for (int64_t u = 0; u < n; ++u)
            for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j)
                grad_w[g->out_eid[j]] = d * lam[g->out_idx[j]] * x[u];
    if (residual) *residual = r;
    free(lam);
    free(nxt);
    return k;
}

/*
 * Gradient with respect to RAW edge weights that are normalised inside the
 * function (not in the paper; the weighted form of the Section 3.1 iteration
 * with P_vu = W_uv / S_u, S_u = sum over u's out-edges of W).  The graph's
 * stored weights are read as the raw W here, not as P.  In order:
 *   1. S_u = sum_{(u->k)} W_uk; P_vu = W_uv / S_u per edge (S_u > 0 whenever
 *      u has an out-edge, since weights are positive);
 *   2. x* = the fixed point x = (1-d) s + d P x (Jacobi sweeps from 1/n until
 *      the L1 change is below tol, at most `iters`);
 *   3. lambda solves (I - d P^T) lambda = g (Jacobi from g, same stop rule);
 *   4. dL/dP_vu = d lambda_v x*_u, and through P_ku = W_uk / S_u (every entry
 *      of u's column depends on W_uv through S_u):
 *        dL/dW_uv = sum_k dL/dP_ku dP_ku/dW_uv
 *                 = d x*_u (lambda_v - sum_{(u->k)} P_ku lambda_k) / S_u;
 *      dL/ds_v = (1-d) lambda_v.
 * s is uniform 1/n when NULL.  Outputs x (the fixed point), lambda, grad_s and
 * grad_W (input edge order).  Returns 0 when both iterations reached tol.
 */
int or_pagerank_adjoint_raw(const or_graph *g, double d, const double *s, const double *gv, int iters, double tol,
                            double *x, double *lambda, double *grad_s, double *grad_W) {
    const int64_t n = g->n, m = g->m;
    double *S = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *P = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    double *a = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *b = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    /* step 1 */
    for (int64_t u = 0; u < n; ++u)
        for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j) S[u] += g->w ? g->w[g->out_eid[j]] : 1.0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j)
            P[g->out_eid[j]] = (g->w ? g->w[g->out_eid[j]] : 1.0) / S[u];
    /* step 2: pull sweeps y[v] = (1-d) s[v] + d sum_{(u->v)} P_vu x[u] */
    int ok = 1;
    for (int64_t v = 0; v < n; ++v) a[v] = 1.0 / (double)n;
    int k = 0;
    double r = INFINITY;
    while (k < iters && !(r < tol)) {
        for (int64_t v = 0; v < n; ++v) {
            double acc = 0.0;
            for (int64_t j = g->in_off[v]; j < g->in_off[v + 1]; ++j) acc += P[g->in_eid[j]] * a[g->in_idx[j]];
            b[v] = (1.0 - d) * (s ? s[v] : 1.0 / (double)n) + d * acc;
        }
        r = 0.0;
        for (int64_t v = 0; v < n; ++v) r += fabs(b[v] - a[v]);
        double *t = a;
        a = b;
        b = t;
        ++k;
    }
    if (!(r < tol)) ok = 0;
    memcpy(x, a, (size_t)n * sizeof(double));
    /* step 3: lambda_u = g_u + d sum_{(u->v)} P_vu lambda_v */
    for (int64_t v = 0; v < n; ++v) a[v] = gv[v];
    k = 0;
    r = INFINITY;
    while (k < iters && !(r < tol)) {
        for (int64_t u = 0; u < n; ++u) {
            double acc = 0.0;
            for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j) acc += P[g->out_eid[j]] * a[g->out_idx[j]];
            b[u] = gv[u] + d * acc;
        }
        r = 0.0;
        for (int64_t v = 0; v < n; ++v) r += fabs(b[v] - a[v]);
        double *t = a;
        a = b;
        b = t;
        ++k;
    }
    if (!(r < tol)) ok = 0;
    memcpy(lambda, a, (size_t)n * sizeof(double));
    /* step 4 */
    for (int64_t v = 0; v < n; ++v) grad_s[v] = (1.0 - d) * lambda[v];
    for (int64_t u = 0; u < n; ++u) {
        double mean = 0.0; /* sum_k P_ku lambda_k over u's out-edges */
        for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j) mean += P[g->out_eid[j]] * lambda[g->out_idx[j]];
        for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j)
            grad_W[g->out_eid[j]] = d * x[u] * (lambda[g->out_idx[j]] - mean) / S[u];
    }
    free(S);
    free(P);
    free(a);
    free(b);
    return ok ? 0 : 1;
}

/* ------------------------------------------------------------------ SSSP */

/* Weight of input edge e for shortest paths: the stored weight, 1 unweighted. */
static inline double or_W(const or_graph *g, int64_t e) { return g->w ? g->w[e] : 1.0; }

typedef struct {
    double key;
    int32_t v;
} or_heap_item;

static void or_heap_push(or_heap_item *h, int64_t *len, double key, int32_t v) {
    int64_t i = (*len)++;
    while (i > 0) {
        const int64_t p = (i - 1) / 2;
        if (h[p].key <= key) break;
        h[i] = h[p];
        i = p;
    }
    h[i].key = key;
    h[i].v = v;
}

static or_heap_item or_heap_pop(or_heap_item *h, int64_t *len) {
    const or_heap_item top = h[0];
    const or_heap_item last = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *len) break;
        if (c + 1 < *len && h[c + 1].key < h[c].key) ++c;
        if (last.key <= h[c].key) break;
        h[i] = h[c];
        i = c;
    }
    if (*len > 0) h[i] = last;
    return top;
}

/*
 * Single-source shortest paths, the plain definition: dist[v] = min over paths
 * r -> ... -> v of the sum of their edge weights, +inf where no path exists.
 * Textbook Dijkstra with a binary heap and lazy deletion, FP64.  pred
 * (nullable) receives the predecessor on the shortest path found (pred[r] = r,
 * -1 unreached).  Weights must be >= 0.  Returns the number of vertices reached.
 */
int64_t or_sssp_dijkstra(const or_graph *g, int32_t r, double *dist, int32_t *pred) {
    const int64_t n = g->n;
    for (int64_t v = 0; v < n; ++v) {
        dist[v] = INFINITY;
        if (pred) pred[v] = -1;
    }
    char *done = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    or_heap_item *h = (or_heap_item *)malloc((size_t)(g->m + 1) * sizeof(or_heap_item));
    int64_t len = 0, reached = 0;
    dist[r] = 0.0;
    if (pred) pred[r] = r;
    or_heap_push(h, &len, 0.0, r);
    while (len > 0) {
        const or_heap_item it = or_heap_pop(h, &len);
        const int32_t u = it.v;
        if (done[u]) continue;
        done[u] = 1;
        ++reached;
        for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j) {
            const int32_t v = g->out_idx[j];
            const double nd = dist[u] + or_W(g, g->out_eid[j]);
            if (nd < dist[v]) {
                dist[v] = nd;
                if (pred) pred[v] = u;
                or_heap_push(h, &len, nd, v);
            }
        }
    }
    free(h);
    free(done);
    return reached;
}

static inline int64_t or_bucket(double d, double delta) { return (int64_t)floor(d / delta); }

/*
 * Delta-Stepping (the paper's push- and pull-based listing), sequential.  Epoch
 * b handles bucket b = the vertices with dist in [b*delta, (b+1)*delta): its
 * relaxation iterations repeat until no vertex of bucket b changed.  Active
 * vertices: every vertex of bucket b in the epoch's first iteration, then the
 * vertices of bucket b whose distance decreased in the previous iteration.
 * Relaxation iteration i of the whole run uses dirs[min(i, ndirs-1)]:
 *   0 push: each active v relaxes its out-edges v->w (dist[w] = min(dist[w],
 *           dist[v] + W));
 *   1 pull: each vertex v not settled in an earlier bucket (dist[v] >=
 *           b*delta, +inf included) takes the minimum of dist[u] + W over its
 *           in-edges u->v from active u.
 * The next epoch is the smallest non-empty bucket above b.  Returns the number
 * of relaxation iterations; *epochs receives the number of epochs.
 */
int64_t or_sssp_delta(const or_graph *g, int32_t r, double delta, const int8_t *dirs, int ndirs, double *dist,
                      int64_t *epochs) {
    const int64_t n = g->n;
    char *act = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    char *nxt = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
    dist[r] = 0.0;
    int64_t b = 0, it = 0, ep = 0;
    for (;;) {
        /* epoch b: every vertex of bucket b is active */
        int64_t nact = 0;
        for (int64_t v = 0; v < n; ++v) {
            act[v] = isfinite(dist[v]) && or_bucket(dist[v], delta) == b;
            nact += act[v];
        }
        ++ep;
        while (nact > 0) {
            const int dir = dirs[it < ndirs ? it : ndirs - 1];
            memset(nxt, 0, (size_t)n);
            if (dir == 0) {
                for (int64_t v = 0; v < n; ++v) {
                    if (!act[v]) continue;
                    for (int64_t j = g->out_off[v]; j < g->out_off[v + 1]; ++j) {
                        const int32_t w = g->out_idx[j];
                        const double nd = dist[v] + or_W(g, g->out_eid[j]);
                        if (nd < dist[w]) {
                            dist[w] = nd;
                            if (or_bucket(nd, delta) == b) nxt[w] = 1;
                        }
                    }
                }
            } else {
                for (int64_t v = 0; v < n; ++v) {
                    if (!(dist[v] >= (double)b * delta)) continue; /* settled in an earlier bucket */
                    double best = dist[v];
                    for (int64_t j = g->in_off[v]; j < g->in_off[v + 1]; ++j) {
                        const int32_t u = g->in_idx[j];
                        if (!act[u]) continue;
                        const double nd = dist[u] + or_W(g, g->in_eid[j]);
                        if (nd < best) best = nd;
                    }
                    if (best < dist[v]) {
                        dist[v] = best;
                        if (or_bucket(best, delta) == b) nxt[v] = 1;
                    }
                }
            }
            ++it;
            char *t = act;
            act = nxt;
            nxt = t;
            nact = 0;
            for (int64_t v = 0; v < n; ++v) nact += act[v];
        }
        /* the next non-empty bucket */
        int64_t nb = -1;
        for (int64_t v = 0; v < n; ++v) {
            if (!isfinite(dist[v])) continue;
            const int64_t bv = or_bucket(dist[v], delta);
            if (bv > b && (nb < 0 || bv < nb)) nb = bv;
        }
        if (nb < 0) break;
        b = nb;
    }
    free(act);
    free(nxt);
    if (epochs) *epochs = ep;
    return it;
}

/* ------------------------------------------------------------------ Frontier-Exploit PageRank */

/*
 * PageRank by propagating pending changes (residuals) from a frontier only.
 * State: ranks x and residuals r, starting at x = s (1/n when s is NULL: the
 * usual start of the iteration) and r = (1-d) s + d P x - x, the change one
 * PageRank sweep would make.  Iteration k: the frontier is F = {u : |r_u| >
 * eps}; every u in F moves its residual into its rank (x_u += r_u) and sends
 * d * P_vu * r_u to each out-neighbour v, all from the residuals at the
 * iteration's start (Jacobi):
 *     r'_v = [v not in F] r_v + d * sum_{u in F, (u->v)} P_vu r_u.
 * x + (I - dP)^-1 r stays equal to the fixed point x* (it does at the start),
 * so on termination (F empty, every |r_u| <= eps) ||x - x*||_1 <= ||r||_1 /
 * (1 - d ||P||_1).  Iteration i uses dirs[min(i, ndirs-1)] (0 push: F's
 * vertices scatter over out-edges; 1 pull: every v gathers over in-edges from
 * F) -- the same sums in another order.  With eps < 0 every vertex stays in F:
 * k iterations give the iterate of k Jacobi sweeps from s.  Runs until F
 * is empty or `iters` iterations.  Returns the iterations done; r_out
 * (nullable) receives the final residuals.
 */
int or_pagerank_fe(const or_graph *g, double d, double eps, int iters, const double *s, const int8_t *dirs, int ndirs,
                   double *x, double *r_out) {
    const int64_t n = g->n;
    double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *rn = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    char *act = (char *)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) x[v] = s ? s[v] : 1.0 / (double)n;
    for (int64_t v = 0; v < n; ++v) { /* r = (1-d) s + d P x - x */
        double acc = 0.0;
        for (int64_t j = g->in_off[v]; j < g->in_off[v + 1]; ++j) {
            const int32_t u = g->in_idx[j];
            acc += or_P(g, g->in_eid[j], u) * x[u];
        }
        r[v] = (1.0 - d) * (s ? s[v] : 1.0 / (double)n) + d * acc - x[v];
    }
    int k = 0;
    while (k < iters) {
        int64_t nf = 0;
        for (int64_t v = 0; v < n; ++v) {
            act[v] = eps < 0.0 || fabs(r[v]) > eps;
            nf += act[v];
        }
        if (nf == 0) break;
        for (int64_t v = 0; v < n; ++v) rn[v] = act[v] ? 0.0 : r[v];
        if (dirs[k < ndirs ? k : ndirs - 1] == 0) {
            for (int64_t u = 0; u < n; ++u) {
                if (!act[u]) continue;
                for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j)
                    rn[g->out_idx[j]] += d * or_P(g, g->out_eid[j], (int32_t)u) * r[u];
            }
        } else {
            for (int64_t v = 0; v < n; ++v) {
                double acc = 0.0;
                for (int64_t j = g->in_off[v]; j < g->in_off[v + 1]; ++j) {
                    const int32_t u = g->in_idx[j];
                    if (act[u]) acc += or_P(g, g->in_eid[j], u) * r[u];
                }
                rn[v] += d * acc;
            }
        }
        for (int64_t u = 0; u < n; ++u)
            if (act[u]) x[u] += r[u];
        double *t = r;
        r = rn;
        rn = t;
        ++k;
    }
    if (r_out)
        for (int64_t v = 0; v < n; ++v) r_out[v] = r[v];
    free(r);
    free(rn);
    free(act);
    return k;
}

/* ------------------------------------------------------------------ betweenness centrality */

/*
 * Betweenness centrality over the given sources (Brandes; the BC listing of
 * Section 3): for each source s, a FIFO BFS over out-edges records each
 * vertex's distance and multiplicity sigma (number of shortest paths from s),
 * the multiplicity of v being the sum of its predecessors' (in-neighbours one
 * level closer); then, in order of decreasing distance, each vertex's partial
 * centrality delta[u] = sum over its successors w (out-neighbours one level
 * further) of sigma[u] / sigma[w] * (1 + delta[w]); bc[u] += delta[u] for
 * u != s.  FP64.  bc (n) is overwritten.  Returns 0.
 */
int or_bc(const or_graph *g, const int32_t *sources, int64_t nsrc, double *bc) {
    const int64_t n = g->n;
    int64_t *dist = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    double *sigma = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *delta = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int32_t *order = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int64_t v = 0; v < n; ++v) bc[v] = 0.0;
    for (int64_t k = 0; k < nsrc; ++k) {
        const int32_t src = sources[k];
        for (int64_t v = 0; v < n; ++v) {
            dist[v] = -1;
            sigma[v] = 0.0;
            delta[v] = 0.0;
        }
        dist[src] = 0;
        sigma[src] = 1.0;
        int64_t head = 0, tail = 0;
        order[tail++] = src;
        while (head < tail) { /* order doubles as the FIFO queue: vertices by distance */
            const int32_t u = order[head++];
            for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j) {
                const int32_t w = g->out_idx[j];
                if (dist[w] < 0) {
                    dist[w] = dist[u] + 1;
                    order[tail++] = w;
                }
                if (dist[w] == dist[u] + 1) sigma[w] += sigma[u];
            }
        }
        for (int64_t i = tail - 1; i >= 0; --i) {
            const int32_t u = order[i];
            for (int64_t j = g->out_off[u]; j < g->out_off[u + 1]; ++j) {
                const int32_t w = g->out_idx[j];
                if (dist[w] == dist[u] + 1) delta[u] += sigma[u] / sigma[w] * (1.0 + delta[w]);
            }
            if (u != src) bc[u] += delta[u];
        }
    }
    free(dist);
    free(sigma);
    free(delta);
    free(order);
    return 0;
}

/* ------------------------------------------------------------------ triangle counting */

static int or_cmp_i32(const void *a, const void *b) {
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* adj(a, b): b is an out-neighbour of a (binary search in a's sorted row of `sorted`). */
static int or_adj(const or_graph *g, const int32_t *sorted, int32_t a, int32_t b) {
    int64_t lo = g->out_off[a], hi = g->out_off[a + 1];
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (sorted[mid] < b)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo < g->out_off[a + 1] && sorted[lo] == b;
}

/*
 * Triangle counts of a simple undirected graph given as its symmetric directed
 * version (self-loops skipped): the NodeIterator listing of Section 3, written
 * out.  For every v, every w1 in N(v) and every w2 in N(v) (w1 != w2, both !=
 * v): if adj(w1, w2), variant 1 (pull) adds one to tc[v] and variant 0 (push)
 * adds one to tc[w1].  Every count is halved at the end (each triangle at a
 * vertex is met as (w1, w2) and as (w2, w1)).  The pull variant runs its outer
 * loop on nthreads threads (each tc[v] has one writer, so the counts do not
 * change).  Returns the number of triangles (sum of tc / 3).
 */
int64_t or_triangles(const or_graph *g, int variant, int64_t *tc, int nthreads) {
    const int64_t n = g->n;
    for (int64_t v = 0; v < n; ++v) tc[v] = 0;
    or_set_threads(nthreads);
    /* rows sorted (a copy) so that adj() is a binary search */
    int32_t *sorted = (int32_t *)malloc((size_t)(g->m > 0 ? g->m : 1) * sizeof(int32_t));
    memcpy(sorted, g->out_idx, (size_t)g->m * sizeof(int32_t));
    for (int64_t v = 0; v < n; ++v)
        qsort(sorted + g->out_off[v], (size_t)(g->out_off[v + 1] - g->out_off[v]), sizeof(int32_t), or_cmp_i32);
    if (variant == 1) {
#pragma omp parallel for schedule(dynamic, 64) if (nthreads > 1)
        for (int64_t v = 0; v < n; ++v) {
            int64_t c = 0;
            for (int64_t i = g->out_off[v]; i < g->out_off[v + 1]; ++i) {
                const int32_t w1 = g->out_idx[i];
                if (w1 == v) continue;
                for (int64_t j = g->out_off[v]; j < g->out_off[v + 1]; ++j) {
                    const int32_t w2 = g->out_idx[j];
                    if (w2 == v || w2 == w1) continue;
                    c += or_adj(g, sorted, w1, w2);
                }
            }
            tc[v] = c;
        }
    } else {
        for (int64_t v = 0; v < n; ++v)
            for (int64_t i = g->out_off[v]; i < g->out_off[v + 1]; ++i) {
                const int32_t w1 = g->out_idx[i];
                if (w1 == v) continue;
                for (int64_t j = g->out_off[v]; j < g->out_off[v + 1]; ++j) {
                    const int32_t w2 = g->out_idx[j];
                    if (w2 == v || w2 == w1) continue;
                    tc[w1] += or_adj(g, sorted, w1, w2);
                }
            }
    }
    free(sorted);
    int64_t total = 0;
    for (int64_t v = 0; v < n; ++v) {
        tc[v] /= 2;
        total += tc[v];
    }
    return total / 3;
}

/* Number of OpenMP threads a parallel region gets (1 without OpenMP). */
int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
