/*
 * oracle/brandes.c -- plain CPU oracle for exact betweenness centrality.
 *
 * TEST INFRASTRUCTURE. Only the tests, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this file's library. The GPU library
 * shares no code with it.
 *
 * What it computes (Kintali, "Betweenness Centrality: Algorithms and Lower
 * Bounds", Section 1.1):
 *   d(s,t)        shortest-path length under positive integer weights,
 *   lambda_st     number of shortest s-t paths (lambda_ss = 1),
 *   P_s(v)        = { u : (u,v) in E, d(s,v) = d(s,u) + w(u,v) }   (predecessors),
 *   delta_s*(v)   dependency of s on v, by Theorem 1.1 (Brandes' recurrence)
 *                 delta_s*(v) = sum_{w : v in P_s(w)} lambda_sv/lambda_sw (1 + delta_s*(w)),
 *   BC(v)         = sum_{s != v} delta_s*(v)  (ordered pairs; the paper halves
 *                 for undirected graphs, the caller may do so).
 * Brandes' algorithm as Section 1.1 describes it: one SSSP per source (BFS when
 * unweighted, Dijkstra with a binary heap when weighted), then the dependencies
 * in reverse settle order, summed into a running score.
 *
 * Directed graphs: the CSR lists out-arcs; P_s(v) takes v's in-arcs, which
 * the caller passes as a second CSR (the transpose, with its weights). When
 * no transpose is given the graph is taken as undirected (symmetric CSR) and
 * the out-arcs serve as in-arcs too.
 *
 * Precision: distances int64; path counts unsigned 128-bit with a flag when a
 * count exceeds 2^64 (the GPU's uint64 wraps there) and another when it would
 * exceed 2^128 (never on the test graphs); dependencies FP64, the ratio
 * lambda_sv/lambda_sw taken as (double)lambda_sv / (double)lambda_sw.
 * Unreachable vertices contribute nothing.
 *
 * Summary values per source (evidence that a device run computed the same
 * rows, without moving them):
 *   hash_sigma(s) = sum_v (lambda_sv mod 2^64) * (v+1)          mod 2^64,
 *   hash_dist(s)  = sum_{v reachable} (d(s,v) + 1) * (v+1)       mod 2^64,
 *   dist_sum(s)   = sum_{v reachable} d(s,v),  reach(s) = #reachable (incl. s),
 *   arcs(s)       = number of (u,v) arcs with u in P_s(v)  (shortest-path DAG size).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

enum { ORC_OVERFLOW64 = 1, ORC_OVERFLOW128 = 2, ORC_BAD_INPUT = 4, ORC_OOM = 8 };

typedef struct {
    int64_t *dist;
    u128 *sigma;
    double *delta;
    int32_t *order;
    int64_t *heap_d;
    int32_t *heap_v;
    int64_t heap_cap;
} work_t;

static int work_init(work_t *ws, int32_t n, int64_t narcs) {
    memset(ws, 0, sizeof(*ws));
    size_t nn = (size_t)(n > 0 ? n : 1);
    ws->dist = (int64_t *)malloc(nn * sizeof(int64_t));
    ws->sigma = (u128 *)malloc(nn * sizeof(u128));
    ws->delta = (double *)malloc(nn * sizeof(double));
    ws->order = (int32_t *)malloc(nn * sizeof(int32_t));
    ws->heap_cap = narcs + 2;
    ws->heap_d = (int64_t *)malloc((size_t)ws->heap_cap * sizeof(int64_t));
    ws->heap_v = (int32_t *)malloc((size_t)ws->heap_cap * sizeof(int32_t));
    return ws->dist && ws->sigma && ws->delta && ws->order && ws->heap_d && ws->heap_v;
}

static void work_free(work_t *ws) {
    free(ws->dist); free(ws->sigma); free(ws->delta); free(ws->order);
    free(ws->heap_d); free(ws->heap_v);
}

/* binary min-heap on (distance, vertex) with lazy deletion */
static void heap_push(work_t *ws, int64_t *size, int64_t d, int32_t v) {
    int64_t i = (*size)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (ws->heap_d[p] < d || (ws->heap_d[p] == d && ws->heap_v[p] <= v)) break;
        ws->heap_d[i] = ws->heap_d[p];
        ws->heap_v[i] = ws->heap_v[p];
        i = p;
    }
    ws->heap_d[i] = d;
    ws->heap_v[i] = v;
}

static void heap_pop(work_t *ws, int64_t *size, int64_t *d, int32_t *v) {
    *d = ws->heap_d[0];
    *v = ws->heap_v[0];
    int64_t n = --(*size);
    int64_t ld = ws->heap_d[n];
    int32_t lv = ws->heap_v[n];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= n) break;
        if (c + 1 < n && (ws->heap_d[c + 1] < ws->heap_d[c] ||
                          (ws->heap_d[c + 1] == ws->heap_d[c] && ws->heap_v[c + 1] < ws->heap_v[c])))
            c++;
        if (ld < ws->heap_d[c] || (ld == ws->heap_d[c] && lv <= ws->heap_v[c])) break;
        ws->heap_d[i] = ws->heap_d[c];
        ws->heap_v[i] = ws->heap_v[c];
        i = c;
    }
    ws->heap_d[i] = ld;
    ws->heap_v[i] = lv;
}

static inline int64_t arc_w(const int32_t *w, int64_t e) { return w ? (int64_t)w[e] : 1; }

/*
 * Forward pass for one source: distances, settle order, path counts.
 * Distances: BFS (unweighted) or Dijkstra (weighted). Path counts by the
 * predecessor definition, vertices taken in settle order (non-decreasing
 * distance, so every predecessor is final first):
 *   lambda_ss = 1,  lambda_sv = sum_{u in P_s(v)} lambda_su.
 * Returns the number of settled (reachable) vertices; *flags gets overflow bits;
 * *arcs the number of predecessor relations.
 */
static int32_t forward(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                       const int32_t *irp, const int32_t *icol, const int32_t *iw,
                       int32_t s, work_t *ws, int32_t *flags, int64_t *arcs) {
    for (int32_t v = 0; v < n; v++) { ws->dist[v] = -1; ws->sigma[v] = 0; }
    int32_t cnt = 0;
    ws->dist[s] = 0;
    if (!w) {
        int32_t head = 0;
        ws->order[cnt++] = s;
        while (head < cnt) {
            int32_t u = ws->order[head++];
            for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
                int32_t v = col[e];
                if (ws->dist[v] < 0) { ws->dist[v] = ws->dist[u] + 1; ws->order[cnt++] = v; }
            }
        }
    } else {
        int64_t hs = 0;
        char *done = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
        if (!done) { *flags |= ORC_OOM; return 0; }
        heap_push(ws, &hs, 0, s);
        while (hs > 0) {
            int64_t d; int32_t u;
            heap_pop(ws, &hs, &d, &u);
            if (done[u] || d > ws->dist[u]) continue;
            done[u] = 1;
            ws->order[cnt++] = u;
            for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
                int32_t v = col[e];
                int64_t nd = d + w[e];
                if (ws->dist[v] < 0 || nd < ws->dist[v]) {
                    ws->dist[v] = nd;
                    if (hs >= ws->heap_cap) { *flags |= ORC_OOM; free(done); return cnt; }
                    heap_push(ws, &hs, nd, v);
                }
            }
        }
        free(done);
    }
    /* path counts over P_s(v): v's in-arcs (u, v) */
    ws->sigma[s] = 1;
    int64_t a = 0;
    for (int32_t i = 1; i < cnt; i++) {
        int32_t v = ws->order[i];
        u128 acc = 0;
        for (int64_t e = irp[v]; e < irp[v + 1]; e++) {
            int32_t u = icol[e];
            if (ws->dist[u] >= 0 && ws->dist[u] + arc_w(iw, e) == ws->dist[v]) {
                u128 nxt = acc + ws->sigma[u];
                if (nxt < acc) *flags |= ORC_OVERFLOW128;
                acc = nxt;
                a++;
            }
        }
        if (acc >> 64) *flags |= ORC_OVERFLOW64;
        ws->sigma[v] = acc;
    }
    *arcs = a;
    return cnt;
}

/*
 * Backward pass (Theorem 1.1): vertices w in reverse settle order push
 * lambda_sv/lambda_sw * (1 + delta_s*(w)) to each predecessor v in P_s(w)
 * (over w's in-arcs (v, w)).
 */
static void backward(const int32_t *irp, const int32_t *icol, const int32_t *iw,
                     int32_t cnt, work_t *ws) {
    for (int32_t i = 0; i < cnt; i++) ws->delta[ws->order[i]] = 0.0;
    for (int32_t i = cnt - 1; i > 0; i--) {
        int32_t x = ws->order[i];
        double sx = (double)ws->sigma[x];
        double f = 1.0 + ws->delta[x];
        for (int64_t e = irp[x]; e < irp[x + 1]; e++) {
            int32_t v = icol[e];
            if (ws->dist[v] >= 0 && ws->dist[v] + arc_w(iw, e) == ws->dist[x])
                ws->delta[v] += ((double)ws->sigma[v] / sx) * f;
        }
    }
}

static int check_csr(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w) {
    if (n < 0 || !rp || (n > 0 && !col)) return 0;
    if (rp[0] != 0) return 0;
    for (int32_t v = 0; v < n; v++) {
        if (rp[v + 1] < rp[v]) return 0;
        for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
            if (col[e] < 0 || col[e] >= n || col[e] == v) return 0;
            if (w && w[e] <= 0) return 0;
        }
    }
    return 1;
}

/*
 * One source, full rows. irp/icol/iw: the in-arc CSR of a directed graph
 * (NULL: undirected, the out-arcs serve). dist: int64[n] (-1 unreachable); sigma_lo/hi: the
 * 128-bit count split in two uint64 (may be NULL); delta: double[n] (may be
 * NULL; delta[s] = reach-1 by the recurrence, which BC excludes); order:
 * int32[n] settle order (may be NULL). Returns the reachable count, or -1 on
 * bad input / allocation failure.
 */
int oracle_source(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                  const int32_t *irp, const int32_t *icol, const int32_t *iw, int32_t s,
                  int64_t *dist, uint64_t *sigma_lo, uint64_t *sigma_hi, double *delta,
                  int32_t *order, int32_t *flags, int64_t *arcs) {
    *flags = 0;
    if (!irp) { irp = rp; icol = col; iw = w; }
    if (!check_csr(n, rp, col, w) || !check_csr(n, irp, icol, iw) || (w == NULL) != (iw == NULL) ||
        s < 0 || s >= n) { *flags = ORC_BAD_INPUT; return -1; }
    work_t ws;
    if (!work_init(&ws, n, (int64_t)rp[n])) { work_free(&ws); *flags = ORC_OOM; return -1; }
    int64_t a = 0;
    int32_t cnt = forward(n, rp, col, w, irp, icol, iw, s, &ws, flags, &a);
    if (delta) backward(irp, icol, iw, cnt, &ws);
    for (int32_t v = 0; v < n; v++) {
        if (dist) dist[v] = ws.dist[v];
        if (sigma_lo) sigma_lo[v] = (uint64_t)ws.sigma[v];
        if (sigma_hi) sigma_hi[v] = (uint64_t)(ws.sigma[v] >> 64);
        if (delta) delta[v] = (ws.dist[v] >= 0) ? ws.delta[v] : 0.0;
    }
    if (order) for (int32_t i = 0; i < cnt; i++) order[i] = ws.order[i];
    if (arcs) *arcs = a;
    work_free(&ws);
    return cnt;
}

/*
 * Betweenness over a source list (sources == NULL: all n vertices);
 * irp/icol/iw as for oracle_source.
 * bc: double[n], the ordered-pair sum over the listed sources. Per-source
 * outputs (each may be NULL, else length nsrc): hash_sigma, hash_dist,
 * dist_sum, reach, arcs. Sources are split statically over nthreads OpenMP
 * threads (<=0: the runtime default); each thread sums into its own vector and
 * the vectors are added in thread order, so a fixed thread count gives a fixed
 * result. *flags ORs the per-source overflow bits. Returns 0, or -1 on bad
 * input or allocation failure.
 */
int oracle_bc(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
              const int32_t *irp, const int32_t *icol, const int32_t *iw,
              const int32_t *sources, int32_t nsrc, int32_t nthreads, double *bc,
              uint64_t *hash_sigma, uint64_t *hash_dist, int64_t *dist_sum, int64_t *reach,
              int64_t *arcs, int32_t *flags) {
    *flags = 0;
    if (!irp) { irp = rp; icol = col; iw = w; }
    if (!check_csr(n, rp, col, w) || !check_csr(n, irp, icol, iw) || (w == NULL) != (iw == NULL)) {
        *flags = ORC_BAD_INPUT;
        return -1;
    }
    int32_t ns = sources ? nsrc : n;
    if (ns < 0) { *flags = ORC_BAD_INPUT; return -1; }
    if (sources)
        for (int32_t i = 0; i < ns; i++)
            if (sources[i] < 0 || sources[i] >= n) { *flags = ORC_BAD_INPUT; return -1; }
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    if (nt < 1) nt = 1;
    double *part = (double *)calloc((size_t)nt * (size_t)(n > 0 ? n : 1), sizeof(double));
    if (!part) { *flags = ORC_OOM; return -1; }
    int32_t gflags = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt) reduction(| : gflags)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = part + (size_t)tid * (size_t)n;
        work_t ws;
        int ok = work_init(&ws, n, (int64_t)rp[n]);
        if (!ok) gflags |= ORC_OOM;
        /* static contiguous split: thread t takes sources [lo, hi) */
        int64_t lo = (int64_t)ns * tid / nt, hi = (int64_t)ns * (tid + 1) / nt;
        for (int64_t i = lo; ok && i < hi; i++) {
            int32_t s = sources ? sources[i] : (int32_t)i;
            int32_t f = 0;
            int64_t a = 0;
            int32_t cnt = forward(n, rp, col, w, irp, icol, iw, s, &ws, &f, &a);
            backward(irp, icol, iw, cnt, &ws);
            gflags |= f;
            uint64_t hs = 0, hd = 0;
            int64_t ds = 0;
            for (int32_t k = 0; k < cnt; k++) {
                int32_t v = ws.order[k];
                hs += (uint64_t)ws.sigma[v] * (uint64_t)(v + 1);
                hd += (uint64_t)(ws.dist[v] + 1) * (uint64_t)(v + 1);
                ds += ws.dist[v];
                if (v != s) my[v] += ws.delta[v];
            }
            if (hash_sigma) hash_sigma[i] = hs;
            if (hash_dist) hash_dist[i] = hd;
            if (dist_sum) dist_sum[i] = ds;
            if (reach) reach[i] = cnt;
            if (arcs) arcs[i] = a;
        }
        work_free(&ws);
    }
    for (int32_t v = 0; v < n; v++) {
        double acc = 0.0;
        for (int t = 0; t < nt; t++) acc += part[(size_t)t * n + v];
        bc[v] = acc;
    }
    free(part);
    *flags = gflags;
    return (gflags & (ORC_OOM | ORC_BAD_INPUT)) ? -1 : 0;
}
