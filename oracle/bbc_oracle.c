/*
 * bbc_oracle.c -- plain CPU oracle for balanced-butterfly counting.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library calls this file; only the tests,
 * the smoke check and the benchmark's CPU-baseline leg load it. It shares no code,
 * header or table with the CUDA path.
 *
 * What it computes (Sec. III, Def. 1 and Def. 2 of the paper): a butterfly is a
 * 4-cycle (u, w in U; x, y in V) with all four edges present; it is balanced when it
 * holds an even number of negative edges. The count is organised as in BB2K
 * (Algorithm 1, Sec. IV) using Lemma 1: for an anchor u and every other endpoint w,
 * the wedges u-v-w are split into symmetric ones (both edge signs equal, Def. 8) and
 * asymmetric ones (Def. 9); with p symmetric and n asymmetric wedges the pair {u, w}
 * closes C(p,2) + C(n,2) balanced butterflies and p*n unbalanced ones.
 *
 * Deliberate differences from the GPU path: anchors are always on side U, vertices
 * keep their ORIGINAL ids (no degree relabelling), the orientation is the raw id
 * order of Algorithm 3 (w > u; orient_low selects w < u), counters are dense arrays
 * indexed by original id with a touched list (in place of BB2K's hash buckets), and
 * every sum is taken in unsigned __int128 so that overflow is detected, not wrapped.
 *
 * Per-vertex counts (the paper defines none; this is the reading used throughout):
 * b(x) is the number of balanced butterflies that contain x.
 *   - anchor side: the pair {u, w} adds f(u,w) = C(p,2) + C(n,2) to b(u) and to b(w);
 *   - centre side: a wedge u-v-w of type t lies in (count_t(u,w) - 1) balanced
 *     butterflies together with another same-type wedge of the pair, so it adds
 *     count_t(u,w) - 1 to b(v).
 *
 * Motif counts (bbco_motif), the same wedge grouping with other per-pair sums:
 *   - sign classes (Sec. VII, Table 7): for a pair {u, w} each common neighbour x is
 *     "pp" (both edges +), "nn" (both -) or "a" (the signs differ). A butterfly is two
 *     such centres, and its class is the unordered pair of centre kinds: coherent ++/++,
 *     ++/--, --/--, incoherent +-/+-, mixed ++/+- and +-/--. Per pair these number
 *     C(pp,2), pp*nn, C(nn,2), C(a,2), pp*a and nn*a;
 *   - balanced (2,k)-bicliques (Def. 5, Algorithm 1): k common neighbours of the pair
 *     with no unbalanced butterfly among them are all symmetric or all asymmetric
 *     (Lemma 1), so the pair closes C(p,k) + C(n,k) balanced ones out of C(p+n,k).
 *   Both depend on which side holds the pair; the anchors are side U here.
 *
 * Mutants: building with -DBBCO_MUTANT=k plants one plausible mistake (k = 1..9); the
 * pin tests compile those variants to show that each one fails at least one pin.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifndef BBCO_MUTANT
#define BBCO_MUTANT 0
#endif

typedef unsigned __int128 u128;

enum { BBCO_OK = 0, BBCO_BAD_INPUT = 1, BBCO_NO_MEMORY = 2, BBCO_OVERFLOW = 3 };

/* Adjacency of one side in plain CSR form, built by a counting pass in input order. */
typedef struct {
    int64_t *off;    /* n + 1 */
    int32_t *nbr;    /* n_edges */
    int8_t *sgn;     /* n_edges, +1 or -1 */
} adj_t;

static void adj_free(adj_t *a) {
    free(a->off);
    free(a->nbr);
    free(a->sgn);
}

static int adj_build(int32_t n, int64_t m, const int32_t *from, const int32_t *to,
                     const int8_t *s, adj_t *a) {
    a->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    a->nbr = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    a->sgn = (int8_t *)malloc((size_t)(m > 0 ? m : 1));
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!a->off || !a->nbr || !a->sgn || !fill) {
        free(fill);
        adj_free(a);
        return BBCO_NO_MEMORY;
    }
    for (int64_t e = 0; e < m; ++e) a->off[from[e] + 1]++;
    for (int32_t i = 0; i < n; ++i) a->off[i + 1] += a->off[i];
    for (int64_t e = 0; e < m; ++e) {
        int32_t x = from[e];
        int64_t slot = a->off[x] + fill[x]++;
        a->nbr[slot] = to[e];
        a->sgn[slot] = s[e];
    }
    free(fill);
    return BBCO_OK;
}

static int check_input(int32_t n_u, int32_t n_v, int64_t m, const int32_t *eu,
                       const int32_t *ev, const int8_t *es) {
    if (n_u < 0 || n_v < 0 || m < 0) return BBCO_BAD_INPUT;
    for (int64_t e = 0; e < m; ++e) {
        if (eu[e] < 0 || eu[e] >= n_u || ev[e] < 0 || ev[e] >= n_v) return BBCO_BAD_INPUT;
        if (es[e] != 1 && es[e] != -1) return BBCO_BAD_INPUT;
    }
    return BBCO_OK;
}

/* C(x, 2) written out. */
static inline u128 choose2(uint64_t x) {
#if BBCO_MUTANT == 4
    return (u128)x * x / 2; /* mutant: drops the -1 */
#else
    return x < 2 ? 0 : (u128)x * (x - 1) / 2;
#endif
}

/* Is w an endpoint for anchor u under the chosen orientation (a strict total order)? */
static inline int oriented(int32_t u, int32_t w, int orient_low) {
#if BBCO_MUTANT == 2
    return orient_low ? (w <= u) : (w >= u); /* mutant: lets u pair with itself */
#else
    return orient_low ? (w < u) : (w > u);
#endif
}

static inline int wedge_symmetric(int8_t s1, int8_t s2) {
#if BBCO_MUTANT == 3
    (void)s1;
    return s2 > 0; /* mutant: the anchor's edge sign is ignored */
#else
    return s1 == s2;
#endif
}

typedef struct {
    /* shared, read-only */
    int32_t n_u, n_v;
    const adj_t *au, *av;
    int orient_low;
    /* shared, written with atomics */
    uint64_t *per_u, *per_v;
    int64_t next_anchor;       /* index into the sampled anchors */
    int64_t anchor_offset, anchor_stride, n_anchors;
    /* per-thread results */
    u128 balanced, unbalanced;
    int status;
} job_t;

typedef struct {
    job_t *job;
    u128 balanced, unbalanced;
    uint64_t wedges;           /* oriented wedges visited in the wedge pass */
    int status;
} worker_t;

static void add_u64(uint64_t *p, u128 x) {
    if (p) __atomic_fetch_add(p, (uint64_t)x, __ATOMIC_RELAXED);
}

static void *worker(void *arg) {
    worker_t *wk = (worker_t *)arg;
    job_t *jb = wk->job;
    const adj_t *au = jb->au, *av = jb->av;
    uint64_t *sym = (uint64_t *)calloc((size_t)jb->n_u + 1, sizeof(uint64_t));
    uint64_t *asym = (uint64_t *)calloc((size_t)jb->n_u + 1, sizeof(uint64_t));
    int32_t *touched = (int32_t *)malloc(((size_t)jb->n_u + 1) * sizeof(int32_t));
    if (!sym || !asym || !touched) {
        free(sym);
        free(asym);
        free(touched);
        wk->status = BBCO_NO_MEMORY;
        return NULL;
    }
    for (;;) {
        int64_t i_anchor = __atomic_fetch_add(&jb->next_anchor, 1, __ATOMIC_RELAXED);
        if (i_anchor >= jb->n_anchors) break;
        int64_t u = jb->anchor_offset + i_anchor * jb->anchor_stride;
        int64_t n_touched = 0;
        /* Wedge pass: bucket every oriented wedge u-v-w by its endpoint and type. */
        for (int64_t i = au->off[u]; i < au->off[u + 1]; ++i) {
            int32_t v = au->nbr[i];
            int8_t s1 = au->sgn[i];
            for (int64_t j = av->off[v]; j < av->off[v + 1]; ++j) {
                int32_t w = av->nbr[j];
                if (!oriented((int32_t)u, w, jb->orient_low)) continue;
                wk->wedges++;
                if (sym[w] == 0 && asym[w] == 0) touched[n_touched++] = w;
                if (wedge_symmetric(s1, av->sgn[j]))
                    sym[w]++;
                else
                    asym[w]++;
            }
        }
        /* Pair pass: Lemma 1 per endpoint. */
        u128 anchor_total = 0;
        for (int64_t k = 0; k < n_touched; ++k) {
            int32_t w = touched[k];
#if BBCO_MUTANT == 1
            u128 f = choose2(sym[w]); /* mutant: asymmetric pairs dropped */
#else
            u128 f = choose2(sym[w]) + choose2(asym[w]);
#endif
            wk->balanced += f;
            wk->unbalanced += (u128)sym[w] * asym[w];
            anchor_total += f;
#if BBCO_MUTANT != 6
            add_u64(jb->per_u ? &jb->per_u[w] : NULL, f);
#endif
        }
        add_u64(jb->per_u ? &jb->per_u[u] : NULL, anchor_total);
        /* Centre pass: each wedge lies in (count of its type - 1) balanced butterflies. */
        if (jb->per_v) {
            for (int64_t i = au->off[u]; i < au->off[u + 1]; ++i) {
                int32_t v = au->nbr[i];
                int8_t s1 = au->sgn[i];
                u128 acc = 0;
                for (int64_t j = av->off[v]; j < av->off[v + 1]; ++j) {
                    int32_t w = av->nbr[j];
                    if (!oriented((int32_t)u, w, jb->orient_low)) continue;
                    uint64_t c = wedge_symmetric(s1, av->sgn[j]) ? sym[w] : asym[w];
#if BBCO_MUTANT == 5
                    acc += c; /* mutant: the wedge itself is counted as a partner */
#elif BBCO_MUTANT == 7
                    acc += (wedge_symmetric(s1, av->sgn[j]) ? asym[w] : sym[w]); /* mutant: wrong counter */
#else
                    acc += c - 1;
#endif
                }
                add_u64(&jb->per_v[v], acc);
            }
        }
        for (int64_t k = 0; k < n_touched; ++k) {
            sym[touched[k]] = 0;
            asym[touched[k]] = 0;
        }
    }
    free(sym);
    free(asym);
    free(touched);
    return NULL;
}

/*
 * Counts, over the anchors u = offset, offset + stride, ... of side U, the balanced and
 * unbalanced butterflies closed at those anchors (with stride 1 and offset 0: all
 * butterflies of the graph). The graph is given by its edge list (ids 0-based per side,
 * signs +1 / -1, no duplicate pairs).
 *   per_u (n_u entries) and per_v (n_v entries) may be NULL; when given they are
 *   overwritten with the per-vertex balanced counts (complete only for stride 1).
 *   n_threads <= 1 runs on the calling thread only.
 *   wedges (may be NULL) receives the number of oriented wedges visited.
 * Returns BBCO_OK, BBCO_BAD_INPUT, BBCO_NO_MEMORY or BBCO_OVERFLOW.
 */
int bbco_count_sample(int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *eu,
                      const int32_t *ev, const int8_t *es, int orient_low, int n_threads,
                      int64_t anchor_offset, int64_t anchor_stride, uint64_t *balanced,
                      uint64_t *unbalanced, uint64_t *per_u, uint64_t *per_v, uint64_t *wedges) {
    if (anchor_stride < 1 || anchor_offset < 0) return BBCO_BAD_INPUT;
    int st = check_input(n_u, n_v, n_edges, eu, ev, es);
    if (st) return st;
    adj_t au, av;
    if (adj_build(n_u, n_edges, eu, ev, es, &au)) return BBCO_NO_MEMORY;
    if (adj_build(n_v, n_edges, ev, eu, es, &av)) {
        adj_free(&au);
        return BBCO_NO_MEMORY;
    }
    if (per_u) memset(per_u, 0, sizeof(uint64_t) * (size_t)n_u);
    if (per_v) memset(per_v, 0, sizeof(uint64_t) * (size_t)n_v);
    job_t jb;
    memset(&jb, 0, sizeof(jb));
    jb.n_u = n_u;
    jb.n_v = n_v;
    jb.au = &au;
    jb.av = &av;
    jb.orient_low = orient_low;
    jb.per_u = per_u;
    jb.per_v = per_v;
    jb.anchor_offset = anchor_offset;
    jb.anchor_stride = anchor_stride;
    jb.n_anchors = anchor_offset < n_u ? (n_u - 1 - anchor_offset) / anchor_stride + 1 : 0;
    if (n_threads < 1) n_threads = 1;
    worker_t *wk = (worker_t *)calloc((size_t)n_threads, sizeof(worker_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!wk || !th) {
        free(wk);
        free(th);
        adj_free(&au);
        adj_free(&av);
        return BBCO_NO_MEMORY;
    }
    for (int t = 0; t < n_threads; ++t) wk[t].job = &jb;
    int started = 0;
    if (n_threads == 1) {
        worker(&wk[0]);
    } else {
        for (int t = 0; t < n_threads; ++t) {
            if (pthread_create(&th[t], NULL, worker, &wk[t]) == 0)
                started++;
            else
                break;
        }
        if (started == 0) worker(&wk[0]);
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    u128 b = 0, ub = 0;
    uint64_t visited = 0;
    st = BBCO_OK;
    for (int t = 0; t < n_threads; ++t) {
        b += wk[t].balanced;
        ub += wk[t].unbalanced;
        visited += wk[t].wedges;
        if (wk[t].status) st = wk[t].status;
    }
    free(wk);
    free(th);
    adj_free(&au);
    adj_free(&av);
    if (st) return st;
    if (b > (u128)UINT64_MAX || ub > (u128)UINT64_MAX) return BBCO_OVERFLOW;
    *balanced = (uint64_t)b;
    *unbalanced = (uint64_t)ub;
    if (wedges) *wedges = visited;
    return BBCO_OK;
}

/* The whole graph: every anchor of U. */
int bbco_count(int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *eu, const int32_t *ev,
               const int8_t *es, int orient_low, int n_threads, uint64_t *balanced,
               uint64_t *unbalanced, uint64_t *per_u, uint64_t *per_v) {
    return bbco_count_sample(n_u, n_v, n_edges, eu, ev, es, orient_low, n_threads, 0, 1,
                             balanced, unbalanced, per_u, per_v, NULL);
}

/*
 * b(x) for one vertex, computed on x's own side: the sum over every other vertex y of
 * the same side of C(p_xy,2) + C(n_xy,2), where p_xy / n_xy count the common
 * neighbours reached by a symmetric / asymmetric wedge x-c-y. side 0 = U, 1 = V.
 * This is the per-vertex definition restated through Lemma 1 on x's side, so for a
 * centre-side vertex it is independent of the centre-pass formula used above.
 */
int bbco_vertex(int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *eu, const int32_t *ev,
                const int8_t *es, int side, int32_t x, uint64_t *out) {
    int st = check_input(n_u, n_v, n_edges, eu, ev, es);
    if (st) return st;
    int32_t n_same = side == 0 ? n_u : n_v;
    if (x < 0 || x >= n_same) return BBCO_BAD_INPUT;
    const int32_t *from = side == 0 ? eu : ev;
    const int32_t *to = side == 0 ? ev : eu;
    int32_t n_other = side == 0 ? n_v : n_u;
    adj_t a_same, a_other;
    if (adj_build(n_same, n_edges, from, to, es, &a_same)) return BBCO_NO_MEMORY;
    if (adj_build(n_other, n_edges, to, from, es, &a_other)) {
        adj_free(&a_same);
        return BBCO_NO_MEMORY;
    }
    uint64_t *sym = (uint64_t *)calloc((size_t)n_same + 1, sizeof(uint64_t));
    uint64_t *asym = (uint64_t *)calloc((size_t)n_same + 1, sizeof(uint64_t));
    if (!sym || !asym) {
        free(sym);
        free(asym);
        adj_free(&a_same);
        adj_free(&a_other);
        return BBCO_NO_MEMORY;
    }
    for (int64_t i = a_same.off[x]; i < a_same.off[x + 1]; ++i) {
        int32_t c = a_same.nbr[i];
        for (int64_t j = a_other.off[c]; j < a_other.off[c + 1]; ++j) {
            int32_t y = a_other.nbr[j];
            if (y == x) continue;
            if (a_same.sgn[i] == a_other.sgn[j])
                sym[y]++;
            else
                asym[y]++;
        }
    }
    u128 total = 0;
    for (int32_t y = 0; y < n_same; ++y) total += choose2(sym[y]) + choose2(asym[y]);
    free(sym);
    free(asym);
    adj_free(&a_same);
    adj_free(&a_other);
    if (total > (u128)UINT64_MAX) return BBCO_OVERFLOW;
    *out = (uint64_t)total;
    return BBCO_OK;
}

/* C(m, k) exactly, or UINT64_MAX + 1 (as a u128) once it exceeds 2^64 - 1. Each step
 * multiplies C(m, i) by (m - i) and divides by (i + 1), which is exact. */
static u128 choose_k(uint64_t m, uint32_t k) {
    const u128 too_big = (u128)UINT64_MAX + 1;
    if (k > m) return 0;
    if (k > m - k) k = (uint32_t)(m - k); /* C(m, k) = C(m, m - k): fewer, smaller steps */
    u128 r = 1;
    for (uint32_t i = 0; i < k; ++i) {
#if BBCO_MUTANT == 9
        r = r * (m - i) / (i + 2); /* mutant: divides by one too many */
#else
        r = r * (m - i) / (i + 1);
#endif
        if (r > (u128)UINT64_MAX) return too_big;
    }
    return r;
}

typedef struct {
    const adj_t *au, *av;
    int32_t n_u;
    int kind;
    uint32_t k;
    int t, nt;
    u128 out[6];
    int overflow;
} motif_job_t;

static void *motif_worker(void *arg) {
    motif_job_t *mj = (motif_job_t *)arg;
    const adj_t *au = mj->au, *av = mj->av;
    const int32_t n_u = mj->n_u;
    /* per endpoint w: common neighbours by kind, and a touched list */
    uint64_t *pp = (uint64_t *)calloc((size_t)n_u + 1, sizeof(uint64_t));
    uint64_t *nn = (uint64_t *)calloc((size_t)n_u + 1, sizeof(uint64_t));
    uint64_t *aa = (uint64_t *)calloc((size_t)n_u + 1, sizeof(uint64_t));
    int32_t *touched = (int32_t *)malloc(((size_t)n_u + 1) * sizeof(int32_t));
    if (!pp || !nn || !aa || !touched) {
        free(pp);
        free(nn);
        free(aa);
        free(touched);
        mj->overflow = -1;
        return NULL;
    }
    for (int32_t u = mj->t; u < n_u; u += mj->nt) {
        int32_t n_touched = 0;
        for (int64_t i = au->off[u]; i < au->off[u + 1]; ++i) {
            const int32_t x = au->nbr[i];
            const int8_t su = au->sgn[i];
            for (int64_t j = av->off[x]; j < av->off[x + 1]; ++j) {
                const int32_t w = av->nbr[j];
                if (w <= u) continue; /* each unordered pair once */
                const int8_t sw = av->sgn[j];
                if (pp[w] == 0 && nn[w] == 0 && aa[w] == 0) touched[n_touched++] = w;
#if BBCO_MUTANT == 8
                if (su == sw) /* mutant: both-negative centres counted as pp */
#else
                if (su == sw && su > 0)
#endif
                    pp[w]++;
                else if (su == sw)
                    nn[w]++;
                else
                    aa[w]++;
            }
        }
        for (int32_t q = 0; q < n_touched; ++q) {
            const int32_t w = touched[q];
            const uint64_t a = pp[w], b = nn[w], c = aa[w];
            if (mj->kind == 1) {
                mj->out[0] += choose2(a);
                mj->out[1] += (u128)a * b;
                mj->out[2] += choose2(b);
                mj->out[3] += choose2(c);
                mj->out[4] += (u128)a * c;
                mj->out[5] += (u128)b * c;
            } else {
                const u128 cp = choose_k(a + b, mj->k), cn = choose_k(c, mj->k);
                const u128 call = choose_k(a + b + c, mj->k);
                if (cp > (u128)UINT64_MAX || cn > (u128)UINT64_MAX || call > (u128)UINT64_MAX)
                    mj->overflow = 1;
                else {
                    mj->out[0] += cp + cn;
                    mj->out[1] += call;
                }
            }
            pp[w] = nn[w] = aa[w] = 0;
        }
    }
    free(pp);
    free(nn);
    free(aa);
    free(touched);
    return NULL;
}

/*
 * Motif totals with the pairs on side U (swap the edge arrays for side V).
 * kind 1: the six sign classes, out[0..5] in the order of Table 7.
 * kind 2: out[0] = balanced (2,k)-bicliques, out[1] = all (2,k)-bicliques, k >= 2.
 * Returns BBCO_OVERFLOW when a total (or one pair's binomial) exceeds 2^64 - 1.
 */
int bbco_motif(int32_t n_u, int32_t n_v, int64_t n_edges, const int32_t *eu, const int32_t *ev,
               const int8_t *es, int kind, uint32_t k, int n_threads, uint64_t *out) {
    int st = check_input(n_u, n_v, n_edges, eu, ev, es);
    if (st) return st;
    if ((kind != 1 && kind != 2) || (kind == 2 && k < 2) || !out) return BBCO_BAD_INPUT;
    if (n_threads < 1) n_threads = 1;
    adj_t au, av;
    if (adj_build(n_u, n_edges, eu, ev, es, &au)) return BBCO_NO_MEMORY;
    if (adj_build(n_v, n_edges, ev, eu, es, &av)) {
        adj_free(&au);
        return BBCO_NO_MEMORY;
    }
    motif_job_t *jobs = (motif_job_t *)calloc((size_t)n_threads, sizeof(motif_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        adj_free(&au);
        adj_free(&av);
        return BBCO_NO_MEMORY;
    }
    for (int t = 0; t < n_threads; ++t) {
        jobs[t].au = &au;
        jobs[t].av = &av;
        jobs[t].n_u = n_u;
        jobs[t].kind = kind;
        jobs[t].k = k;
        jobs[t].t = t;
        jobs[t].nt = n_threads;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, motif_worker, &jobs[t]);
    motif_worker(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    u128 tot[6] = {0, 0, 0, 0, 0, 0};
    int overflow = 0, nomem = 0;
    for (int t = 0; t < n_threads; ++t) {
        for (int i = 0; i < 6; ++i) tot[i] += jobs[t].out[i];
        if (jobs[t].overflow > 0) overflow = 1;
        if (jobs[t].overflow < 0) nomem = 1;
    }
    free(jobs);
    free(th);
    adj_free(&au);
    adj_free(&av);
    if (nomem) return BBCO_NO_MEMORY;
    for (int i = 0; i < 6; ++i)
        if (tot[i] > (u128)UINT64_MAX) overflow = 1;
    if (overflow) return BBCO_OVERFLOW;
    for (int i = 0; i < 6; ++i) out[i] = (uint64_t)tot[i];
    return BBCO_OK;
}

int bbco_mutant(void) { return BBCO_MUTANT; }
