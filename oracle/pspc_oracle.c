/*
 * CPU oracle for the shortest-path-counting (SPC) 2-hop hub-label index.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do. It shares no code, header or table with the CUDA
 * library.
 *
 * What it computes (Section "PSPC algorithm description from the Covering
 * Side": the ESPC construction by trough shortest paths; Theorem "Trough
 * Path Property"; Theorem "L^SPC = L^PSPC"): for a graph G and a total
 * order (rank 0 = highest), the label of v is
 *     L(v) = { (w, sd(v,w), tau(v,w)) : w = v or w ranks above v, tau > 0 }
 * where tau(v,w) counts the shortest v-w paths on which every vertex other
 * than w ranks below w (tau(v,v) = 1). Entries are listed by hub rank.
 *
 * Labeler: the sequential hub-pushing construction (HP-SPC, Section
 * "Order Property" and Lemma "Order Dependency"): hubs are taken in rank
 * order; each runs a breadth-first search from the hub w over w and the
 * vertices ranked below w. A popped vertex x is pruned when the query over
 * the labels built so far returns a distance q < D[x]; otherwise the entry
 * (w, D[x], C[x]) is appended to L(x) (canonical when q > D[x],
 * non-canonical when q == D[x]) and x expands. C[x] is the breadth-first
 * path count over the non-pruned search, which equals tau(x,w); the
 * paper's "count + c1" wording for non-canonical entries is not used.
 *
 * Query: Eq. (1)-(2): over the common hubs h of L(s) and L(t) take the
 * minimum of sd(s,h) + sd(h,t) and sum tau(s,h) * tau(t,h) over the hubs
 * that reach it.
 *
 * Counts: uint64 arithmetic wraps modulo 2^64, and every count carries a
 * sticky overflow flag that is set iff the exact value is >= 2^64 (all
 * exact counts are >= 1, so a flagged term forces a flagged sum/product).
 * Sum: flag |= carry. Product: flag |= (high 64 bits of the 128-bit
 * product != 0).
 *
 * Conventions: SPC(s,s) = (0, 1); no common hub = (0xFFFF, 0, 0).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_UNREACHED 0xFFFFu
#define ORC_INF_DIST 0x3FFFFFFF

typedef struct {
    int32_t hub;   /* hub as a rank position during the build */
    uint16_t dist;
    uint8_t ovf;
    uint8_t pad;
    uint64_t cnt;
} orc_entry;

typedef struct {
    orc_entry* e;
    int64_t len, cap;
} orc_label;

typedef struct {
    int64_t n;
    int32_t* rank;  /* rank[v] */
    int32_t* order; /* order[r] = v */
    orc_label* L;   /* indexed by vertex id */
    int64_t entries;
    int64_t hubs_done; /* hubs 0..hubs_done-1 (by rank) have been pushed */
    int truncated;
    double seconds;
    int max_dist;
} orc_index;

static int label_push(orc_label* l, int32_t hub, uint16_t dist, uint64_t cnt, uint8_t ovf) {
    if (l->len == l->cap) {
        int64_t nc = l->cap ? l->cap * 2 : 4;
        orc_entry* ne = (orc_entry*)realloc(l->e, (size_t)nc * sizeof(orc_entry));
        if (!ne) return -1;
        l->e = ne;
        l->cap = nc;
    }
    orc_entry* x = &l->e[l->len++];
    x->hub = hub;
    x->dist = dist;
    x->ovf = ovf;
    x->pad = 0;
    x->cnt = cnt;
    return 0;
}

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

void orc_free(orc_index* ix) {
    if (!ix) return;
    if (ix->L) {
        for (int64_t v = 0; v < ix->n; ++v) free(ix->L[v].e);
        free(ix->L);
    }
    free(ix->rank);
    free(ix->order);
    free(ix);
}

/*
 * Build the index with hub pushing in rank order. max_hubs < 0 pushes every
 * hub; otherwise only the max_hubs highest-ranked hubs are pushed, which
 * yields exactly the restriction of the full index to those hubs (the
 * labels of a hub never depend on lower-ranked hubs). time_cap_s > 0 stops
 * after the hub during which the cap is passed (truncated = 1).
 * Returns NULL on allocation failure or if a distance exceeds 32767.
 */
orc_index* orc_build(int64_t n, const int64_t* row_ptr, const int32_t* col,
                     const int32_t* rank, int64_t max_hubs, double time_cap_s) {
    double t0 = now_s();
    orc_index* ix = (orc_index*)calloc(1, sizeof(orc_index));
    if (!ix) return NULL;
    ix->n = n;
    ix->rank = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    ix->order = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    ix->L = (orc_label*)calloc((size_t)(n ? n : 1), sizeof(orc_label));
    int32_t* D = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint64_t* C = (uint64_t*)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    uint8_t* F = (uint8_t*)malloc((size_t)(n ? n : 1));
    int32_t* T = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t)); /* dist of hub r in L(w) */
    int32_t* queue = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int ok = ix->rank && ix->order && ix->L && D && C && F && T && queue;
    if (ok) {
        memcpy(ix->rank, rank, (size_t)n * sizeof(int32_t));
        for (int64_t v = 0; v < n; ++v) ix->order[rank[v]] = (int32_t)v;
        for (int64_t v = 0; v < n; ++v) {
            D[v] = ORC_INF_DIST;
            T[v] = ORC_INF_DIST;
        }
    }
    int64_t hubs = (max_hubs < 0 || max_hubs > n) ? n : max_hubs;
    for (int64_t r = 0; ok && r < hubs; ++r) {
        int32_t w = ix->order[r];
        /* dense view of the current L(w), indexed by hub rank */
        orc_label* Lw = &ix->L[w];
        for (int64_t i = 0; i < Lw->len; ++i) T[Lw->e[i].hub] = Lw->e[i].dist;
        int64_t qh = 0, qt = 0;
        queue[qt++] = w;
        D[w] = 0;
        C[w] = 1;
        F[w] = 0;
        while (qh < qt) {
            int32_t x = queue[qh++];
            int32_t dx = D[x];
            /* query over the labels built so far: any common hub h with
             * dist(w,h) + dist(x,h) < D[x] prunes x */
            orc_label* Lx = &ix->L[x];
            int pruned = 0;
            for (int64_t i = 0; i < Lx->len; ++i) {
                int32_t th = T[Lx->e[i].hub];
                if (th != ORC_INF_DIST && th + (int32_t)Lx->e[i].dist < dx) {
                    pruned = 1;
                    break;
                }
            }
            if (pruned) continue;
            if (dx > 32767) {
                ok = 0;
                break;
            }
            if (label_push(Lx, (int32_t)r, (uint16_t)dx, C[x], F[x])) {
                ok = 0;
                break;
            }
            ix->entries++;
            if (dx > ix->max_dist) ix->max_dist = dx;
            for (int64_t a = row_ptr[x]; a < row_ptr[x + 1]; ++a) {
                int32_t y = col[a];
                if (rank[y] <= r) continue; /* only w and vertices ranked below w */
                if (D[y] == ORC_INF_DIST) {
                    D[y] = dx + 1;
                    C[y] = C[x];
                    F[y] = F[x];
                    queue[qt++] = y;
                } else if (D[y] == dx + 1) {
                    uint64_t s = C[y] + C[x];
                    F[y] |= (uint8_t)(F[x] | (s < C[x]));
                    C[y] = s;
                }
            }
        }
        for (int64_t i = 0; i < qt; ++i) D[queue[i]] = ORC_INF_DIST;
        for (int64_t i = 0; i < Lw->len; ++i) T[Lw->e[i].hub] = ORC_INF_DIST;
        ix->hubs_done = r + 1;
        if (time_cap_s > 0 && now_s() - t0 > time_cap_s && r + 1 < hubs) {
            ix->truncated = 1;
            break;
        }
    }
    free(D);
    free(C);
    free(F);
    free(T);
    free(queue);
    if (!ok) {
        orc_free(ix);
        return NULL;
    }
    ix->seconds = now_s() - t0;
    return ix;
}

int64_t orc_entries(const orc_index* ix) { return ix->entries; }
int64_t orc_hubs_done(const orc_index* ix) { return ix->hubs_done; }
int orc_truncated(const orc_index* ix) { return ix->truncated; }
double orc_seconds(const orc_index* ix) { return ix->seconds; }
int orc_max_dist(const orc_index* ix) { return ix->max_dist; }

/* Export in caller vertex ids: off[n+1], then per vertex its entries by hub
 * rank, with hubs written as caller vertex ids. */
void orc_export(const orc_index* ix, int64_t* off, int32_t* hub, uint16_t* dist,
                uint64_t* cnt, uint8_t* ovf) {
    int64_t p = 0;
    for (int64_t v = 0; v < ix->n; ++v) {
        off[v] = p;
        const orc_label* l = &ix->L[v];
        for (int64_t i = 0; i < l->len; ++i, ++p) {
            hub[p] = ix->order[l->e[i].hub];
            dist[p] = l->e[i].dist;
            cnt[p] = l->e[i].cnt;
            ovf[p] = l->e[i].ovf;
        }
    }
    off[ix->n] = p;
}

/* Eq. (1)-(2) on one pair of labels (vertex ids). */
static void orc_query_one(const orc_index* ix, int32_t s, int32_t t, uint16_t* od,
                          uint64_t* oc, uint8_t* of) {
    if (s == t) {
        *od = 0;
        *oc = 1;
        *of = 0;
        return;
    }
    const orc_label* a = &ix->L[s];
    const orc_label* b = &ix->L[t];
    int64_t i = 0, j = 0;
    int32_t best = ORC_INF_DIST;
    uint64_t sum = 0;
    uint8_t flag = 0;
    while (i < a->len && j < b->len) {
        int32_t ha = a->e[i].hub, hb = b->e[j].hub;
        if (ha < hb) {
            ++i;
        } else if (hb < ha) {
            ++j;
        } else {
            int32_t d = (int32_t)a->e[i].dist + (int32_t)b->e[j].dist;
            unsigned __int128 pr = (unsigned __int128)a->e[i].cnt * b->e[j].cnt;
            uint64_t lo = (uint64_t)pr;
            uint8_t pf = (uint8_t)(a->e[i].ovf | b->e[j].ovf | ((uint64_t)(pr >> 64) != 0));
            if (d < best) {
                best = d;
                sum = lo;
                flag = pf;
            } else if (d == best) {
                uint64_t s2 = sum + lo;
                flag |= (uint8_t)(pf | (s2 < lo));
                sum = s2;
            }
            ++i;
            ++j;
        }
    }
    if (best == ORC_INF_DIST) {
        *od = ORC_UNREACHED;
        *oc = 0;
        *of = 0;
    } else {
        *od = (uint16_t)best;
        *oc = sum;
        *of = flag;
    }
}

/* Answer q pairs given in caller vertex ids (pairs[2i], pairs[2i+1]).
 * Parallel over pairs with OpenMP when compiled with it. Returns the number
 * of threads used. */
int orc_query(const orc_index* ix, const int32_t* pairs, int64_t q, uint16_t* dist,
              uint64_t* cnt, uint8_t* ovf) {
    int threads = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        threads = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1024)
#endif
    for (int64_t k = 0; k < q; ++k)
        orc_query_one(ix, pairs[2 * k], pairs[2 * k + 1], &dist[k], &cnt[k], &ovf[k]);
    return threads;
}

/* Breadth-first shortest-path counting from s: dist[v] (-1 unreachable),
 * cnt[v] mod 2^64, ovf[v] set iff the exact count is >= 2^64. */
void orc_bfs_count(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t s,
                   int32_t* dist, uint64_t* cnt, uint8_t* ovf, int32_t* queue,
                   const int32_t* rank, int32_t rank_floor) {
    /* rank/rank_floor: when rank != NULL only s and vertices with
     * rank[v] > rank_floor are traversed (the subgraph of s and the vertices
     * ranked below it when rank_floor = rank[s]). */
    for (int64_t v = 0; v < n; ++v) {
        dist[v] = -1;
        cnt[v] = 0;
        ovf[v] = 0;
    }
    int64_t qh = 0, qt = 0;
    queue[qt++] = s;
    dist[s] = 0;
    cnt[s] = 1;
    while (qh < qt) {
        int32_t x = queue[qh++];
        for (int64_t a = row_ptr[x]; a < row_ptr[x + 1]; ++a) {
            int32_t y = col[a];
            if (rank && rank[y] <= rank_floor) continue;
            if (dist[y] < 0) {
                dist[y] = dist[x] + 1;
                cnt[y] = cnt[x];
                ovf[y] = ovf[x];
                queue[qt++] = y;
            } else if (dist[y] == dist[x] + 1) {
                uint64_t s2 = cnt[y] + cnt[x];
                ovf[y] |= (uint8_t)(ovf[x] | (s2 < cnt[x]));
                cnt[y] = s2;
            }
        }
    }
}

/*
 * Hub column of w straight from the definition: the entry of hub w in L(v)
 * for every v. A true BFS from w gives sd(v,w); a BFS over w and the
 * vertices ranked below w gives the trough distance and the trough path
 * count. v has an entry (w, sd, tau) iff v is reached in the restricted
 * search at distance sd(v,w). Writes dist 0xFFFF where there is no entry.
 */
int orc_hub_column(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* rank,
                   int32_t w, uint16_t* out_dist, uint64_t* out_cnt, uint8_t* out_ovf) {
    int32_t* d_true = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* d_tr = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    uint64_t* c_true = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    uint8_t* f_true = (uint8_t*)malloc((size_t)n);
    int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!d_true || !d_tr || !c_true || !f_true || !queue) {
        free(d_true); free(d_tr); free(c_true); free(f_true); free(queue);
        return -1;
    }
    orc_bfs_count(n, row_ptr, col, w, d_true, c_true, f_true, queue, NULL, 0);
    orc_bfs_count(n, row_ptr, col, w, d_tr, out_cnt, out_ovf, queue, rank, rank[w]);
    for (int64_t v = 0; v < n; ++v) {
        if (d_tr[v] >= 0 && d_tr[v] == d_true[v]) {
            out_dist[v] = (uint16_t)d_tr[v];
        } else {
            out_dist[v] = ORC_UNREACHED;
            out_cnt[v] = 0;
            out_ovf[v] = 0;
        }
    }
    free(d_true); free(d_tr); free(c_true); free(f_true); free(queue);
    return 0;
}

/*
 * SPC of many pairs straight from the definition: one breadth-first path
 * count per distinct source, answering every pair with that source.
 * Sources run in parallel with OpenMP (each thread with its own search
 * arrays). Same conventions as orc_query: SPC(s,s) = (0,1), unreachable =
 * (0xFFFF, 0, 0). Returns the threads used, or -1 on allocation failure.
 */
int orc_spc_pairs(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* pairs, int64_t q,
                  uint16_t* out_dist, uint64_t* out_cnt, uint8_t* out_ovf) {
    int64_t* first = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t)); /* pairs of source s: bucket s */
    int64_t* by_src = (int64_t*)malloc((size_t)(q ? q : 1) * sizeof(int64_t));
    int32_t* srcs = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!first || !by_src || !srcs) {
        free(first); free(by_src); free(srcs);
        return -1;
    }
    for (int64_t k = 0; k < q; ++k) first[pairs[2 * k] + 1]++;
    int64_t ns = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (first[v + 1]) srcs[ns++] = (int32_t)v;
        first[v + 1] += first[v];
    }
    {
        int64_t* fill = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
        if (!fill) {
            free(first); free(by_src); free(srcs);
            return -1;
        }
        memcpy(fill, first, (size_t)n * sizeof(int64_t));
        for (int64_t k = 0; k < q; ++k) by_src[fill[pairs[2 * k]]++] = k;
        free(fill);
    }
    int threads = 1, failed = 0;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
#ifdef _OPENMP
#pragma omp single
        threads = omp_get_num_threads();
#endif
        int32_t* d = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        uint64_t* c = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
        uint8_t* f = (uint8_t*)malloc((size_t)n);
        int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        if (!d || !c || !f || !queue) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t i = 0; i < ns; ++i) {
            if (!d || !c || !f || !queue) continue;
            const int32_t s = srcs[i];
            orc_bfs_count(n, row_ptr, col, s, d, c, f, queue, NULL, 0);
            for (int64_t j = first[s]; j < first[s + 1]; ++j) {
                const int64_t k = by_src[j];
                const int32_t t = pairs[2 * k + 1];
                if (d[t] < 0) {
                    out_dist[k] = ORC_UNREACHED;
                    out_cnt[k] = 0;
                    out_ovf[k] = 0;
                } else {
                    out_dist[k] = (uint16_t)d[t];
                    out_cnt[k] = c[t];
                    out_ovf[k] = f[t];
                }
            }
        }
        free(d); free(c); free(f); free(queue);
    }
    free(first); free(by_src); free(srcs);
    return failed ? -1 : threads;
}

/*
 * Whole-index check from the definition, parallel over hubs: for every hub
 * w of hubs[0..nh) (caller ids) the column of w is computed as in
 * orc_hub_column (a true and a restricted breadth-first search) and
 * compared with the exported index (off, hub, dist, cnt, ovf: per vertex
 * its entries in strictly increasing hub rank, hubs as caller ids), where
 * the entry of w in L(v) is found by binary search on rank. An entry that
 * the definition gives and the index lacks, or holds with another
 * distance, count or flag, is a mismatch. *entries receives the number of
 * entries the definition gives for these hubs: for all n hubs it must
 * equal the index size, and then, every expected entry having been found
 * at its own position, the index holds nothing else. Returns the number of
 * mismatching (hub, vertex) pairs (the first `max_bad` of them in
 * bad_w/bad_v), or -1 on allocation failure.
 */
int64_t orc_check_columns(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* rank,
                          const int32_t* hubs, int64_t nh, const int64_t* off, const int32_t* hub,
                          const uint16_t* dist, const uint64_t* cnt, const uint8_t* ovf, int64_t* entries,
                          int32_t* bad_w, int32_t* bad_v, int64_t max_bad) {
    int64_t nbad = 0, ent = 0;
    int failed = 0;
#ifdef _OPENMP
#pragma omp parallel reduction(+ : ent)
#endif
    {
        int32_t* dt = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        int32_t* dr = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        uint64_t* ct = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
        uint64_t* cr = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
        uint8_t* ft = (uint8_t*)malloc((size_t)n);
        uint8_t* fr = (uint8_t*)malloc((size_t)n);
        int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        const int ok = dt && dr && ct && cr && ft && fr && queue;
        if (!ok) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t i = 0; i < nh; ++i) {
            if (!ok) continue;
            const int32_t w = hubs[i];
            const int32_t rw = rank[w];
            orc_bfs_count(n, row_ptr, col, w, dt, ct, ft, queue, NULL, 0);
            orc_bfs_count(n, row_ptr, col, w, dr, cr, fr, queue, rank, rw);
            for (int64_t v = 0; v < n; ++v) {
                const int expect = dr[v] >= 0 && dr[v] == dt[v];
                if (!expect) continue;
                /* entry of w in L(v): labels are sorted by hub rank */
                int64_t lo = off[v], hi = off[v + 1];
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (rank[hub[mid]] < rw) lo = mid + 1; else hi = mid;
                }
                const int have = lo < off[v + 1] && hub[lo] == w;
                const int bad = !have || dist[lo] != (uint16_t)dr[v] || cnt[lo] != cr[v] || ovf[lo] != fr[v];
                ent += 1;
                if (bad) {
                    int64_t k;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
                    k = nbad++;
                    if (k < max_bad) {
                        bad_w[k] = w;
                        bad_v[k] = (int32_t)v;
                    }
                }
            }
        }
        free(dt); free(dr); free(ct); free(cr); free(ft); free(fr); free(queue);
    }
    *entries = ent;
    return failed ? -1 : nbad;
}

/*
 * Columns of many hubs at once, as orc_hub_column computes one, in
 * parallel over the hubs: row i of out_dist/out_cnt/out_ovf (n values each)
 * is the column of hubs[i]. Returns the threads used, or -1 on allocation
 * failure.
 */
int orc_hub_columns(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* rank,
                    const int32_t* hubs, int64_t nh, uint16_t* out_dist, uint64_t* out_cnt, uint8_t* out_ovf) {
    int threads = 1, failed = 0;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
#ifdef _OPENMP
#pragma omp single
        threads = omp_get_num_threads();
#endif
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t i = 0; i < nh; ++i) {
            if (orc_hub_column(n, row_ptr, col, rank, hubs[i], out_dist + i * n, out_cnt + i * n, out_ovf + i * n)) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                failed = 1;
            }
        }
    }
    return failed ? -1 : threads;
}
