/*
 * pspc.h -- C ABI of the GB300 shortest-path-counting (SPC) hub-label
 * library: parallel construction of the 2-hop SPC index of an undirected,
 * unweighted graph, and batched SPC(s,t) queries on it.
 *
 * Paper: "PSPC: Efficient Parallel Shortest Path Counting on Large-Scale
 * Graphs" (Peng, Yu, Wang; arXiv 2212.00977).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Vertices are ids 0..n-1 chosen by the caller. The caller also supplies a
 *   total order as rank[v] in [0,n), a permutation, rank 0 = highest (the
 *   order "w <= v means w ranks higher" of Section "PSPC algorithm
 *   description from the Covering Side").
 * - Label entries are (hub, dist, count, overflow): dist = sd(v,hub) is exact,
 *   count = the number of trough shortest paths between v and hub (hub ranked
 *   above every other vertex on them) modulo 2^64, overflow = 1 iff that
 *   exact number is >= 2^64. Query counts follow the same rule.
 * - Pointers may be host or device memory unless stated otherwise; the
 *   library detects which with cudaPointerGetAttributes and stages host
 *   buffers through device memory inside the call (host <-> device copies
 *   are then part of the call).
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream). Calls return after their work on `stream` has completed.
 * - Every entry point returns an int status (PSPC_OK = 0); no exception or
 *   longjmp crosses this boundary. pspc_strerror() names a status.
 * - Only one GPU is used: the device current on the calling thread when
 *   pspc_build is called; later calls on that index switch to it.
 */
#ifndef PSPC_H
#define PSPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define PSPC_OK 0
#define PSPC_E_INVAL 1   /* malformed graph, rank, pair or argument */
#define PSPC_E_NOMEM 2   /* device or host allocation failed */
#define PSPC_E_CUDA 3    /* a CUDA runtime call or kernel failed */
/* 4 is not used: no kernel of the library waits on another kernel, a flag
 * or a peer, so there is no device-side wait that could time out. */
#define PSPC_E_DIST 5    /* a label distance exceeds the limit (32767 or
                            pspc_opts.max_levels) */

/* Unreachable marker in query and export distances. */
#define PSPC_UNREACHED 0xFFFFu

/* Undirected graph as symmetric CSR over caller vertex ids.
 * row_ptr: int64[n+1], row_ptr[0] = 0, non-decreasing.
 * col:     int32[row_ptr[n]]; the neighbours of v are col[row_ptr[v] ..
 *          row_ptr[v+1]), strictly ascending (so no duplicate arcs), no
 *          self-loop, and every arc u->v has its reverse v->u.
 * 1 <= n < 2^24. Violations make pspc_build return PSPC_E_INVAL. The
 * strictly ascending rows are how the library rejects duplicate arcs (an
 * undirected simple graph, Section "Preliminaries"); the library then
 * relabels the vertices by rank and sorts each row again in rank space. */
typedef struct {
    int64_t n;
    const int64_t* row_ptr;
    const int32_t* col;
} pspc_csr;

/* Build options; pass NULL for defaults. Zero fields take their default. */
typedef struct {
    int32_t cand_capacity;   /* on-chip candidate hash slots per vertex
                                (power of two, 1024..16384; default 4096) */
    int32_t label_capacity;  /* on-chip label hash slots per vertex (power of
                                two, 1024..16384; default 8192). The two
                                tables take 12*cand + max(6*label, 8*cand)
                                bytes of shared memory per CTA; sizes that do
                                not fit the device give PSPC_E_INVAL */
    int64_t arena_entries;   /* initial label arena capacity in entries
                                (default 32 * arcs + 4 * n; grows on demand) */
    int32_t max_levels;      /* distance limit: the build fails with
                                PSPC_E_DIST when some label entry would
                                have a distance above it (default and
                                largest value 32767; distances are stored
                                in 15 bits) */
    int32_t verbose;         /* 1: per-level line on stderr */
    int32_t map_kind;        /* how a level tests membership in L(u):
                                0 = automatic (bitmaps when (d-1) bitmaps
                                of n bits fit on chip, else 3),
                                1 = per-level bitmaps (falls back to 3 when
                                they do not fit), 2 = on-chip hash of the
                                label (labels that do not fit go to device
                                scratch), 3 = binary search in the two
                                level segments that can hold the hub */
    int32_t max_ctas;        /* cap on the CTAs of the build's persistent
                                kernels (0 = fill the GPU) */
    int32_t granular;        /* 1: launch the level kernel with one CTA per
                                vertex instead of persistent CTAs, so that
                                work on a higher-priority stream (a query
                                batch next to a build) gets SMs as soon as
                                any vertex finishes; same results */
    int32_t landmarks;       /* landmark filter of pruning rule 2 (Section
                                "Landmark-Based Filtering"): K landmarks
                                per graph, the highest-ranked vertices
                                (past the first 32 of a single large
                                graph, spread ones: see pspc_landmarks);
                                their exact BFS distances to every vertex
                                (two bytes each) let the prune step drop a
                                candidate h of u at level d at once when
                                sd(u,l) + sd(l,h) < d for some landmark l,
                                and keep it unscanned when
                                |sd(u,l) - sd(l,h)| >= d. 0 = default
                                (K = 128; 64 in pspc_build_batch), -1 =
                                off, 1..128 = K (at most 64 in
                                pspc_build_batch); levels below 16 test at
                                most the first 32. Results do not depend
                                on it */
    int32_t reduce_shell;    /* 1: reduction by 1-shell (Section "Index
                                Size Reduction"): vertices of degree 1 are
                                peeled repeatedly, the index is built on the
                                rest (the core), and a peeled vertex is
                                answered through the core vertex its tree
                                hangs from. pspc_query gives the same
                                answers; pspc_query_async, _noalloc, export,
                                hub_column and landmarks are not available
                                on such an index (PSPC_E_INVAL). pspc_build
                                only */
    int32_t paradigm;        /* 0 = pull (Algorithm PULL, the default);
                                1 = push (Algorithm PUSH): each level, every
                                vertex first sends its entries to the
                                buckets of its neighbours in device memory,
                                then each vertex merges, prunes and appends
                                from its bucket. Same index; the buckets
                                hold a level's pulled entries (12 bytes
                                each), PSPC_E_NOMEM when they do not fit */
    int32_t warp_levels;     /* vertices with fewer than 64 pulled entries
                                run one warp per vertex (no CTA barrier) at
                                levels 2..warp_levels, and in 128-thread
                                CTAs above; 0 = automatic (levels 2 and 3,
                                and up to level 127 while the previous
                                level had under 32 candidates per active
                                vertex), -1 = never. Same results */
} pspc_opts;

/* Per-level counters of the last build (level d = distance d). */
typedef struct {
    int64_t raw_candidates;    /* pulled entries (h, d-1, c) with h above u
                                  (rule 1), including those below u's dense
                                  prefix that the kernel skips unread */
    int64_t unique_candidates; /* distinct (u, h) after count merging */
    int64_t entries;           /* survivors appended as level d */
    int64_t active_vertices;   /* vertices with at least one pulled entry */
    int64_t active_arcs;       /* CSR arcs of those vertices */
    float ms;                  /* device time of the whole level */
    float kernel_ms;           /* device time of the level's gather/merge/
                                  prune/append kernel launches only */
    int64_t landmark_pruned;   /* candidates the landmark filter dropped */
    int64_t landmark_proven;   /* candidates the landmarks proved to survive
                                  (the rest went through the label scan) */
    int64_t offchip_vertices;  /* vertices whose tables did not fit on chip
                                  and ran in device memory */
    float offchip_ms;          /* device time of their kernel launches */
    int64_t routed_vertices;   /* of those, vertices sent there without an
                                  on-chip attempt, their size class having
                                  mostly overflowed the on-chip table */
} pspc_level_stat_t;

typedef struct {
    int64_t n;
    int64_t arcs;        /* directed arcs = 2m */
    int64_t entries;     /* total label entries */
    int32_t levels;      /* number of non-empty levels (max distance + 1) */
    int32_t device;      /* CUDA device ordinal holding the index */
    int64_t index_bytes; /* device bytes held by the finished index */
    int64_t overflow_entries; /* entries whose exact count is >= 2^64 */
    int64_t kernel_launches; /* CUDA kernels launched by pspc_build */
    int64_t query_kernel_launches; /* CUDA kernels launched by all pspc_query
                                      calls on this index so far */
    int32_t graphs;      /* graphs the index was built from (1, or k of a batch) */
    float build_ms;      /* device time of pspc_build, input checks included */
    int32_t landmarks;   /* landmarks per graph used by the build (0: none) */
    float landmark_ms;   /* device time of the landmark BFS within build_ms */
    int64_t shell_vertices; /* vertices peeled by reduce_shell (their labels
                               are not stored; entries counts the core's) */
} pspc_stats_t;

/* One graph of a batch: symmetric CSR as in pspc_csr, plus its order. */
typedef struct {
    int64_t n;
    const int64_t* row_ptr;
    const int32_t* col;
    const int32_t* rank;
} pspc_graph;

typedef struct pspc_index pspc_index;

/*
 * pspc_build -- construct the SPC hub-label index of g under `rank`.
 *
 * Computes, for every vertex v, L(v) = {(w, sd(v,w), tau(v,w))} over w = v
 * and the vertices w ranked above v with tau(v,w) > 0, where tau counts the
 * trough shortest paths (the ESPC construction of Section "PSPC algorithm
 * description from the Covering Side"; by Theorem "L^SPC = L^PSPC" this is
 * the index of the sequential hub-pushing method).
 * Method: level-synchronous pull propagation by distance d (Theorem
 * "Distance Dependency", Lemma "Propagation", Algorithm PULL): each vertex u
 * gathers its neighbours' level-(d-1) entries whose hub ranks above u
 * (pruning rule 1), merges counts per hub (Label Merging), drops hubs for
 * which a query over the labels of distance < d gives a shorter distance
 * (pruning rule 2), and appends the rest as level d. The build stops after
 * the first level with no entry.
 *
 * g, rank:  host or device memory, borrowed for the call only.
 * opts:     NULL or host pointer.
 * out:      host pointer; receives an index owned by the library until
 *           pspc_free. On failure *out is set to NULL.
 * Errors:   PSPC_E_INVAL (bad CSR or rank, n out of range), PSPC_E_NOMEM,
 *           PSPC_E_CUDA, PSPC_E_DIST (distance above 32767 or max_levels).
 */
int pspc_build(const pspc_csr* g, const int32_t* rank, const pspc_opts* opts,
               pspc_index** out, void* stream);

/*
 * pspc_build_batch -- build the indexes of k graphs in one pass: one level
 * loop and one set of kernel launches per level serve all of them (the
 * batched form of pspc_build; the paper builds one graph at a time).
 *
 * The result is ONE index over the disjoint union of the graphs: vertex v
 * of graph g has the id base_g + v, base_g = n_0 + ... + n_{g-1}. Each
 * graph keeps its own order, so the labels of graph g are exactly those
 * pspc_build gives for it alone (hubs as union ids). Queries take union ids;
 * a pair from two different graphs is unreachable. Every graph must satisfy
 * the rules of pspc_csr and rank; sum of n < 2^24.
 * graphs: host array of k descriptors; their arrays may be host or device
 * memory, borrowed for the call. Errors: as pspc_build.
 */
int pspc_build_batch(const pspc_graph* graphs, int32_t k, const pspc_opts* opts, pspc_index** out,
                     void* stream);

/*
 * pspc_query -- answer q SPC(s,t) queries (Eq. (1)-(2)): over the common
 * hubs h of L(s) and L(t), dist = min sd(s,h) + sd(h,t) and count = sum of
 * tau(s,h) * tau(h,t) over the hubs reaching that minimum, modulo 2^64;
 * overflow = 1 iff the exact count is >= 2^64.
 *
 * pairs: int32[q][2] caller vertex ids (s, t), host or device.
 * dist:  uint16[q] out; PSPC_UNREACHED when s and t are not connected.
 * count: uint64[q] out; 0 when unreachable; SPC(s,s) = (0, 1).
 * overflow: uint8[q] out (may be NULL).
 * Outputs are caller-allocated, host or device (all of one kind).
 * q = 0 is a no-op. Errors: PSPC_E_INVAL (NULL index/pointer, q < 0, a
 * vertex id outside [0,n); outputs are then unspecified), PSPC_E_CUDA,
 * PSPC_E_NOMEM.
 */
int pspc_query(const pspc_index* ix, const int32_t* pairs, int64_t q, uint16_t* dist,
               uint64_t* count, uint8_t* overflow, void* stream);

/*
 * pspc_query_async -- pspc_query in stream order, for CUDA-graph capture
 * and pipelines: it enqueues its work on `stream` and returns without
 * waiting, allocates nothing and never synchronises, so a capture of the
 * stream records it. pairs, dist, count, overflow (may be NULL) and err
 * must be device memory of the index's device, and the calling thread's
 * current device must be the index's. *err (device int32) is cleared, then
 * set to 1 if a pair holds a vertex id outside [0,n) (those outputs are
 * unspecified); read it after the stream completes. Same answers as
 * pspc_query. Errors (returned at once): PSPC_E_INVAL, PSPC_E_CUDA.
 */
int pspc_query_async(const pspc_index* ix, const int32_t* pairs, int64_t q, uint16_t* dist,
                     uint64_t* count, uint8_t* overflow, int32_t* err, void* stream);

/*
 * pspc_export -- copy the index to host arrays, by caller vertex id, each
 * label listed by hub rank (highest first), hubs given as caller ids: the
 * layout of the paper's Table "Shortest Path Counting Labels", where each
 * vertex's entries (hub, distance, count) follow the vertex order.
 * off: int64[n+1]; hub: int32[E]; dist: uint16[E]; cnt: uint64[E];
 * ovf: uint8[E] (E = pspc_stats().entries). All host memory owned by the
 * caller. Errors: PSPC_E_INVAL, PSPC_E_NOMEM, PSPC_E_CUDA.
 */
int pspc_export(const pspc_index* ix, int64_t* off, int32_t* hub, uint16_t* dist,
                uint64_t* cnt, uint8_t* ovf);

/*
 * pspc_export_vertices -- the labels of k selected caller vertices, gathered
 * on the device, in the layout of pspc_export: off[k+1] (host) receives the
 * offsets; hub/dist/cnt/ovf (host, off[k] entries) receive the entries, hubs
 * as caller ids in hub-rank order. With hub = NULL only off is filled (to
 * size the buffers). verts: host int32[k]. Errors: PSPC_E_INVAL (vertex out
 * of range, NULL pointers), PSPC_E_NOMEM, PSPC_E_CUDA.
 */
int pspc_export_vertices(const pspc_index* ix, const int32_t* verts, int64_t k, int64_t* off,
                         int32_t* hub, uint16_t* dist, uint64_t* cnt, uint8_t* ovf);

/*
 * pspc_hub_column -- the column of hub w (caller id): for every caller
 * vertex v, the entry of w in L(v) -- dist[v] = sd(v,w), cnt[v] =
 * tau(v,w) mod 2^64, ovf[v] -- or dist[v] = PSPC_UNREACHED, cnt 0, ovf 0
 * when w is not a hub of v. Host arrays of n elements. Errors:
 * PSPC_E_INVAL, PSPC_E_NOMEM, PSPC_E_CUDA.
 */
int pspc_hub_column(const pspc_index* ix, int32_t w, uint16_t* dist, uint64_t* cnt, uint8_t* ovf);

/* pspc_stats -- sizes and timings of an index (host struct): vertices,
 * arcs, label entries (the index size the paper reports in Section
 * "Experiments"), levels (the largest label distance + 1, Theorem "Distance
 * Dependency"), device bytes, kernel launches and device times. */
int pspc_stats(const pspc_index* ix, pspc_stats_t* s);

/* pspc_level_stats -- copy up to `cap` per-level records (level 1 first) to
 * host memory; *levels receives the number of levels built after level 0. */
int pspc_level_stats(const pspc_index* ix, pspc_level_stat_t* out, int32_t cap,
                     int32_t* levels);

/*
 * pspc_set_query_group -- tuning hook for pspc_query: how one pair is
 * merge-joined. 8, 16 or 32 = that many lanes compare 32-bit hub words held
 * in registers; 64, 128 or 256 = one warp stages chunks of that many
 * entries of both labels in shared memory; PSPC_QUERY_BY_SOURCE = pairs
 * sorted by source, L(s) held on chip for every pair of that source and
 * each pair streams only L(t): as a table of every vertex's position in
 * L(s) when 2 bytes per vertex plus 2 per entry of the largest label fit
 * in 224 KB, else as a hash of L(s); PSPC_QUERY_BY_SOURCE_HASH = the hash
 * form even where the table fits. Both apply when the call groups its
 * pairs by source (q >= 4096 and q >= n/4); the hash needs a largest label
 * of at most 12,287 entries. Where the chosen form does not apply, 0
 * applies. 0 = PSPC_QUERY_BY_SOURCE when it applies and q >= 64 n, else
 * chosen from the average label size. Results do not depend on it.
 * Errors: PSPC_E_INVAL.
 */
#define PSPC_QUERY_BY_SOURCE 1
#define PSPC_QUERY_BY_SOURCE_HASH 2
int pspc_set_query_group(pspc_index* ix, int32_t lanes);

/*
 * pspc_query_noalloc -- pspc_query for callers that cannot allocate device
 * memory during a query (for example an engine whose device memory is all
 * owned by another allocator, or a latency-critical serving loop that must
 * never enter the driver's allocator). The paper has no counterpart: this
 * is a deployment variant of pspc_query, with the same answers.
 *
 * It allocates nothing: no cudaMalloc, cudaFree or pool allocation. Its
 * working memory lives in one static device array of
 * PSPC_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU which loads the
 * library holds until the process exits. Like pspc_query, a call groups its
 * pairs by source only when q >= 4096 and q >= n/4; such a call needs, in
 * the array, the error flag (256 bytes), n+2 per-source bins of 8 bytes,
 * the scan's partial sums (8 bytes per 4096 bins, rounded up), and q pair
 * indices of 4 bytes, each part rounded up to 256 bytes. A grouped call
 * that does not fit returns PSPC_E_INVAL: about 4.06M pairs for n = 65,536,
 * and none for n above about 2.09M (the bins alone fill the array). A call
 * that does not group uses only the error flag and has no size limit
 * (q < 2^40). pairs, dist, count and overflow (may be NULL) must be device
 * memory of the index's device; host pointers would need staging buffers
 * and are rejected. The call waits for its stream before it returns. The
 * first call on a device looks up the array's device address; make that
 * first call before any stream capture. Every call shares the array and
 * clears what it counts in; calls that overlap on the GPU (on different
 * streams, or from different threads) race on it and must be serialized by
 * the caller. Errors: PSPC_E_INVAL (as pspc_query, plus the size and
 * pointer rules above), PSPC_E_CUDA.
 */
#define PSPC_NOALLOC_SCRATCH_BYTES (16u << 20)
int pspc_query_noalloc(const pspc_index* ix, const int32_t* pairs, int64_t q, uint16_t* dist,
                       uint64_t* count, uint8_t* overflow, void* stream);

/*
 * pspc_landmarks -- the landmarks and landmark distances the build used for
 * its landmark filter (Section "Landmark-Based Filtering"). Landmarks
 * 0 .. min(k, 32)-1 of a graph are its highest-ranked vertices, the
 * paper's degree threshold under a degree order. For an index of one graph
 * with k > 32 and more than 4k vertices, landmarks 32 .. k-1 are spread
 * over the graph instead (the filter tests them from level 16 on, where
 * they prove most survivors of high-diameter graphs): each in turn is the
 * vertex that maximises the smaller of its distance to landmarks 0..31 and
 * the landmark lower bound max_j |sd(v,l_j) - sd(p,l_j)|, j < 32, of its
 * distance to every spread landmark p before it, ties to the smaller id.
 * k:      host int32 out; the landmarks per graph (0 when the filter was
 *         off).
 * dist:   NULL, or host uint16[n][k] out by caller vertex id:
 *         dist[v*k + j] = sd(v, landmark j of v's graph), or 0xFFFF when
 *         the two are not connected or v's graph has no landmark j.
 * vertex: NULL, or host int32[k] out for an index of one graph: the caller
 *         id of landmark j (-1: none).
 * Errors: PSPC_E_INVAL (NULL index or k, vertex for a batch or 1-shell
 * index), PSPC_E_NOMEM, PSPC_E_CUDA.
 */
int pspc_landmarks(const pspc_index* ix, int32_t* k, uint16_t* dist, int32_t* vertex);

/*
 * pspc_inject_alloc_failure -- fault injection for tests of the library's
 * error paths (the paper has no counterpart). After this call the
 * library's next `after` device allocations succeed and every later one
 * fails, reporting `status`: PSPC_E_NOMEM as if the device were out of
 * memory, or PSPC_E_CUDA as another CUDA error. The call that needed the
 * allocation returns that status, releases what it holds, and leaves
 * *out = NULL for a build. after < 0 removes the limit (the default).
 * Process-wide, for every device; pspc_query_noalloc allocates nothing and
 * is unaffected. Errors: PSPC_E_INVAL (another status).
 */
int pspc_inject_alloc_failure(int64_t after, int32_t status);

/* pspc_free -- release an index and all its device memory; NULL is a no-op. */
void pspc_free(pspc_index* ix);

/* pspc_strerror -- static, human-readable name of a status code. */
const char* pspc_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* PSPC_H */
