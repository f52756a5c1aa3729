// Internal interface between the build orchestration (pspc_build.cu) and
// the per-level kernels (pspc_level.cu): status record, kernel arguments,
// the on-chip table layout and the host-side launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pspc_internal.cuh"

namespace pspc {

constexpr int kLevelThreads = 512;  // CTA of the level kernel for heavy vertices
constexpr int kLightThreads = 128;  // CTA of the level kernel for light vertices
constexpr uint32_t kLightCap = 1024;  // candidate slots of a light vertex
constexpr uint32_t kOffStartCap = 16384;    // first off-chip table size
constexpr uint32_t kOffSlabCap = 1u << 17;  // off-chip slab of the first pass, in candidate slots
constexpr int kMicroThreads = 256;    // the warp-per-vertex level kernel: 8 vertices per CTA
constexpr int kMicroBucket = 6;       // micro: fewer than 2^6 pulled entries (64 fit a warp's registers)
constexpr int kLightBucket = 9;       // light: fewer than 2^9 pulled entries, so at most 2 * 511 < kLightCap
                                      // slots are asked for, and the table never overflows
constexpr int kWarpLevelsMax = 127;   // automatic warp-per-vertex levels: at most this deep,
constexpr int kWarpLevelsFew = 32;    // and while the last level had under this many candidates per vertex
constexpr int kArcChunk = kLevelThreads;  // arcs staged per gather chunk (the CTA size)

// Resident CTAs per SM each kernel size is built for (64 registers a thread).
__host__ __device__ constexpr int level_min_blocks(int nt) { return nt >= 512 ? 2 : 8; }
constexpr int kBuckets = 64;
constexpr size_t kBitmapBudget = 40 * 1024;  // on-chip bytes for the level bitmaps
constexpr int kLmkShallow = 32;    // landmarks the filter tests below level kLmkDeepLevel
constexpr int kLmkDeepLevel = 16;  // from this level on, the filter tests every landmark

struct LevelStatus {
    unsigned long long raw_total;
    unsigned long long unique_total;
    unsigned long long bump;        // arena fill after this level
    unsigned long long need_cap_c;  // largest candidate table of the off-chip class
    unsigned long long need_cap_u;  // largest label table of the off-chip class
    unsigned long long active_arcs;
    int n_active;
    int n_smem;
    int n_global;
    int n_retry;
    unsigned long long prefix_skipped;  // rule-1 entries skipped below the dense prefixes
    unsigned long long lmk_pruned;  // candidates dropped by the landmark filter
    unsigned long long lmk_proven;  // candidates the landmarks proved to survive
    int arena_overflow;
    int work_smem;
    int work_global;
    int work_light;
    int n_giant;     // off-chip vertices whose candidates overflow the slab
    int work_giant;
    int work_micro;
    // on-chip attempts and overflows of vertices that can overflow, by
    // floor(log2 pulled entries): where most overflow, the rest go straight
    // to the off-chip pass
    unsigned int route_att[kBuckets];
    unsigned int route_ovf[kBuckets];
    int bucket_cnt[kBuckets];
    int bucket_base[kBuckets];
    int bucket_fill[kBuckets];
};

struct LevelArgs {
    int d;
    int64_t n;
    const int64_t* rp;
    const int32_t* col;
    const uint32_t* cnt_arc;
    const uint32_t* arc_lo;  // first pulled entry of each arc's segment (dense-prefix skip), or NULL
    const int32_t* hpre;     // dense prefix per vertex when arc_lo is set
    // Push paradigm: the entries sent to u this level lie in
    // push_hub/push_cnt[push_off[rp[u]] .. push_off[rp[u+1]]) (NULL: pull).
    const uint32_t* push_hub;
    const uint64_t* push_cnt;
    const int64_t* push_off;
    const uint64_t* seg;  // [levels][n]
    uint64_t* seg_out;    // row d
    uint32_t* hub_arena;
    uint64_t* cnt_arena;
    unsigned long long arena_cap;
    const int64_t* raw_u;
    const int64_t* lab_size;
    const int32_t* items;
    int n_items;
    int* work;
    LevelStatus* stt;
    int32_t* retry_list;  // appended at retry_list[k]
    int32_t* giant_list;  // off chip: vertices for the final pass with full-size slabs
    uint32_t off_start_cap;  // off chip: first table size (0: the full bound)
    uint32_t cap_c_max;   // candidate table slots (on chip, or per-CTA scratch)
    uint32_t cap_u_max;   // label hash slots (hash map kind)
    uint32_t bm_words;    // words per level bitmap (bitmap map kind)
    const int32_t* comp_base;  // first rank-space id of each vertex's graph in a batch (NULL: 0)
    int granular;              // 1: CTA b handles item b only (grid = n_items); 0: persistent
    uint8_t* gscratch;    // per-CTA table memory when the tables are off chip
    size_t gscratch_stride;
    const uint8_t* lmk;   // [n][lmk_stride] bytes of uint16 landmark distances, or NULL (no filter)
    int lmk_stride;       // bytes per row: a multiple of 16, <= 2 kLmkMax
    int lmk_words;        // 16-byte words of each row the filter tests at this level
};

// Table layout (on chip, or in per-CTA device scratch). The map region also
// holds the survivor sort buffer once the prune step is done.
struct LevelLayout {
    size_t cnt, key, map, list, st, pfx, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline LevelLayout level_layout(uint32_t cap_c, size_t map_bytes, int nt = kLevelThreads) {
    LevelLayout L;
    size_t p = 0;
    L.cnt = p;
    p += (size_t)cap_c * 8;
    L.key = p;
    p = align16(p + (size_t)cap_c * 4);
    L.map = p;
    p = align16(p + (map_bytes > (size_t)cap_c * 8 ? map_bytes : (size_t)cap_c * 8));
    L.list = p;
    p = align16(p + (size_t)cap_c * 4);
    L.st = p;
    p = align16(p + (size_t)nt * 8);
    L.pfx = p;
    p = align16(p + (size_t)(nt + 1) * 8);
    L.total = p;
    return L;
}

__host__ __device__ inline size_t bitmap_bytes(int d, uint32_t bm_words) { return (size_t)(d - 1) * bm_words * 4; }
__host__ __device__ inline size_t hashmap_bytes(uint32_t cap_u) { return (size_t)cap_u * 6; }

__host__ __device__ inline uint32_t cand_cap_for(int64_t raw, int64_t u, uint32_t cap_max) {
    const int64_t bound = raw < u ? raw : u;  // distinct hubs <= pulled entries, and < u
    const uint64_t want = (uint64_t)(2 * bound) < 64ull ? 64ull : (uint64_t)(2 * bound);
    return want >= cap_max ? cap_max : pow2_ceil(want);
}
__host__ __device__ inline uint32_t label_cap_for(int64_t lab) {
    const uint64_t want = (uint64_t)(lab + lab / 3 + 1);
    return pow2_ceil(want < 64ull ? 64ull : want);
}

enum MapKind { kMapBitmap = 0, kMapHash = 1, kMapSeg = 2 };

// Bytes of the label-map region for a map kind (host plan and kernel must
// agree: the kernel carves its tables with exactly this size).
__host__ __device__ inline size_t level_map_bytes(int kind, int d, uint32_t bm_words, uint32_t cap_u) {
    return kind == kMapBitmap ? bitmap_bytes(d, bm_words) : kind == kMapHash ? hashmap_bytes(cap_u) : 0;
}

// Landmark distances (Section "Landmark-Based Filtering"): the first
// min(k, kLmkShallow) landmarks of every graph are its highest-ranked
// vertices (id comp_base + j, or j when comp_base is NULL); for one graph
// (comp_base NULL) with k > kLmkShallow and more than 4k vertices the others
// are spread out over the graph (chosen one by one, each far from the
// landmarks before it). ld is [n][stride] bytes, k uint16 distances per
// row, 0xFFFF where the distance is undefined (unreached, or no such
// landmark). ids (NULL, or host int32[64] out): the id of landmark j, -1 for
// none. Synchronises st every few BFS levels.
int landmark_bfs(int64_t n, const int64_t* rp, const int32_t* col, const int32_t* comp_base, int k, int stride,
                 uint8_t* ld, int32_t* ids, cudaStream_t st, int64_t* launches);

// Push paradigm (Algorithm PUSH): every arc u->v sends u the entries of
// L_{d-1}(v) that the pull would read for it (cnt_arc[a] of them from
// arc_lo[a], or from 0), into u's bucket at push_off[a]. Warp per arc.
cudaError_t launch_push_scatter(int64_t arcs, const int32_t* col, const uint64_t* seg_prev,
                                const uint32_t* hub_arena, const uint64_t* cnt_arena, const uint32_t* cnt_arc,
                                const uint32_t* arc_lo, const int64_t* push_off, uint32_t* push_hub,
                                uint64_t* push_cnt, cudaStream_t st);
cudaError_t launch_arc_counts(int64_t arcs, const uint32_t* cnt_arc, int64_t* out, cudaStream_t st);

// Launchers (pspc_level.cu). Each returns a CUDA error code of the launch.
cudaError_t launch_arc_src(const int64_t* rp, int64_t n, int32_t* arc_src, cudaStream_t st);
// Dense prefix of every vertex (k_dense_prefix): hpre[u] = the smallest rank
// id x >= (first id of u's graph) not in L_<d(u), at most u, looking at the
// first kDensePrefixWindow ids. Every pulled entry whose hub is below it is
// in L_<d(u), so the membership filter would drop it; the cost pass then
// starts each arc's pull after those entries.
constexpr int kDensePrefixWindow = 1024;
constexpr int kDensePrefixMaxLevel = 8;  // deeper levels: no skip (cost grows with d)
constexpr double kDensePrefixMinGain = 0.10;  // stop skipping once it saves less than this share of a level's pulls
cudaError_t launch_dense_prefix(int d, int64_t n, const uint64_t* seg, const uint32_t* hub_arena,
                                const int32_t* comp_base, int32_t* hpre, cudaStream_t st);
// hpre NULL: no skip (arc_lo is not written).
cudaError_t launch_cost(int d, int64_t n, int64_t arcs, const int64_t* rp, const int32_t* col,
                        const int32_t* arc_src, const uint64_t* seg_prev, const uint32_t* hub_arena,
                        const int32_t* hpre, uint32_t* arc_lo, uint32_t* cnt_arc, int64_t* raw_u,
                        int64_t* lab_size, LevelStatus* stt, int64_t label_limit, int32_t* glist, int32_t* items,
                        cudaStream_t st, int64_t* launches);
cudaError_t level_kernel_attrs(int map_kind, size_t smem_bytes, int* occupancy, int nt = kLevelThreads);
cudaError_t launch_level(int map_kind, bool offchip, int grid, size_t smem_bytes, const LevelArgs& A,
                         cudaStream_t st, int nt = kLevelThreads);
// The warp-per-vertex variant for vertices with fewer than 2^kMicroBucket
// pulled entries (k_level_micro).
cudaError_t micro_kernel_occupancy(int* occupancy);
cudaError_t launch_level_micro(int grid, const LevelArgs& A, cudaStream_t st);

}  // namespace pspc
