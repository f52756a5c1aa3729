// One distance level d of the pull construction (Algorithm PULL; Theorem
// "Distance Dependency"; Lemma "Propagation"; pruning rules 1 and 2; Label
// Elimination and Label Merging; cost-function schedule).
//
// k_dense_prefix / k_cost_arcs / k_cost_vertices
//   For every arc u->v: how many entries of L_{d-1}(v) have a hub ranked
//   above u. Level segments are hub-sorted, so rule 1 keeps a prefix, found
//   by binary search. The pull of the arc also skips the entries whose hub
//   lies below u's dense prefix (every rank id up to it is a hub of
//   L_<d(u), so the membership test of step 2 would drop those entries),
//   found by a second binary search. Per vertex the sum is the
//   pulled-entry count (the paper's cost function); active vertices are
//   bucketed by it so that the most expensive ones start first.
//
// k_level  (one CTA per vertex, persistent CTAs taking vertices in bucket
//   order from a work counter, or one CTA per vertex when granular)
//   1. The label map of u: which hubs x are in L_<d(u), and at which
//      distance. Cumulative bitmaps B_j = {x : d_u(x) <= j}, j = 1..d-1,
//      when they fit on chip; otherwise a binary search in u's level
//      segments, with per-level bitmaps over the highest-ranked ids cached
//      on chip; or (on request) an open-addressing hash x -> d_u(x).
//   2. Pull: the arcs of u are staged in chunks, their pulled-entry counts
//      prefix-summed, and the flattened entries split evenly over the
//      warps. An entry (h, d-1, c) whose hub h is already in L_<d(u) is
//      dropped before its count is read: then Query(h, u) <= d_u(h) < d,
//      so rule 2 would prune it (Label Elimination at no cost). The others
//      are merged per hub in an on-chip hash (count += c mod 2^64; the
//      overflow flag takes the entry's flag and the carry: Label Merging).
//   3a. d = 3: rule 2 asks for a common neighbour of u and h ranked above
//      h; the rows of u's higher-ranked neighbours are walked once and the
//      candidates met there are marked.
//   3. Otherwise: landmark filter (Section "Landmark-Based Filtering"),
//      when the build has landmark distances: a candidate h with
//      sd(u,l) + sd(l,h) < d for a landmark l is pruned at once, one with
//      |sd(u,l) - sd(l,h)| >= d survives at once; the others are compacted
//      and go on. Prune (rule 2) for every remaining candidate h. A common
//      hub x of L_<d(u) and L_<d(h) with d_u(x) + d_h(x) < d exists iff
//      some x in L_k(h), 1 <= k <= d-2, has d_u(x) <= d-1-k (the case
//      k = 0, x = h, was handled in step 2; entries of h at distance d-1
//      cannot help because d_u(x) >= 1 for x != u). Groups of lanes take
//      candidates from a shared counter and scan these segments in level
//      order with early exit: 8 lanes level by level when u has many
//      candidates; 16 or 32 lanes over G levels' descriptors read at once,
//      scanned as one list, when it has few (deep levels of high-diameter
//      graphs), so that their lanes stay busy.
//   4. Survivors are put in hub order (the rank of a hub is a popcount over
//      a bitmap of the survivors, or a bitonic sort when that bitmap does
//      not fit) and appended to the label arena as L_d(u); the arena slot
//      comes from one atomic add.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "pspc_level.cuh"

namespace cg = cooperative_groups;

namespace pspc {

constexpr int kProbeUnroll = 4;  // loads in flight per lane in the prune scan
constexpr uint32_t kSegCacheMinWords = 1024;  // narrowest useful level cache (32K ids)
constexpr uint32_t kSegCacheMaxWords = 8192;  // widest (the off-chip tables can be far larger)
constexpr int kGatherUnroll = 4; // loads in flight per lane in the pull
constexpr unsigned kRouteSamples = 64;  // on-chip attempts per size class before routing by their outcome
constexpr uint32_t kPrunedBit = 0x80000000u;  // list entry: candidate pruned by rule 2
constexpr uint32_t kProvenBit = 0x40000000u;  // list entry: survival proven by the landmarks
constexpr uint32_t kSlotMask = 0x3FFFFFFFu;

// ---------------------------------------------------------------------------
// Cost (rule 1 prefix per arc) and classification.

__global__ void k_arc_src(const int64_t* __restrict__ rp, int64_t n, int32_t* __restrict__ arc_src) {
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    for (int64_t a = rp[u] + lane; a < rp[u + 1]; a += 32) arc_src[a] = (int32_t)u;
}

// First index of the hub-sorted segment h[0..len) whose hub is >= x.
__device__ __forceinline__ uint32_t seg_lower_bound(const uint32_t* h, uint32_t len, uint32_t x) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((__ldg(h + mid) & kHubMask) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_cost_arcs(int64_t arcs, const int32_t* __restrict__ arc_src, const int32_t* __restrict__ col,
                            const uint64_t* __restrict__ seg_prev, const uint32_t* __restrict__ hub_arena,
                            const int32_t* __restrict__ hpre, uint32_t* __restrict__ arc_lo,
                            uint32_t* __restrict__ cnt_arc, unsigned long long* __restrict__ raw_u,
                            unsigned long long* __restrict__ skipped) {
    __shared__ unsigned long long s_skip;
    if (threadIdx.x == 0) s_skip = 0;
    __syncthreads();
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < arcs) {
        const uint32_t u = (uint32_t)arc_src[a];
        const uint64_t s = __ldg(seg_prev + col[a]);
        const uint32_t* h = hub_arena + seg_start(s);
        const uint32_t end = seg_lower_bound(h, seg_len(s), u);  // rule 1: hubs ranked above u
        uint32_t lo = 0;
        if (hpre) {
            lo = seg_lower_bound(h, end, (uint32_t)__ldg(hpre + u));
            arc_lo[a] = lo;
            if (lo) atomicAdd(&s_skip, (unsigned long long)lo);
        }
        cnt_arc[a] = end - lo;
        if (end > lo) atomicAdd(raw_u + u, (unsigned long long)(end - lo));
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_skip) atomicAdd(skipped, s_skip);
}

// Warp per vertex: a bitmap of the first kDensePrefixWindow ids of u's
// graph, set for every hub of L_0(u) .. L_{d-1}(u) in that window (the
// segments are hub-sorted, so each lane stops at the window's end); the
// first clear bit is the dense prefix.
constexpr int kPrefixWarps = 8;

__global__ void __launch_bounds__(kPrefixWarps * 32)
    k_dense_prefix(int d, int64_t n, const uint64_t* __restrict__ seg, const uint32_t* __restrict__ hub_arena,
                   const int32_t* __restrict__ comp_base, int32_t* __restrict__ hpre) {
    __shared__ uint32_t bits[kPrefixWarps][kDensePrefixWindow / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t u = (int64_t)blockIdx.x * kPrefixWarps + w;
    if (u >= n) return;  // the whole warp
    const uint32_t cb = comp_base ? (uint32_t)__ldg(comp_base + u) : 0u;
    const uint32_t lim = cb + kDensePrefixWindow;
    bits[w][lane] = 0u;
    __syncwarp();
    for (int l = 0; l < d; ++l) {
        const uint64_t s = __ldg(seg + (int64_t)l * n + u);
        const uint32_t len = seg_len(s);
        const uint32_t* hs = hub_arena + seg_start(s);
        for (uint32_t i = lane; i < len; i += 32) {
            const uint32_t x = __ldg(hs + i) & kHubMask;
            if (x >= lim) break;
            atomicOr(&bits[w][(x - cb) >> 5], 1u << ((x - cb) & 31));
        }
    }
    __syncwarp();
    const uint32_t word = bits[w][lane];
    const unsigned open = __ballot_sync(0xFFFFFFFFu, word != 0xFFFFFFFFu);
    uint32_t H = lim;
    if (open) {
        const int k = __ffs(open) - 1;
        const uint32_t wk = __shfl_sync(0xFFFFFFFFu, word, k);
        H = cb + 32u * k + (uint32_t)(__ffs(~wk) - 1);
    }
    if (lane == 0) hpre[u] = (int32_t)(H < (uint32_t)u ? H : (uint32_t)u);
}

__global__ void k_cost_vertices(int64_t n, const int64_t* __restrict__ rp, const uint64_t* __restrict__ seg_prev,
                                const int64_t* __restrict__ raw_u, int64_t* __restrict__ lab_size, LevelStatus* stt,
                                int64_t label_limit, int32_t* __restrict__ glist) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int64_t ls = lab_size[u] + seg_len(seg_prev[u]);
    lab_size[u] = ls;
    const int64_t raw = raw_u[u];
    if (raw == 0) return;
    atomicAdd(&stt->raw_total, (unsigned long long)raw);
    atomicAdd(&stt->active_arcs, (unsigned long long)(rp[u + 1] - rp[u]));
    atomicAdd(&stt->n_active, 1);
    if (ls <= label_limit) {
        atomicAdd(&stt->n_smem, 1);
        atomicAdd(&stt->bucket_cnt[63 - __clzll((unsigned long long)raw)], 1);
    } else {
        const int p = atomicAdd(&stt->n_global, 1);
        glist[p] = (int32_t)u;
        atomicMax(&stt->need_cap_u, (unsigned long long)label_cap_for(ls));
        atomicMax(&stt->need_cap_c, (unsigned long long)cand_cap_for(raw, u, 1u << 30));
    }
}

__global__ void k_bucket_base(LevelStatus* stt) {
    if (threadIdx.x != 0) return;
    int run = 0;
    for (int b = kBuckets - 1; b >= 0; --b) {  // most expensive vertices first
        stt->bucket_base[b] = run;
        run += stt->bucket_cnt[b];
        stt->bucket_fill[b] = 0;
    }
}

__global__ void k_bucket_fill(int64_t n, const int64_t* __restrict__ raw_u, const int64_t* __restrict__ lab_size,
                              LevelStatus* stt, int64_t label_limit, int32_t* __restrict__ items) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int64_t raw = raw_u[u];
    if (raw == 0 || lab_size[u] > label_limit) return;
    const int b = 63 - __clzll((unsigned long long)raw);
    items[stt->bucket_base[b] + atomicAdd(&stt->bucket_fill[b], 1)] = (int32_t)u;
}

// ---------------------------------------------------------------------------
// Label maps of L_<d(u).

struct BitMap {
    uint32_t* bits;  // (d-1) bitmaps of `words` words; bitmap j-1 = {x : d_u(x) <= j}
    uint32_t words;
    int d;
    uint32_t base;   // first id of u's graph: bits index x - base
    __device__ void clear() const {
        const uint32_t total = (uint32_t)(d - 1) * words;
        for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) bits[i] = 0u;
    }
    __device__ void insert(uint32_t x, int l) const {
        if (l == 0) return;  // u itself is never a candidate or a witness
        x -= base;
        const uint32_t m = 1u << (x & 31);
        for (int j = l; j <= d - 1; ++j) atomicOr(&bits[(uint32_t)(j - 1) * words + (x >> 5)], m);
    }
    __device__ bool within(uint32_t x, int thr) const {  // d_u(x) <= thr, 1 <= thr <= d-1
        x -= base;
        return (bits[(uint32_t)(thr - 1) * words + (x >> 5)] >> (x & 31)) & 1u;
    }
    __device__ bool member(uint32_t x) const { return d > 1 && within(x, d - 1); }
};

struct HashMap {
    uint32_t* keys;
    uint16_t* lvl;
    uint32_t cap;
    __device__ void clear() const {
        for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) keys[i] = kEmpty;
    }
    __device__ void insert(uint32_t x, int l) const {
        uint32_t slot = hash_hub(x) & (cap - 1);
        for (uint32_t probe = 0; probe < cap; ++probe) {
            const uint32_t k = atomicCAS(&keys[slot], kEmpty, x);
            if (k == kEmpty || k == x) {
                lvl[slot] = (uint16_t)l;
                return;
            }
            slot = (slot + 1) & (cap - 1);
        }
    }
    __device__ uint32_t lookup(uint32_t x) const {
        uint32_t slot = hash_hub(x) & (cap - 1);
        for (uint32_t probe = 0; probe < cap; ++probe) {
            const uint32_t k = keys[slot];
            if (k == x) return lvl[slot];
            if (k == kEmpty) return 0xFFFFu;
            slot = (slot + 1) & (cap - 1);
        }
        return 0xFFFFu;
    }
    __device__ bool within(uint32_t x, int thr) const { return lookup(x) <= (uint32_t)thr; }
    __device__ bool member(uint32_t x) const { return lookup(x) != 0xFFFFu; }
};

// No map at all: a pulled hub h can only be in L(u) at distance d-2 or d-1
// (it is at distance d-1 from a neighbour), and a witness x in L_k(h) can
// only be at distance d-2-k or d-1-k from u (triangle inequality with
// sd(u,h) >= d-2). So two binary searches in u's hub-sorted level segments
// answer every test, and nothing is built per vertex.
struct SegMap {
    const uint64_t* seg;
    const uint32_t* hub_arena;
    int64_t n, u;
    int d;
    // Optional on-chip cache: one bitmap per level 1..d-1 over the ids
    // base .. base + 32*cwords - 1 (the highest-ranked hubs, which hold
    // most label entries of power-law graphs); NULL when not built.
    const uint32_t* cache;
    uint32_t cwords;
    uint32_t base;
    __device__ bool in_level(uint32_t x, int l) const {
        if (l < 1) return false;  // level 0 is u itself
        if (cache && x - base < 32u * cwords) {
            const uint32_t r = x - base;
            return (cache[(uint32_t)(l - 1) * cwords + (r >> 5)] >> (r & 31)) & 1u;
        }
        const uint64_t s = __ldg(seg + (int64_t)l * n + u);
        const uint32_t* h = hub_arena + seg_start(s);
        uint32_t lo = 0, hi = seg_len(s);
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if ((__ldg(h + mid) & kHubMask) < x) lo = mid + 1; else hi = mid;
        }
        return lo < seg_len(s) && (__ldg(h + lo) & kHubMask) == x;
    }
    __device__ bool within(uint32_t x, int thr) const { return in_level(x, thr) || in_level(x, thr - 1); }
    __device__ bool member(uint32_t x) const { return in_level(x, d - 1) || in_level(x, d - 2); }
};

// ---------------------------------------------------------------------------
// Block helpers.

__device__ __forceinline__ bool cand_insert(uint32_t* keys, unsigned long long* cnts, uint32_t cap, uint32_t limit,
                                            uint32_t h, uint64_t c, uint32_t ovf, int* nkeys, int* abort_flag) {
    uint32_t slot = hash_hub(h) & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        uint32_t k = ((volatile uint32_t*)keys)[slot];
        if (k == kEmpty) {
            if (*(volatile int*)abort_flag) return false;
            k = atomicCAS(&keys[slot], kEmpty, h);
            if (k == kEmpty) {
                if ((uint32_t)(atomicAdd(nkeys, 1) + 1) > limit) *(volatile int*)abort_flag = 1;
                k = h;
            }
        }
        if ((k & kHubMask) == h) {
            const unsigned long long old = atomicAdd(&cnts[slot], (unsigned long long)c);
            if (ovf | (old + c < old)) atomicOr(&keys[slot], kOvfBit);
            return true;
        }
        slot = (slot + 1) & (cap - 1);
    }
    *(volatile int*)abort_flag = 1;
    return false;
}

__device__ __forceinline__ long long warp_incl_scan64(long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of a[0..n) (n <= blockDim.x) in place; a[n] = total.
__device__ long long block_excl_scan(long long* a, int n, long long* wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const long long v = tid < n ? a[tid] : 0;
    const long long incl = warp_incl_scan64(v);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long t = lane < nw ? wsum[lane] : 0;
        t = warp_incl_scan64(t);
        if (lane < nw) wsum[lane] = t;
    }
    __syncthreads();
    const long long total = wsum[nw - 1];
    if (tid < n) a[tid] = incl - v + (warp ? wsum[warp - 1] : 0);
    if (tid == 0) a[n] = total;
    __syncthreads();
    return total;
}

// Exclusive prefix of popcounts of bits[0..W) into wp[0..W); returns the
// total number of set bits. Each thread owns a contiguous run of words.
__device__ long long block_excl_scan_popc(const uint32_t* bits, uint32_t* wp, uint32_t W, long long* wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const uint32_t per = (W + blockDim.x - 1) / blockDim.x;
    const uint32_t w0 = tid * per, w1 = w0 + per < W ? w0 + per : W;
    long long v = 0;
    for (uint32_t i = w0; i < w1; ++i) v += __popc(bits[i]);
    const long long incl = warp_incl_scan64(v);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long t = lane < nw ? wsum[lane] : 0;
        t = warp_incl_scan64(t);
        if (lane < nw) wsum[lane] = t;
    }
    __syncthreads();
    const long long total = wsum[nw - 1];
    long long run = incl - v + (warp ? wsum[warp - 1] : 0);
    for (uint32_t i = w0; i < w1; ++i) {
        wp[i] = (uint32_t)run;
        run += __popc(bits[i]);
    }
    __syncthreads();
    return total;
}

// Rule 2 over levels klo..khi of L(h) for one candidate h, by one group of
// G lanes. Lane j reads the descriptor of level k0 + j (G at a time); the
// lengths are prefix-summed over the group and the concatenated entries
// scanned in level order, kProbeUnroll loads in flight per lane. The level of
// entry i is the last lane whose exclusive prefix is <= i (a binary search
// by shuffles). An entry x of level k is a witness iff d_u(x) <= d-1-k.
// Returns whether the group found a witness; it also stops (returning
// false) once *stop, shared with other groups scanning other levels of the
// same candidate, is set.
template <int G, class Map>
__device__ bool scan_levels(const Map& mp, const uint64_t* __restrict__ seg, const uint32_t* __restrict__ hub_arena,
                            int64_t n, int d, uint32_t h, int klo, int khi, const int* stop) {
    auto tile = cg::tiled_partition<G>(cg::this_thread_block());
    const int gl = tile.thread_rank();
    bool pruned = false, halt = false;
    for (int k0 = klo; k0 <= khi && !pruned && !halt; k0 += G) {
        const int k = k0 + gl;
        const uint64_t s = k <= khi ? __ldg(seg + (int64_t)k * n + h) : 0ull;
        const uint32_t len = seg_len(s);
        const unsigned long long start = seg_start(s);
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const uint32_t t = tile.shfl_up(incl, o);
            if (gl >= o) incl += t;
        }
        const uint32_t excl = incl - len;
        const uint32_t total = tile.shfl(incl, G - 1);
        for (uint32_t b = 0; b < total && !pruned && !halt; b += G * kProbeUnroll) {
            uint32_t x[kProbeUnroll];
            int thr[kProbeUnroll];
#pragma unroll
            for (int t = 0; t < kProbeUnroll; ++t) {
                const uint32_t i = b + t * G + gl;
                int j = 0;
#pragma unroll
                for (int step = G >> 1; step > 0; step >>= 1) {
                    const uint32_t e = tile.shfl(excl, j + step);
                    if (e <= i) j += step;
                }
                const unsigned long long sj = tile.shfl(start, j);
                const uint32_t ej = tile.shfl(excl, j);
                thr[t] = d - 1 - (k0 + j);
                x[t] = i < total ? (__ldg(hub_arena + sj + (i - ej)) & kHubMask) : kEmpty;
            }
            bool hit = false;
#pragma unroll
            for (int t = 0; t < kProbeUnroll; ++t)
                if (x[t] != kEmpty) hit |= mp.within(x[t], thr[t]);
            pruned = tile.any(hit);
            if (stop) halt = tile.any(*(volatile const int*)stop != 0);
        }
    }
    return pruned;
}

// Rule 2 for the candidates list[0..M): G lanes per candidate h take
// candidates from a shared counter and scan levels 1..d-2 of L(h).
template <int G, class Map>
__device__ void prune_candidates(const Map& mp, const uint64_t* __restrict__ seg,
                                 const uint32_t* __restrict__ hub_arena, int64_t n, int d, uint32_t* list,
                                 const uint32_t* ckeys, int M, int* next) {
    auto tile = cg::tiled_partition<G>(cg::this_thread_block());
    const int gl = tile.thread_rank();
    for (;;) {
        int c = 0;
        if (gl == 0) c = atomicAdd(next, 1);
        c = tile.shfl(c, 0);
        if (c >= M) break;
        const uint32_t slot = list[c];
        if (slot & kProvenBit) continue;
        const uint32_t h = ckeys[slot] & kHubMask;
        const bool pruned = scan_levels<G>(mp, seg, hub_arena, n, d, h, 1, d - 2, nullptr);
        if (pruned && gl == 0) list[c] = slot | kPrunedBit;
    }
}

// Rule 2 when fewer candidates remain to be scanned than the CTA has warps
// (P < NT/32: the deep levels of high-diameter graphs, where each scan is
// long): the warps form P' >= P groups of wpc = (NT/32) / P' warps, group g takes
// the g-th candidate still undecided, and its warps split levels 1..d-2
// into wpc contiguous ranges. A warp that finds a witness sets the group's
// flag, and the others stop at their next step. Every warp reaches the
// barriers (the call is made by the whole CTA).
template <int NT, class Map>
__device__ void prune_split(const Map& mp, const uint64_t* __restrict__ seg, const uint32_t* __restrict__ hub_arena,
                            int64_t n, int d, uint32_t* list, const uint32_t* ckeys, int M, int P, int* s_flag) {
    constexpr int kWarps = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int wpc = 1;
    while (wpc * 2 * P <= kWarps) wpc *= 2;
    const int groups = kWarps / wpc, g = warp / wpc, j = warp % wpc;
    if (tid < kWarps) s_flag[tid] = 0;
    __syncthreads();
    // position in list of the g-th candidate that is not proven
    int c = -1;
    if (g < P) {
        int seen = 0;
        for (int base = 0; base < M && c < 0; base += 32) {
            const int i = base + lane;
            const bool open = i < M && !(list[i] & kProvenBit);
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, open);
            const int cnt = __popc(bal);
            if (seen + cnt > g) {
                unsigned m = bal;
                for (int r = g - seen; r > 0; --r) m &= m - 1;
                c = base + __ffs(m) - 1;
            }
            seen += cnt;
        }
    }
    if (c >= 0) {
        const uint32_t h = ckeys[list[c] & kSlotMask] & kHubMask;
        const int levels = d - 2;
        const int klo = 1 + (int)((int64_t)levels * j / wpc), khi = (int)((int64_t)levels * (j + 1) / wpc);
        if (klo <= khi && scan_levels<32>(mp, seg, hub_arena, n, d, h, klo, khi, &s_flag[g]) && lane == 0)
            atomicExch(&s_flag[g], 1);
    }
    __syncthreads();
    if (c >= 0 && j == 0 && lane == 0 && s_flag[g]) list[c] |= kPrunedBit;
    (void)groups;
}

// Rule 2 level by level: G lanes per candidate scan L_1(h), then L_2(h), ...
// (one descriptor read per level), kProbeUnroll loads in flight per lane.
// A witness x in L_k(h) has sd(h,x) = k, and sd(u,h) >= d-2, so d_u(x) is
// d-2-k or d-1-k: x lies in one of u's two level segments thr-1, thr
// (thr = d-1-k; level 0 is u itself, never in L(h)). When those two are
// much shorter than L_k(h), the group scans them instead and looks each
// entry up in L_k(h) (hub-sorted) by binary search. useg holds u's level
// descriptors for levels 0 .. kUSideLevels-1 (NULL: always scan L_k(h)).
constexpr int kUSideLevels = 16;

__device__ __forceinline__ bool seg_contains(const uint32_t* xs, uint32_t len, uint32_t x) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((__ldg(xs + mid) & kHubMask) < x) lo = mid + 1; else hi = mid;
    }
    return lo < len && (__ldg(xs + lo) & kHubMask) == x;
}

template <int G, class Map>
__device__ void prune_by_level(const Map& mp, const uint64_t* __restrict__ seg,
                               const uint32_t* __restrict__ hub_arena, int64_t n, int d, uint32_t* list,
                               const uint32_t* ckeys, int M, int* next, const uint64_t* useg) {
    auto tile = cg::tiled_partition<G>(cg::this_thread_block());
    const int gl = tile.thread_rank();
    for (;;) {
        int c = 0;
        if (gl == 0) c = atomicAdd(next, 1);
        c = tile.shfl(c, 0);
        if (c >= M) break;
        const uint32_t slot = list[c];
        if (slot & kProvenBit) continue;
        const uint32_t h = ckeys[slot] & kHubMask;
        bool pruned = false;
        for (int k = 1; k <= d - 2 && !pruned; ++k) {
            const uint64_t s = __ldg(seg + (int64_t)k * n + h);
            const uint32_t len = seg_len(s);
            const uint32_t* xs = hub_arena + seg_start(s);
            const int thr = d - 1 - k;
            if (useg && thr < kUSideLevels && len > 0) {
                const uint64_t ua = thr >= 2 ? useg[thr - 1] : 0ull, ub = useg[thr];
                const uint32_t la = seg_len(ua), lb = seg_len(ub);
                const uint32_t steps = 32 - __clz(len);  // binary-search steps in L_k(h)
                if ((uint64_t)(la + lb) * steps < len) {
                    const uint32_t* xa = hub_arena + seg_start(ua);
                    const uint32_t* xb = hub_arena + seg_start(ub);
                    for (uint32_t b = 0; b < la + lb && !pruned; b += G * kProbeUnroll) {
                        bool hit = false;
#pragma unroll
                        for (int t = 0; t < kProbeUnroll; ++t) {
                            const uint32_t i = b + t * G + gl;
                            if (i < la + lb) {
                                const uint32_t x = __ldg(i < la ? xa + i : xb + (i - la)) & kHubMask;
                                hit |= seg_contains(xs, len, x);
                            }
                        }
                        pruned = tile.any(hit);
                    }
                    continue;
                }
            }
            for (uint32_t b = 0; b < len && !pruned; b += G * kProbeUnroll) {
                uint32_t x[kProbeUnroll];
#pragma unroll
                for (int t = 0; t < kProbeUnroll; ++t) {
                    const uint32_t i = b + t * G + gl;
                    x[t] = i < len ? (__ldg(xs + i) & kHubMask) : kEmpty;
                }
                bool hit = false;
#pragma unroll
                for (int t = 0; t < kProbeUnroll; ++t)
                    if (x[t] != kEmpty) hit |= mp.within(x[t], thr);
                pruned = tile.any(hit);
            }
        }
        if (pruned && gl == 0) list[c] = slot | kPrunedBit;
    }
}

// Many candidates: 8 lanes each, level by level (most are pruned within the
// first entries of L_1(h), so reading further descriptors up front only
// costs loads). Few candidates: wider groups over the concatenated levels,
// so that the long scans of deep levels keep all lanes busy.
template <int NT, class Map>
__device__ __forceinline__ void prune_all(const Map& mp, const uint64_t* seg, const uint32_t* hub_arena, int64_t n,
                                          int d, uint32_t* list, const uint32_t* ckeys, int M, int to_scan,
                                          int* next, const uint64_t* useg, int* s_flag) {
    if (to_scan >= 64) prune_by_level<8>(mp, seg, hub_arena, n, d, list, ckeys, M, next, useg);
    else if (to_scan >= NT / 32) prune_candidates<16>(mp, seg, hub_arena, n, d, list, ckeys, M, next);
    else prune_split<NT>(mp, seg, hub_arena, n, d, list, ckeys, M, to_scan, s_flag);
}

// Landmark filter (Section "Landmark-Based Filtering"). For a candidate h
// of u at level d, rule 2 prunes h exactly when sd(u,h) < d. Each landmark
// l bounds sd(u,h) from both sides: sd(u,h) <= sd(u,l) + sd(l,h), and
// sd(u,h) >= |sd(u,l) - sd(l,h)|. An upper bound below d prunes h at once;
// a lower bound of at least d proves that h survives (it keeps its list
// entry, marked kProvenBit, and skips the label scan). Distances are uint16
// (0xFFFF = unknown): the sum is taken with saturation and compared with d
// (at most 32767), so an unknown or saturated sum never prunes, and 0xFFFF
// on either side gives no lower bound. The candidates not pruned are
// compacted to list[0..kept) in the same order (in rounds of one candidate
// per thread: every read of a round precedes its writes, and no write
// reaches past the round's reads). Returns kept; *n_proven receives the
// proven ones among them.
template <int NT>
__device__ int landmark_filter(const LevelArgs& A, const uint32_t* s_lmk, int d, uint32_t* list,
                               const uint32_t* ckeys, int M, int* s_wcnt, int* s_kept, int* n_proven) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t dd = (uint32_t)d * 0x00010001u;  // d <= 32767 in both halfwords
    const int words = A.lmk_words;
    int kept = 0, proven = 0;
    for (int base = 0; base < M; base += NT) {
        const int c = base + tid;
        uint32_t slot = 0;
        bool keep = false, sure = false;
        if (c < M) {
            slot = list[c];
            const uint4* row = (const uint4*)(A.lmk + (size_t)(ckeys[slot] & kHubMask) * A.lmk_stride);
            uint32_t hit = 0, far = 0;
            // two uint16 distances per word; 0xFFFF (undefined) saturates
            // the sum and is masked out of the difference test
#pragma unroll
            for (int w = 0; w < kLmkMax / 8; ++w)
                if (w < words) {
                    const uint4 b4 = __ldg(row + w);
                    const uint32_t bw[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t a = s_lmk[4 * w + q], b = bw[q];
                        hit |= __vcmpltu2(__vaddus2(a, b), dd);
                        const uint32_t known = ~(__vcmpeq2(a, 0xFFFFFFFFu) | __vcmpeq2(b, 0xFFFFFFFFu));
                        far |= __vcmpgeu2(__vabsdiffu2(a, b), dd) & known;
                    }
                }
            keep = hit == 0u;
            sure = keep && far != 0u;
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
        const unsigned bsure = __ballot_sync(0xFFFFFFFFu, sure);
        if (lane == 0) s_wcnt[warp] = __popc(bal) | (__popc(bsure) << 16);
        __syncthreads();
        int before = 0, round = 0, round_sure = 0;
        for (int w = 0; w < NT / 32; ++w) {
            const int v = s_wcnt[w];
            before += w < warp ? (v & 0xFFFF) : 0;
            round += v & 0xFFFF;
            round_sure += v >> 16;
        }
        if (keep) list[kept + before + __popc(bal & ((1u << lane) - 1u))] = slot | (sure ? kProvenBit : 0u);
        kept += round;
        proven += round_sure;
        __syncthreads();
    }
    if (tid == 0) *s_kept = kept;
    *n_proven = proven;
    return kept;
}

__device__ void block_bitonic_sort(unsigned long long* buf, uint32_t P) {
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = buf[i], b = buf[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        buf[i] = b;
                        buf[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// The level kernel.

template <int kMap, bool kOffChip, int NT>
__global__ void __launch_bounds__(NT, level_min_blocks(NT)) k_level(const LevelArgs A) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_item, s_nkeys, s_abort, s_m, s_next, s_nsurv, s_kept, s_route;
    __shared__ uint32_t s_lmk[kLmkMax / 2];  // u's landmark distances (uint16 pairs)
    __shared__ uint64_t s_useg[kUSideLevels];  // u's level descriptors for the rule-2 scan
    __shared__ int s_wcnt[NT / 32];
    __shared__ unsigned long long s_base;
    __shared__ long long s_wsum[NT / 32];

    const int d = A.d;
    const int64_t n = A.n;
    const size_t map_bytes = level_map_bytes(kMap, d, A.bm_words, A.cap_u_max);
    const LevelLayout L = level_layout(A.cap_c_max, map_bytes, NT);
    uint8_t* base = kOffChip ? A.gscratch + (size_t)blockIdx.x * A.gscratch_stride : smem;
    unsigned long long* ccnt = (unsigned long long*)(base + L.cnt);
    uint32_t* ckeys = (uint32_t*)(base + L.key);
    uint8_t* mapr = base + L.map;
    unsigned long long* sortbuf = (unsigned long long*)mapr;
    uint32_t* list = (uint32_t*)(base + L.list);
    uint64_t* st = (uint64_t*)(base + L.st);
    long long* pfx = (long long*)(base + L.pfx);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = NT / 32;
    const uint64_t* seg_prev = A.seg + (int64_t)(d - 1) * n;

    for (int round = 0;; ++round) {
        if (tid == 0) s_item = A.granular ? (round == 0 ? (int)blockIdx.x : A.n_items) : atomicAdd(A.work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= A.n_items) break;
        const int64_t u = A.items[item];
        const uint32_t cbase = A.comp_base ? (uint32_t)__ldg(A.comp_base + u) : 0u;
        const int64_t raw = A.raw_u[u];
        // On chip a vertex whose candidates overflow the table is handed to
        // the off-chip pass. Off chip the table starts at A.off_start_cap
        // slots (0: the full bound) and doubles, the pull redone, whenever
        // it fills to three quarters, up to the bound 2 min(raw, u) clipped
        // to the slab (A.cap_c_max); a vertex that still overflows then goes
        // to the final off-chip pass, whose slabs hold the full bound.
        const uint32_t full_cap = cand_cap_for(raw, u, A.cap_c_max);
        uint32_t cap_c = (kOffChip && A.off_start_cap) ? min(full_cap, A.off_start_cap) : full_cap;
        // A vertex whose bound does not fit the on-chip table may overflow
        // it; an overflowing attempt reads about half its entries for
        // nothing. Once at least kRouteSamples such attempts in its size
        // class (floor(log2 pulled entries)) have been made at this level
        // and more than two thirds overflowed, it goes to the off-chip pass
        // without an attempt (the same labels either way).
        const bool may_overflow = !kOffChip && full_cap >= A.cap_c_max;
        const int rb = 63 - __clzll((unsigned long long)raw | 1ull);
        if (may_overflow) {
            if (tid == 0) {
                const unsigned a = *(volatile unsigned*)&A.stt->route_att[rb];
                const unsigned o = *(volatile unsigned*)&A.stt->route_ovf[rb];
                s_route = a >= kRouteSamples && 3ull * o > 2ull * a;
                if (s_route) {
                    const int p = atomicAdd(&A.stt->n_retry, 1);
                    A.retry_list[p] = (int32_t)u;
                    atomicMax(&A.stt->need_cap_c, (unsigned long long)cand_cap_for(raw, u, 1u << 30));
                    atomicMax(&A.stt->need_cap_u, (unsigned long long)label_cap_for(A.lab_size[u]));
                }
            }
            __syncthreads();
            if (s_route) {
                __syncthreads();  // s_route and s_item are rewritten by the next item
                continue;
            }
        }

        BitMap bm;
        HashMap hm;
        SegMap sm;
        sm.seg = A.seg;
        sm.hub_arena = A.hub_arena;
        sm.n = n;
        sm.u = u;
        sm.d = d;
        sm.cache = nullptr;
        sm.cwords = 0;
        sm.base = cbase;
        if (kMap == kMapSeg) {
        } else if (kMap == kMapBitmap) {
            bm.bits = (uint32_t*)mapr;
            bm.words = A.bm_words;
            bm.base = cbase;
            bm.d = d;
        } else {
            hm.cap = label_cap_for(A.lab_size[u]);
            hm.keys = (uint32_t*)mapr;
            hm.lvl = (uint16_t*)(mapr + (size_t)hm.cap * 4);
        }

        for (uint32_t i = tid; i < cap_c; i += NT) {
            ckeys[i] = kEmpty;
            ccnt[i] = 0ull;
        }
        uint32_t limit = kOffChip ? cap_c - cap_c / 4 : (cap_c < A.cap_c_max ? cap_c : cap_c - NT - 64);
        if (kMap == kMapBitmap) bm.clear();
        else if (kMap == kMapHash) hm.clear();
        if (tid == 0) {
            s_nkeys = 0;
            s_abort = 0;
            s_m = 0;
            s_next = 0;
            s_nsurv = 0;
        }
        if (A.lmk && tid < A.lmk_stride / 4) s_lmk[tid] = __ldg((const uint32_t*)(A.lmk + u * A.lmk_stride) + tid);
        __syncthreads();

        // 1. label map of L_<d(u)
        for (int l = 0; l < d && kMap != kMapSeg; ++l) {
            const uint64_t s = __ldg(A.seg + (int64_t)l * n + u);
            const uint32_t len = seg_len(s);
            const uint32_t* hs = A.hub_arena + seg_start(s);
            for (uint32_t i = tid; i < len; i += NT) {
                const uint32_t x = __ldg(hs + i) & kHubMask;
                if (kMap == kMapBitmap) bm.insert(x, l); else hm.insert(x, l);
            }
        }
        __syncthreads();

        // 1b. segment-search map: cache the levels of u on chip over the
        // first ids that the table region can hold (the region is free
        // until the prune step is done). Each thread walks hub-sorted
        // segments, so it stops at the first hub beyond the window.
        if (kMap == kMapSeg && d > 1) {
            uint32_t cw = (uint32_t)((L.list - L.map) / 4) / (uint32_t)(d - 1);
            cw = cw < kSegCacheMaxWords ? cw : kSegCacheMaxWords;
            if (cw >= kSegCacheMinWords) {
                uint32_t* cache = (uint32_t*)mapr;
                for (uint32_t i = tid; i < (uint32_t)(d - 1) * cw; i += NT) cache[i] = 0u;
                __syncthreads();
                for (int l = 1; l < d; ++l) {
                    const uint64_t s = __ldg(A.seg + (int64_t)l * n + u);
                    const uint32_t len = seg_len(s);
                    const uint32_t* hs = A.hub_arena + seg_start(s);
                    for (uint32_t i = tid; i < len; i += NT) {
                        const uint32_t r = (__ldg(hs + i) & kHubMask) - cbase;
                        if (r >= 32u * cw) break;
                        atomicOr(&cache[(uint32_t)(l - 1) * cw + (r >> 5)], 1u << (r & 31));
                    }
                }
                __syncthreads();
                sm.cache = cache;
                sm.cwords = cw;
            }
        }

        // 2. pull with the membership filter, merged per hub. In the push
        // paradigm the entries sent to u lie in one bucket, read as a
        // single segment.
        for (;;) {
            const bool push = A.push_hub != nullptr;
            const uint32_t* ghub = push ? A.push_hub : A.hub_arena;
            const unsigned long long* gcnt =
                push ? (const unsigned long long*)A.push_cnt : (const unsigned long long*)A.cnt_arena;
            const int64_t a0 = push ? 0 : A.rp[u], a1 = push ? 1 : A.rp[u + 1];
            for (int64_t ca = a0; ca < a1; ca += NT) {
                const int nc = (int)((a1 - ca) < NT ? (a1 - ca) : NT);
                if (tid < nc) {
                    if (push) {
                        const int64_t b0 = __ldg(A.push_off + A.rp[u]);
                        pfx[tid] = __ldg(A.push_off + A.rp[u + 1]) - b0;
                        st[tid] = (uint64_t)b0;
                    } else {
                        const uint32_t c = __ldg(A.cnt_arc + ca + tid);
                        pfx[tid] = c;
                        st[tid] = c ? seg_start(__ldg(seg_prev + __ldg(A.col + ca + tid))) +
                                          (A.arc_lo ? __ldg(A.arc_lo + ca + tid) : 0u)
                                    : 0ull;
                    }
                }
                __syncthreads();
                const long long total = block_excl_scan(pfx, nc, s_wsum);
                for (long long cb = (long long)warp * 32 * kGatherUnroll; cb < total;
                     cb += (long long)kWarps * 32 * kGatherUnroll) {
                    if (__shfl_sync(0xFFFFFFFFu, *(volatile int*)&s_abort, 0)) break;
                    int lo = 0, hi = nc;  // last arc whose first entry is <= cb
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (pfx[mid] <= cb) lo = mid; else hi = mid;
                    }
                    int j = lo;
                    uint32_t hw[kGatherUnroll];
                    uint64_t pos[kGatherUnroll];
                    bool ok[kGatherUnroll];
    #pragma unroll
                    for (int t = 0; t < kGatherUnroll; ++t) {
                        const long long i = cb + t * 32 + lane;
                        ok[t] = i < total;
                        if (ok[t]) {
                            while (pfx[j + 1] <= i) ++j;
                            pos[t] = st[j] + (uint64_t)(i - pfx[j]);
                            hw[t] = __ldg(ghub + pos[t]);
                        }
                    }
    #pragma unroll
                    for (int t = 0; t < kGatherUnroll; ++t)
                        if (ok[t]) {
                            const uint32_t h = hw[t] & kHubMask;
                            ok[t] = !(kMap == kMapBitmap ? bm.member(h) : kMap == kMapHash ? hm.member(h) : sm.member(h));
                        }
                    uint64_t cv[kGatherUnroll];
    #pragma unroll
                    for (int t = 0; t < kGatherUnroll; ++t)
                        if (ok[t]) cv[t] = __ldg(gcnt + pos[t]);
    #pragma unroll
                    for (int t = 0; t < kGatherUnroll; ++t)
                        if (ok[t]) cand_insert(ckeys, ccnt, cap_c, limit, hw[t] & kHubMask, cv[t], hw[t] >> 31, &s_nkeys,
                                               &s_abort);
                }
                __syncthreads();
                if (s_abort) break;
            }
            __syncthreads();
            if (!kOffChip || !s_abort || cap_c >= full_cap) break;
            // off chip: a larger table, and the pull again
            cap_c = min(2 * cap_c, full_cap);
            limit = cap_c - cap_c / 4;
            for (uint32_t i = tid; i < cap_c; i += NT) {
                ckeys[i] = kEmpty;
                ccnt[i] = 0ull;
            }
            __syncthreads();
            if (tid == 0) {
                s_nkeys = 0;
                s_abort = 0;
            }
            __syncthreads();
        }
        __syncthreads();
        if (s_abort) {
            if (tid == 0) {
                if (kOffChip) {
                    A.giant_list[atomicAdd(&A.stt->n_giant, 1)] = (int32_t)u;
                } else {
                    if (may_overflow) {
                        atomicAdd(&A.stt->route_att[rb], 1u);
                        atomicAdd(&A.stt->route_ovf[rb], 1u);
                    }
                    const int p = atomicAdd(&A.stt->n_retry, 1);
                    A.retry_list[p] = (int32_t)u;
                    atomicMax(&A.stt->need_cap_c, (unsigned long long)cand_cap_for(raw, u, 1u << 30));
                    atomicMax(&A.stt->need_cap_u, (unsigned long long)label_cap_for(A.lab_size[u]));
                }
            }
            __syncthreads();
            continue;
        }

        // candidate list
        for (uint32_t slot = tid; slot < cap_c; slot += NT)
            if (ckeys[slot] != kEmpty) list[atomicAdd(&s_m, 1)] = slot;
        __syncthreads();
        int M = s_m;

        // 3a. d = 3: rule 2 asks for a common neighbour x of u and h ranked
        // above h (x in L_1(u) and x in L_1(h)). Walk, for every x in L_1(u),
        // the range (x, u) of x's sorted row; a hub met there that is a
        // candidate (bitmap cand_bm) is marked pruned (bitmap mk). This replaces
        // scanning L_1(h) for every candidate h.
        bool marked = false;
        const uint32_t Wm = (uint32_t)((u - cbase + 31) >> 5);
        if (d == 3 && (size_t)Wm * 8 <= (size_t)(L.list - L.map) && M > 0) {
            uint32_t* cand_bm = (uint32_t*)mapr;
            uint32_t* mk = cand_bm + Wm;
            for (uint32_t i = tid; i < 2 * Wm; i += NT) cand_bm[i] = 0u;
            __syncthreads();
            for (int c = tid; c < M; c += NT) {
                const uint32_t h = (ckeys[list[c]] & kHubMask) - cbase;
                atomicOr(&cand_bm[h >> 5], 1u << (h & 31));
            }
            const uint64_t s1 = __ldg(A.seg + n + u);
            const uint32_t len1 = seg_len(s1);
            const uint32_t* xs = A.hub_arena + seg_start(s1);
            __syncthreads();
            for (uint32_t c0 = 0; c0 < len1; c0 += NT) {
                const int nc = (int)(len1 - c0 < (uint32_t)NT ? len1 - c0 : (uint32_t)NT);
                if (tid < nc) {
                    const uint32_t x = __ldg(xs + c0 + tid) & kHubMask;
                    // below u's dense prefix every id is in L_<3(u), so no
                    // candidate: start the walk at the prefix when it is past x
                    const uint32_t from = A.hpre && (uint32_t)__ldg(A.hpre + u) > x + 1 ? (uint32_t)__ldg(A.hpre + u) - 1 : x;
                    const int64_t r1 = A.rp[x + 1];
                    int64_t lo = A.rp[x], hi = r1;
                    while (lo < hi) {  // first neighbour of x ranked below both x and the prefix
                        const int64_t mid = (lo + hi) >> 1;
                        if ((uint32_t)__ldg(A.col + mid) <= from) lo = mid + 1; else hi = mid;
                    }
                    const int64_t first = lo;
                    hi = r1;
                    while (lo < hi) {  // first neighbour of x not ranked above u
                        const int64_t mid = (lo + hi) >> 1;
                        if ((int64_t)__ldg(A.col + mid) < u) lo = mid + 1; else hi = mid;
                    }
                    pfx[tid] = lo - first;
                    st[tid] = (uint64_t)first;
                }
                __syncthreads();
                const long long total = block_excl_scan(pfx, nc, s_wsum);
                for (long long cb = (long long)warp * 32 * kGatherUnroll; cb < total;
                     cb += (long long)kWarps * 32 * kGatherUnroll) {
                    int lo = 0, hi = nc;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (pfx[mid] <= cb) lo = mid; else hi = mid;
                    }
                    int j = lo;
                    int32_t hv[kGatherUnroll];
#pragma unroll
                    for (int t = 0; t < kGatherUnroll; ++t) {
                        const long long i = cb + t * 32 + lane;
                        hv[t] = -1;
                        if (i < total) {
                            while (pfx[j + 1] <= i) ++j;
                            hv[t] = __ldg(A.col + st[j] + (uint64_t)(i - pfx[j]));
                        }
                    }
#pragma unroll
                    for (int t = 0; t < kGatherUnroll; ++t)
                        if (hv[t] >= 0) {
                            const uint32_t hr = (uint32_t)hv[t] - cbase;
                            const uint32_t bit = 1u << (hr & 31);
                            if (cand_bm[hr >> 5] & bit) atomicOr(&mk[hr >> 5], bit);
                        }
                }
                __syncthreads();
            }
            for (int c = tid; c < M; c += NT) {
                const uint32_t slot = list[c];
                const uint32_t h = (ckeys[slot] & kHubMask) - cbase;
                if ((mk[h >> 5] >> (h & 31)) & 1u) list[c] = slot | kPrunedBit;
            }
            __syncthreads();
            marked = true;
        }

        // 3. prune rule 2 over levels 1..d-2 of each candidate's label
        int M_scan = M, n_proven = 0;
        if (d >= 3 && !marked && M > 0 && A.lmk) {
            M_scan = landmark_filter<NT>(A, s_lmk, d, list, ckeys, M, s_wcnt, &s_kept, &n_proven);
            if (tid == 0 && M_scan < M) atomicAdd(&A.stt->lmk_pruned, (unsigned long long)(M - M_scan));
            if (tid == 0 && n_proven) atomicAdd(&A.stt->lmk_proven, (unsigned long long)n_proven);
        }
        if (d >= 3 && !marked && M_scan > n_proven) {
            const int ns = M_scan - n_proven;
            // u's level descriptors, for scanning u's side when it is shorter
            // (not with bitmaps: their probes cost one on-chip read)
            const bool useg_on = kMap != kMapBitmap && d - 2 < kUSideLevels;
            if (useg_on && tid < d - 1) s_useg[tid] = __ldg(A.seg + (int64_t)tid * n + u);
            __syncthreads();
            const uint64_t* useg = useg_on ? s_useg : nullptr;
            if constexpr (kMap == kMapBitmap)
                prune_all<NT>(bm, A.seg, A.hub_arena, n, d, list, ckeys, M_scan, ns, &s_next, useg, s_wcnt);
            else if constexpr (kMap == kMapHash)
                prune_all<NT>(hm, A.seg, A.hub_arena, n, d, list, ckeys, M_scan, ns, &s_next, useg, s_wcnt);
            else prune_all<NT>(sm, A.seg, A.hub_arena, n, d, list, ckeys, M_scan, ns, &s_next, useg, s_wcnt);
            __syncthreads();
        }
        M = M_scan;  // list[0..M) now holds every candidate that can survive

        // 4. survivors, hub-sorted, appended as L_d(u). Candidate hubs are < u:
        // when a bitmap of u bits and its word prefix fit the map region, a
        // survivor's rank is the prefix of its word plus a popcount; else a
        // bitonic sort.
        const uint32_t W = (uint32_t)((u - cbase + 31) >> 5);
        const size_t region = (L.list - L.map);
        if ((size_t)W * 8 <= region) {
            uint32_t* sb = (uint32_t*)mapr;
            uint32_t* wp = sb + W;
            for (uint32_t i = tid; i < W; i += NT) sb[i] = 0u;
            __syncthreads();
            for (int c = tid; c < M; c += NT) {
                const uint32_t slot = list[c];
                if (!(slot & kPrunedBit)) {
                    const uint32_t h = (ckeys[slot & kSlotMask] & kHubMask) - cbase;
                    atomicOr(&sb[h >> 5], 1u << (h & 31));
                }
            }
            __syncthreads();
            const int S = (int)block_excl_scan_popc(sb, wp, W, s_wsum);
            if (S > 0) {
                if (tid == 0) {
                    const unsigned long long b0 = atomicAdd(&A.stt->bump, (unsigned long long)S);
                    if (b0 + S > A.arena_cap) atomicOr(&A.stt->arena_overflow, 1);
                    s_base = b0;
                }
                __syncthreads();
                const unsigned long long b0 = s_base;
                if (b0 + S <= A.arena_cap) {
                    for (int c = tid; c < M; c += NT) {
                        const uint32_t e = list[c];
                        if (e & kPrunedBit) continue;
                        const uint32_t slot = e & kSlotMask;
                        const uint32_t key = ckeys[slot];
                        const uint32_t h = key & kHubMask;
                        const uint32_t hr = h - cbase;
                        const uint32_t r = wp[hr >> 5] + __popc(sb[hr >> 5] & ((1u << (hr & 31)) - 1u));
                        A.hub_arena[b0 + r] = h | (key & kOvfBit);
                        A.cnt_arena[b0 + r] = ccnt[slot];
                    }
                    if (tid == 0) A.seg_out[u] = seg_pack(b0, (uint32_t)S);
                }
            }
        } else {
            for (int c = tid; c < M; c += NT) {
                const uint32_t e = list[c];
                if (!(e & kPrunedBit))
                    sortbuf[atomicAdd(&s_nsurv, 1)] =
                        ((unsigned long long)(ckeys[e & kSlotMask] & kHubMask) << 32) | (e & kSlotMask);
            }
            __syncthreads();
            const int S = s_nsurv;
            if (S > 0) {
                const uint32_t P = pow2_ceil((uint64_t)S);
                for (uint32_t i = S + tid; i < P; i += NT) sortbuf[i] = ~0ull;
                __syncthreads();
                block_bitonic_sort(sortbuf, P);
                if (tid == 0) {
                    const unsigned long long b0 = atomicAdd(&A.stt->bump, (unsigned long long)S);
                    if (b0 + S > A.arena_cap) atomicOr(&A.stt->arena_overflow, 1);
                    s_base = b0;
                }
                __syncthreads();
                const unsigned long long b0 = s_base;
                if (b0 + S <= A.arena_cap) {
                    for (int i = tid; i < S; i += NT) {
                        const uint32_t slot = (uint32_t)sortbuf[i];
                        const uint32_t key = ckeys[slot];
                        A.hub_arena[b0 + i] = (key & kHubMask) | (key & kOvfBit);
                        A.cnt_arena[b0 + i] = ccnt[slot];
                    }
                    if (tid == 0) A.seg_out[u] = seg_pack(b0, (uint32_t)S);
                }
            }
        }
        if (tid == 0) atomicAdd(&A.stt->unique_total, (unsigned long long)s_nkeys);
        if (tid == 0 && may_overflow) atomicAdd(&A.stt->route_att[rb], 1u);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The level for tiny vertices (fewer than 2^kMicroBucket pulled entries):
// one warp per vertex and no CTA barrier, so that many such vertices (the
// deep levels of high-diameter graphs, the tails of power-law graphs) are in
// flight per SM. The warp stages the pulled entries on chip, drops those
// whose hub is already in L_<d(u) (segment search), sorts the rest by hub
// (a 64-element bitonic sort in registers, two elements per lane) and sums
// the counts of equal hubs with a segmented scan (mod 2^64; the flag takes
// the entries' flags and every carry: Label Merging). Rule 2 then runs per
// candidate: the landmark filter, and for the undecided ones a scan of
// levels 1..d-2 of L(h) by the whole warp. Survivors are already in hub
// order and are appended as L_d(u).
constexpr int kMicroWarps = kMicroThreads / 32;

__device__ __forceinline__ void add_count(uint64_t& sum, uint32_t& flag, uint64_t c, uint32_t f) {
    const uint64_t s = sum + c;
    flag |= f | (uint32_t)(s < c);
    sum = s;
}

__global__ void __launch_bounds__(kMicroThreads) k_level_micro(const LevelArgs A) {
    __shared__ uint32_t s_hub[kMicroWarps][64];
    __shared__ unsigned long long s_cnt[kMicroWarps][64];
    __shared__ uint32_t s_lmkw[kMicroWarps][kLmkMax / 2];
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d = A.d;
    const int64_t n = A.n;
    const uint64_t* seg_prev = A.seg + (int64_t)(d - 1) * n;
    uint32_t* hb = s_hub[w];
    unsigned long long* cbuf = s_cnt[w];
    uint32_t* ul = s_lmkw[w];
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long n_uniq = 0, n_lpr = 0, n_lpv = 0;
    for (int round = 0;; ++round) {
        int item;
        if (A.granular) {
            item = round == 0 ? (int)(blockIdx.x * kMicroWarps + w) : A.n_items;
        } else {
            item = 0;
            if (lane == 0) item = atomicAdd(A.work, 1);
            item = __shfl_sync(FULL, item, 0);
        }
        if (item >= A.n_items) break;
        const int64_t u = A.items[item];
        SegMap sm;
        sm.seg = A.seg;
        sm.hub_arena = A.hub_arena;
        sm.n = n;
        sm.u = u;
        sm.d = d;
        sm.cache = nullptr;
        sm.cwords = 0;
        sm.base = 0;

        // 1. stage the pulled entries (fewer than 64)
        int total = 0;
        if (A.push_hub) {
            const int64_t b0 = __ldg(A.push_off + A.rp[u]);
            total = (int)(__ldg(A.push_off + A.rp[u + 1]) - b0);
            for (int i = lane; i < total; i += 32) {
                hb[i] = __ldg(A.push_hub + b0 + i);
                cbuf[i] = __ldg((const unsigned long long*)A.push_cnt + b0 + i);
            }
        } else {
            const int64_t a0 = A.rp[u], a1 = A.rp[u + 1];
            for (int64_t ca = a0; ca < a1; ca += 32) {
                const int64_t a = ca + lane;
                uint32_t c = 0;
                uint64_t st = 0;
                if (a < a1) {
                    c = __ldg(A.cnt_arc + a);
                    if (c) st = seg_start(__ldg(seg_prev + __ldg(A.col + a))) + (A.arc_lo ? __ldg(A.arc_lo + a) : 0u);
                }
                uint32_t incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += t;
                }
                const int base = total + (int)(incl - c);
                for (uint32_t i = 0; i < c; ++i) {
                    hb[base + i] = __ldg(A.hub_arena + st + i);
                    cbuf[base + i] = __ldg((const unsigned long long*)A.cnt_arena + st + i);
                }
                total += (int)__shfl_sync(FULL, incl, 31);
            }
        }
        __syncwarp();

        // 2. membership filter and sort keys: hub << 6 | entry, 0xFFFFFFFF
        // for dropped and absent entries (they sort last)
        uint32_t key[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int e = lane + 32 * j;
            key[j] = 0xFFFFFFFFu;
            if (e < total) {
                const uint32_t h = hb[e] & kHubMask;
                if (!sm.member(h)) key[j] = (h << 6) | (uint32_t)e;
            }
        }
#pragma unroll
        for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                if (jj == 32) {  // partners in the same lane
                    const bool asc = (lane & k) == 0;
                    const uint32_t lo = min(key[0], key[1]), hi = max(key[0], key[1]);
                    key[0] = asc ? lo : hi;
                    key[1] = asc ? hi : lo;
                } else {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int e = lane + 32 * j;
                        const uint32_t other = __shfl_xor_sync(FULL, key[j], jj);
                        const bool lower = (e & jj) == 0, asc = (e & k) == 0;
                        key[j] = (lower == asc) ? min(key[j], other) : max(key[j], other);
                    }
                }
            }
        }

        // 3. segmented sums over runs of equal hubs, in sorted order
        uint32_t hub[2], flg[2];
        uint64_t sum[2];
        bool valid[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            valid[j] = key[j] != 0xFFFFFFFFu;
            hub[j] = valid[j] ? key[j] >> 6 : 0xFFFFFFFFu;
            const int src = (int)(key[j] & 63u);
            sum[j] = valid[j] ? (uint64_t)cbuf[src] : 0ull;
            flg[j] = valid[j] ? (hb[src] >> 31) : 0u;
        }
        // a run starts where the previous element (in sorted order) has
        // another hub; row 1's lane 0 follows row 0's lane 31
        const uint32_t prev0 = __shfl_up_sync(FULL, hub[0], 1);
        const uint32_t last0 = __shfl_sync(FULL, hub[0], 31);
        const uint32_t prev1 = __shfl_up_sync(FULL, hub[1], 1);
        const bool head0 = valid[0] && (lane == 0 || prev0 != hub[0]);
        const bool head1 = valid[1] && (lane == 0 ? last0 != hub[1] : prev1 != hub[1]);
        const unsigned h0 = __ballot_sync(FULL, head0), h1 = __ballot_sync(FULL, head1);
        const int id0 = __popc(h0 & (lt | (1u << lane)));                       // segment id (1-based)
        const int id1 = __popc(h0) + __popc(h1 & (lt | (1u << lane)));
        int id[2] = {id0, id1};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t sv = __shfl_up_sync(FULL, sum[j], o);
                const uint32_t fv = __shfl_up_sync(FULL, flg[j], o);
                const int iv = __shfl_up_sync(FULL, id[j], o);
                if (lane >= o && iv == id[j] && valid[j]) add_count(sum[j], flg[j], sv, fv);
            }
        }
        {  // row 1's first run may continue row 0's last one (every lane
           // takes part in the shuffles; only then do lanes branch)
            const uint64_t s31 = __shfl_sync(FULL, sum[0], 31);
            const uint32_t f31 = __shfl_sync(FULL, flg[0], 31);
            const int i31 = __shfl_sync(FULL, id[0], 31);
            const int v31 = __shfl_sync(FULL, (int)valid[0], 31);
            if (valid[1] && v31 && id[1] == i31) add_count(sum[1], flg[1], s31, f31);
        }
        // the last element of each run holds its total
        const uint32_t next0 = __shfl_down_sync(FULL, hub[0], 1);
        const uint32_t first1 = __shfl_sync(FULL, hub[1], 0);
        const uint32_t next1 = __shfl_down_sync(FULL, hub[1], 1);
        bool cand[2];
        cand[0] = valid[0] && (lane == 31 ? first1 != hub[0] : next0 != hub[0]);
        cand[1] = valid[1] && (lane == 31 || next1 != hub[1]);
        const int uniq = __popc(h0) + __popc(h1);
        n_uniq += (unsigned long long)uniq;

        // 4. rule 2: the landmark filter, then the undecided candidates' scans
        bool surv[2] = {cand[0], cand[1]};
        if (d >= 3 && uniq > 0) {
            bool und[2] = {cand[0], cand[1]};
            if (A.lmk) {
                for (int i = lane; i < A.lmk_stride / 4; i += 32) ul[i] = __ldg((const uint32_t*)(A.lmk + u * A.lmk_stride) + i);
                __syncwarp();
                const uint32_t dd = (uint32_t)d * 0x00010001u;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (!cand[j]) continue;
                    const uint4* row = (const uint4*)(A.lmk + (size_t)hub[j] * A.lmk_stride);
                    uint32_t hit = 0, far = 0;
                    for (int q4 = 0; q4 < A.lmk_words; ++q4) {
                        const uint4 b4 = __ldg(row + q4);
                        const uint32_t bw[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t a = ul[4 * q4 + q], b = bw[q];
                            hit |= __vcmpltu2(__vaddus2(a, b), dd);
                            const uint32_t known = ~(__vcmpeq2(a, 0xFFFFFFFFu) | __vcmpeq2(b, 0xFFFFFFFFu));
                            far |= __vcmpgeu2(__vabsdiffu2(a, b), dd) & known;
                        }
                    }
                    if (hit) {
                        surv[j] = false;
                        und[j] = false;
                        ++n_lpr;
                    } else if (far) {
                        und[j] = false;
                        ++n_lpv;
                    }
                }
                __syncwarp();
            }
            unsigned u0 = __ballot_sync(FULL, und[0]), u1 = __ballot_sync(FULL, und[1]);
            while (u0 | u1) {
                const int j = u0 ? 0 : 1;
                const unsigned m = j ? u1 : u0;
                const int src = __ffs(m) - 1;
                const uint32_t h = __shfl_sync(FULL, hub[j], src);
                const bool pruned = scan_levels<32>(sm, A.seg, A.hub_arena, n, d, h, 1, d - 2, nullptr);
                if (pruned && lane == src) surv[j] = false;
                if (j) u1 &= m - 1; else u0 &= m - 1;
            }
        }

        // 5. append the survivors in hub order
        const unsigned s0 = __ballot_sync(FULL, surv[0]), s1 = __ballot_sync(FULL, surv[1]);
        const int S = __popc(s0) + __popc(s1);
        if (S > 0) {
            unsigned long long b0 = 0;
            if (lane == 0) {
                b0 = atomicAdd(&A.stt->bump, (unsigned long long)S);
                if (b0 + S > A.arena_cap) atomicOr(&A.stt->arena_overflow, 1);
            }
            b0 = __shfl_sync(FULL, b0, 0);
            if (b0 + S <= A.arena_cap) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (!surv[j]) continue;
                    const int pos = j ? __popc(s0) + __popc(s1 & lt) : __popc(s0 & lt);
                    A.hub_arena[b0 + pos] = hub[j] | (flg[j] ? kOvfBit : 0u);
                    A.cnt_arena[b0 + pos] = sum[j];
                }
                if (lane == 0) A.seg_out[u] = seg_pack(b0, (uint32_t)S);
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (n_uniq) atomicAdd(&A.stt->unique_total, n_uniq);
        if (n_lpr) atomicAdd(&A.stt->lmk_pruned, n_lpr);
        if (n_lpv) atomicAdd(&A.stt->lmk_proven, n_lpv);
    }
}

// ---------------------------------------------------------------------------
// Push paradigm.

__global__ void k_arc_counts(int64_t arcs, const uint32_t* __restrict__ cnt_arc, int64_t* __restrict__ out) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < arcs) out[a] = cnt_arc[a];
}

// Warp per arc u->v: the entries of L_{d-1}(v) that u receives go to u's
// bucket in the order they lie in v's segment.
__global__ void k_push_scatter(int64_t arcs, const int32_t* __restrict__ col, const uint64_t* __restrict__ seg_prev,
                               const uint32_t* __restrict__ hub_arena, const uint64_t* __restrict__ cnt_arena,
                               const uint32_t* __restrict__ cnt_arc, const uint32_t* __restrict__ arc_lo,
                               const int64_t* __restrict__ push_off, uint32_t* __restrict__ push_hub,
                               uint64_t* __restrict__ push_cnt) {
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a >= arcs) return;
    const uint32_t c = cnt_arc[a];
    if (!c) return;
    const uint64_t src = seg_start(__ldg(seg_prev + col[a])) + (arc_lo ? arc_lo[a] : 0u);
    const int64_t dst = push_off[a];
    for (uint32_t i = lane; i < c; i += 32) {
        push_hub[dst + i] = __ldg(hub_arena + src + i);
        push_cnt[dst + i] = __ldg((const unsigned long long*)cnt_arena + src + i);
    }
}

cudaError_t launch_arc_counts(int64_t arcs, const uint32_t* cnt_arc, int64_t* out, cudaStream_t st) {
    if (arcs > 0) k_arc_counts<<<(unsigned)((arcs + 255) / 256), 256, 0, st>>>(arcs, cnt_arc, out);
    return cudaGetLastError();
}

cudaError_t launch_push_scatter(int64_t arcs, const int32_t* col, const uint64_t* seg_prev,
                                const uint32_t* hub_arena, const uint64_t* cnt_arena, const uint32_t* cnt_arc,
                                const uint32_t* arc_lo, const int64_t* push_off, uint32_t* push_hub,
                                uint64_t* push_cnt, cudaStream_t st) {
    if (arcs > 0)
        k_push_scatter<<<(unsigned)((arcs * 32 + 255) / 256), 256, 0, st>>>(arcs, col, seg_prev, hub_arena, cnt_arena,
                                                                          cnt_arc, arc_lo, push_off, push_hub,
                                                                          push_cnt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers.

cudaError_t launch_arc_src(const int64_t* rp, int64_t n, int32_t* arc_src, cudaStream_t st) {
    k_arc_src<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(rp, n, arc_src);
    return cudaGetLastError();
}

cudaError_t launch_dense_prefix(int d, int64_t n, const uint64_t* seg, const uint32_t* hub_arena,
                                const int32_t* comp_base, int32_t* hpre, cudaStream_t st) {
    k_dense_prefix<<<(unsigned)((n + kPrefixWarps - 1) / kPrefixWarps), kPrefixWarps * 32, 0, st>>>(
        d, n, seg, hub_arena, comp_base, hpre);
    return cudaGetLastError();
}

cudaError_t launch_cost(int d, int64_t n, int64_t arcs, const int64_t* rp, const int32_t* col,
                        const int32_t* arc_src, const uint64_t* seg_prev, const uint32_t* hub_arena,
                        const int32_t* hpre, uint32_t* arc_lo, uint32_t* cnt_arc, int64_t* raw_u,
                        int64_t* lab_size, LevelStatus* stt, int64_t label_limit, int32_t* glist, int32_t* items,
                        cudaStream_t st, int64_t* launches) {
    cudaError_t e = cudaMemsetAsync(raw_u, 0, n * 8, st);
    if (e != cudaSuccess) return e;
    if (arcs > 0)
        k_cost_arcs<<<(unsigned)((arcs + 255) / 256), 256, 0, st>>>(arcs, arc_src, col, seg_prev, hub_arena, hpre,
                                                                     arc_lo, cnt_arc, (unsigned long long*)raw_u,
                                                                     &stt->prefix_skipped);
    k_cost_vertices<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, rp, seg_prev, raw_u, lab_size, stt, label_limit,
                                                                  glist);
    k_bucket_base<<<1, 32, 0, st>>>(stt);
    k_bucket_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, raw_u, lab_size, stt, label_limit, items);
    if (launches) *launches += (arcs > 0) + 3;
    return cudaGetLastError();
}

template <int NT>
static const void* level_fn(int map_kind, bool offchip) {
    if (offchip) return map_kind == kMapSeg ? (const void*)k_level<kMapSeg, true, NT> : (const void*)k_level<kMapHash, true, NT>;
    return map_kind == kMapBitmap ? (const void*)k_level<kMapBitmap, false, NT>
           : map_kind == kMapHash ? (const void*)k_level<kMapHash, false, NT>
                                  : (const void*)k_level<kMapSeg, false, NT>;
}

// The kernel's dynamic shared-memory limit is raised to the device's
// opt-in maximum, the same value on every call: builds that run at the same
// time on other threads never see it lowered under a launch.
cudaError_t level_kernel_attrs(int map_kind, size_t smem_bytes, int* occupancy, int nt) {
    const void* f = nt == kLightThreads ? level_fn<kLightThreads>(map_kind, false) : level_fn<kLevelThreads>(map_kind, false);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    const size_t max_dyn = (size_t)optin - fa.sharedSizeBytes;
    if (smem_bytes > max_dyn) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dyn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, f, nt, smem_bytes);
}

template <int NT>
static void launch_level_nt(int map_kind, bool offchip, int grid, size_t smem_bytes, const LevelArgs& A,
                            cudaStream_t st) {
    if (offchip && map_kind == kMapSeg)
        k_level<kMapSeg, true, NT><<<grid, NT, 0, st>>>(A);
    else if (offchip)
        k_level<kMapHash, true, NT><<<grid, NT, 0, st>>>(A);
    else if (map_kind == kMapBitmap)
        k_level<kMapBitmap, false, NT><<<grid, NT, smem_bytes, st>>>(A);
    else if (map_kind == kMapHash)
        k_level<kMapHash, false, NT><<<grid, NT, smem_bytes, st>>>(A);
    else
        k_level<kMapSeg, false, NT><<<grid, NT, smem_bytes, st>>>(A);
}

cudaError_t micro_kernel_occupancy(int* occupancy) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, (const void*)k_level_micro, kMicroThreads, 0);
}

cudaError_t launch_level_micro(int grid, const LevelArgs& A, cudaStream_t st) {
    k_level_micro<<<grid, kMicroThreads, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_level(int map_kind, bool offchip, int grid, size_t smem_bytes, const LevelArgs& A,
                         cudaStream_t st, int nt) {
    if (nt == kLightThreads && !offchip) launch_level_nt<kLightThreads>(map_kind, false, grid, smem_bytes, A, st);
    else launch_level_nt<kLevelThreads>(map_kind, offchip, grid, smem_bytes, A, st);
    return cudaGetLastError();
}

}  // namespace pspc
