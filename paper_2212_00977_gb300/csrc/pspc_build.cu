// Level-synchronous pull construction of the SPC 2-hop hub-label index
// (PSPC, arXiv 2212.00977): Theorem "Distance Dependency", Lemma
// "Propagation", pruning rules 1 and 2, Label Merging, and Algorithm PULL.
//
// Vertices are relabelled so that id = rank (0 = highest). Level d of every
// vertex is stored as one hub-sorted segment of a label arena (hub word with
// the overflow flag in bit 31, uint64 count; the distance is the level).
// Per level:
//   k_cost      per arc u->v: how many entries of L_{d-1}(v) have a hub
//               ranked above u (a prefix, segments are hub-sorted: rule 1);
//               per vertex the sum (the paper's cost function) and a class.
//   k_bucket_*  orders active vertices by decreasing cost (dynamic schedule).
//   k_level     one CTA per vertex, persistent with a work counter: gathers
//               the pulled entries into an on-chip hash keyed by hub, adding
//               counts mod 2^64 with a sticky overflow flag (Label Merging);
//               tests every candidate hub h with the distance-bounded prune
//               query (rule 2), sorts the survivors by hub and appends them.
// After the last non-empty level, k_finalize merges each vertex's level
// segments into one hub-sorted label (Table "Shortest Path Counting Labels"
// order).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pspc_internal.cuh"

namespace cg = cooperative_groups;

namespace pspc {

constexpr int kLevelThreads = 512;
constexpr int kProbeGroup = 8;  // lanes that scan one candidate's label segment
constexpr int kBuckets = 64;
constexpr int kFinThreads = 256;
constexpr int kFinSmemKeys = 8192;  // labels up to this size are merged on chip

struct LevelStatus {
    unsigned long long raw_total;
    unsigned long long unique_total;
    unsigned long long bump;       // arena fill after this level
    unsigned long long need_cap_c; // largest candidate table of the off-chip class
    unsigned long long need_cap_u; // largest label table of the off-chip class
    unsigned long long active_arcs;
    int n_active;
    int n_smem;
    int n_global;
    int n_retry;
    int arena_overflow;
    int work_smem;
    int work_global;
    int pad;
    int bucket_cnt[kBuckets];
    int bucket_base[kBuckets];
    int bucket_fill[kBuckets];
};

// ---------------------------------------------------------------------------
// Input checks (the ABI rejects malformed graphs and orders).

__global__ void k_check_rank(const int32_t* __restrict__ rank, int64_t n, uint32_t* seen, int* err) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t r = rank[v];
    if (r < 0 || r >= n) {
        atomicOr(err, 1);
        return;
    }
    if (atomicExch(&seen[r], 1u) != 0u) atomicOr(err, 1);
}

__global__ void k_check_rowptr(const int64_t* __restrict__ rp, int64_t n, int* err) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v > n) return;
    if (v == 0 && rp[0] != 0) atomicOr(err, 1);
    if (v < n && rp[v] > rp[v + 1]) atomicOr(err, 1);
}

// Warp per vertex: ids in range, no self-loop, rows strictly ascending, and
// every arc has its reverse (binary search in the neighbour's row).
__global__ void k_check_arcs(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                             int* err) {
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    const int64_t a0 = rp[u], a1 = rp[u + 1];
    for (int64_t a = a0 + lane; a < a1; a += 32) {
        const int32_t v = col[a];
        if (v < 0 || v >= n || v == u || (a + 1 < a1 && col[a + 1] <= v)) {
            atomicOr(err, 1);
            continue;
        }
        int64_t lo = rp[v], hi = rp[v + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (col[mid] < u) lo = mid + 1; else hi = mid;
        }
        if (lo == rp[v + 1] || col[lo] != (int32_t)u) atomicOr(err, 1);
    }
}

// ---------------------------------------------------------------------------
// Relabel by rank (id = rank): row lengths, inverse permutation, arcs.

__global__ void k_deg_perm(const int64_t* __restrict__ rp, const int32_t* __restrict__ rank, int64_t n,
                           int64_t* rp_r, int32_t* order) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t r = rank[v];
    rp_r[r] = rp[v + 1] - rp[v];
    order[r] = (int32_t)v;
}

__global__ void k_relabel_arcs(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ rank, int64_t n, const int64_t* __restrict__ rp_r,
                               int32_t* __restrict__ col_r) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    const int64_t a0 = rp[v], deg = rp[v + 1] - a0;
    const int64_t b0 = rp_r[rank[v]];
    for (int64_t i = lane; i < deg; i += 32) col_r[b0 + i] = rank[col[a0 + i]];
}

// Level 0: L_0(v) = {(v, 0, 1)}.
__global__ void k_level0(int64_t n, uint32_t* hub_arena, uint64_t* cnt_arena, uint64_t* seg0) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    hub_arena[v] = (uint32_t)v;
    cnt_arena[v] = 1ull;
    seg0[v] = seg_pack((uint64_t)v, 1u);
}

// ---------------------------------------------------------------------------
// Per-level cost and classification.

__device__ __forceinline__ uint32_t cand_cap_for(int64_t raw, int64_t u, uint32_t cap_max) {
    const int64_t bound = raw < u ? raw : u;  // distinct hubs <= pulled entries, and < u
    const uint64_t want = (uint64_t)(2 * bound) < 64ull ? 64ull : (uint64_t)(2 * bound);
    return want >= cap_max ? cap_max : pow2_ceil(want);
}
__device__ __forceinline__ uint32_t label_cap_for(int64_t lab) {
    const uint64_t want = (uint64_t)(lab + lab / 3 + 1);
    return pow2_ceil(want < 64ull ? 64ull : want);
}

// Warp per vertex u: updates |L_<d(u)| with level d-1, and for every arc
// u->v counts the entries of L_{d-1}(v) whose hub ranks above u.
__global__ void k_cost(int d, int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const uint64_t* __restrict__ seg_prev, const uint32_t* __restrict__ hub_arena,
                       uint32_t* __restrict__ cnt_arc, int64_t* __restrict__ raw_u, int64_t* __restrict__ lab_size,
                       LevelStatus* stt, uint32_t cap_u_smem, int32_t* __restrict__ glist) {
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    int64_t raw = 0;
    for (int64_t a = rp[u] + lane; a < rp[u + 1]; a += 32) {
        const int32_t v = col[a];
        const uint64_t s = seg_prev[v];
        const uint32_t* h = hub_arena + seg_start(s);
        uint32_t lo = 0, hi = seg_len(s);
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if ((__ldg(h + mid) & kHubMask) < (uint32_t)u) lo = mid + 1; else hi = mid;
        }
        cnt_arc[a] = lo;
        raw += lo;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) raw += __shfl_xor_sync(0xFFFFFFFFu, raw, o);
    if (lane != 0) return;
    const int64_t ls = lab_size[u] + seg_len(seg_prev[u]);
    lab_size[u] = ls;
    raw_u[u] = raw;
    if (raw == 0) return;
    atomicAdd(&stt->raw_total, (unsigned long long)raw);
    atomicAdd(&stt->active_arcs, (unsigned long long)(rp[u + 1] - rp[u]));
    atomicAdd(&stt->n_active, 1);
    if (label_cap_for(ls) <= cap_u_smem) {
        atomicAdd(&stt->n_smem, 1);
        atomicAdd(&stt->bucket_cnt[63 - __clzll((unsigned long long)raw)], 1);
    } else {
        const int p = atomicAdd(&stt->n_global, 1);
        glist[p] = (int32_t)u;
        const uint64_t cu = label_cap_for(ls);
        const uint64_t cc = cand_cap_for(raw, u, 1u << 30);
        atomicMax(&stt->need_cap_u, (unsigned long long)cu);
        atomicMax(&stt->need_cap_c, (unsigned long long)cc);
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
                              LevelStatus* stt, uint32_t cap_u_smem, int32_t* __restrict__ items) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int64_t raw = raw_u[u];
    if (raw == 0 || label_cap_for(lab_size[u]) > cap_u_smem) return;
    const int b = 63 - __clzll((unsigned long long)raw);
    items[stt->bucket_base[b] + atomicAdd(&stt->bucket_fill[b], 1)] = (int32_t)u;
}

// ---------------------------------------------------------------------------
// The level kernel.

struct LevelArgs {
    int d;
    int64_t n;
    const int64_t* rp;
    const int32_t* col;
    const uint32_t* cnt_arc;
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
    int32_t* retry_list;  // appended at retry_list[n_global + k]
    uint32_t cap_c_max;   // candidate table slots (on chip, or per-CTA scratch)
    uint32_t cap_u_max;   // label table slots
    uint8_t* gscratch;    // per-CTA table memory when tables are off chip
    size_t gscratch_stride;
};

__host__ __device__ inline size_t table_region_bytes(uint32_t cap_c, uint32_t cap_u) {
    const size_t a = (size_t)cap_u * 6, b = (size_t)cap_c * 8;
    return a > b ? a : b;
}

__host__ __device__ inline size_t level_table_bytes(uint32_t cap_c, uint32_t cap_u) {
    const size_t region = table_region_bytes(cap_c, cap_u);
    return (size_t)cap_c * 8 + ((region + 15) & ~(size_t)15) + (size_t)cap_c * 4;
}

__device__ __forceinline__ bool cand_insert(uint32_t* keys, unsigned long long* cnts, uint32_t cap, uint32_t limit,
                                            uint32_t h, uint64_t c, uint32_t ovf, int* nkeys, volatile int* abort_flag) {
    uint32_t slot = hash_hub(h) & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        uint32_t k = ((volatile uint32_t*)keys)[slot];
        if (k == kEmpty) {
            if (*abort_flag) return false;
            k = atomicCAS(&keys[slot], kEmpty, h);
            if (k == kEmpty) {
                if ((uint32_t)(atomicAdd(nkeys, 1) + 1) > limit) *abort_flag = 1;
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
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void label_insert(uint32_t* keys, uint16_t* lvl, uint32_t cap, uint32_t x, uint16_t l) {
    uint32_t slot = hash_hub(x) & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        const uint32_t k = atomicCAS(&keys[slot], kEmpty, x);
        if (k == kEmpty || k == x) {
            lvl[slot] = l;
            return;
        }
        slot = (slot + 1) & (cap - 1);
    }
}

__device__ __forceinline__ uint32_t label_lookup(const uint32_t* keys, const uint16_t* lvl, uint32_t cap, uint32_t x) {
    uint32_t slot = hash_hub(x) & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        const uint32_t k = keys[slot];
        if (k == x) return lvl[slot];
        if (k == kEmpty) return 0xFFFFu;
        slot = (slot + 1) & (cap - 1);
    }
    return 0xFFFFu;
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

template <bool kOffChip>
__global__ void __launch_bounds__(kLevelThreads) k_level(const LevelArgs A) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_item, s_nkeys, s_abort, s_nsurv, s_pos;
    __shared__ unsigned long long s_base;

    uint8_t* tables = kOffChip ? A.gscratch + (size_t)blockIdx.x * A.gscratch_stride : smem;
    unsigned long long* ccnt = (unsigned long long*)tables;
    const size_t region = table_region_bytes(A.cap_c_max, A.cap_u_max);
    uint8_t* reg = tables + (size_t)A.cap_c_max * 8;
    uint32_t* ukeys = (uint32_t*)reg;
    unsigned long long* sortbuf = (unsigned long long*)reg;
    uint32_t* ckeys = (uint32_t*)(reg + ((region + 15) & ~(size_t)15));

    const int tid = threadIdx.x;
    const int d = A.d;
    const int64_t n = A.n;
    auto tile = cg::tiled_partition<kProbeGroup>(cg::this_thread_block());
    const int group = tile.meta_group_rank();
    const int ngroups = kLevelThreads / kProbeGroup;
    const int warp = tid >> 5, lane = tid & 31;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(A.work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= A.n_items) break;
        const int64_t u = A.items[item];
        const int64_t raw = A.raw_u[u];
        const int64_t lab = A.lab_size[u];
        const uint32_t cap_u = label_cap_for(lab);
        const uint32_t cap_c = cand_cap_for(raw, u, A.cap_c_max);
        // Off chip the table is sized for every distinct hub; on chip a
        // vertex whose candidates overflow is handed to the off-chip pass.
        const uint32_t limit = (kOffChip || cap_c < A.cap_c_max) ? cap_c : cap_c - kLevelThreads - 64;
        uint16_t* ulvl = (uint16_t*)(reg + (size_t)cap_u * 4);

        for (uint32_t i = tid; i < cap_c; i += kLevelThreads) {
            ckeys[i] = kEmpty;
            ccnt[i] = 0ull;
        }
        for (uint32_t i = tid; i < cap_u; i += kLevelThreads) ukeys[i] = kEmpty;
        if (tid == 0) {
            s_nkeys = 0;
            s_abort = 0;
            s_nsurv = 0;
            s_pos = 0;
        }
        __syncthreads();

        // L_<d(u) as hub -> level (levels 0..d-1).
        for (int l = 0; l < d; ++l) {
            const uint64_t s = __ldg(A.seg + (int64_t)l * n + u);
            const uint32_t len = seg_len(s);
            const uint32_t* hs = A.hub_arena + seg_start(s);
            for (uint32_t i = tid; i < len; i += kLevelThreads)
                label_insert(ukeys, ulvl, cap_u, __ldg(hs + i) & kHubMask, (uint16_t)l);
        }

        // Pull: entries of L_{d-1}(v), v in N(u), with hub above u (a prefix),
        // merged per hub.
        {
            const int64_t a0 = A.rp[u], a1 = A.rp[u + 1];
            const uint64_t* segp = A.seg + (int64_t)(d - 1) * n;
            for (int64_t a = a0 + warp; a < a1; a += kLevelThreads / 32) {
                if (*(volatile int*)&s_abort) break;
                const uint32_t c = __ldg(A.cnt_arc + a);
                if (c == 0) continue;
                const uint64_t s = __ldg(segp + __ldg(A.col + a));
                const uint64_t st = seg_start(s);
                for (uint32_t i = lane; i < c; i += 32) {
                    const uint32_t hw = __ldg(A.hub_arena + st + i);
                    const uint64_t cc = __ldg((const unsigned long long*)A.cnt_arena + st + i);
                    if (!cand_insert(ckeys, ccnt, cap_c, limit, hw & kHubMask, cc, hw >> 31, &s_nkeys, &s_abort))
                        break;
                }
            }
        }
        __syncthreads();
        if (s_abort) {
            if (tid == 0) {
                const int p = atomicAdd(&A.stt->n_retry, 1);
                A.retry_list[p] = (int32_t)u;
                atomicMax(&A.stt->need_cap_c, (unsigned long long)cand_cap_for(raw, u, 1u << 30));
                atomicMax(&A.stt->need_cap_u, (unsigned long long)cap_u);
            }
            __syncthreads();
            continue;
        }

        // Prune rule 2, distance-bounded: a hub x of L_k(h) (k <= d-2) is a
        // witness iff x in L(u) at level <= d-1-k; k = 0 is x = h itself.
        for (uint32_t slot = group; slot < cap_c; slot += ngroups) {
            const uint32_t key = ckeys[slot];
            if (key == kEmpty) continue;
            const uint32_t h = key & kHubMask;
            bool pruned = label_lookup(ukeys, ulvl, cap_u, h) != 0xFFFFu;
            for (int k = 1; k <= d - 2 && !pruned; ++k) {
                const uint64_t s = __ldg(A.seg + (int64_t)k * n + h);
                const uint32_t len = seg_len(s);
                const uint32_t* xs = A.hub_arena + seg_start(s);
                const uint32_t thr = (uint32_t)(d - 1 - k);
                for (uint32_t b = 0; b < len && !pruned; b += kProbeGroup) {
                    const uint32_t i = b + tile.thread_rank();
                    bool hit = false;
                    if (i < len) hit = label_lookup(ukeys, ulvl, cap_u, __ldg(xs + i) & kHubMask) <= thr;
                    pruned = tile.any(hit);
                }
            }
            if (!pruned && tile.thread_rank() == 0) {
                ckeys[slot] = key | kMarkBit;
                atomicAdd(&s_nsurv, 1);
            }
        }
        __syncthreads();

        const int S = s_nsurv;
        if (S > 0) {
            const uint32_t P = pow2_ceil((uint64_t)S);
            for (uint32_t slot = tid; slot < cap_c; slot += kLevelThreads) {
                const uint32_t key = ckeys[slot];
                if (key != kEmpty && (key & kMarkBit)) {
                    const int p = atomicAdd(&s_pos, 1);
                    sortbuf[p] = ((unsigned long long)(key & kHubMask) << 32) | slot;
                }
            }
            for (uint32_t i = S + tid; i < P; i += kLevelThreads) sortbuf[i] = ~0ull;
            __syncthreads();
            block_bitonic_sort(sortbuf, P);
            if (tid == 0) {
                const unsigned long long base = atomicAdd(&A.stt->bump, (unsigned long long)S);
                if (base + S > A.arena_cap) atomicOr(&A.stt->arena_overflow, 1);
                s_base = base;
            }
            __syncthreads();
            const unsigned long long base = s_base;
            if (base + S <= A.arena_cap) {
                for (int i = tid; i < S; i += kLevelThreads) {
                    const uint32_t slot = (uint32_t)sortbuf[i];
                    const uint32_t key = ckeys[slot];
                    A.hub_arena[base + i] = (key & kHubMask) | (key & kOvfBit);
                    A.cnt_arena[base + i] = ccnt[slot];
                }
                if (tid == 0) A.seg_out[u] = seg_pack(base, (uint32_t)S);
            }
        }
        if (tid == 0) atomicAdd(&A.stt->unique_total, (unsigned long long)s_nkeys);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Finalize: merge each vertex's level segments into one hub-sorted label.

__global__ void k_fin_sizes(int64_t n, int levels, const uint64_t* __restrict__ seg, int64_t* __restrict__ off,
                            int32_t* __restrict__ big, int* n_big) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int64_t t = 0;
    for (int l = 0; l < levels; ++l) t += seg_len(seg[(int64_t)l * n + u]);
    off[u] = t;
    if (t > kFinSmemKeys) big[atomicAdd(n_big, 1)] = (int32_t)u;
}

struct FinArgs {
    int64_t n;
    int levels;
    const uint64_t* seg;
    const uint32_t* hub_arena;
    const uint64_t* cnt_arena;
    const unsigned long long* lvl_base;  // [levels+1] arena start of each level
    const int64_t* off;
    int32_t* hub;
    uint16_t* dist;
    uint64_t* cnt;
    const int32_t* list;  // vertices for the off-chip variant
    int n_list;
    int* work;
    unsigned long long* n_ovf;
    unsigned long long* gscratch;
    size_t gscratch_stride;  // keys per CTA
};

template <bool kOffChip>
__global__ void __launch_bounds__(kFinThreads) k_finalize(const FinArgs F) {
    extern __shared__ __align__(16) unsigned long long s_keys[];
    __shared__ int s_item;
    __shared__ unsigned long long s_ovf;
    unsigned long long* keys = kOffChip ? F.gscratch + (size_t)blockIdx.x * F.gscratch_stride : s_keys;
    const int tid = threadIdx.x;
    if (tid == 0) s_ovf = 0;
    for (int64_t it = kOffChip ? 0 : blockIdx.x;; it += kOffChip ? 0 : gridDim.x) {
        int64_t u;
        if (kOffChip) {
            if (tid == 0) s_item = atomicAdd(F.work, 1);
            __syncthreads();
            if (s_item >= F.n_list) break;
            u = F.list[s_item];
        } else {
            if (it >= F.n) break;
            u = it;
        }
        const int64_t o0 = F.off[u];
        const int64_t T = F.off[u + 1] - o0;
        if (!kOffChip && T > kFinSmemKeys) {
            __syncthreads();
            continue;
        }
        int64_t f0 = 0;
        for (int l = 0; l < F.levels; ++l) {
            const uint64_t s = F.seg[(int64_t)l * F.n + u];
            const uint32_t len = seg_len(s);
            const uint64_t st = seg_start(s);
            for (uint32_t i = tid; i < len; i += kFinThreads)
                keys[f0 + i] = ((unsigned long long)(__ldg(F.hub_arena + st + i) & kHubMask) << 40) | (st + i);
            f0 += len;
        }
        const uint32_t P = pow2_ceil((uint64_t)T);
        for (uint32_t i = (uint32_t)T + tid; i < P; i += kFinThreads) keys[i] = ~0ull;
        __syncthreads();
        block_bitonic_sort(keys, P);
        unsigned long long novf = 0;
        for (int64_t i = tid; i < T; i += kFinThreads) {
            const unsigned long long k = keys[i];
            const uint64_t pos = k & ((1ull << 40) - 1);
            int lo = 0, hi = F.levels;  // level = last l with lvl_base[l] <= pos
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (F.lvl_base[mid] <= pos) lo = mid; else hi = mid;
            }
            const uint32_t ovf = __ldg(F.hub_arena + pos) >> 31;
            novf += ovf;
            F.hub[o0 + i] = (int32_t)(k >> 40);
            F.dist[o0 + i] = (uint16_t)(lo | (ovf << 15));
            F.cnt[o0 + i] = __ldg((const unsigned long long*)F.cnt_arena + pos);
        }
        if (novf) atomicAdd(&s_ovf, novf);
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0 && s_ovf) atomicAdd(F.n_ovf, s_ovf);
}

// ---------------------------------------------------------------------------
// Host orchestration.

template <typename T>
static cudaError_t dalloc(T** p, size_t count, cudaStream_t st) {
    return cudaMallocAsync((void**)p, std::max<size_t>(count, 1) * sizeof(T), st);
}
template <typename T>
static void dfree(T*& p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
}

struct Builder {
    cudaStream_t st;
    int dev = 0, sms = 0;
    pspc_opts o;
    int64_t n = 0, arcs = 0;
    // staged inputs
    int64_t* rp_in = nullptr;
    int32_t* col_in = nullptr;
    int32_t* rank_in = nullptr;
    bool own_rp = false, own_col = false, own_rank = false;
    const int64_t* rp = nullptr;
    const int32_t* col = nullptr;
    const int32_t* rank = nullptr;
    // build state
    int64_t* rp_r = nullptr;
    int32_t* col_r = nullptr;
    int32_t* order = nullptr;
    uint32_t* hub_arena = nullptr;
    uint64_t* cnt_arena = nullptr;
    unsigned long long arena_cap = 0;
    uint64_t* seg = nullptr;
    int seg_levels_cap = 0;
    uint32_t* cnt_arc = nullptr;
    int64_t* raw_u = nullptr;
    int64_t* lab_size = nullptr;
    int32_t* items = nullptr;
    int32_t* glist = nullptr;
    LevelStatus* stt = nullptr;
    LevelStatus* hstt = nullptr;  // pinned
    int* err = nullptr;
    uint8_t* gscratch = nullptr;
    size_t gscratch_bytes = 0;
    std::vector<unsigned long long> lvl_base;
    Index out;
    cudaEvent_t ek0 = nullptr, ek1 = nullptr;
    float kernel_ms = 0.f;  // level-kernel time of the current level

    ~Builder() {
        dfree(rp_in, st);
        dfree(col_in, st);
        dfree(rank_in, st);
        dfree(rp_r, st);
        dfree(col_r, st);
        dfree(order, st);
        dfree(hub_arena, st);
        dfree(cnt_arena, st);
        dfree(seg, st);
        dfree(cnt_arc, st);
        dfree(raw_u, st);
        dfree(lab_size, st);
        dfree(items, st);
        dfree(glist, st);
        dfree(stt, st);
        dfree(err, st);
        dfree(gscratch, st);
        if (hstt) cudaFreeHost(hstt);
        if (ek0) cudaEventDestroy(ek0);
        if (ek1) cudaEventDestroy(ek1);
        cudaFree(out.rank);
        cudaFree(out.order);
        cudaFree(out.off);
        cudaFree(out.hub);
        cudaFree(out.dist);
        cudaFree(out.cnt);
        cudaStreamSynchronize(st);
    }

    int read_status() {
        PSPC_TRY_CUDA(cudaMemcpyAsync(hstt, stt, sizeof(LevelStatus), cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        return PSPC_OK;
    }

    int stage_inputs(const pspc_csr* g, const int32_t* rank_user) {
        n = g->n;
        if (is_device_ptr(g->row_ptr)) {
            rp = g->row_ptr;
            PSPC_TRY_CUDA(cudaMemcpyAsync(&arcs, g->row_ptr + n, 8, cudaMemcpyDeviceToHost, st));
            PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        } else {
            arcs = g->row_ptr[n];
            PSPC_TRY_CUDA(dalloc(&rp_in, n + 1, st));
            PSPC_TRY_CUDA(cudaMemcpyAsync(rp_in, g->row_ptr, (n + 1) * 8, cudaMemcpyHostToDevice, st));
            rp = rp_in;
        }
        if (arcs < 0 || arcs >= (int64_t)1 << 40) return PSPC_E_INVAL;
        if (arcs > 0 && !g->col) return PSPC_E_INVAL;
        if (arcs > 0 && is_device_ptr(g->col)) {
            col = g->col;
        } else {
            PSPC_TRY_CUDA(dalloc(&col_in, arcs, st));
            if (arcs)
                PSPC_TRY_CUDA(cudaMemcpyAsync(col_in, g->col, arcs * 4, cudaMemcpyHostToDevice, st));
            col = col_in;
        }
        if (is_device_ptr(rank_user)) {
            rank = rank_user;
        } else {
            PSPC_TRY_CUDA(dalloc(&rank_in, n, st));
            PSPC_TRY_CUDA(cudaMemcpyAsync(rank_in, rank_user, n * 4, cudaMemcpyHostToDevice, st));
            rank = rank_in;
        }
        return PSPC_OK;
    }

    int validate() {
        PSPC_TRY_CUDA(dalloc(&err, 1, st));
        PSPC_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        uint32_t* seen = nullptr;
        PSPC_TRY_CUDA(dalloc(&seen, n, st));
        PSPC_TRY_CUDA(cudaMemsetAsync(seen, 0, n * 4, st));
        k_check_rank<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rank, n, seen, err);
        k_check_rowptr<<<(unsigned)((n + 256) / 256), 256, 0, st>>>(rp, n, err);
        out.launches += 2;
        dfree(seen, st);
        int h = 0;
        PSPC_TRY_CUDA(cudaGetLastError());
        PSPC_TRY_CUDA(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        if (h) return PSPC_E_INVAL;
        k_check_arcs<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(rp, col, n, err);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        PSPC_TRY_CUDA(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        return h ? PSPC_E_INVAL : PSPC_OK;
    }

    int relabel() {
        PSPC_TRY_CUDA(dalloc(&rp_r, n + 1, st));
        PSPC_TRY_CUDA(dalloc(&col_r, arcs, st));
        PSPC_TRY_CUDA(dalloc(&order, n, st));
        k_deg_perm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rp, rank, n, rp_r, order);
        out.launches += 2;
        PSPC_TRY_CUDA(cudaGetLastError());
        int rc = exclusive_scan_i64(rp_r, n, st, &out.launches);
        if (rc) return rc;
        k_relabel_arcs<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(rp, col, rank, n, rp_r, col_r);
        return cuda_status(cudaGetLastError());
    }

    int grow_arena(unsigned long long need, unsigned long long keep) {
        unsigned long long cap = std::max<unsigned long long>(arena_cap * 2, need + need / 4);
        uint32_t* h2 = nullptr;
        uint64_t* c2 = nullptr;
        PSPC_TRY_CUDA(dalloc(&h2, cap, st));
        cudaError_t e = dalloc(&c2, cap, st);
        if (e != cudaSuccess) {
            dfree(h2, st);
            return cuda_status(e);
        }
        if (keep) {
            PSPC_TRY_CUDA(cudaMemcpyAsync(h2, hub_arena, keep * 4, cudaMemcpyDeviceToDevice, st));
            PSPC_TRY_CUDA(cudaMemcpyAsync(c2, cnt_arena, keep * 8, cudaMemcpyDeviceToDevice, st));
        }
        dfree(hub_arena, st);
        dfree(cnt_arena, st);
        hub_arena = h2;
        cnt_arena = c2;
        arena_cap = cap;
        return PSPC_OK;
    }

    int ensure_seg_levels(int need) {
        if (need <= seg_levels_cap) return PSPC_OK;
        int cap = std::max(need, seg_levels_cap ? seg_levels_cap * 2 : 16);
        uint64_t* s2 = nullptr;
        PSPC_TRY_CUDA(dalloc(&s2, (size_t)cap * n, st));
        if (seg)
            PSPC_TRY_CUDA(cudaMemcpyAsync(s2, seg, (size_t)seg_levels_cap * n * 8, cudaMemcpyDeviceToDevice, st));
        dfree(seg, st);
        seg = s2;
        seg_levels_cap = cap;
        return PSPC_OK;
    }

    int ensure_gscratch(size_t bytes) {
        if (bytes <= gscratch_bytes) return PSPC_OK;
        dfree(gscratch, st);
        gscratch_bytes = 0;
        PSPC_TRY_CUDA(dalloc(&gscratch, bytes, st));
        gscratch_bytes = bytes;
        return PSPC_OK;
    }

    int run_level_kernels(int d, uint32_t cap_c_smem, uint32_t cap_u_smem, size_t smem_bytes, int occ_smem,
                          int& n_offchip) {
        LevelArgs A;
        memset(&A, 0, sizeof(A));
        A.d = d;
        A.n = n;
        A.rp = rp_r;
        A.col = col_r;
        A.cnt_arc = cnt_arc;
        A.seg = seg;
        A.seg_out = seg + (int64_t)d * n;
        A.hub_arena = hub_arena;
        A.cnt_arena = cnt_arena;
        A.arena_cap = arena_cap;
        A.raw_u = raw_u;
        A.lab_size = lab_size;
        A.stt = stt;
        A.retry_list = glist + hstt->n_global;
        if (hstt->n_smem > 0) {
            A.items = items;
            A.n_items = hstt->n_smem;
            A.work = &stt->work_smem;
            A.cap_c_max = cap_c_smem;
            A.cap_u_max = cap_u_smem;
            const int grid = std::min(hstt->n_smem, sms * occ_smem);
            cudaEventRecord(ek0, st);
            k_level<false><<<grid, kLevelThreads, smem_bytes, st>>>(A);
            cudaEventRecord(ek1, st);
            out.launches += 1;
            PSPC_TRY_CUDA(cudaGetLastError());
        }
        int rc = read_status();
        if (rc) return rc;
        if (hstt->n_smem > 0) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ek0, ek1);
            kernel_ms += ms;
        }
        const int n_off = hstt->n_global + hstt->n_retry;
        n_offchip = n_off;
        if (n_off > 0) {
            const uint32_t cc = (uint32_t)std::max<unsigned long long>(hstt->need_cap_c, 64);
            const uint32_t cu = (uint32_t)std::max<unsigned long long>(hstt->need_cap_u, 64);
            const size_t stride = (level_table_bytes(cc, cu) + 255) & ~(size_t)255;
            const size_t budget = (size_t)4 << 30;
            int grid = (int)std::min<size_t>((size_t)n_off, std::max<size_t>(1, budget / stride));
            grid = std::min(grid, sms * 2);
            rc = ensure_gscratch(stride * grid);
            if (rc) return rc;
            A.items = glist;
            A.n_items = n_off;
            A.work = &stt->work_global;
            A.cap_c_max = cc;
            A.cap_u_max = cu;
            A.gscratch = gscratch;
            A.gscratch_stride = stride;
            cudaEventRecord(ek0, st);
            k_level<true><<<grid, kLevelThreads, 0, st>>>(A);
            cudaEventRecord(ek1, st);
            out.launches += 1;
            PSPC_TRY_CUDA(cudaGetLastError());
            rc = read_status();
            if (rc) return rc;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ek0, ek1);
            kernel_ms += ms;
        }
        return PSPC_OK;
    }

    int build_levels() {
        const uint32_t cap_c_smem = (uint32_t)o.cand_capacity;
        const uint32_t cap_u_smem = (uint32_t)o.label_capacity;
        const size_t smem_bytes = level_table_bytes(cap_c_smem, cap_u_smem);
        int smem_optin = 0;
        PSPC_TRY_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (smem_bytes + 1024 > (size_t)smem_optin) return PSPC_E_INVAL;  // tables must fit on chip
        PSPC_TRY_CUDA(cudaFuncSetAttribute(k_level<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes));
        int occ = 0;
        PSPC_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_level<false>, kLevelThreads, smem_bytes));
        if (occ < 1) return PSPC_E_INVAL;

        int rc = ensure_seg_levels(16);
        if (rc) return rc;
        const unsigned long long cap0 = o.arena_entries > 0 ? (unsigned long long)o.arena_entries
                                                            : (unsigned long long)(32 * arcs + 4 * n);
        rc = grow_arena(std::max<unsigned long long>(cap0, (unsigned long long)n + 1024), 0);
        if (rc) return rc;
        PSPC_TRY_CUDA(dalloc(&cnt_arc, arcs, st));
        PSPC_TRY_CUDA(dalloc(&raw_u, n, st));
        PSPC_TRY_CUDA(dalloc(&lab_size, n, st));
        PSPC_TRY_CUDA(dalloc(&items, n, st));
        PSPC_TRY_CUDA(dalloc(&glist, 2 * n, st));
        PSPC_TRY_CUDA(dalloc(&stt, 1, st));
        PSPC_TRY_CUDA(cudaMallocHost((void**)&hstt, sizeof(LevelStatus)));
        PSPC_TRY_CUDA(cudaMemsetAsync(lab_size, 0, n * 8, st));

        k_level0<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, hub_arena, cnt_arena, seg);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        lvl_base.assign({0ull, (unsigned long long)n});
        unsigned long long bump = (unsigned long long)n;
        cudaEvent_t e0, e1;
        PSPC_TRY_CUDA(cudaEventCreate(&e0));
        PSPC_TRY_CUDA(cudaEventCreate(&e1));
        PSPC_TRY_CUDA(cudaEventCreate(&ek0));
        PSPC_TRY_CUDA(cudaEventCreate(&ek1));
        int levels = 1;
        for (int d = 1;; ++d) {
            if (d > o.max_levels || d > kMaxDist) {
                rc = PSPC_E_DIST;
                break;
            }
            if ((rc = ensure_seg_levels(d + 1))) break;
            cudaEventRecord(e0, st);
            cudaMemsetAsync(seg + (int64_t)d * n, 0, n * 8, st);
            cudaMemsetAsync(stt, 0, sizeof(LevelStatus), st);
            cudaMemcpyAsync(&stt->bump, &lvl_base[d], 8, cudaMemcpyHostToDevice, st);
            k_cost<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(d, n, rp_r, col_r, seg + (int64_t)(d - 1) * n,
                                                                       hub_arena, cnt_arc, raw_u, lab_size, stt,
                                                                       cap_u_smem, glist);
            k_bucket_base<<<1, 32, 0, st>>>(stt);
            k_bucket_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, raw_u, lab_size, stt, cap_u_smem, items);
            out.launches += 3;
            if ((rc = cuda_status(cudaGetLastError()))) break;
            if ((rc = read_status())) break;
            if (hstt->n_active == 0) break;
            const long long raw_total = (long long)hstt->raw_total;
            const long long active_arcs = (long long)hstt->active_arcs;
            int n_off = 0;
            kernel_ms = 0.f;
            for (int attempt = 0;; ++attempt) {
                if ((rc = run_level_kernels(d, cap_c_smem, cap_u_smem, smem_bytes, occ, n_off))) break;
                if (!hstt->arena_overflow) break;
                kernel_ms = 0.f;
                if (attempt > 4) {
                    rc = PSPC_E_NOMEM;
                    break;
                }
                // Arena too small: grow it keeping levels < d, then redo level d.
                if ((rc = grow_arena(hstt->bump, lvl_base[d]))) break;
                cudaMemsetAsync(seg + (int64_t)d * n, 0, n * 8, st);
                LevelStatus keep = *hstt;
                keep.bump = lvl_base[d];
                keep.unique_total = 0;
                keep.n_retry = 0;
                keep.arena_overflow = 0;
                keep.work_smem = keep.work_global = 0;
                cudaMemcpyAsync(stt, &keep, sizeof(LevelStatus), cudaMemcpyHostToDevice, st);
                *hstt = keep;
            }
            if (rc) break;
            cudaEventRecord(e1, st);
            bump = hstt->bump;
            const long long added = (long long)(bump - lvl_base[d]);
            float ms = 0.f;
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            pspc_level_stat_t ls;
            ls.raw_candidates = raw_total;
            ls.unique_candidates = (long long)hstt->unique_total;
            ls.entries = added;
            ls.active_vertices = hstt->n_active;
            ls.active_arcs = active_arcs;
            ls.ms = ms;
            ls.kernel_ms = kernel_ms;
            out.lstats.push_back(ls);
            if (o.verbose)
                fprintf(stderr, "pspc level %d: raw %lld unique %lld entries %lld active %d (off-chip %d) %.3f ms\n",
                        d, raw_total, (long long)hstt->unique_total, added, hstt->n_active, n_off, ms);
            if (added == 0) break;
            lvl_base.push_back(bump);
            levels = d + 1;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        out.levels = levels;
        return PSPC_OK;
    }

    int finalize() {
        const int L = out.levels;
        PSPC_TRY_CUDA(cudaMalloc(&out.off, (n + 1) * 8));
        int32_t* big = nullptr;
        int* ctr = nullptr;  // [0] = n_big, [1] = work
        unsigned long long* d_lvl = nullptr;
        unsigned long long* n_ovf = nullptr;
        PSPC_TRY_CUDA(dalloc(&big, n, st));
        PSPC_TRY_CUDA(dalloc(&ctr, 2, st));
        PSPC_TRY_CUDA(dalloc(&d_lvl, lvl_base.size(), st));
        PSPC_TRY_CUDA(dalloc(&n_ovf, 1, st));
        PSPC_TRY_CUDA(cudaMemsetAsync(ctr, 0, 8, st));
        PSPC_TRY_CUDA(cudaMemsetAsync(n_ovf, 0, 8, st));
        PSPC_TRY_CUDA(cudaMemcpyAsync(d_lvl, lvl_base.data(), lvl_base.size() * 8, cudaMemcpyHostToDevice, st));
        k_fin_sizes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, L, seg, out.off, big, ctr);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        int rc = exclusive_scan_i64(out.off, n, st, &out.launches);
        if (rc) return rc;
        int hbig[2] = {0, 0};
        PSPC_TRY_CUDA(cudaMemcpyAsync(&out.entries, out.off + n, 8, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaMemcpyAsync(hbig, ctr, 8, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        const int64_t E = out.entries;
        PSPC_TRY_CUDA(cudaMalloc(&out.hub, std::max<int64_t>(E, 1) * 4));
        PSPC_TRY_CUDA(cudaMalloc(&out.dist, std::max<int64_t>(E, 1) * 2));
        PSPC_TRY_CUDA(cudaMalloc(&out.cnt, std::max<int64_t>(E, 1) * 8));
        FinArgs F;
        memset(&F, 0, sizeof(F));
        F.n = n;
        F.levels = L;
        F.seg = seg;
        F.hub_arena = hub_arena;
        F.cnt_arena = cnt_arena;
        F.lvl_base = d_lvl;
        F.off = out.off;
        F.hub = out.hub;
        F.dist = out.dist;
        F.cnt = out.cnt;
        F.n_ovf = n_ovf;
        const size_t fin_smem = (size_t)kFinSmemKeys * 8;
        PSPC_TRY_CUDA(cudaFuncSetAttribute(k_finalize<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fin_smem));
        const int grid = (int)std::min<int64_t>(n, (int64_t)sms * 8);
        k_finalize<false><<<grid, kFinThreads, fin_smem, st>>>(F);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        if (hbig[0] > 0) {
            // Labels longer than the on-chip buffer: sort them in device memory.
            int64_t maxT = 0;
            std::vector<int32_t> hb(hbig[0]);
            std::vector<int64_t> hoff(n + 1);
            PSPC_TRY_CUDA(cudaMemcpyAsync(hb.data(), big, hbig[0] * 4, cudaMemcpyDeviceToHost, st));
            PSPC_TRY_CUDA(cudaMemcpyAsync(hoff.data(), out.off, (n + 1) * 8, cudaMemcpyDeviceToHost, st));
            PSPC_TRY_CUDA(cudaStreamSynchronize(st));
            for (int32_t u : hb) maxT = std::max(maxT, hoff[u + 1] - hoff[u]);
            const size_t stride = pow2_ceil((uint64_t)maxT);
            const int g2 = std::min(hbig[0], sms);
            if ((rc = ensure_gscratch(stride * 8 * g2))) return rc;
            F.list = big;
            F.n_list = hbig[0];
            F.work = ctr + 1;
            F.gscratch = (unsigned long long*)gscratch;
            F.gscratch_stride = stride;
            k_finalize<true><<<g2, kFinThreads, 0, st>>>(F);
            out.launches += 1;
            PSPC_TRY_CUDA(cudaGetLastError());
        }
        unsigned long long hovf = 0;
        PSPC_TRY_CUDA(cudaMemcpyAsync(&hovf, n_ovf, 8, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        out.overflow_entries = (int64_t)hovf;
        dfree(big, st);
        dfree(ctr, st);
        dfree(d_lvl, st);
        dfree(n_ovf, st);
        // the index keeps its own copy of the order
        PSPC_TRY_CUDA(cudaMalloc(&out.rank, n * 4));
        PSPC_TRY_CUDA(cudaMalloc(&out.order, n * 4));
        PSPC_TRY_CUDA(cudaMemcpyAsync(out.rank, rank, n * 4, cudaMemcpyDeviceToDevice, st));
        PSPC_TRY_CUDA(cudaMemcpyAsync(out.order, order, n * 4, cudaMemcpyDeviceToDevice, st));
        return PSPC_OK;
    }
};

}  // namespace pspc

using namespace pspc;

static void fill_defaults(pspc_opts& o, const pspc_opts* user) {
    memset(&o, 0, sizeof(o));
    if (user) o = *user;
    if (o.cand_capacity <= 0) o.cand_capacity = 4096;
    if (o.label_capacity <= 0) o.label_capacity = 8192;
    if (o.max_levels <= 0) o.max_levels = kMaxDist;
}

static bool pow2_in(int32_t v, int32_t lo, int32_t hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

extern "C" int pspc_build(const pspc_csr* g, const int32_t* rank, const pspc_opts* opts, pspc_index** out,
                          void* stream) {
    if (!out) return PSPC_E_INVAL;
    *out = nullptr;
    if (!g || !rank || !g->row_ptr) return PSPC_E_INVAL;
    if (g->n < 1 || g->n > kMaxVertices) return PSPC_E_INVAL;
    Builder B;
    B.st = (cudaStream_t)stream;
    fill_defaults(B.o, opts);
    if (!pow2_in(B.o.cand_capacity, 1024, 16384) || !pow2_in(B.o.label_capacity, 1024, 16384)) return PSPC_E_INVAL;
    PSPC_TRY_CUDA(cudaGetDevice(&B.dev));
    PSPC_TRY_CUDA(cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, B.dev));
    cudaEvent_t t0, t1;
    PSPC_TRY_CUDA(cudaEventCreate(&t0));
    PSPC_TRY_CUDA(cudaEventCreate(&t1));
    cudaEventRecord(t0, B.st);
    int rc = B.stage_inputs(g, rank);
    if (!rc) rc = B.validate();
    if (!rc) rc = B.relabel();
    if (!rc) {
        B.out.n = B.n;
        B.out.arcs = B.arcs;
        B.out.device = B.dev;
        rc = B.build_levels();
    }
    if (!rc) rc = B.finalize();
    if (!rc) {
        cudaEventRecord(t1, B.st);
        cudaError_t e = cudaEventSynchronize(t1);
        if (e != cudaSuccess) rc = cuda_status(e);
        cudaEventElapsedTime(&B.out.build_ms, t0, t1);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc) {
        cudaGetLastError();
        return rc;
    }
    pspc_index* h = new (std::nothrow) pspc_index;
    if (!h) return PSPC_E_NOMEM;
    h->ix = B.out;
    // ownership of the index arrays moves to h
    B.out.rank = B.out.order = nullptr;
    B.out.off = nullptr;
    B.out.hub = nullptr;
    B.out.dist = nullptr;
    B.out.cnt = nullptr;
    *out = h;
    return PSPC_OK;
}
