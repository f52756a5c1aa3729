// pspc_build: construction of the SPC 2-hop hub-label index (PSPC, arXiv
// 2212.00977) on one GPU -- input checks, relabelling by rank, the level
// loop of the pull construction (Theorem "Distance Dependency": level d
// depends only on levels < d, so levels are built one after another, each
// fully parallel over vertices), and the final merge of each vertex's level
// segments into one hub-sorted label (the order of Table "Shortest Path
// Counting Labels").
//
// Vertices are relabelled so that id = rank (0 = highest). Level d of every
// vertex is one hub-sorted segment of a label arena: a hub word (bits 0-23
// hub, bit 31 overflow flag) and a uint64 count; the distance is the level.
// The per-level kernels live in pspc_level.cu, the landmark BFS in
// pspc_landmark.cu, and the 1-shell reduction in pspc_shell.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pspc_internal.cuh"
#include "pspc_level.cuh"
#include "pspc_shell.cuh"

namespace pspc {

constexpr int kFinThreads = 256;
constexpr int kFinSmemKeys = 8192;  // labels up to this size are merged on chip

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

// Thread per arc u->v: ids in range, no self-loop, rows strictly ascending,
// and the reverse arc v->u exists (binary search in the row of v).
__global__ void k_check_arcs(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ arc_src, int64_t arcs, int64_t n, int* err) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= arcs) return;
    const int32_t u = arc_src[a];
    const int32_t v = col[a];
    if (v < 0 || v >= n || v == u || (a + 1 < rp[u + 1] && col[a + 1] <= v)) {
        atomicOr(err, 1);
        return;
    }
    int64_t lo = rp[v], hi = rp[v + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < u) lo = mid + 1; else hi = mid;
    }
    if (lo == rp[v + 1] || col[lo] != u) atomicOr(err, 1);
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

// Rank-space rows sorted ascending (highest-ranked neighbours first). Rows
// of up to 32 arcs are sorted by one warp in registers, up to kRowSmem on
// chip by the block; longer rows are listed for k_sort_big_rows.
constexpr int kRowThreads = 128;
constexpr int kRowSmem = 4096;

__global__ void __launch_bounds__(kRowThreads) k_sort_rows(const int64_t* __restrict__ rp, int32_t* __restrict__ col,
                                                           int64_t n, int32_t* __restrict__ big, int* n_big) {
    __shared__ int32_t s[kRowSmem];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t a0 = rp[r];
        const int64_t deg = rp[r + 1] - a0;
        if (deg <= 1) continue;
        if (deg <= 32) {
            if (tid < 32) {
                int32_t v = lane < deg ? col[a0 + lane] : INT32_MAX;
                for (int k = 2; k <= 32; k <<= 1)
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        const int32_t w = __shfl_xor_sync(0xFFFFFFFFu, v, j);
                        const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
                        v = keep_min ? min(v, w) : max(v, w);
                    }
                if (lane < deg) col[a0 + lane] = v;
            }
        } else if (deg <= kRowSmem) {
            const uint32_t P = pow2_ceil((uint64_t)deg);
            for (uint32_t i = tid; i < P; i += kRowThreads) s[i] = i < deg ? col[a0 + i] : INT32_MAX;
            __syncthreads();
            for (uint32_t k = 2; k <= P; k <<= 1)
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    for (uint32_t i = tid; i < P; i += kRowThreads) {
                        const uint32_t ixj = i ^ j;
                        if (ixj > i) {
                            const int32_t x = s[i], y = s[ixj];
                            if ((x > y) == ((i & k) == 0)) {
                                s[i] = y;
                                s[ixj] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            for (uint32_t i = tid; i < deg; i += kRowThreads) col[a0 + i] = s[i];
            __syncthreads();
        } else if (tid == 0) {
            big[atomicAdd(n_big, 1)] = (int32_t)r;
        }
    }
}

// Long rows: ids in a row are distinct, so a bitmap over [0, n) in device
// scratch, read back in order with a popcount prefix, sorts the row.
__global__ void __launch_bounds__(kRowThreads) k_sort_big_rows(const int64_t* __restrict__ rp, int32_t* __restrict__ col,
                                                               int64_t n, const int32_t* __restrict__ big, int n_big,
                                                               uint32_t* __restrict__ scratch) {
    __shared__ long long s_run[kRowThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t W = (uint32_t)((n + 31) >> 5);
    uint32_t* bm = scratch + (size_t)blockIdx.x * W;
    for (int b = blockIdx.x; b < n_big; b += gridDim.x) {
        const int64_t r = big[b];
        const int64_t a0 = rp[r], deg = rp[r + 1] - a0;
        for (uint32_t i = tid; i < W; i += kRowThreads) bm[i] = 0u;
        __syncthreads();
        for (int64_t i = tid; i < deg; i += kRowThreads) {
            const int32_t v = col[a0 + i];
            atomicOr(&bm[v >> 5], 1u << (v & 31));
        }
        __syncthreads();
        const uint32_t per = (W + kRowThreads - 1) / kRowThreads;
        const uint32_t w0 = tid * per, w1 = w0 + per < W ? w0 + per : W;
        long long cnt = 0;
        for (uint32_t i = w0; i < w1; ++i) cnt += __popc(bm[i]);
        long long incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_run[warp] = incl;
        __syncthreads();
        long long run = incl - cnt;
        for (int w = 0; w < warp; ++w) run += s_run[w];
        for (uint32_t i = w0; i < w1; ++i) {
            uint32_t bits = bm[i];
            while (bits) {
                const int bit = __ffs(bits) - 1;
                bits &= bits - 1;
                col[a0 + run++] = (int32_t)(i * 32 + bit);
            }
        }
        __syncthreads();
    }
}

// Level 1 without a pull: L_1(u) is the set of neighbours ranked above u,
// each with one path -- the prefix of u's sorted row below u.
__global__ void k_level1_counts(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                                int64_t* __restrict__ len1, unsigned long long* active) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int64_t lo = rp[u], hi = rp[u + 1];
    const int64_t a0 = lo;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < u) lo = mid + 1; else hi = mid;
    }
    len1[u] = lo - a0;
    if (lo > a0) {
        atomicAdd(&active[0], 1ull);
        atomicAdd(&active[1], (unsigned long long)(rp[u + 1] - a0));
    }
}

__global__ void k_level1_write(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                               const int64_t* __restrict__ pos1, unsigned long long base,
                               uint32_t* __restrict__ hub_arena, uint64_t* __restrict__ cnt_arena,
                               uint64_t* __restrict__ seg1, int64_t* __restrict__ lab_size) {
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    const int64_t p0 = pos1[u], len = pos1[u + 1] - p0;
    const int64_t a0 = rp[u];
    for (int64_t i = lane; i < len; i += 32) {
        hub_arena[base + p0 + i] = (uint32_t)col[a0 + i];
        cnt_arena[base + p0 + i] = 1ull;
    }
    if (lane == 0) {
        seg1[u] = len ? seg_pack(base + p0, (uint32_t)len) : 0ull;
        lab_size[u] = 1;  // L_<2(u) before level 1 is added: the level-0 entry
    }
}

// Batches: the disjoint union of k graphs. Graph g's vertex v becomes
// vbase_g + v, its arcs shift by abase_g, and its order maps to ranks
// vbase_g + rank_g(v), so every graph keeps its own order and occupies one
// contiguous rank range (whose start is the component base of its vertices).
struct GraphDesc {
    int64_t n, vbase, abase;
    const int64_t* rp;
    const int32_t* col;
    const int32_t* rank;
};

__global__ void k_union(const GraphDesc* __restrict__ G, int k, int64_t N, int64_t A, int64_t* __restrict__ rp_u,
                        int32_t* __restrict__ col_u, int32_t* __restrict__ rank_u, int32_t* __restrict__ comp_base,
                        int* err) {
    for (int g = blockIdx.x; g < k; g += gridDim.x) {
        const GraphDesc d = G[g];
        for (int64_t i = threadIdx.x; i < d.n; i += blockDim.x) {
            rp_u[d.vbase + i] = d.rp[i] + d.abase;
            const int32_t r = d.rank[i];
            if (r < 0 || r >= d.n) atomicOr(err, 1);
            rank_u[d.vbase + i] = (int32_t)(d.vbase + r);
            comp_base[d.vbase + i] = (int32_t)d.vbase;
        }
        const int64_t arcs = d.rp[d.n] - d.rp[0];
        if (d.rp[0] != 0) atomicOr(err, 1);
        for (int64_t j = threadIdx.x; j < arcs; j += blockDim.x) {
            const int32_t v = d.col[j];
            col_u[d.abase + j] = (v < 0 || v >= d.n) ? -1 : (int32_t)(v + d.vbase);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rp_u[N] = A;
}

// Level 0: L_0(v) = {(v, 0, 1)}.
__global__ void k_level0(int64_t n, uint32_t* hub_arena, uint64_t* cnt_arena, uint64_t* seg0) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    hub_arena[v] = (uint32_t)v;
    cnt_arena[v] = 1ull;
    seg0[v] = seg_pack((uint64_t)v, 1u);
}

// Bitonic sort of buf[0..P) (P a power of two) by the whole block.
__device__ void fin_bitonic_sort(unsigned long long* buf, uint32_t P) {
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
// Finalize: merge each vertex's level segments into one hub-sorted label.

// Label sizes (into off, scanned later), the vertices whose labels need the
// off-chip finalize, and the largest label size (max_lab, by warp maxima).
__global__ void k_fin_sizes(int64_t n, int levels, const uint64_t* __restrict__ seg, int64_t* __restrict__ off,
                            int32_t* __restrict__ big, int* n_big, unsigned long long* max_lab) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t t = 0;
    if (u < n) {
        for (int l = 0; l < levels; ++l) t += seg_len(seg[(int64_t)l * n + u]);
        off[u] = t;
        if (t > kFinSmemKeys) big[atomicAdd(n_big, 1)] = (int32_t)u;
    }
    unsigned long long m = (unsigned long long)t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xFFFFFFFFu, m, o);
        m = x > m ? x : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(max_lab, m);
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
    const int32_t* comp_base;  // batches: first id of each vertex's graph (NULL: 0)
    uint32_t rank_words;       // k_finalize_rank: bitmap words per CTA
    int merge_keys;            // k_finalize_merge: hub words on chip (longer labels are skipped)
};

// Exclusive scan of one value per thread of a kFinThreads block into pre[];
// returns the total. Ends with a barrier.
__device__ int fin_block_scan(uint32_t v, int* pre, int* wtot) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int incl = (int)v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kFinThreads / 32; ++w) {
        before += w < warp ? wtot[w] : 0;
        total += wtot[w];
    }
    pre[tid] = before + incl - (int)v;
    __syncthreads();
    return total;
}

template <bool kOffChip>
__global__ void __launch_bounds__(kFinThreads) k_finalize(const FinArgs F) {
    extern __shared__ __align__(16) unsigned long long s_keys[];
    __shared__ int s_item;
    __shared__ unsigned long long s_ovf;
    __shared__ int s_pre[kFinThreads];
    __shared__ int s_wtot[kFinThreads / 32];
    __shared__ uint64_t s_st[kFinThreads];
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
        // Level descriptors are read kFinThreads at a time (one per thread)
        // and prefix-summed, so that a vertex of a high-diameter graph does
        // not walk its levels one by one.
        int64_t f0 = 0;
        for (int l0 = 0; l0 < F.levels; l0 += kFinThreads) {
            const int l = l0 + tid;
            const uint64_t s = l < F.levels ? F.seg[(int64_t)l * F.n + u] : 0ull;
            const int total = fin_block_scan(seg_len(s), s_pre, s_wtot);
            s_st[tid] = seg_start(s);
            __syncthreads();
            for (int i = tid; i < total; i += kFinThreads) {
                int lo = 0, hi = kFinThreads - 1;  // last level j of the chunk with s_pre[j] <= i
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_pre[mid] <= i) lo = mid; else hi = mid - 1;
                }
                const uint64_t pos = s_st[lo] + (uint64_t)(i - s_pre[lo]);
                keys[f0 + i] = ((unsigned long long)(__ldg(F.hub_arena + pos) & kHubMask) << 40) | pos;
            }
            f0 += total;
            __syncthreads();
        }
        const uint32_t P = pow2_ceil((uint64_t)T);
        for (uint32_t i = (uint32_t)T + tid; i < P; i += kFinThreads) keys[i] = ~0ull;
        __syncthreads();
        fin_bitonic_sort(keys, P);
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

// Many levels: each level segment of a vertex is hub-sorted, and its hubs
// are distinct ids in [cbase, u] (ranked above u, or u itself). The final
// slot of an entry is the number of the vertex's hubs below it: a bitmap of
// them over ids cbase..u on chip, its popcount prefix, then every entry is
// written at its rank, with its level as the distance and its count read
// in segment order (no sort, no gather of counts, no level search).
constexpr uint32_t kFinRankWords = 12288;  // ids up to 393,216 per graph

__global__ void __launch_bounds__(kFinThreads) k_finalize_rank(const FinArgs F) {
    extern __shared__ __align__(16) uint32_t s_bits[];  // rank_words bitmap words, then their prefixes
    __shared__ int s_pre[kFinThreads];
    __shared__ int s_wtot[kFinThreads / 32];
    __shared__ uint64_t s_st[kFinThreads];
    __shared__ unsigned long long s_ovf;
    const int tid = threadIdx.x;
    if (tid == 0) s_ovf = 0;
    uint32_t* bits = s_bits;
    uint32_t* wp = s_bits + F.rank_words;
    unsigned long long novf = 0;
    for (int64_t u = blockIdx.x; u < F.n; u += gridDim.x) {
        const int64_t o0 = F.off[u];
        const uint32_t cb = F.comp_base ? (uint32_t)__ldg(F.comp_base + u) : 0u;
        const uint32_t W = (uint32_t)((u - cb) >> 5) + 1;
        for (uint32_t i = tid; i < W; i += kFinThreads) bits[i] = 0u;
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {  // popcount prefix of the bitmap, a run of words per thread
                const uint32_t per = (W + kFinThreads - 1) / kFinThreads;
                const uint32_t w0 = tid * per < W ? tid * per : W, w1 = w0 + per < W ? w0 + per : W;
                uint32_t v = 0;
                for (uint32_t i = w0; i < w1; ++i) v += __popc(bits[i]);
                fin_block_scan(v, s_pre, s_wtot);
                uint32_t run = (uint32_t)s_pre[tid];
                for (uint32_t i = w0; i < w1; ++i) {
                    wp[i] = run;
                    run += __popc(bits[i]);
                }
                __syncthreads();
            }
            // the level descriptors kFinThreads at a time, prefix-summed
            for (int l0 = 0; l0 < F.levels; l0 += kFinThreads) {
                const int l = l0 + tid;
                const uint64_t sd = l < F.levels ? F.seg[(int64_t)l * F.n + u] : 0ull;
                const int total = fin_block_scan(seg_len(sd), s_pre, s_wtot);
                s_st[tid] = seg_start(sd);
                __syncthreads();
                for (int i = tid; i < total; i += kFinThreads) {
                    int lo = 0, hi = kFinThreads - 1;  // last level j of the chunk with s_pre[j] <= i
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_pre[mid] <= i) lo = mid; else hi = mid - 1;
                    }
                    const uint64_t pos = s_st[lo] + (uint64_t)(i - s_pre[lo]);
                    const uint32_t hw = __ldg(F.hub_arena + pos);
                    const uint32_t r = (hw & kHubMask) - cb;
                    if (pass == 0) {
                        atomicOr(&bits[r >> 5], 1u << (r & 31));
                    } else {
                        const uint32_t rank = wp[r >> 5] + __popc(bits[r >> 5] & ((1u << (r & 31)) - 1u));
                        const uint32_t ovf = hw >> 31;
                        novf += ovf;
                        F.hub[o0 + rank] = (int32_t)(hw & kHubMask);
                        F.dist[o0 + rank] = (uint16_t)((uint32_t)(l0 + lo) | (ovf << 15));
                        F.cnt[o0 + rank] = __ldg((const unsigned long long*)F.cnt_arena + pos);
                    }
                }
                __syncthreads();
            }
        }
    }
    if (novf) atomicAdd(&s_ovf, novf);
    __syncthreads();
    if (tid == 0 && s_ovf) atomicAdd(F.n_ovf, s_ovf);
}

// Few levels: every level segment of a vertex is already hub-sorted, so the
// final slot of an entry is its index in its own segment plus, for every
// other level, the number of hubs there that rank above it (binary search
// over an on-chip copy of the vertex's hubs). Hubs are unique per vertex.
constexpr int kFinMergeLevels = 16;

__global__ void __launch_bounds__(kFinThreads) k_finalize_merge(const FinArgs F) {
    extern __shared__ __align__(16) uint32_t s_hub[];  // F.merge_keys hub words
    __shared__ unsigned long long s_st[kFinMergeLevels];
    __shared__ int s_off[kFinMergeLevels + 1];
    __shared__ unsigned long long s_ovf;
    const int tid = threadIdx.x;
    const int L = F.levels;
    if (tid == 0) s_ovf = 0;
    unsigned long long novf = 0;
    // every vertex, or (F.list) the long labels with a larger on-chip buffer
    const int64_t items = F.list ? (int64_t)F.n_list : F.n;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t u = F.list ? (int64_t)F.list[it] : it;
        const int64_t o0 = F.off[u];
        const int T = (int)(F.off[u + 1] - o0);
        if (T > F.merge_keys) continue;  // uniform: placed by a later launch
        if (T == 1) {  // only (u, 0, 1): an isolated vertex, no merge
            if (tid == 0) {
                const uint64_t s = __ldg(F.seg + u);
                F.hub[o0] = (int32_t)(__ldg(F.hub_arena + seg_start(s)) & kHubMask);
                F.dist[o0] = 0;
                F.cnt[o0] = __ldg((const unsigned long long*)F.cnt_arena + seg_start(s));
            }
            continue;
        }
        if (tid < L) {
            const uint64_t s = __ldg(F.seg + (int64_t)tid * F.n + u);
            s_st[tid] = seg_start(s);
            s_off[tid + 1] = (int)seg_len(s);
        }
        __syncthreads();
        if (tid == 0) {
            s_off[0] = 0;
            for (int l = 0; l < L; ++l) s_off[l + 1] += s_off[l];
        }
        __syncthreads();
        for (int i = tid; i < T; i += kFinThreads) {
            int l = 0;
            while (s_off[l + 1] <= i) ++l;
            s_hub[i] = __ldg(F.hub_arena + s_st[l] + (i - s_off[l]));
        }
        __syncthreads();
        for (int i = tid; i < T; i += kFinThreads) {
            int l = 0;
            while (s_off[l + 1] <= i) ++l;
            const uint32_t w = s_hub[i];
            const uint32_t h = w & kHubMask;
            const unsigned long long c = __ldg((const unsigned long long*)F.cnt_arena + s_st[l] + (i - s_off[l]));
            int pos = i - s_off[l];
            for (int l2 = 0; l2 < L; ++l2) {
                if (l2 == l) continue;
                int lo = s_off[l2], hi = s_off[l2 + 1];
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if ((s_hub[mid] & kHubMask) < h) lo = mid + 1; else hi = mid;
                }
                pos += lo - s_off[l2];
            }
            const uint32_t ovf = w >> 31;
            novf += ovf;
            F.hub[o0 + pos] = (int32_t)h;
            F.dist[o0 + pos] = (uint16_t)(l | (ovf << 15));
            F.cnt[o0 + pos] = c;
        }
        __syncthreads();
    }
    if (novf) atomicAdd(&s_ovf, novf);
    __syncthreads();
    if (tid == 0 && s_ovf) atomicAdd(F.n_ovf, s_ovf);
}

// ---------------------------------------------------------------------------
// Host orchestration.

template <typename T>
static cudaError_t dalloc(T** p, size_t count, cudaStream_t st) {
    return dev_alloc((void**)p, std::max<size_t>(count, 1) * sizeof(T), st);
}
template <typename T>
static void dfree(T*& p, cudaStream_t st) {
    dev_free(p, st);
    p = nullptr;
}

struct LevelPlan {
    int map_kind = kMapBitmap;
    uint32_t cap_c = 0, cap_u = 0, bm_words = 0;
    int64_t label_limit = 0;
    size_t smem_bytes = 0;
    int occupancy = 0;
    size_t light_smem_bytes = 0;  // light vertices: kLightThreads CTAs, segment-search map
    int light_occupancy = 0;
    int micro_occupancy = 0;      // tiny vertices: the warp-per-vertex kernel
};

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
    uint32_t* arc_lo = nullptr;    // first pulled entry per arc (dense-prefix skip)
    int32_t* hpre = nullptr;       // dense prefix per vertex
    bool skip_prefix = false;      // the current level uses arc_lo
    bool prefix_pays = true;       // the last level that skipped saved enough to go on
    int64_t* push_off = nullptr;   // push paradigm: bucket offset per arc [arcs+1]
    uint32_t* push_hub = nullptr;  // push paradigm: the buckets (hub words, counts)
    uint64_t* push_cnt = nullptr;
    int64_t push_cap = 0;
    bool push_level = false;       // the current level runs from the buckets
    int32_t* arc_src = nullptr;
    int32_t* comp_base = nullptr;  // batches: first rank-space id of each vertex's graph
    int64_t max_comp = 0;          // largest graph (bits per level bitmap)
    int64_t* raw_u = nullptr;
    int64_t* lab_size = nullptr;
    int32_t* items = nullptr;
    int32_t* glist = nullptr;
    LevelStatus* stt = nullptr;
    LevelStatus hs;               // host copy of the level status
    LevelStatus* hstt = &hs;
    int* err = nullptr;
    uint8_t* gscratch = nullptr;
    size_t gscratch_bytes = 0;
    std::vector<unsigned long long> lvl_base;
    Index out;
    cudaEvent_t ek0 = nullptr, ek1 = nullptr;
    float kernel_ms = 0.f;  // level-kernel time of the current level
    float offchip_ms = 0.f; // of which the off-chip variant
    int smem_optin = 0;

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
        dfree(arc_lo, st);
        dfree(hpre, st);
        dfree(push_off, st);
        dfree(push_hub, st);
        dfree(push_cnt, st);
        dfree(arc_src, st);
        dfree(comp_base, st);
        dfree(raw_u, st);
        dfree(lab_size, st);
        dfree(items, st);
        dfree(glist, st);
        dfree(stt, st);
        dfree(err, st);
        dfree(gscratch, st);
        if (ek0) cudaEventDestroy(ek0);
        if (ek1) cudaEventDestroy(ek1);
        dfree(out.rank, st);
        dfree(out.order, st);
        dfree(out.off, st);
        dfree(out.hub, st);
        dfree(out.dist, st);
        dfree(out.cnt, st);
        dfree(out.lmk, st);
        cudaStreamSynchronize(st);
    }

    int read_status() {
        PSPC_TRY_CUDA(cudaMemcpyAsync(hstt, stt, sizeof(LevelStatus), cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        return PSPC_OK;
    }

    int stage_inputs(const pspc_csr* g, const int32_t* rank_user) {
        n = g->n;
        max_comp = n;
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

    // Assembles the disjoint union of k graphs (host or device arrays) in
    // device memory; rank and CSR checks then run on the union.
    int stage_batch(const pspc_graph* graphs, int32_t k) {
        std::vector<GraphDesc> desc(k);
        std::vector<int64_t*> rp_tmp(k, nullptr);
        std::vector<int32_t*> col_tmp(k, nullptr), rank_tmp(k, nullptr);
        int64_t N = 0, A = 0;
        int rc = PSPC_OK;
        for (int32_t g = 0; g < k && rc == PSPC_OK; ++g) {
            const pspc_graph& G = graphs[g];
            if (G.n < 1 || !G.row_ptr || !G.rank) {
                rc = PSPC_E_INVAL;
                break;
            }
            int64_t arcs_g = 0;
            const bool dev_rp = is_device_ptr(G.row_ptr);
            if (dev_rp) {
                cudaError_t e = cudaMemcpy(&arcs_g, G.row_ptr + G.n, 8, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) return cuda_status(e);
            } else {
                arcs_g = G.row_ptr[G.n];
            }
            if (arcs_g < 0 || (arcs_g > 0 && !G.col)) {
                rc = PSPC_E_INVAL;
                break;
            }
            desc[g].n = G.n;
            desc[g].vbase = N;
            desc[g].abase = A;
            desc[g].rp = G.row_ptr;
            desc[g].col = G.col;
            desc[g].rank = G.rank;
            if (!dev_rp) {
                PSPC_TRY_CUDA(dalloc(&rp_tmp[g], G.n + 1, st));
                PSPC_TRY_CUDA(cudaMemcpyAsync(rp_tmp[g], G.row_ptr, (G.n + 1) * 8, cudaMemcpyHostToDevice, st));
                desc[g].rp = rp_tmp[g];
            }
            if (arcs_g > 0 && !is_device_ptr(G.col)) {
                PSPC_TRY_CUDA(dalloc(&col_tmp[g], arcs_g, st));
                PSPC_TRY_CUDA(cudaMemcpyAsync(col_tmp[g], G.col, arcs_g * 4, cudaMemcpyHostToDevice, st));
                desc[g].col = col_tmp[g];
            }
            if (!is_device_ptr(G.rank)) {
                PSPC_TRY_CUDA(dalloc(&rank_tmp[g], G.n, st));
                PSPC_TRY_CUDA(cudaMemcpyAsync(rank_tmp[g], G.rank, G.n * 4, cudaMemcpyHostToDevice, st));
                desc[g].rank = rank_tmp[g];
            }
            N += G.n;
            A += arcs_g;
            max_comp = std::max(max_comp, G.n);
            if (N > kMaxVertices || A >= ((int64_t)1 << 40)) rc = PSPC_E_INVAL;
        }
        if (rc == PSPC_OK) {
            n = N;
            arcs = A;
            GraphDesc* d_desc = nullptr;
            PSPC_TRY_CUDA(dalloc(&rp_in, n + 1, st));
            PSPC_TRY_CUDA(dalloc(&col_in, arcs, st));
            PSPC_TRY_CUDA(dalloc(&rank_in, n, st));
            PSPC_TRY_CUDA(dalloc(&comp_base, n, st));
            PSPC_TRY_CUDA(dalloc(&err, 1, st));
            PSPC_TRY_CUDA(dalloc(&d_desc, k, st));
            PSPC_TRY_CUDA(cudaMemcpyAsync(d_desc, desc.data(), k * sizeof(GraphDesc), cudaMemcpyHostToDevice, st));
            PSPC_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
            k_union<<<std::min(k, sms * 8), 256, 0, st>>>(d_desc, k, n, arcs, rp_in, col_in, rank_in, comp_base, err);
            out.launches += 1;
            PSPC_TRY_CUDA(cudaGetLastError());
            int h = 0;
            PSPC_TRY_CUDA(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st));
            PSPC_TRY_CUDA(cudaStreamSynchronize(st));
            dfree(d_desc, st);
            if (h) rc = PSPC_E_INVAL;
            rp = rp_in;
            col = col_in;
            rank = rank_in;
        }
        for (int32_t g = 0; g < k; ++g) {
            dfree(rp_tmp[g], st);
            dfree(col_tmp[g], st);
            dfree(rank_tmp[g], st);
        }
        return rc;
    }

    int validate() {
        if (!err) PSPC_TRY_CUDA(dalloc(&err, 1, st));
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
        PSPC_TRY_CUDA(dalloc(&arc_src, arcs, st));
        if (arcs > 0) {
            PSPC_TRY_CUDA(launch_arc_src(rp, n, arc_src, st));
            k_check_arcs<<<(unsigned)((arcs + 255) / 256), 256, 0, st>>>(rp, col, arc_src, arcs, n, err);
            out.launches += 2;
        }
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
        PSPC_TRY_CUDA(cudaGetLastError());
        return sort_rows();
    }

    // Sorts every rank-space row ascending (highest-ranked neighbour first).
    int sort_rows() {
        int32_t* big = nullptr;
        int* nbig = nullptr;
        PSPC_TRY_CUDA(dalloc(&big, n, st));
        PSPC_TRY_CUDA(dalloc(&nbig, 1, st));
        PSPC_TRY_CUDA(cudaMemsetAsync(nbig, 0, sizeof(int), st));
        int grid = (int)std::min<int64_t>(n, (int64_t)sms * 16);
        if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
        k_sort_rows<<<grid, kRowThreads, 0, st>>>(rp_r, col_r, n, big, nbig);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        int hbig = 0;
        PSPC_TRY_CUDA(cudaMemcpyAsync(&hbig, nbig, sizeof(int), cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        int rc = PSPC_OK;
        if (hbig > 0) {
            const int g2 = std::min(hbig, sms);
            const size_t W = (size_t)((n + 31) / 32);
            uint32_t* scratch = nullptr;
            PSPC_TRY_CUDA(dalloc(&scratch, W * g2, st));
            k_sort_big_rows<<<g2, kRowThreads, 0, st>>>(rp_r, col_r, n, big, hbig, scratch);
            out.launches += 1;
            rc = cuda_status(cudaGetLastError());
            dfree(scratch, st);
        }
        dfree(big, st);
        dfree(nbig, st);
        return rc;
    }

    // Level 1 (distance 1): the prefix of each sorted row below the vertex.
    int level1(unsigned long long& bump, pspc_level_stat_t& ls) {
        int64_t* len1 = nullptr;
        unsigned long long* act = nullptr;
        PSPC_TRY_CUDA(dalloc(&len1, n + 1, st));
        PSPC_TRY_CUDA(dalloc(&act, 2, st));
        PSPC_TRY_CUDA(cudaMemsetAsync(act, 0, 16, st));
        k_level1_counts<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rp_r, col_r, n, len1, act);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        int rc = exclusive_scan_i64(len1, n, st, &out.launches);
        if (rc) return rc;
        int64_t total = 0;
        unsigned long long hact[2] = {0, 0};
        PSPC_TRY_CUDA(cudaMemcpyAsync(&total, len1 + n, 8, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaMemcpyAsync(hact, act, 16, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        if (bump + (unsigned long long)total > arena_cap) {
            if ((rc = grow_arena(bump + total, bump))) return rc;
        }
        k_level1_write<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(rp_r, col_r, n, len1, bump, hub_arena,
                                                                          cnt_arena, seg + n, lab_size);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        dfree(len1, st);
        dfree(act, st);
        bump += (unsigned long long)total;
        ls.raw_candidates = total;
        ls.unique_candidates = total;
        ls.entries = total;
        ls.active_vertices = (int64_t)hact[0];
        ls.active_arcs = (int64_t)hact[1];
        ls.kernel_ms = 0.f;
        return PSPC_OK;
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
        // rows for levels 0 .. kMaxDist + 1 at most (the level after the
        // storage limit is run to learn whether it is empty)
        int cap = std::max(need, std::min(seg_levels_cap ? seg_levels_cap * 2 : 16, kMaxDist + 2));
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

    // Launches the on-chip level kernel over the bucketed vertices, then the
    // off-chip variant over the vertices whose labels or candidates do not
    // fit on chip. Reads the level status after each.
    int run_level_kernels(int d, const LevelPlan& plan, int& n_offchip) {
        LevelArgs A;
        memset(&A, 0, sizeof(A));
        A.d = d;
        A.n = n;
        A.rp = rp_r;
        A.col = col_r;
        A.cnt_arc = cnt_arc;
        A.arc_lo = skip_prefix ? arc_lo : nullptr;
        A.hpre = skip_prefix ? hpre : nullptr;
        A.push_hub = push_level ? push_hub : nullptr;
        A.push_cnt = push_level ? push_cnt : nullptr;
        A.push_off = push_level ? push_off : nullptr;
        A.seg = seg;
        A.seg_out = seg + (int64_t)d * n;
        A.hub_arena = hub_arena;
        A.cnt_arena = cnt_arena;
        A.arena_cap = arena_cap;
        A.raw_u = raw_u;
        A.lab_size = lab_size;
        A.stt = stt;
        A.retry_list = glist + hstt->n_global;
        A.comp_base = comp_base;
        A.lmk = out.lmk;
        A.lmk_stride = out.lmk_stride;
        // shallow levels test the first kLmkShallow landmarks only: their
        // short distances seldom prove survival, and half the row is read
        A.lmk_words = d < kLmkDeepLevel ? std::min(out.lmk_stride / 16, 2 * kLmkShallow / 16) : out.lmk_stride / 16;
        if (hstt->n_smem > 0) {
            // Items are bucketed heaviest first. Light vertices (fewer than
            // 2^kLightBucket pulled entries) run in small CTAs with small
            // tables and the segment-search map, so that many of them share
            // an SM; the others in full-size CTAs.
            int n_light = 0, n_micro = 0;
            // Automatic: one warp per tiny vertex at levels 2 and 3, and
            // deeper (up to level 127) while the last level had few
            // candidates per vertex: there the warp's own rule-2 scans are
            // short or rare.
            bool warp_level = o.warp_levels > 0 && d <= o.warp_levels;
            if (o.warp_levels == 0 && !out.lstats.empty()) {
                const pspc_level_stat_t& pl = out.lstats.back();
                warp_level = d <= 3 || (d <= kWarpLevelsMax && pl.active_vertices > 0 &&
                                        pl.unique_candidates < kWarpLevelsFew * pl.active_vertices);
            }
            for (int b = 0; b < kLightBucket; ++b)
                (warp_level && b < kMicroBucket ? n_micro : n_light) += hstt->bucket_cnt[b];
            const int n_heavy = hstt->n_smem - n_light - n_micro;
            A.granular = o.granular ? 1 : 0;
            cudaEventRecord(ek0, st);
            cudaError_t e = cudaSuccess;
            if (n_heavy > 0) {
                A.items = items;
                A.n_items = n_heavy;
                A.work = &stt->work_smem;
                A.cap_c_max = plan.cap_c;
                A.cap_u_max = plan.cap_u;
                A.bm_words = plan.bm_words;
                int grid = std::min(n_heavy, sms * plan.occupancy);
                if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
                if (o.granular) grid = n_heavy;
                e = launch_level(plan.map_kind, false, grid, plan.smem_bytes, A, st);
                out.launches += 1;
            }
            if (e == cudaSuccess && n_light > 0) {
                A.items = items + n_heavy;
                A.n_items = n_light;
                A.work = &stt->work_light;
                A.cap_c_max = kLightCap;
                A.cap_u_max = plan.cap_u;
                A.bm_words = plan.bm_words;
                int grid = std::min(n_light, sms * plan.light_occupancy);
                if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
                if (o.granular) grid = n_light;
                e = launch_level(kMapSeg, false, grid, plan.light_smem_bytes, A, st, kLightThreads);
                out.launches += 1;
            }
            if (e == cudaSuccess && n_micro > 0) {  // one warp per vertex
                A.items = items + n_heavy + n_light;
                A.n_items = n_micro;
                A.work = &stt->work_micro;
                const int per_cta = kMicroThreads / 32;
                int grid = (n_micro + per_cta - 1) / per_cta;
                if (!o.granular) grid = std::min(grid, sms * plan.micro_occupancy);
                if (o.max_ctas > 0 && !o.granular) grid = std::min(grid, o.max_ctas);
                e = launch_level_micro(grid, A, st);
                out.launches += 1;
            }
            cudaEventRecord(ek1, st);
            PSPC_TRY_CUDA(e);
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
            // first pass: slabs of at most kOffSlabCap candidate slots, tables
            // grown from kOffStartCap; vertices beyond the slab go to a second
            // pass with slabs of the full bound
            const uint32_t cc_full = (uint32_t)std::max<unsigned long long>(hstt->need_cap_c, 64);
            const uint32_t cu = (uint32_t)std::max<unsigned long long>(hstt->need_cap_u, 64);
            const int off_kind = plan.map_kind == kMapSeg ? kMapSeg : kMapHash;
            const size_t budget = (size_t)4 << 30;
            for (int pass = 0; pass < 2; ++pass) {
                const int count = pass == 0 ? n_off : hstt->n_giant;
                if (count == 0) break;
                const uint32_t cc = pass == 0 ? std::min(cc_full, kOffSlabCap) : cc_full;
                const size_t stride =
                    (level_layout(cc, level_map_bytes(off_kind, d, 0, cu)).total + 255) & ~(size_t)255;
                int grid = (int)std::min<size_t>((size_t)count, std::max<size_t>(1, budget / stride));
                // granular builds leave every SM half free for concurrent work
                grid = std::min(grid, o.granular ? sms : sms * 2);
                if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
                rc = ensure_gscratch(stride * grid);
                if (rc) return rc;
                A.items = pass == 0 ? glist : glist + n;
                A.n_items = count;
                A.work = pass == 0 ? &stt->work_global : &stt->work_giant;
                A.cap_c_max = cc;
                A.cap_u_max = cu;
                A.off_start_cap = pass == 0 ? kOffStartCap : 0u;
                A.giant_list = glist + n;
                A.gscratch = gscratch;
                A.gscratch_stride = stride;
                A.granular = 0;  // off-chip scratch slabs are per persistent CTA
                cudaEventRecord(ek0, st);
                cudaError_t e = launch_level(off_kind, true, grid, 0, A, st);
                cudaEventRecord(ek1, st);
                out.launches += 1;
                PSPC_TRY_CUDA(e);
                rc = read_status();
                if (rc) return rc;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ek0, ek1);
                kernel_ms += ms;
                offchip_ms += ms;
            }
        }
        return PSPC_OK;
    }

    // How level d runs on chip: level bitmaps when (d-1) bitmaps of n bits
    // fit the bitmap budget, else a label hash of cap_u slots (labels that
    // need more go off chip).
    int plan_level(int d, LevelPlan& plan) {
        plan.cap_c = (uint32_t)o.cand_capacity;
        plan.cap_u = (uint32_t)o.label_capacity;
        plan.bm_words = (uint32_t)((max_comp + 31) / 32);
        const bool bm_fits = bitmap_bytes(d, plan.bm_words) <= kBitmapBudget;
        if ((o.map_kind == 0 || o.map_kind == 1) && bm_fits) {
            plan.map_kind = kMapBitmap;
            plan.label_limit = INT64_MAX;
        } else if (o.map_kind == 2) {
            plan.map_kind = kMapHash;
            int64_t lo = 0, hi = plan.cap_u;  // largest label size whose hash fits cap_u slots
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) / 2;
                if (label_cap_for(mid) <= plan.cap_u) lo = mid; else hi = mid - 1;
            }
            plan.label_limit = lo;
        } else {
            plan.map_kind = kMapSeg;
            plan.label_limit = INT64_MAX;
        }
        plan.smem_bytes = level_layout(plan.cap_c, level_map_bytes(plan.map_kind, d, plan.bm_words, plan.cap_u)).total;
        if (plan.smem_bytes + 1024 > (size_t)smem_optin) return PSPC_E_INVAL;  // tables must fit on chip
        PSPC_TRY_CUDA(level_kernel_attrs(plan.map_kind, plan.smem_bytes, &plan.occupancy));
        if (plan.occupancy < 1) return PSPC_E_INVAL;
        plan.light_smem_bytes = level_layout(kLightCap, level_map_bytes(kMapSeg, d, 0, 0), kLightThreads).total;
        PSPC_TRY_CUDA(level_kernel_attrs(kMapSeg, plan.light_smem_bytes, &plan.light_occupancy, kLightThreads));
        if (plan.light_occupancy < 1) return PSPC_E_INVAL;
        PSPC_TRY_CUDA(micro_kernel_occupancy(&plan.micro_occupancy));
        if (plan.micro_occupancy < 1) return PSPC_E_INVAL;
        return PSPC_OK;
    }

    // Landmark labelling (Section "Landmark-Based Filtering"): distances
    // from o.landmarks landmarks per graph (the highest-ranked vertices;
    // past the first kLmkShallow, spread ones for a large single graph),
    // kept with the index.
    int landmarks() {
        out.lmk_k = o.landmarks;
        out.lmk_stride = (2 * o.landmarks + 15) / 16 * 16;
        PSPC_TRY_CUDA(dalloc(&out.lmk, n * out.lmk_stride, st));
        cudaEvent_t a, b;
        PSPC_TRY_CUDA(cudaEventCreate(&a));
        PSPC_TRY_CUDA(cudaEventCreate(&b));
        cudaEventRecord(a, st);
        int rc = landmark_bfs(n, rp_r, col_r, comp_base, out.lmk_k, out.lmk_stride, out.lmk, out.lmk_ids, st,
                              &out.launches);
        cudaEventRecord(b, st);
        if (!rc) {
            cudaEventSynchronize(b);
            cudaEventElapsedTime(&out.lmk_ms, a, b);
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return rc;
    }

    // Push paradigm (Algorithm PUSH): bucket offsets from a scan of the
    // per-arc counts of the cost pass, then every arc copies its entries.
    int push_entries(int d) {
        if (!push_off) PSPC_TRY_CUDA(dalloc(&push_off, arcs + 1, st));
        PSPC_TRY_CUDA(launch_arc_counts(arcs, cnt_arc, push_off, st));
        int rc = exclusive_scan_i64(push_off, arcs, st, &out.launches);
        if (rc) return rc;
        int64_t total = 0;
        PSPC_TRY_CUDA(cudaMemcpyAsync(&total, push_off + arcs, 8, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        if (total > push_cap) {
            dfree(push_hub, st);
            dfree(push_cnt, st);
            push_hub = nullptr;
            push_cnt = nullptr;
            push_cap = 0;
            PSPC_TRY_CUDA(dalloc(&push_hub, total + total / 4 + 1, st));
            PSPC_TRY_CUDA(dalloc(&push_cnt, total + total / 4 + 1, st));
            push_cap = total + total / 4 + 1;
        }
        PSPC_TRY_CUDA(launch_push_scatter(arcs, col_r, seg + (int64_t)(d - 1) * n, hub_arena, cnt_arena, cnt_arc,
                                          skip_prefix ? arc_lo : nullptr, push_off, push_hub, push_cnt, st));
        out.launches += 3;
        return PSPC_OK;
    }

    int build_levels() {
        PSPC_TRY_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        LevelPlan plan;
        int rc = plan_level(1, plan);  // rejects option sizes that cannot run at all
        if (rc) return rc;
        if ((rc = ensure_seg_levels(16))) return rc;
        const unsigned long long cap0 = o.arena_entries > 0 ? (unsigned long long)o.arena_entries
                                                            : (unsigned long long)(32 * arcs + 4 * n);
        rc = grow_arena(std::max<unsigned long long>(cap0, (unsigned long long)n + 1024), 0);
        if (rc) return rc;
        PSPC_TRY_CUDA(dalloc(&cnt_arc, arcs, st));
        PSPC_TRY_CUDA(dalloc(&arc_lo, arcs, st));
        PSPC_TRY_CUDA(dalloc(&hpre, n, st));
        PSPC_TRY_CUDA(dalloc(&raw_u, n, st));
        PSPC_TRY_CUDA(dalloc(&lab_size, n, st));
        PSPC_TRY_CUDA(dalloc(&items, n, st));
        PSPC_TRY_CUDA(dalloc(&glist, 2 * n, st));
        PSPC_TRY_CUDA(dalloc(&stt, 1, st));
        PSPC_TRY_CUDA(cudaMemsetAsync(lab_size, 0, n * 8, st));
        PSPC_TRY_CUDA(launch_arc_src(rp_r, n, arc_src, st));
        out.launches += 1;

        k_level0<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, hub_arena, cnt_arena, seg);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        if (o.landmarks > 0 && (rc = landmarks())) return rc;
        lvl_base.assign({0ull, (unsigned long long)n});
        unsigned long long bump = (unsigned long long)n;
        cudaEvent_t e0, e1;
        PSPC_TRY_CUDA(cudaEventCreate(&e0));
        PSPC_TRY_CUDA(cudaEventCreate(&e1));
        PSPC_TRY_CUDA(cudaEventCreate(&ek0));
        PSPC_TRY_CUDA(cudaEventCreate(&ek1));
        int levels = 1;
        // Distances are stored in 15 bits: a level beyond the limit that
        // adds an entry ends the build with PSPC_E_DIST (one that adds
        // nothing is the normal end).
        const int dist_limit = std::min(o.max_levels, kMaxDist);
        for (int d = 1;; ++d) {
            if ((rc = ensure_seg_levels(d + 1))) break;
            if ((rc = plan_level(d, plan))) break;
            cudaEventRecord(e0, st);
            if (d == 1) {
                pspc_level_stat_t ls{};
                cudaMemsetAsync(seg + n, 0, n * 8, st);
                if ((rc = level1(bump, ls))) break;
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ls.ms, e0, e1);
                out.lstats.push_back(ls);
                if (o.verbose)
                    fprintf(stderr, "pspc level 1: entries %lld active %lld %.3f ms\n", (long long)ls.entries,
                            (long long)ls.active_vertices, ls.ms);
                if (ls.entries == 0) break;
                if (d > dist_limit) {
                    rc = PSPC_E_DIST;
                    break;
                }
                lvl_base.push_back(bump);
                levels = 2;
                continue;
            }
            cudaMemsetAsync(seg + (int64_t)d * n, 0, n * 8, st);
            cudaMemsetAsync(stt, 0, sizeof(LevelStatus), st);
            cudaMemcpyAsync(&stt->bump, &lvl_base[d], 8, cudaMemcpyHostToDevice, st);
            // Dense-prefix skip on the shallow levels (the prefix pass reads
            // d segments per vertex; deep levels of high-diameter graphs gain
            // little from it).
            skip_prefix = d >= 3 && d <= kDensePrefixMaxLevel && prefix_pays;
            cudaError_t ce = cudaSuccess;
            if (skip_prefix) {
                ce = launch_dense_prefix(d, n, seg, hub_arena, comp_base, hpre, st);
                out.launches += 1;
            }
            if (ce == cudaSuccess)
                ce = launch_cost(d, n, arcs, rp_r, col_r, arc_src, seg + (int64_t)(d - 1) * n, hub_arena,
                                 skip_prefix ? hpre : nullptr, arc_lo, cnt_arc, raw_u, lab_size, stt,
                                 plan.label_limit, glist, items, st, &out.launches);
            if ((rc = cuda_status(ce))) break;
            if ((rc = read_status())) break;
            if (hstt->n_active == 0) break;
            const long long raw_total = (long long)hstt->raw_total;
            // Push paradigm: the arcs send their entries into per-vertex
            // buckets before the level kernel merges them.
            push_level = o.paradigm == 1;
            if (push_level && (rc = push_entries(d))) break;
            if (skip_prefix)  // on the graphs measured, the share saved only fell after its first level
                prefix_pays = (double)hstt->prefix_skipped >=
                              kDensePrefixMinGain * (double)(hstt->prefix_skipped + hstt->raw_total);
            const long long active_arcs = (long long)hstt->active_arcs;
            // Size the arena for this level before running it: the level
            // adds at most one entry per distinct pulled (u, h), bounded here
            // by the pulled count and by four times what exists so far.
            {
                const unsigned long long used = lvl_base[d];
                const unsigned long long add =
                    std::min<unsigned long long>((unsigned long long)raw_total, 4 * used + (unsigned long long)n);
                if (used + add > arena_cap && (rc = grow_arena(used + add, used))) break;
            }
            int n_off = 0;
            kernel_ms = 0.f;
            offchip_ms = 0.f;
            for (int attempt = 0;; ++attempt) {
                if ((rc = run_level_kernels(d, plan, n_off))) break;
                if (!hstt->arena_overflow) break;
                kernel_ms = 0.f;
                offchip_ms = 0.f;
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
                keep.lmk_pruned = 0;
                keep.lmk_proven = 0;
                keep.n_retry = 0;
                keep.arena_overflow = 0;
                keep.work_smem = keep.work_global = keep.work_light = keep.work_giant = keep.work_micro = 0;
                keep.n_giant = 0;
                memset(keep.route_att, 0, sizeof(keep.route_att));  // the level is re-run from scratch
                memset(keep.route_ovf, 0, sizeof(keep.route_ovf));
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
            pspc_level_stat_t ls{};
            ls.raw_candidates = raw_total + (long long)hstt->prefix_skipped;
            ls.unique_candidates = (long long)hstt->unique_total;
            ls.entries = added;
            ls.active_vertices = hstt->n_active;
            ls.active_arcs = active_arcs;
            ls.ms = ms;
            ls.kernel_ms = kernel_ms;
            ls.landmark_pruned = (long long)hstt->lmk_pruned;
            ls.landmark_proven = (long long)hstt->lmk_proven;
            ls.offchip_vertices = n_off;
            ls.offchip_ms = offchip_ms;
            // the retry list holds the overflowed attempts (counted per size
            // class) and the routed vertices
            long long ovf_attempts = 0;
            for (int b = 0; b < kBuckets; ++b) ovf_attempts += hstt->route_ovf[b];
            ls.routed_vertices = std::max(0LL, (long long)hstt->n_retry - ovf_attempts);
            out.lstats.push_back(ls);
            if (o.verbose)
                fprintf(stderr, "pspc level %d: raw %lld unique %lld entries %lld active %d (off-chip %d) %.3f ms\n",
                        d, raw_total, (long long)hstt->unique_total, added, hstt->n_active, n_off, ms);
            if (added == 0) break;
            if (d > dist_limit) {
                rc = PSPC_E_DIST;
                break;
            }
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
        PSPC_TRY_CUDA(dalloc(&out.off, n + 1, st));
        int32_t* big = nullptr;
        int* ctr = nullptr;  // [0] = n_big, [1] = work
        unsigned long long* d_lvl = nullptr;
        unsigned long long* n_ovf = nullptr;
        PSPC_TRY_CUDA(dalloc(&big, n, st));
        PSPC_TRY_CUDA(dalloc(&ctr, 2, st));
        PSPC_TRY_CUDA(dalloc(&d_lvl, lvl_base.size(), st));
        PSPC_TRY_CUDA(dalloc(&n_ovf, 2, st));  // [0] overflow entries, [1] largest label
        PSPC_TRY_CUDA(cudaMemsetAsync(ctr, 0, 8, st));
        PSPC_TRY_CUDA(cudaMemsetAsync(n_ovf, 0, 16, st));
        PSPC_TRY_CUDA(cudaMemcpyAsync(d_lvl, lvl_base.data(), lvl_base.size() * 8, cudaMemcpyHostToDevice, st));
        k_fin_sizes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, L, seg, out.off, big, ctr, n_ovf + 1);
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        int rc = exclusive_scan_i64(out.off, n, st, &out.launches);
        if (rc) return rc;
        int hbig[2] = {0, 0};
        PSPC_TRY_CUDA(cudaMemcpyAsync(&out.entries, out.off + n, 8, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaMemcpyAsync(hbig, ctr, 8, cudaMemcpyDeviceToHost, st));
        unsigned long long hmax = 0;
        PSPC_TRY_CUDA(cudaMemcpyAsync(&hmax, n_ovf + 1, 8, cudaMemcpyDeviceToHost, st));
        PSPC_TRY_CUDA(cudaStreamSynchronize(st));
        out.max_label = (int64_t)hmax;
        const int64_t E = out.entries;
        PSPC_TRY_CUDA(dalloc(&out.hub, E, st));
        PSPC_TRY_CUDA(dalloc(&out.dist, E, st));
        PSPC_TRY_CUDA(dalloc(&out.cnt, E, st));
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
        const uint32_t rank_words = (uint32_t)((max_comp + 31) / 32 + 1);
        const bool by_rank = L > kFinMergeLevels && rank_words <= kFinRankWords;
        if (by_rank) {  // every vertex, whatever its label size
            F.comp_base = comp_base;
            F.rank_words = rank_words;
            const size_t fin_smem = (size_t)rank_words * 8;
            PSPC_TRY_CUDA(cudaFuncSetAttribute(k_finalize_rank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)fin_smem));
            int grid = (int)std::min<int64_t>(n, (int64_t)sms * 8);
            if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
            k_finalize_rank<<<grid, kFinThreads, fin_smem, st>>>(F);
        } else if (L <= kFinMergeLevels) {
            const size_t fin_smem = (size_t)kFinSmemKeys * 4;
            PSPC_TRY_CUDA(cudaFuncSetAttribute(k_finalize_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(2 * fin_smem)));
            int grid = (int)std::min<int64_t>(n, (int64_t)sms * 8);
            if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
            F.merge_keys = kFinSmemKeys;
            k_finalize_merge<<<grid, kFinThreads, fin_smem, st>>>(F);
        } else {
            const size_t fin_smem = (size_t)kFinSmemKeys * 8;
            PSPC_TRY_CUDA(cudaFuncSetAttribute(k_finalize<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)fin_smem));
            int grid = (int)std::min<int64_t>(n, (int64_t)sms * 8);
            if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
            k_finalize<false><<<grid, kFinThreads, fin_smem, st>>>(F);
        }
        out.launches += 1;
        PSPC_TRY_CUDA(cudaGetLastError());
        // Long labels of a few-level index: the merge again, with twice the
        // on-chip buffer, over those vertices only.
        const bool big_by_merge = hbig[0] > 0 && !by_rank && L <= kFinMergeLevels &&
                                  out.max_label <= 2 * (int64_t)kFinSmemKeys;
        if (big_by_merge) {
            int grid = std::min(hbig[0], sms * 2);
            if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
            F.list = big;
            F.n_list = hbig[0];
            F.merge_keys = 2 * kFinSmemKeys;
            k_finalize_merge<<<grid, kFinThreads, (size_t)kFinSmemKeys * 8, st>>>(F);
            F.list = nullptr;
            F.n_list = 0;
            out.launches += 1;
            PSPC_TRY_CUDA(cudaGetLastError());
        }
        if (hbig[0] > 0 && !by_rank && !big_by_merge) {
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
        PSPC_TRY_CUDA(dalloc(&out.rank, n, st));
        PSPC_TRY_CUDA(dalloc(&out.order, n, st));
        PSPC_TRY_CUDA(cudaMemcpyAsync(out.rank, rank, n * 4, cudaMemcpyDeviceToDevice, st));
        PSPC_TRY_CUDA(cudaMemcpyAsync(out.order, order, n * 4, cudaMemcpyDeviceToDevice, st));
        return PSPC_OK;
    }
};

}  // namespace pspc

using namespace pspc;

// Default landmarks: 128 for one graph (32 highest-ranked and 96 spread),
// 64 highest-ranked per graph in a batch (one BFS round).
static void fill_defaults(pspc_opts& o, const pspc_opts* user, bool batch = false) {
    memset(&o, 0, sizeof(o));
    if (user) o = *user;
    if (o.cand_capacity <= 0) o.cand_capacity = 4096;
    if (o.label_capacity <= 0) o.label_capacity = 8192;
    if (o.max_levels <= 0) o.max_levels = kMaxDist;
    if (o.landmarks == 0) o.landmarks = batch ? 64 : kLmkMax;
}

static bool opts_ok(const pspc_opts& o) {
    return o.map_kind >= 0 && o.map_kind <= 3 && o.max_ctas >= 0 && (o.granular == 0 || o.granular == 1) &&
           o.landmarks >= -1 && o.landmarks <= kLmkMax && (o.paradigm == 0 || o.paradigm == 1) && o.warp_levels >= -1;
}

static bool pow2_in(int32_t v, int32_t lo, int32_t hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// Common driver: stage the input (one graph or a batch), check it, relabel,
// build the levels, finalize, and hand the index to the caller.
template <typename Stage>
static int run_build(const pspc_opts* opts, pspc_index** out, void* stream, int32_t graphs, Stage stage,
                     bool batch = false) {
    Builder B;
    B.st = (cudaStream_t)stream;
    fill_defaults(B.o, opts, batch);
    if (!pow2_in(B.o.cand_capacity, 1024, 16384) || !pow2_in(B.o.label_capacity, 1024, 16384) || !opts_ok(B.o))
        return PSPC_E_INVAL;
    PSPC_TRY_CUDA(cudaGetDevice(&B.dev));
    PSPC_TRY_CUDA(cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, B.dev));
    cudaEvent_t t0, t1;
    PSPC_TRY_CUDA(cudaEventCreate(&t0));
    PSPC_TRY_CUDA(cudaEventCreate(&t1));
    cudaEventRecord(t0, B.st);
    int rc = stage(B);
    if (!rc) rc = B.validate();
    if (!rc) rc = B.relabel();
    if (!rc) {
        B.out.n = B.n;
        B.out.arcs = B.arcs;
        B.out.device = B.dev;
        B.out.graphs = graphs;
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
    B.out.lmk = nullptr;
    *out = h;
    return PSPC_OK;
}

// Reduction by 1-shell: peel G, build the index of the core (an ordinary
// index over core ids), and wrap it with the per-vertex roots and depths.
static int build_reduced(const pspc_csr* g, const int32_t* rank, const pspc_opts* opts, pspc_index** out,
                         void* stream) {
    Builder B;
    B.st = (cudaStream_t)stream;
    fill_defaults(B.o, opts);
    if (!pow2_in(B.o.cand_capacity, 1024, 16384) || !pow2_in(B.o.label_capacity, 1024, 16384) || !opts_ok(B.o))
        return PSPC_E_INVAL;
    PSPC_TRY_CUDA(cudaGetDevice(&B.dev));
    cudaEvent_t t0, t1;
    PSPC_TRY_CUDA(cudaEventCreate(&t0));
    PSPC_TRY_CUDA(cudaEventCreate(&t1));
    cudaEventRecord(t0, B.st);
    int rc = B.stage_inputs(g, rank);
    if (!rc) rc = B.validate();
    ShellParts P;
    if (!rc) rc = shell_reduce(B.n, B.rp, B.col, B.rank, P, B.st, &B.out.launches);
    pspc_index* core = nullptr;
    if (!rc) {
        pspc_csr cg;
        cg.n = P.n_core;
        cg.row_ptr = P.rp;
        cg.col = P.col;
        pspc_opts co = B.o;
        co.reduce_shell = 0;
        rc = pspc_build(&cg, P.rank, &co, &core, stream);
    }
    shell_free(P, B.st);
    pspc_index* h = nullptr;
    if (!rc) {
        cudaEventRecord(t1, B.st);
        cudaError_t e = cudaEventSynchronize(t1);
        h = new (std::nothrow) pspc_index;
        if (e != cudaSuccess) rc = cuda_status(e);
        else if (!h) rc = PSPC_E_NOMEM;
    }
    if (rc) {
        if (core) pspc_free(core);
        delete h;
        dfree(P.parent, B.st);
        dfree(P.root, B.st);
        dfree(P.depth, B.st);
        dfree(P.core_id, B.st);
    } else {
        Index& ix = h->ix;
        const Index& c = core->ix;
        ix.device = c.device;
        ix.n = B.n;
        ix.arcs = B.arcs;
        ix.entries = c.entries;
        ix.max_label = c.max_label;
        ix.levels = c.levels;
        ix.overflow_entries = c.overflow_entries;
        ix.launches = B.out.launches + c.launches;
        ix.lstats = c.lstats;
        ix.lmk_k = c.lmk ? c.lmk_k : 0;
        memcpy(ix.lmk_ids, c.lmk_ids, sizeof(ix.lmk_ids));
        ix.lmk_ms = c.lmk_ms;
        cudaEventElapsedTime(&ix.build_ms, t0, t1);
        ix.core = core;
        ix.sh_core = P.core_id;
        ix.sh_root = P.root;
        ix.sh_depth = P.depth;
        ix.sh_parent = P.parent;
        ix.shell_vertices = P.removed;
        *out = h;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return rc;
}

extern "C" int pspc_build(const pspc_csr* g, const int32_t* rank, const pspc_opts* opts, pspc_index** out,
                          void* stream) {
    if (!out) return PSPC_E_INVAL;
    *out = nullptr;
    if (!g || !rank || !g->row_ptr) return PSPC_E_INVAL;
    if (g->n < 1 || g->n > kMaxVertices) return PSPC_E_INVAL;
    if (opts && opts->reduce_shell) {
        if (opts->reduce_shell != 1) return PSPC_E_INVAL;
        return build_reduced(g, rank, opts, out, stream);
    }
    return run_build(opts, out, stream, 1, [&](Builder& B) { return B.stage_inputs(g, rank); });
}

extern "C" int pspc_build_batch(const pspc_graph* graphs, int32_t k, const pspc_opts* opts, pspc_index** out,
                                void* stream) {
    if (!out) return PSPC_E_INVAL;
    *out = nullptr;
    // a batch keeps one BFS round of landmarks: at most 64 per graph
    if (!graphs || k < 1 || (opts && (opts->reduce_shell || opts->landmarks > 64))) return PSPC_E_INVAL;
    return run_build(opts, out, stream, k, [&](Builder& B) { return B.stage_batch(graphs, k); }, true);
}
