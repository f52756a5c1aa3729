// SPC(s,t) queries on the hub-label index: Eq. (1)-(2) of the paper
// (Section "2-Hop Labeling for Shortest Path Counting"), evaluated as a
// merge-join of the two hub-sorted labels; queries are independent
// (Section "Reduction by Equivalence Relation", parallel query evaluation).
//
// Kernels: k_query<G> (G lanes per pair, 32-bit hub words in registers,
// binary search by shuffles), k_query_chunked<CH> (a warp per pair, chunks
// of CH entries of both labels staged in shared memory, binary search per
// entry; the side whose last hub is smaller advances), k_query_by_source
// (pairs sorted by source; L(s) hashed on chip once per run of pairs with
// that source, each warp streams L(t)). In each, a match h gives
// dist_s(h) + dist_t(h); counts (and their 128-bit product) are read only
// for matches that reach the lane's running minimum. The warp then keeps
// the global minimum and adds the products of the hubs that reach it,
// modulo 2^64, with a sticky overflow flag (flag of a factor, high word of
// a product, carry of a sum).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "pspc_internal.cuh"
#include "pspc_shell.cuh"

namespace cg = cooperative_groups;

namespace pspc {

constexpr int kQueryThreads = 256;
constexpr uint32_t kNoHub = 0xFFFFFFFFu;

struct QueryArgs {
    int64_t n;
    const int32_t* rank;
    const int64_t* off;
    const int32_t* hub;
    const uint16_t* dist;
    const uint64_t* cnt;
    const int32_t* pairs;
    const int32_t* perm;  // processing order of the pairs (grouped by source), or NULL
    const unsigned long long* src_end;  // with perm: end of each source's pairs in it (bucket n: invalid ids)
    int64_t q;
    uint16_t* out_dist;
    uint64_t* out_cnt;
    uint8_t* out_ovf;
    int* err;
};

__device__ __forceinline__ void add_term(uint64_t& sum, uint32_t& flag, uint64_t term, uint32_t tflag) {
    const uint64_t s = sum + term;
    flag |= tflag | (uint32_t)(s < term);
    sum = s;
}

// Warp-wide end of one pair: the minimum distance over the lanes, the sum
// (mod 2^64, sticky flag) of the lanes' partial sums at that minimum, and
// lane 0 writes the answer of pair p.
__device__ __forceinline__ void finish_pair_warp(const QueryArgs& Q, int64_t p, uint32_t best, uint64_t sum,
                                                 uint32_t flag, int lane) {
    uint32_t gbest = best;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gbest = min(gbest, __shfl_xor_sync(0xFFFFFFFFu, gbest, o));
    if (best != gbest) {
        sum = 0;
        flag = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t os = __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        const uint32_t of = __shfl_xor_sync(0xFFFFFFFFu, flag, o);
        add_term(sum, flag, os, of);
    }
    if (lane == 0) {
        if (gbest == 0xFFFFFFFFu) {
            Q.out_dist[p] = PSPC_UNREACHED;
            Q.out_cnt[p] = 0;
            if (Q.out_ovf) Q.out_ovf[p] = 0;
        } else {
            Q.out_dist[p] = (uint16_t)gbest;
            Q.out_cnt[p] = sum;
            if (Q.out_ovf) Q.out_ovf[p] = (uint8_t)(flag != 0);
        }
    }
}

__device__ __forceinline__ void write_fixed(const QueryArgs& Q, int64_t p, uint16_t d, uint64_t c) {
    Q.out_dist[p] = d;
    Q.out_cnt[p] = c;
    if (Q.out_ovf) Q.out_ovf[p] = 0;
}

template <int G>
__global__ void __launch_bounds__(kQueryThreads) k_query(const QueryArgs Q) {
    auto tile = cg::tiled_partition<G>(cg::this_thread_block());
    const int lane = tile.thread_rank();
    const int64_t ngroups = (int64_t)gridDim.x * (kQueryThreads / G);
    for (int64_t k = ((int64_t)blockIdx.x * kQueryThreads + threadIdx.x) / G; k < Q.q; k += ngroups) {
        const int64_t p = Q.perm ? (int64_t)__ldg(Q.perm + k) : k;
        const int32_t s = __ldg(Q.pairs + 2 * p), t = __ldg(Q.pairs + 2 * p + 1);
        if (s < 0 || s >= Q.n || t < 0 || t >= Q.n) {
            if (lane == 0) {
                atomicOr(Q.err, 1);
                Q.out_dist[p] = PSPC_UNREACHED;
                Q.out_cnt[p] = 0;
                if (Q.out_ovf) Q.out_ovf[p] = 0;
            }
            continue;
        }
        if (s == t) {
            if (lane == 0) {
                Q.out_dist[p] = 0;
                Q.out_cnt[p] = 1;
                if (Q.out_ovf) Q.out_ovf[p] = 0;
            }
            continue;
        }
        const int32_t rs = __ldg(Q.rank + s), rt = __ldg(Q.rank + t);
        int64_t ia = __ldg(Q.off + rs);
        const int64_t ea = __ldg(Q.off + rs + 1);
        int64_t ib = __ldg(Q.off + rt);
        const int64_t eb = __ldg(Q.off + rt + 1);
        uint32_t best = 0xFFFFFFFFu;
        uint64_t sum = 0;
        uint32_t flag = 0;
        while (ia < ea && ib < eb) {
            const bool va = ia + lane < ea, vb = ib + lane < eb;
            const uint32_t ha = va ? (uint32_t)__ldg(Q.hub + ia + lane) : kNoHub;
            const uint32_t hb = vb ? (uint32_t)__ldg(Q.hub + ib + lane) : kNoHub;
            const uint16_t db = vb ? __ldg(Q.dist + ib + lane) : 0;
            const int la = ea - ia > G ? G - 1 : (int)(ea - ia - 1);
            const int lb = eb - ib > G ? G - 1 : (int)(eb - ib - 1);
            const uint32_t amax = tile.shfl(ha, la);
            const uint32_t bmax = tile.shfl(hb, lb);
            // largest j with hb_j <= ha (hb is ascending over the lanes)
            int j = 0;
#pragma unroll
            for (int step = G / 2; step > 0; step >>= 1) {
                const uint32_t v = tile.shfl(hb, j + step);
                if (v <= ha) j += step;
            }
            const uint32_t hj = tile.shfl(hb, j);
            const uint16_t dj = tile.shfl(db, j);
            if (va && hj == ha) {
                const uint16_t da = __ldg(Q.dist + ia + lane);
                const uint32_t dsum = (uint32_t)(da & 0x7FFF) + (uint32_t)(dj & 0x7FFF);
                if (dsum <= best) {
                    const uint64_t ca = __ldg((const unsigned long long*)Q.cnt + ia + lane);
                    const uint64_t cb = __ldg((const unsigned long long*)Q.cnt + ib + j);
                    const uint64_t lo = ca * cb;
                    const uint32_t tf =
                        (uint32_t)(da >> 15) | (uint32_t)(dj >> 15) | (uint32_t)(__umul64hi(ca, cb) != 0);
                    if (dsum < best) {
                        best = dsum;
                        sum = lo;
                        flag = tf;
                    } else {
                        add_term(sum, flag, lo, tf);
                    }
                }
            }
            if (amax <= bmax) ia += G;
            if (bmax <= amax) ib += G;
        }
        uint32_t gbest = best;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) gbest = min(gbest, tile.shfl_xor(gbest, o));
        if (best != gbest) {
            sum = 0;
            flag = 0;
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const uint64_t os = tile.shfl_xor(sum, o);
            const uint32_t of = tile.shfl_xor(flag, o);
            add_term(sum, flag, os, of);
        }
        if (lane == 0) {
            if (gbest == 0xFFFFFFFFu) {
                Q.out_dist[p] = PSPC_UNREACHED;
                Q.out_cnt[p] = 0;
                if (Q.out_ovf) Q.out_ovf[p] = 0;
            } else {
                Q.out_dist[p] = (uint16_t)gbest;
                Q.out_cnt[p] = sum;
                if (Q.out_ovf) Q.out_ovf[p] = (uint8_t)(flag != 0);
            }
        }
    }
}

// Warp per pair over chunks of CH entries staged in the warp's slice of
// shared memory (one load round trip per chunk instead of one per 32
// entries). Each lane looks up its A hubs in the B chunk by binary search;
// the side whose last hub is smaller advances, and only that side is
// reloaded.
constexpr int kChunkWarps = kQueryThreads / 32;

// At most 40 registers, so that 6 CTAs (48 warps) fit an SM: the kernel
// waits on loads, and more resident warps hide more of that (measured:
// 5.50 -> 5.15 ms for 10^6 pairs on R-MAT 16, without spills).
template <int CH>
__global__ void __launch_bounds__(kQueryThreads, 6) k_query_chunked(const QueryArgs Q) {
    __shared__ uint32_t s_ha[kChunkWarps][CH], s_hb[kChunkWarps][CH];
    __shared__ uint16_t s_da[kChunkWarps][CH], s_db[kChunkWarps][CH];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* ha_s = s_ha[w];
    uint32_t* hb_s = s_hb[w];
    uint16_t* da_s = s_da[w];
    uint16_t* db_s = s_db[w];
    const int64_t nwarps = (int64_t)gridDim.x * kChunkWarps;
    for (int64_t k = (int64_t)blockIdx.x * kChunkWarps + w; k < Q.q; k += nwarps) {
        const int64_t p = Q.perm ? (int64_t)__ldg(Q.perm + k) : k;
        const int32_t s = __ldg(Q.pairs + 2 * p), t = __ldg(Q.pairs + 2 * p + 1);
        if (s < 0 || s >= Q.n || t < 0 || t >= Q.n) {
            if (lane == 0) {
                atomicOr(Q.err, 1);
                Q.out_dist[p] = PSPC_UNREACHED;
                Q.out_cnt[p] = 0;
                if (Q.out_ovf) Q.out_ovf[p] = 0;
            }
            continue;
        }
        if (s == t) {
            if (lane == 0) {
                Q.out_dist[p] = 0;
                Q.out_cnt[p] = 1;
                if (Q.out_ovf) Q.out_ovf[p] = 0;
            }
            continue;
        }
        const int32_t rs = __ldg(Q.rank + s), rt = __ldg(Q.rank + t);
        int64_t ia = __ldg(Q.off + rs);
        const int64_t ea = __ldg(Q.off + rs + 1);
        int64_t ib = __ldg(Q.off + rt);
        const int64_t eb = __ldg(Q.off + rt + 1);
        uint32_t best = 0xFFFFFFFFu;
        uint64_t sum = 0;
        uint32_t flag = 0;
        bool load_a = true, load_b = true;
        while (ia < ea && ib < eb) {
            const int na = ea - ia < CH ? (int)(ea - ia) : CH;
            const int nb = eb - ib < CH ? (int)(eb - ib) : CH;
            if (load_a)
                for (int i = lane; i < CH; i += 32) {
                    ha_s[i] = i < na ? (uint32_t)__ldg(Q.hub + ia + i) : kNoHub;
                    da_s[i] = i < na ? __ldg(Q.dist + ia + i) : (uint16_t)0;
                }
            if (load_b)
                for (int i = lane; i < CH; i += 32) {
                    hb_s[i] = i < nb ? (uint32_t)__ldg(Q.hub + ib + i) : kNoHub;
                    db_s[i] = i < nb ? __ldg(Q.dist + ib + i) : (uint16_t)0;
                }
            __syncwarp();
            const uint32_t amax = ha_s[na - 1], bmax = hb_s[nb - 1];
#pragma unroll
            for (int r = 0; r < CH / 32; ++r) {
                const int i = lane + 32 * r;
                const uint32_t ha = ha_s[i];
                if (i >= na || ha > bmax) continue;
                int lo = 0, hi = nb;  // first B hub >= ha
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (hb_s[mid] < ha) lo = mid + 1; else hi = mid;
                }
                if (lo < nb && hb_s[lo] == ha) {
                    const uint16_t da = da_s[i], dbv = db_s[lo];
                    const uint32_t dsum = (uint32_t)(da & 0x7FFF) + (uint32_t)(dbv & 0x7FFF);
                    if (dsum <= best) {
                        const uint64_t ca = __ldg((const unsigned long long*)Q.cnt + ia + i);
                        const uint64_t cb = __ldg((const unsigned long long*)Q.cnt + ib + lo);
                        const uint64_t prod = ca * cb;
                        const uint32_t tf =
                            (uint32_t)(da >> 15) | (uint32_t)(dbv >> 15) | (uint32_t)(__umul64hi(ca, cb) != 0);
                        if (dsum < best) {
                            best = dsum;
                            sum = prod;
                            flag = tf;
                        } else {
                            add_term(sum, flag, prod, tf);
                        }
                    }
                }
            }
            __syncwarp();
            load_a = amax <= bmax;
            load_b = bmax <= amax;
            if (load_a) ia += na;
            if (load_b) ib += nb;
        }
        finish_pair_warp(Q, p, best, sum, flag, lane);
    }
}

// Pairs grouped by source (perm sorted by s; sources outside [0, n) last).
// The sorted pairs are cut into items of kBySourceItem; a CTA takes items
// in turn and walks each item's runs of pairs with one source s. For a run
// it puts L(s) into an on-chip hash (slot = hub | distance << 24 | entry
// index << 40), then each of its warps answers one pair of the run at a
// time by streaming L(t), kBySourceUnroll loads in flight per lane, and
// probing the hash for each hub. L(s) is read once per run instead of once
// per pair, and no warp waits on a second list. The table has a power of
// two >= 4/3 |L(s)| slots (at most max_slots, which the host sizes from the
// largest label), so it is at most three quarters full and a probe always
// ends at an empty slot.
constexpr int kBySourceItem = 512;
constexpr int kBySourceThreads = 1024;  // CTA size with large tables (one CTA per SM); 256 with small ones
constexpr int kBySourceUnroll = 8;
constexpr unsigned long long kEmptySlot = ~0ull;

__host__ __device__ inline uint32_t by_source_table(uint64_t label) {
    const uint32_t s = pow2_ceil(label + label / 3 + 1);
    return s < 64u ? 64u : s;
}

__global__ void __launch_bounds__(kBySourceThreads) k_query_by_source(const QueryArgs Q, uint32_t max_slots) {
    extern __shared__ unsigned long long tab[];
    __shared__ int32_t s_src[kBySourceItem];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t items = (Q.q + kBySourceItem - 1) / kBySourceItem;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t kb = item * kBySourceItem;
        const int m = (int)(Q.q - kb < kBySourceItem ? Q.q - kb : kBySourceItem);
        for (int i = tid; i < m; i += blockDim.x) s_src[i] = __ldg(Q.pairs + 2 * (int64_t)__ldg(Q.perm + kb + i));
        __syncthreads();
        for (int r0 = 0; r0 < m;) {
            const int32_t s = s_src[r0];
            int r1 = r0 + 1;
            while (r1 < m && s_src[r1] == s) ++r1;
            if (s < 0 || s >= Q.n) {  // the sort puts every invalid source in this bucket
                for (int r = r0 + tid; r < r1; r += blockDim.x) {
                    const int64_t p = __ldg(Q.perm + kb + r);
                    atomicOr(Q.err, 1);
                    write_fixed(Q, p, PSPC_UNREACHED, 0);
                }
                r0 = r1;
                continue;
            }
            const int32_t rs = __ldg(Q.rank + s);
            const int64_t a0 = __ldg(Q.off + rs);
            const uint32_t la = (uint32_t)(__ldg(Q.off + rs + 1) - a0);
            uint32_t slots = by_source_table(la);
            slots = slots > max_slots ? max_slots : slots;
            const uint32_t mask = slots - 1;
            for (uint32_t i = tid; i < slots; i += blockDim.x) tab[i] = kEmptySlot;
            __syncthreads();
            for (uint32_t i = tid; i < la; i += blockDim.x) {
                const uint32_t h = (uint32_t)__ldg(Q.hub + a0 + i);
                const unsigned long long v = (unsigned long long)h | ((unsigned long long)__ldg(Q.dist + a0 + i) << 24) |
                                             ((unsigned long long)i << 40);
                uint32_t slot = hash_hub(h) & mask;
                for (uint32_t probe = 0; probe < slots; ++probe) {
                    if (atomicCAS(&tab[slot], kEmptySlot, v) == kEmptySlot) break;
                    slot = (slot + 1) & mask;
                }
            }
            __syncthreads();
            for (int r = r0 + w; r < r1; r += (int)(blockDim.x >> 5)) {
                const int64_t p = __ldg(Q.perm + kb + r);
                const int32_t t = __ldg(Q.pairs + 2 * p + 1);
                if (t < 0 || t >= Q.n) {
                    if (lane == 0) {
                        atomicOr(Q.err, 1);
                        write_fixed(Q, p, PSPC_UNREACHED, 0);
                    }
                    continue;
                }
                if (t == s) {
                    if (lane == 0) write_fixed(Q, p, 0, 1);
                    continue;
                }
                const int32_t rt = __ldg(Q.rank + t);
                const int64_t b0 = __ldg(Q.off + rt);
                const int64_t lb = __ldg(Q.off + rt + 1) - b0;
                uint32_t best = 0xFFFFFFFFu;
                uint64_t sum = 0;
                uint32_t flag = 0;
                for (int64_t j0 = 0; j0 < lb; j0 += 32 * kBySourceUnroll) {
                    uint32_t hb[kBySourceUnroll];
                    uint16_t db[kBySourceUnroll];
#pragma unroll
                    for (int u = 0; u < kBySourceUnroll; ++u) {
                        const int64_t j = j0 + 32 * u + lane;
                        hb[u] = j < lb ? (uint32_t)__ldg(Q.hub + b0 + j) : kNoHub;
                        db[u] = j < lb ? __ldg(Q.dist + b0 + j) : (uint16_t)0;
                    }
#pragma unroll
                    for (int u = 0; u < kBySourceUnroll; ++u) {
                        if (hb[u] == kNoHub) continue;
                        uint32_t slot = hash_hub(hb[u]) & mask;
                        unsigned long long e = tab[slot];
                        for (uint32_t probe = 0; e != kEmptySlot && (uint32_t)(e & 0xFFFFFFu) != hb[u] && probe < slots;
                             ++probe) {
                            slot = (slot + 1) & mask;
                            e = tab[slot];
                        }
                        if (e == kEmptySlot || (uint32_t)(e & 0xFFFFFFu) != hb[u]) continue;
                        const uint16_t da = (uint16_t)(e >> 24);
                        const uint32_t dsum = (uint32_t)(da & 0x7FFF) + (uint32_t)(db[u] & 0x7FFF);
                        if (dsum > best) continue;
                        const uint64_t ca = __ldg((const unsigned long long*)Q.cnt + a0 + (uint32_t)(e >> 40));
                        const uint64_t cb = __ldg((const unsigned long long*)Q.cnt + b0 + j0 + 32 * u + lane);
                        const uint64_t prod = ca * cb;
                        const uint32_t tf =
                            (uint32_t)(da >> 15) | (uint32_t)(db[u] >> 15) | (uint32_t)(__umul64hi(ca, cb) != 0);
                        if (dsum < best) {
                            best = dsum;
                            sum = prod;
                            flag = tf;
                        } else {
                            add_term(sum, flag, prod, tf);
                        }
                    }
                }
                finish_pair_warp(Q, p, best, sum, flag, lane);
            }
            __syncthreads();
            r0 = r1;
        }
        __syncthreads();  // s_src is rewritten by the next item
    }
}

// One step of L(t) for a lane: entries j0 + 32 u + lane (hub kNoHub past
// the end of the label).
__device__ __forceinline__ void load_step(const int32_t* __restrict__ hubt, const uint16_t* __restrict__ distt,
                                          uint32_t j0, uint32_t lb, int lane, uint32_t (&hb)[kBySourceUnroll],
                                          uint32_t (&db)[kBySourceUnroll]) {
    if (j0 + 32 * kBySourceUnroll <= lb) {
#pragma unroll
        for (int u = 0; u < kBySourceUnroll; ++u) {
            hb[u] = (uint32_t)__ldg(hubt + j0 + 32 * u + lane);
            db[u] = __ldg(distt + j0 + 32 * u + lane);
        }
    } else {
#pragma unroll
        for (int u = 0; u < kBySourceUnroll; ++u) {
            const uint32_t j = j0 + 32 * u + lane;
            hb[u] = j < lb ? (uint32_t)__ldg(hubt + j) : kNoHub;
            db[u] = j < lb ? __ldg(distt + j) : 0u;
        }
    }
}

// Source bucket of sorted pair r (n for a source outside [0, n)).
__device__ __forceinline__ int64_t run_bucket(const QueryArgs& Q, int64_t r) {
    const int32_t v = __ldg(Q.pairs + 2 * (int64_t)__ldg(Q.perm + r));
    return (v >= 0 && v < Q.n) ? (int64_t)v : Q.n;
}

// Entries of the by-source candidate list of a warp: matches at the pair's
// running minimum (position in L(t) << 16 | position in L(s) << 1 | a
// factor's flag), whose counts are read together once the list is full or
// the pair is done.
constexpr uint32_t kBySourceCand = 256;

// Adds the count products of the warp's list to the lanes' partial sums:
// lane i takes entries i, i + 32, ..., so the loads are independent.
__device__ __forceinline__ void add_candidates(const QueryArgs& Q, int64_t a0, const unsigned long long* cntt,
                                               const uint32_t* cw, uint32_t nc, int lane, uint64_t& sum,
                                               uint32_t& flag) {
    __syncwarp();
    for (uint32_t c = lane; c < nc; c += 32) {
        const uint32_t v = cw[c];
        const uint64_t ca = __ldg((const unsigned long long*)Q.cnt + a0 + ((v >> 1) & 0x7FFFu));
        const uint64_t cb = __ldg(cntt + (v >> 16));
        add_term(sum, flag, ca * cb, (v & 1u) | (uint32_t)(__umul64hi(ca, cb) != 0));
    }
    __syncwarp();
}

// The by-source query with direct addressing, for graphs whose vertex
// count fits on chip: pos[h] is the position of hub h in L(s) (0xFFFF:
// absent) and sd[i] the distance of L(s) entry i. Hubs are ranks in
// [0, n), so a lookup is one 2-byte shared-memory read with no probe chain
// (the hash above has chains of several 8-byte reads whose length varies
// across the lanes of a warp). pos is cleared once per CTA; a run sets the
// positions of its L(s) and resets them to 0xFFFF when its pairs are done.
// An item of kBySourceItem sorted pairs owns the runs that start in it and
// takes each whole (its end comes from the grouping sort's bucket ends),
// so every source's L(s) is set up once. The run's pairs are handed to
// warps from a shared counter. Per pair, L(t) streams in steps of
// 32 x kBySourceUnroll entries with the next step's loads in flight; a
// step finds, from shared memory alone, the smallest distance sum among its
// matches over the whole warp, and the matches at the pair's running
// minimum join a per-warp list in shared memory. Counts are read only for
// the list, once per pair (or when it fills), all loads independent: reads
// at every match that reached a lane's minimum so far cost one 32-byte
// sector each and one load round trip each inside the stream.
__global__ void __launch_bounds__(kBySourceThreads)
    k_query_by_source_direct(const QueryArgs Q, uint32_t n_pad, uint32_t label_pad) {
    extern __shared__ uint16_t dsm[];
    uint16_t* pos = dsm;         // n_pad entries (even)
    uint16_t* sd = dsm + n_pad;  // entries of the largest label (label_pad: even)
    __shared__ unsigned long long s_next;
    const int tid = threadIdx.x, lane = tid & 31;
    uint32_t* cw = (uint32_t*)(dsm + n_pad + label_pad) + (tid >> 5) * kBySourceCand;  // the warp's list
    for (uint32_t i = tid; i < n_pad; i += blockDim.x) pos[i] = 0xFFFFu;
    __syncthreads();
    const int64_t items = (Q.q + kBySourceItem - 1) / kBySourceItem;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        // the runs that start in [kb, ke), each in full (one L(s) setup per source)
        const int64_t kb = item * kBySourceItem;
        const int64_t ke = Q.q - kb < kBySourceItem ? Q.q : kb + kBySourceItem;
        int64_t r0 = kb;
        {
            const int64_t b = run_bucket(Q, r0);
            const int64_t start = b > 0 ? (int64_t)__ldg(Q.src_end + b - 1) : 0;
            if (start < kb) r0 = (int64_t)__ldg(Q.src_end + b);  // that run belongs to an earlier item
        }
        while (r0 < ke) {
            const int64_t b = run_bucket(Q, r0);
            const int64_t r1 = (int64_t)__ldg(Q.src_end + b);
            const int32_t s = (int32_t)b;
            if (b >= Q.n) {  // the sort puts every invalid source in bucket n
                for (int64_t r = r0 + tid; r < r1; r += blockDim.x) {
                    const int64_t p = __ldg(Q.perm + r);
                    atomicOr(Q.err, 1);
                    write_fixed(Q, p, PSPC_UNREACHED, 0);
                }
                r0 = r1;
                continue;
            }
            const int32_t rs = __ldg(Q.rank + s);
            const int64_t a0 = __ldg(Q.off + rs);
            const uint32_t la = (uint32_t)(__ldg(Q.off + rs + 1) - a0);
            for (uint32_t i = tid; i < la; i += blockDim.x) {
                pos[__ldg(Q.hub + a0 + i)] = (uint16_t)i;
                sd[i] = __ldg(Q.dist + a0 + i);
            }
            if (tid == 0) s_next = (unsigned long long)r0;
            __syncthreads();
            for (;;) {
                unsigned long long r = 0;
                if (lane == 0) r = atomicAdd(&s_next, 1ull);
                r = __shfl_sync(0xFFFFFFFFu, r, 0);
                if ((int64_t)r >= r1) break;
                const int64_t p = __ldg(Q.perm + r);
                const int32_t t = __ldg(Q.pairs + 2 * p + 1);
                if (t < 0 || t >= Q.n) {
                    if (lane == 0) {
                        atomicOr(Q.err, 1);
                        write_fixed(Q, p, PSPC_UNREACHED, 0);
                    }
                    continue;
                }
                if (t == s) {
                    if (lane == 0) write_fixed(Q, p, 0, 1);
                    continue;
                }
                const int32_t rt = __ldg(Q.rank + t);
                const int64_t b0 = __ldg(Q.off + rt);
                const int64_t lb = __ldg(Q.off + rt + 1) - b0;
                const int32_t* hubt = Q.hub + b0;
                const uint16_t* distt = Q.dist + b0;
                const unsigned long long* cntt = (const unsigned long long*)Q.cnt + b0;
                uint32_t best = 0xFFFFu;  // the pair's minimum distance sum so far (0xFFFF: none)
                uint64_t sum = 0;
                uint32_t flag = 0;
                uint32_t nc = 0;  // entries in the warp's list (warp-uniform)
                // L(t) in steps of 32 x kBySourceUnroll entries; the next step's
                // loads are in flight while this step probes
                const uint32_t lbu = (uint32_t)lb;
                uint32_t nh[kBySourceUnroll], nd[kBySourceUnroll];
                load_step(hubt, distt, 0, lbu, lane, nh, nd);
                for (uint32_t j0 = 0; j0 < lbu; j0 += 32 * kBySourceUnroll) {
                    uint32_t hb[kBySourceUnroll], db[kBySourceUnroll];
#pragma unroll
                    for (int u = 0; u < kBySourceUnroll; ++u) {
                        hb[u] = nh[u];
                        db[u] = nd[u];
                    }
                    if (j0 + 32 * kBySourceUnroll < lbu) load_step(hubt, distt, j0 + 32 * kBySourceUnroll, lbu, lane, nh, nd);
                    // key of a match: distance sum << 16 | L(s) position (15 bits) << 1 | a factor's flag
                    uint32_t key[kBySourceUnroll];
                    uint32_t kmin = 0xFFFFFFFFu;
#pragma unroll
                    for (int u = 0; u < kBySourceUnroll; ++u) {
                        const uint32_t ia = hb[u] == kNoHub ? 0xFFFFu : (uint32_t)pos[hb[u]];
                        const uint32_t da = ia == 0xFFFFu ? 0u : (uint32_t)sd[ia];
                        key[u] = ia == 0xFFFFu ? 0xFFFFFFFFu
                                               : ((da & 0x7FFFu) + (db[u] & 0x7FFFu)) << 16 | ia << 1 | ((da | db[u]) >> 15);
                        kmin = min(kmin, key[u]);
                    }
                    // the matches at the running minimum join the warp's list
                    uint32_t cmin = kmin >> 16;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cmin = min(cmin, __shfl_xor_sync(0xFFFFFFFFu, cmin, o));
                    if (cmin == 0xFFFFu || cmin > best) continue;  // warp-uniform
                    if (cmin < best) {  // a smaller sum: what the list and the sum hold is superseded
                        best = cmin;
                        nc = 0;
                        sum = 0;
                        flag = 0;
                    }
#pragma unroll
                    for (int u = 0; u < kBySourceUnroll; ++u) {
                        const bool hit = (key[u] >> 16) == best;
                        const uint32_t m = __ballot_sync(0xFFFFFFFFu, hit);
                        if (m == 0) continue;
                        if (nc + (uint32_t)__popc(m) > kBySourceCand) {  // rare: a full list
                            add_candidates(Q, a0, cntt, cw, nc, lane, sum, flag);
                            nc = 0;
                        }
                        if (hit)
                            cw[nc + (uint32_t)__popc(m & ((1u << lane) - 1u))] =
                                (j0 + 32 * u + lane) << 16 | (key[u] & 0xFFFFu);
                        nc += (uint32_t)__popc(m);
                    }
                }
                add_candidates(Q, a0, cntt, cw, nc, lane, sum, flag);
                finish_pair_warp(Q, p, best == 0xFFFFu ? 0xFFFFFFFFu : best, sum, flag, lane);
            }
            __syncthreads();
            for (uint32_t i = tid; i < la; i += blockDim.x) pos[__ldg(Q.hub + a0 + i)] = 0xFFFFu;
            __syncthreads();
            r0 = r1;
        }
    }
}

// Grouping by source: a counting sort of the pair indices by s, so that the
// pairs sharing a source run back to back and reuse L(s) from cache. Ids
// outside [0, n) go to an extra bucket n (they are rejected later).
__global__ void k_pair_hist(const int32_t* __restrict__ pairs, int64_t q, int64_t n,
                            unsigned long long* __restrict__ cnt) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= q) return;
    const int32_t s = pairs[2 * p];
    atomicAdd(cnt + ((s >= 0 && s < n) ? s : n), 1ull);
}

__global__ void k_pair_scatter(const int32_t* __restrict__ pairs, int64_t q, int64_t n,
                               unsigned long long* __restrict__ pos, int32_t* __restrict__ perm) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= q) return;
    const int32_t s = pairs[2 * p];
    perm[atomicAdd(pos + ((s >= 0 && s < n) ? s : n), 1ull)] = (int32_t)p;
}

// All query kernels prefer the largest shared-memory carve-out, the
// configuration the build kernels run in, so that query blocks can share
// SMs with a build running on another stream instead of waiting for those
// SMs to drain and change configuration.
static void prefer_max_shared(const void* fn) {
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

static std::once_flag g_carveout_once;

constexpr uint32_t kBySourceMaxSlots = 16384;  // 128 KB of table
// Shared memory the direct-address variant may take: 2 bytes per vertex and
// per entry of the largest label (within the 227 KB a CTA can have, less
// the kernel's static arrays).
constexpr size_t kBySourceDirectBytes = 224 * 1024;

static void set_query_carveouts() {
    std::call_once(g_carveout_once, [] {
        prefer_max_shared((const void*)k_query_by_source);
        cudaFuncSetAttribute((const void*)k_query_by_source, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kBySourceMaxSlots * 8));
        prefer_max_shared((const void*)k_query_by_source_direct);
        cudaFuncSetAttribute((const void*)k_query_by_source_direct, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBySourceDirectBytes);
        prefer_max_shared((const void*)k_query<8>);
        prefer_max_shared((const void*)k_query<16>);
        prefer_max_shared((const void*)k_query<32>);
        prefer_max_shared((const void*)k_query_chunked<64>);
        prefer_max_shared((const void*)k_query_chunked<128>);
        prefer_max_shared((const void*)k_query_chunked<256>);
    });
}

// Table slots the by-source kernel needs for the largest label (0: it does
// not fit on chip).
static uint32_t by_source_slots(const Index& ix) {
    const uint32_t s = by_source_table((uint64_t)(ix.max_label > 0 ? ix.max_label : 1));
    return s <= kBySourceMaxSlots ? s : 0u;
}

// Positions of the largest label the direct-address by-source kernel keeps
// in shared memory (rounded up to even, so the lists after them are 4-byte
// aligned).
static uint32_t by_source_label_pad(const Index& ix) {
    return (uint32_t)(((ix.max_label > 0 ? ix.max_label : 1) + 1) & ~(int64_t)1);
}

// Shared-memory bytes of the direct-address by-source kernel's vertex
// positions and largest label (0: with the candidate lists of a 1024-thread
// CTA they do not fit on chip, or a position does not fit the 15 bits the
// kernel keeps of it).
static size_t by_source_direct_bytes(const Index& ix) {
    if (ix.max_label > 0x7FFF) return 0;
    const size_t b = 2 * (size_t)((ix.n + 1) & ~(int64_t)1) + 2 * (size_t)by_source_label_pad(ix);
    return b + (size_t)(kBySourceThreads / 32) * kBySourceCand * 4 <= kBySourceDirectBytes ? b : 0;
}

// The query kernel. Automatic choice: by source when the pairs are grouped,
// L(s) fits on chip and sources repeat often (q >= 64 n: each table build
// serves many pairs; with fewer pairs per source the staged merge-join,
// whose L(s) reads mostly hit L2 after the grouping sort, measured faster);
// otherwise lanes per pair from the label sizes: wide groups for long
// labels (fewer merge steps), narrow groups for short ones (more pairs in
// flight per warp), warp-staged chunks of 256 entries for long labels.
static int query_group_for(const Index& ix, bool grouped, int64_t q) {
    const bool by_source_ok = grouped && (by_source_direct_bytes(ix) > 0 || by_source_slots(ix) > 0);
    if (ix.query_group == PSPC_QUERY_BY_SOURCE && by_source_ok) return PSPC_QUERY_BY_SOURCE;
    if (ix.query_group == PSPC_QUERY_BY_SOURCE_HASH && grouped && by_source_slots(ix) > 0)
        return PSPC_QUERY_BY_SOURCE_HASH;
    if (ix.query_group && ix.query_group != PSPC_QUERY_BY_SOURCE && ix.query_group != PSPC_QUERY_BY_SOURCE_HASH)
        return ix.query_group;
    if (ix.query_group == 0 && by_source_ok && q >= 64 * ix.n) return PSPC_QUERY_BY_SOURCE;
    const double avg = ix.n ? (double)ix.entries / (double)ix.n : 0.0;
    return avg >= 128.0 ? 256 : (avg >= 24.0 ? 16 : 8);
}

// Whether a call groups its pairs by source (both pspc_query and
// pspc_query_noalloc): when sources repeat enough for L(s) to be reused.
static bool groups_by_source(const Index& ix, int64_t q) {
    return q >= 4096 && q >= ix.n / 4 && q < ((int64_t)1 << 31);
}

// Launches the query kernel chosen for the index (Q.perm is the grouping
// sort's order, or NULL). Counts the launch on the index.
static cudaError_t launch_query(Index& ix, const QueryArgs& Q, cudaStream_t st) {
    set_query_carveouts();
    const int G = query_group_for(ix, Q.perm != nullptr, Q.q);
    int sms = 0, occ = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix.device);
    if (e != cudaSuccess) return e;
    __atomic_fetch_add(&ix.query_launches, (int64_t)1, __ATOMIC_RELAXED);
    if (G == PSPC_QUERY_BY_SOURCE && by_source_direct_bytes(ix) > 0) {
        // positions above a ninth of the shared memory leave room for one CTA
        // per SM: make it a large one; smaller tables share SMs
        const size_t base = by_source_direct_bytes(ix);
        const int threads = base > (size_t)24 * 1024 ? kBySourceThreads : kQueryThreads;
        const size_t smem = base + (size_t)(threads / 32) * kBySourceCand * 4;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_query_by_source_direct, threads, smem);
        if (e != cudaSuccess) return e;
        const int64_t items = (Q.q + kBySourceItem - 1) / kBySourceItem;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)sms * std::max(occ, 1)));
        k_query_by_source_direct<<<grid, threads, smem, st>>>(Q, (uint32_t)((ix.n + 1) & ~(int64_t)1),
                                                             by_source_label_pad(ix));
        return cudaGetLastError();
    }
    if (G == PSPC_QUERY_BY_SOURCE || G == PSPC_QUERY_BY_SOURCE_HASH) {
        const uint32_t slots = by_source_slots(ix);
        const size_t smem = (size_t)slots * 8;
        // tables above a quarter of the shared memory leave room for one CTA
        // per SM: make it a large one; smaller tables share SMs
        const int threads = smem > (size_t)56 * 1024 ? kBySourceThreads : kQueryThreads;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_query_by_source, threads, smem);
        if (e != cudaSuccess) return e;
        const int64_t items = (Q.q + kBySourceItem - 1) / kBySourceItem;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)sms * std::max(occ, 1)));
        k_query_by_source<<<grid, threads, smem, st>>>(Q, slots);
        return cudaGetLastError();
    }
    const void* fn = G == 8 ? (const void*)k_query<8>
                     : G == 16 ? (const void*)k_query<16>
                     : G == 32 ? (const void*)k_query<32>
                     : G == 64 ? (const void*)k_query_chunked<64>
                     : G == 128 ? (const void*)k_query_chunked<128>
                                : (const void*)k_query_chunked<256>;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kQueryThreads, 0);
    if (e != cudaSuccess) return e;
    const int64_t per_block = G >= 64 ? kChunkWarps : kQueryThreads / G;
    const int64_t want = (Q.q + per_block - 1) / per_block;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * std::max(occ, 1)));
    if (G == 8) k_query<8><<<grid, kQueryThreads, 0, st>>>(Q);
    else if (G == 16) k_query<16><<<grid, kQueryThreads, 0, st>>>(Q);
    else if (G == 32) k_query<32><<<grid, kQueryThreads, 0, st>>>(Q);
    else if (G == 64) k_query_chunked<64><<<grid, kQueryThreads, 0, st>>>(Q);
    else if (G == 128) k_query_chunked<128><<<grid, kQueryThreads, 0, st>>>(Q);
    else k_query_chunked<256><<<grid, kQueryThreads, 0, st>>>(Q);
    return cudaGetLastError();
}

}  // namespace pspc

using namespace pspc;

// A query batch on an index built with the 1-shell reduction: pairs with
// s = t or a common root are answered by the tree path; the rest become
// the pairs of their roots in core ids, go through pspc_query on the core
// index, and get their depths added.
static int query_reduced(const Index& ix, const int32_t* pairs, int64_t q, uint16_t* dist, uint64_t* count,
                         uint8_t* overflow, cudaStream_t st) {
    const bool dev_in = is_device_ptr(pairs), dev_out = is_device_ptr(dist);
    if (dev_out != is_device_ptr(count) || (overflow && dev_out != is_device_ptr(overflow))) return PSPC_E_INVAL;
    int32_t *d_pairs = nullptr, *cpairs = nullptr, *extra = nullptr;
    uint16_t *d_dist = nullptr, *cd = nullptr;
    uint64_t *d_cnt = nullptr, *cc = nullptr;
    uint8_t *d_ovf = nullptr, *co = nullptr;
    int* d_err = nullptr;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = dev_alloc(p, bytes, st);
    };
    alloc((void**)&d_err, sizeof(int));
    if (!dev_in) alloc((void**)&d_pairs, (size_t)q * 8);
    if (!dev_out) {
        alloc((void**)&d_dist, (size_t)q * 2);
        alloc((void**)&d_cnt, (size_t)q * 8);
        alloc((void**)&d_ovf, (size_t)q);
    }
    alloc((void**)&cpairs, (size_t)q * 8);
    alloc((void**)&extra, (size_t)q * 4);
    alloc((void**)&cd, (size_t)q * 2);
    alloc((void**)&cc, (size_t)q * 8);
    alloc((void**)&co, (size_t)q);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess && !dev_in) e = cudaMemcpyAsync(d_pairs, pairs, (size_t)q * 8, cudaMemcpyHostToDevice, st);
    const int32_t* pin = dev_in ? pairs : d_pairs;
    uint16_t* od = dev_out ? dist : d_dist;
    uint64_t* oc = dev_out ? count : d_cnt;
    uint8_t* oo = dev_out ? overflow : d_ovf;
    if (e == cudaSuccess) e = launch_shell_pairs(ix, pin, q, cpairs, extra, od, oc, oo, d_err, st);
    int rc = PSPC_OK;
    if (e == cudaSuccess) rc = pspc_query(ix.core, cpairs, q, cd, cc, co, st);
    if (e == cudaSuccess && rc == PSPC_OK) e = launch_shell_combine(q, extra, cd, cc, co, od, oc, oo, d_err, st);
    if (e == cudaSuccess && rc == PSPC_OK && !dev_out) {
        e = cudaMemcpyAsync(dist, d_dist, (size_t)q * 2, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(count, d_cnt, (size_t)q * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && overflow)
            e = cudaMemcpyAsync(overflow, d_ovf, (size_t)q, cudaMemcpyDeviceToHost, st);
    }
    int herr = 0;
    if (e == cudaSuccess && rc == PSPC_OK) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_status(e);
    else if (rc == PSPC_OK && (herr & 1)) rc = PSPC_E_INVAL;
    else if (rc == PSPC_OK && (herr & 2)) rc = PSPC_E_DIST;
    dev_free(d_err, st);
    dev_free(d_pairs, st);
    dev_free(d_dist, st);
    dev_free(d_cnt, st);
    dev_free(d_ovf, st);
    dev_free(cpairs, st);
    dev_free(extra, st);
    dev_free(cd, st);
    dev_free(cc, st);
    dev_free(co, st);
    return rc;
}

extern "C" int pspc_query(const pspc_index* hc, const int32_t* pairs, int64_t q, uint16_t* dist, uint64_t* count,
                          uint8_t* overflow, void* stream) {
    if (!hc || q < 0) return PSPC_E_INVAL;
    if (q == 0) return PSPC_OK;
    if (hc->ix.core) {
        if (!pairs || !dist || !count) return PSPC_E_INVAL;
        int prev = 0;
        cudaGetDevice(&prev);
        if (prev != hc->ix.device) PSPC_TRY_CUDA(cudaSetDevice(hc->ix.device));
        const int rc = query_reduced(hc->ix, pairs, q, dist, count, overflow, (cudaStream_t)stream);
        if (prev != hc->ix.device) cudaSetDevice(prev);
        return rc;
    }
    pspc_index* h = const_cast<pspc_index*>(hc);  // only the launch counter changes
    if (!pairs || !dist || !count) return PSPC_E_INVAL;
    const Index& ix = h->ix;
    cudaStream_t st = (cudaStream_t)stream;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ix.device) PSPC_TRY_CUDA(cudaSetDevice(ix.device));
    const bool dev_in = is_device_ptr(pairs);
    const bool dev_out = is_device_ptr(dist);
    if (dev_out != is_device_ptr(count) || (overflow && dev_out != is_device_ptr(overflow))) {
        if (prev != ix.device) cudaSetDevice(prev);
        return PSPC_E_INVAL;
    }
    int32_t* d_pairs = nullptr;
    uint16_t* d_dist = nullptr;
    uint64_t* d_cnt = nullptr;
    uint8_t* d_ovf = nullptr;
    int* d_err = nullptr;
    int rc = PSPC_OK;
    cudaError_t e = dev_alloc((void**)&d_err, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess && !dev_in) {
        e = dev_alloc((void**)&d_pairs, (size_t)q * 8, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_pairs, pairs, (size_t)q * 8, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && !dev_out) {
        e = dev_alloc((void**)&d_dist, (size_t)q * 2, st);
        if (e == cudaSuccess) e = dev_alloc((void**)&d_cnt, (size_t)q * 8, st);
        if (e == cudaSuccess && overflow) e = dev_alloc((void**)&d_ovf, (size_t)q, st);
    }
    // Group by source when sources repeat enough for L(s) to be reused.
    int32_t* d_perm = nullptr;
    int64_t* d_bins = nullptr;
    const bool group = groups_by_source(ix, q);
    if (e == cudaSuccess && group) {
        const int32_t* pin = dev_in ? pairs : d_pairs;
        e = dev_alloc((void**)&d_perm, (size_t)q * 4, st);
        if (e == cudaSuccess) e = dev_alloc((void**)&d_bins, (size_t)(ix.n + 2) * 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_bins, 0, (size_t)(ix.n + 2) * 8, st);
        if (e == cudaSuccess) {
            k_pair_hist<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(pin, q, ix.n, (unsigned long long*)d_bins);
            __atomic_fetch_add(&h->ix.query_launches, (int64_t)2, __ATOMIC_RELAXED);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            int64_t scan_launches = 0;
            rc = exclusive_scan_i64(d_bins, ix.n + 1, st, &scan_launches);
            __atomic_fetch_add(&h->ix.query_launches, scan_launches, __ATOMIC_RELAXED);
        }
        if (e == cudaSuccess && rc == PSPC_OK) {
            k_pair_scatter<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(pin, q, ix.n, (unsigned long long*)d_bins,
                                                                       d_perm);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && rc == PSPC_OK) {
        QueryArgs Q;
        Q.perm = d_perm;
        Q.src_end = (const unsigned long long*)d_bins;
        Q.n = ix.n;
        Q.rank = ix.rank;
        Q.off = ix.off;
        Q.hub = ix.hub;
        Q.dist = ix.dist;
        Q.cnt = ix.cnt;
        Q.pairs = dev_in ? pairs : d_pairs;
        Q.q = q;
        Q.out_dist = dev_out ? dist : d_dist;
        Q.out_cnt = dev_out ? count : d_cnt;
        Q.out_ovf = dev_out ? overflow : d_ovf;
        Q.err = d_err;
        e = launch_query(h->ix, Q, st);
    }
    if (e == cudaSuccess && !dev_out) {
        e = cudaMemcpyAsync(dist, d_dist, (size_t)q * 2, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(count, d_cnt, (size_t)q * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && overflow) e = cudaMemcpyAsync(overflow, d_ovf, (size_t)q, cudaMemcpyDeviceToHost, st);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_status(e);
    else if (herr && rc == PSPC_OK) rc = PSPC_E_INVAL;
    dev_free(d_perm, st);
    dev_free(d_bins, st);
    dev_free(d_pairs, st);
    dev_free(d_dist, st);
    dev_free(d_cnt, st);
    dev_free(d_ovf, st);
    dev_free(d_err, st);
    if (prev != ix.device) cudaSetDevice(prev);
    return rc;
}

extern "C" int pspc_set_query_group(pspc_index* h, int32_t lanes) {
    if (!h || !(lanes == 0 || lanes == PSPC_QUERY_BY_SOURCE || lanes == PSPC_QUERY_BY_SOURCE_HASH || lanes == 8 ||
                lanes == 16 || lanes == 32 || lanes == 64 || lanes == 128 || lanes == 256))
        return PSPC_E_INVAL;
    h->ix.query_group = lanes;
    if (h->ix.core) h->ix.core->ix.query_group = lanes;  // the core index runs the queries
    return PSPC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free queries.
//
// pspc_query allocates its working memory (the source-grouping permutation,
// the per-source bins, the error flag, staging for host buffers) from the
// library's device pool. Some callers cannot allow any device allocation
// during a query: an engine whose device memory is entirely owned by
// another allocator, a latency-critical serving loop that must not touch
// the driver's allocator, or a process that has reserved all device memory
// up front. pspc_query_noalloc answers the same queries with the same
// kernels, but its working memory is one file-scope device array of
// kNoallocScratchBytes that every GPU loading this library holds until the
// process exits.

namespace pspc {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;  // PSPC_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the host-side symbol is not a device address).
static cudaError_t noalloc_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace pspc

extern "C" int pspc_query_noalloc(const pspc_index* hc, const int32_t* pairs, int64_t q, uint16_t* dist,
                                  uint64_t* count, uint8_t* overflow, void* stream) {
    if (!hc || q < 0 || q >= ((int64_t)1 << 40)) return PSPC_E_INVAL;
    if (q == 0) return PSPC_OK;
    if (!pairs || !dist || !count || hc->ix.core) return PSPC_E_INVAL;
    pspc_index* h = const_cast<pspc_index*>(hc);  // only the launch counter changes
    const Index& ix = h->ix;
    // Scratch layout: error flag | n+2 source bins | scan partials | q pair
    // indices. Only calls that group by source use more than the flag.
    const bool group = groups_by_source(ix, q);
    const size_t bins_off = 256;
    const size_t part_off = bins_off + (((size_t)(ix.n + 2) * 8 + 255) & ~(size_t)255);
    const size_t perm_off = part_off + (((size_t)scan_scratch_entries(ix.n + 2) * 8 + 255) & ~(size_t)255);
    if (group && perm_off + (size_t)q * 4 > kNoallocScratchBytes) return PSPC_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ix.device) PSPC_TRY_CUDA(cudaSetDevice(ix.device));
    int rc = PSPC_OK;
    if (!is_device_ptr(pairs) || !is_device_ptr(dist) || !is_device_ptr(count) ||
        (overflow && !is_device_ptr(overflow)))
        rc = PSPC_E_INVAL;  // host buffers would need staging memory
    unsigned char* scratch = nullptr;
    cudaError_t e = cudaSuccess;
    if (rc == PSPC_OK) e = noalloc_scratch(ix.device, &scratch);
    if (rc == PSPC_OK && e == cudaSuccess) {
        int* d_err = (int*)scratch;
        int64_t* d_bins = (int64_t*)(scratch + bins_off);
        int64_t* d_part = (int64_t*)(scratch + part_off);
        int32_t* d_perm = group ? (int32_t*)(scratch + perm_off) : nullptr;
        // The array keeps the previous call's contents: clear what is counted.
        e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
        if (e == cudaSuccess && group) e = cudaMemsetAsync(d_bins, 0, (size_t)(ix.n + 2) * 8, st);
        if (e == cudaSuccess && group) {
            k_pair_hist<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(pairs, q, ix.n, (unsigned long long*)d_bins);
            __atomic_fetch_add(&h->ix.query_launches, (int64_t)2, __ATOMIC_RELAXED);
            e = cudaGetLastError();
            if (e == cudaSuccess) {
                int64_t scan_launches = 0;
                rc = exclusive_scan_i64(d_bins, ix.n + 1, st, &scan_launches, d_part);
                __atomic_fetch_add(&h->ix.query_launches, scan_launches, __ATOMIC_RELAXED);
            }
            if (e == cudaSuccess && rc == PSPC_OK) {
                k_pair_scatter<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(pairs, q, ix.n,
                                                                           (unsigned long long*)d_bins, d_perm);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess && rc == PSPC_OK) {
            QueryArgs Q;
            Q.n = ix.n;
            Q.rank = ix.rank;
            Q.off = ix.off;
            Q.hub = ix.hub;
            Q.dist = ix.dist;
            Q.cnt = ix.cnt;
            Q.pairs = pairs;
            Q.perm = d_perm;
            Q.src_end = (const unsigned long long*)d_bins;
            Q.q = q;
            Q.out_dist = dist;
            Q.out_cnt = count;
            Q.out_ovf = overflow;
            Q.err = d_err;
            e = launch_query(h->ix, Q, st);
        }
        int herr = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && herr && rc == PSPC_OK) rc = PSPC_E_INVAL;
    }
    if (e != cudaSuccess) rc = cuda_status(e);
    if (prev != ix.device) cudaSetDevice(prev);
    return rc;
}

// ---------------------------------------------------------------------------
// Stream-ordered queries for CUDA graphs: no host synchronisation, no
// allocation, errors reported through a caller-provided device flag.

extern "C" int pspc_query_async(const pspc_index* hc, const int32_t* pairs, int64_t q, uint16_t* dist,
                                uint64_t* count, uint8_t* overflow, int32_t* err, void* stream) {
    if (!hc || q < 0 || q >= ((int64_t)1 << 40)) return PSPC_E_INVAL;
    if (q == 0) return PSPC_OK;
    if (!pairs || !dist || !count || !err || hc->ix.core) return PSPC_E_INVAL;
    pspc_index* h = const_cast<pspc_index*>(hc);  // only the launch counter changes
    const Index& ix = h->ix;
    int cur = 0;
    PSPC_TRY_CUDA(cudaGetDevice(&cur));
    if (cur != ix.device) return PSPC_E_INVAL;  // the stream belongs to the index's device
    if (!is_device_ptr(pairs) || !is_device_ptr(dist) || !is_device_ptr(count) || !is_device_ptr(err) ||
        (overflow && !is_device_ptr(overflow)))
        return PSPC_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    PSPC_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    QueryArgs Q;
    Q.n = ix.n;
    Q.rank = ix.rank;
    Q.off = ix.off;
    Q.hub = ix.hub;
    Q.dist = ix.dist;
    Q.cnt = ix.cnt;
    Q.pairs = pairs;
    Q.perm = nullptr;
    Q.src_end = nullptr;
    Q.q = q;
    Q.out_dist = dist;
    Q.out_cnt = count;
    Q.out_ovf = overflow;
    Q.err = err;
    return cuda_status(launch_query(h->ix, Q, st));
}
