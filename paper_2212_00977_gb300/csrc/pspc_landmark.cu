// Landmark labelling for the landmark filter of pruning rule 2 (Section
// "Landmark-Based Filtering"). The first landmarks of a graph (up to
// kLmkShallow) are its highest-ranked vertices; under a degree order these
// are the vertices whose degree reaches the k-th largest degree, the
// paper's degree threshold. The filter needs sd(v, l) for every vertex v and
// landmark l: the searches of a round run together, one BFS level per
// launch. Every vertex keeps a 64-bit mask of the round's landmarks that
// have reached it; at level t it takes the OR of its neighbours' frontier
// masks, and the bits new to it get distance t.
//
// The remaining landmarks of a single graph (k > kLmkShallow; the filter
// tests them from level kLmkDeepLevel on) are spread out instead: a
// survivor h of u at level d is proven by landmark l when
// |sd(u,l) - sd(h,l)| >= d, that is when l lies behind h on a shortest path
// from u (or behind u), and for far-apart u and h that region is near the
// graph's periphery, where high-ranked vertices of a high-diameter graph
// seldom lie. Each spread landmark, chosen in turn, maximises over the
// vertices reached in the first round the smaller of (a) its distance to
// the first round's landmarks and (b) the landmark lower bound
// max_j |sd(v,l_j) - sd(p,l_j)| of its distance to every spread landmark p
// chosen before it (ties to the smaller id), so it is far from all of
// them; a second round of searches gives their distances. When no vertex
// is farther than D from the first landmarks and 2D < kLmkDeepLevel, the
// labels they cover stop short of the levels that test spread landmarks,
// and none are placed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "pspc_level.cuh"

namespace pspc {

constexpr int kLmkGroup = 8;         // lanes per vertex in a BFS level
constexpr int kLmkThreads = 256;
constexpr int kLmkLevelsPerCheck = 4;  // BFS levels launched between host checks
constexpr int kLmkMaxDist = 65534;   // 0xFFFF marks "unreached" (or no such landmark)

// Row v of the distance table: `stride` bytes holding k uint16 distances.
__device__ __forceinline__ uint16_t* lmk_row(uint8_t* ld, int64_t v, int stride) {
    return (uint16_t*)(ld + v * stride);
}

__global__ void k_lmk_init(int64_t n, int k, int stride, const int32_t* __restrict__ comp_base,
                           uint64_t* __restrict__ visited, uint64_t* __restrict__ frontier, uint8_t* __restrict__ ld) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    uint4* row = (uint4*)(ld + v * stride);
    for (int w = 0; w < stride / 16; ++w) row[w] = make_uint4(~0u, ~0u, ~0u, ~0u);
    const int64_t j = v - (comp_base ? (int64_t)comp_base[v] : 0);
    const bool is_lmk = j < k;
    visited[v] = is_lmk ? (1ull << j) : 0ull;
    frontier[v] = visited[v];
    if (is_lmk) lmk_row(ld, v, stride)[j] = 0;
}

// One BFS level for all landmarks of a round: kLmkGroup lanes per vertex OR
// the frontier masks of its neighbours; bit j is landmark slot slot0 + j.
__global__ void __launch_bounds__(kLmkThreads)
    k_lmk_level(int64_t n, int stride, int level, uint64_t full, int slot0, const int64_t* __restrict__ rp,
                const int32_t* __restrict__ col, const uint64_t* __restrict__ frontier, uint64_t* __restrict__ next,
                uint64_t* __restrict__ visited, uint8_t* __restrict__ ld, int* __restrict__ changed) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kLmkGroup;
    const int gl = threadIdx.x % kLmkGroup;
    uint64_t acc = 0, vis = full;
    if (v < n) {
        vis = visited[v];
        if (vis != full)
            for (int64_t a = rp[v] + gl; a < rp[v + 1]; a += kLmkGroup) acc |= __ldg(frontier + __ldg(col + a));
    }
#pragma unroll
    for (int o = kLmkGroup / 2; o > 0; o >>= 1) acc |= __shfl_xor_sync(0xFFFFFFFFu, acc, o, kLmkGroup);
    if (v >= n) return;
    const uint64_t fresh = acc & ~vis;
    if (gl == 0) {
        next[v] = fresh;
        if (fresh) {
            visited[v] = vis | fresh;
            *changed = 1;
        }
    }
    for (int j = gl; j < 64; j += kLmkGroup)
        if ((fresh >> j) & 1ull) lmk_row(ld, v, stride)[slot0 + j] = (uint16_t)level;
}

// Spread landmarks. cur[v]: the score of v (the smaller of its distance to
// the first round's k1 landmarks and its lower bounds to the spread ones
// chosen so far); 0 for vertices no first-round landmark reached. dmax: the
// largest distance of any vertex from a first-round landmark.
__global__ void k_lmk_score(int64_t n, int stride, int k1, const uint8_t* __restrict__ ld, uint32_t* __restrict__ cur,
                            unsigned* __restrict__ dmax) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t m = 0xFFFFFFFFu, far = 0;
    if (v < n) {
        const uint16_t* r = (const uint16_t*)(ld + v * stride);
        for (int j = 0; j < k1; ++j)
            if (r[j] != 0xFFFFu) {
                m = min(m, (uint32_t)r[j]);
                far = max(far, (uint32_t)r[j]);
            }
        cur[v] = m == 0xFFFFFFFFu ? 0u : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) far = max(far, __shfl_xor_sync(0xFFFFFFFFu, far, o));
    if ((threadIdx.x & 31) == 0 && far) atomicMax(dmax, far);
}

// The largest score, ties to the smaller id: key = score << 32 | ~v.
__global__ void k_lmk_argmax(int64_t n, const uint32_t* __restrict__ cur, unsigned long long* __restrict__ key) {
    unsigned long long best = 0ull;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        best = max(best, (unsigned long long)cur[v] << 32 | (0xFFFFFFFFull - (unsigned long long)v));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

// Takes the chosen vertex p as spread landmark `slot` (ids[slot]) and
// lowers every score to the landmark lower bound of sd(v, p) (0xFFFF when
// exactly one of v, p was reached by some first-round landmark: they are
// not connected).
__global__ void k_lmk_take(int64_t n, int stride, int k1, const uint8_t* __restrict__ ld, uint32_t* __restrict__ cur,
                           const unsigned long long* __restrict__ key, int32_t* __restrict__ ids, int slot) {
    const int64_t p = (int64_t)(0xFFFFFFFFull - (*key & 0xFFFFFFFFull));
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v == 0) ids[slot] = (int32_t)p;
    if (v >= n || p >= n) return;
    const uint16_t* rv = (const uint16_t*)(ld + v * stride);
    const uint16_t* rp = (const uint16_t*)(ld + p * stride);
    uint32_t lb = 0;
    for (int j = 0; j < k1; ++j) {
        const uint32_t a = rv[j], b = rp[j];
        if (a == 0xFFFFu && b == 0xFFFFu) continue;
        if (a == 0xFFFFu || b == 0xFFFFu) {
            lb = 0xFFFFu;
            break;
        }
        lb = max(lb, a > b ? a - b : b - a);
    }
    cur[v] = min(cur[v], lb);
}

// Sources of a later round: landmark slot s0 + j at vertex ids[s0 + j]
// (none for -1).
__global__ void k_lmk_seed(int64_t n, int s0, int count, int stride, const int32_t* __restrict__ ids,
                           uint64_t* __restrict__ visited, uint64_t* __restrict__ frontier, uint8_t* __restrict__ ld) {
    const int j = threadIdx.x;
    if (j >= count) return;
    const int64_t v = ids[s0 + j];
    if (v < 0 || v >= n) return;
    atomicOr((unsigned long long*)&visited[v], 1ull << j);
    atomicOr((unsigned long long*)&frontier[v], 1ull << j);
    lmk_row(ld, v, stride)[s0 + j] = 0;
}

// The searches of one round: bits of `full` from the round's sources
// (already set in visited and fa), distances into slots slot0 + j.
static cudaError_t lmk_round(int64_t n, const int64_t* rp, const int32_t* col, int stride, uint64_t full, int slot0,
                             uint8_t* ld, uint64_t* visited, uint64_t* fa, uint64_t* fb, int* changed, cudaStream_t st,
                             int64_t* nl) {
    cudaError_t e = cudaSuccess;
    const unsigned blocks = (unsigned)((n * kLmkGroup + kLmkThreads - 1) / kLmkThreads);
    for (int level = 1; level <= kLmkMaxDist;) {
        if ((e = cudaMemsetAsync(changed, 0, sizeof(int), st)) != cudaSuccess) return e;
        // A level after the last one that reaches anything changes nothing,
        // so a few levels run between host checks.
        for (int t = 0; t < kLmkLevelsPerCheck && level <= kLmkMaxDist; ++t, ++level) {
            k_lmk_level<<<blocks, kLmkThreads, 0, st>>>(n, stride, level, full, slot0, rp, col, fa, fb, visited, ld,
                                                        changed);
            std::swap(fa, fb);
            ++*nl;
        }
        int h = 0;
        if ((e = cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (!h) break;
    }
    return cudaGetLastError();
}

int landmark_bfs(int64_t n, const int64_t* rp, const int32_t* col, const int32_t* comp_base, int k, int stride,
                 uint8_t* ld, int32_t* ids, cudaStream_t st, int64_t* launches) {
    if (k < 1 || k > kLmkMax || (comp_base && k > 64) || stride % 16 || stride < 2 * k) return PSPC_E_INVAL;
    // slots 0..k1-1: the highest-ranked vertices; k1..k-1: spread landmarks,
    // only for one graph large enough to place them
    const int k1 = (comp_base || k <= kLmkShallow || n <= 4 * (int64_t)k) ? k : kLmkShallow;
    void* mem = nullptr;
    const size_t masks = (size_t)n * 8;
    cudaError_t e = dev_alloc(&mem, 3 * masks + (size_t)n * 4 + kLmkMax * 12 + 256, st);
    if (e != cudaSuccess) return cuda_status(e);
    uint64_t* visited = (uint64_t*)mem;
    uint64_t* fa = visited + n;
    uint64_t* fb = fa + n;
    unsigned long long* keys = (unsigned long long*)(fb + n);
    int32_t* d_ids = (int32_t*)(keys + kLmkMax);
    uint32_t* cur = (uint32_t*)(d_ids + kLmkMax);
    int* changed = (int*)(cur + n);
    int32_t h_ids[kLmkMax];
    for (int j = 0; j < kLmkMax; ++j) h_ids[j] = j < k1 && j < n ? j : -1;
    int64_t nl = 1;
    const unsigned vb = (unsigned)((n + kLmkThreads - 1) / kLmkThreads);
    // first search batch: the first (up to 64) highest-ranked vertices of every graph
    const int r1 = k1 < 64 ? k1 : 64;
    k_lmk_init<<<vb, kLmkThreads, 0, st>>>(n, r1, stride, comp_base, visited, fa, ld);
    e = cudaMemcpyAsync(d_ids, h_ids, sizeof(h_ids), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = lmk_round(n, rp, col, stride, r1 == 64 ? ~0ull : ((1ull << r1) - 1), 0, ld, visited, fa, fb, changed, st,
                      &nl);
    // Spread landmarks, from the first round's distances (k1 <= 64). The
    // filter tests them from level kLmkDeepLevel on; when every distance
    // from the first landmarks is at most D with 2D < kLmkDeepLevel, labels
    // between vertices they reach stop short of that level, and the spread
    // ones are left out (slots k1..k-1 stay empty).
    int kk = k;
    if (e == cudaSuccess && k1 < k) {
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned ab = (unsigned)std::min<int64_t>(vb, std::max(sms, 1) * 4);
        if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0, kLmkMax * 8, st);
        unsigned dmax = 0;
        if (e == cudaSuccess) e = cudaMemsetAsync(changed, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) {
            k_lmk_score<<<vb, kLmkThreads, 0, st>>>(n, stride, k1, ld, cur, (unsigned*)changed);
            nl += 1;
            e = cudaMemcpyAsync(&dmax, changed, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && 2 * dmax < (unsigned)kLmkDeepLevel) kk = k1;
        }
        if (e == cudaSuccess && kk > k1) {
            for (int j = k1; j < k; ++j) {
                k_lmk_argmax<<<ab, kLmkThreads, 0, st>>>(n, cur, keys + j);
                k_lmk_take<<<vb, kLmkThreads, 0, st>>>(n, stride, k1, ld, cur, keys + j, d_ids, j);
                nl += 2;
            }
            e = cudaGetLastError();
        }
    }
    // later search batches: slots r1.. in groups of 64, from their vertices in d_ids
    for (int s0 = r1; e == cudaSuccess && s0 < kk; s0 += 64) {
        const int cnt = kk - s0 < 64 ? kk - s0 : 64;
        e = cudaMemsetAsync(visited, 0, 2 * masks, st);
        if (e == cudaSuccess) {
            k_lmk_seed<<<1, 64, 0, st>>>(n, s0, cnt, stride, d_ids, visited, fa, ld);
            nl += 1;
            e = lmk_round(n, rp, col, stride, cnt == 64 ? ~0ull : ((1ull << cnt) - 1), s0, ld, visited, fa, fb,
                          changed, st, &nl);
        }
    }
    if (e == cudaSuccess && ids) {
        e = cudaMemcpyAsync(h_ids, d_ids, sizeof(h_ids), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess)
            for (int j = 0; j < kLmkMax; ++j) ids[j] = j < kk ? h_ids[j] : -1;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    const int rc = e == cudaSuccess ? PSPC_OK : cuda_status(e);
    dev_free(mem, st);
    if (launches) *launches += nl;
    return rc;
}

}  // namespace pspc
