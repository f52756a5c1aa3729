// Landmark labelling for the landmark filter of pruning rule 2 (Section
// "Landmark-Based Filtering"). The landmarks of a graph are its k
// highest-ranked vertices; under a degree order these are the vertices whose
// degree reaches the k-th largest degree, the paper's degree threshold. The
// filter needs sd(v, l) for every vertex v and landmark l: all k
// breadth-first searches run together, one BFS level per launch. Every
// vertex keeps a 64-bit mask of the landmarks that have reached it; at level
// t it takes the OR of its neighbours' frontier masks, and the bits new to it
// get distance t.
#include <cuda_runtime.h>
#include <stdint.h>

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

// One BFS level for all landmarks: kLmkGroup lanes per vertex OR the
// frontier masks of its neighbours.
__global__ void __launch_bounds__(kLmkThreads)
    k_lmk_level(int64_t n, int stride, int level, uint64_t full, const int64_t* __restrict__ rp,
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
        if ((fresh >> j) & 1ull) lmk_row(ld, v, stride)[j] = (uint16_t)level;
}

int landmark_bfs(int64_t n, const int64_t* rp, const int32_t* col, const int32_t* comp_base, int k, int stride,
                 uint8_t* ld, cudaStream_t st, int64_t* launches) {
    if (k < 1 || k > 64 || stride % 16 || stride < 2 * k) return PSPC_E_INVAL;
    void* mem = nullptr;
    const size_t masks = (size_t)n * 8;
    cudaError_t e = dev_alloc(&mem, 3 * masks + 256, st);
    if (e != cudaSuccess) return cuda_status(e);
    uint64_t* visited = (uint64_t*)mem;
    uint64_t* fa = visited + n;
    uint64_t* fb = fa + n;
    int* changed = (int*)(fb + n);
    const uint64_t full = k == 64 ? ~0ull : ((1ull << k) - 1);
    int rc = PSPC_OK;
    k_lmk_init<<<(unsigned)((n + kLmkThreads - 1) / kLmkThreads), kLmkThreads, 0, st>>>(n, k, stride, comp_base,
                                                                                         visited, fa, ld);
    int64_t nl = 1;
    const unsigned blocks = (unsigned)((n * kLmkGroup + kLmkThreads - 1) / kLmkThreads);
    for (int level = 1; level <= kLmkMaxDist && rc == PSPC_OK;) {
        if ((e = cudaMemsetAsync(changed, 0, sizeof(int), st)) != cudaSuccess) break;
        // A level after the last one that reaches anything changes nothing,
        // so a few levels run between host checks.
        for (int t = 0; t < kLmkLevelsPerCheck && level <= kLmkMaxDist; ++t, ++level) {
            k_lmk_level<<<blocks, kLmkThreads, 0, st>>>(n, stride, level, full, rp, col, fa, fb, visited, ld, changed);
            std::swap(fa, fb);
            ++nl;
        }
        int h = 0;
        if ((e = cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        if (!h) break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_status(e);
    dev_free(mem, st);
    if (launches) *launches += nl;
    return rc;
}

}  // namespace pspc
