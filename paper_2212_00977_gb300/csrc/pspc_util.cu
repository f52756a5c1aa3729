// Host utilities of the SPC hub-label library: pointer classification,
// status mapping, a device exclusive scan, and the small ABI entry points
// (pspc_stats, pspc_level_stats, pspc_export, pspc_free, pspc_strerror).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "pspc_internal.cuh"

namespace pspc {

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64];
static bool g_pool_ok[64];

// Allocation-failure injection (pspc_inject_alloc_failure): the number of
// library device allocations still allowed to succeed, or -1 (no limit).
static std::atomic<int64_t> g_alloc_budget{-1};
static std::atomic<int> g_alloc_error{(int)cudaErrorMemoryAllocation};  // what an injected failure returns

static bool alloc_allowed() {
    int64_t b = g_alloc_budget.load(std::memory_order_relaxed);
    while (b >= 0) {
        if (b == 0) return false;
        if (g_alloc_budget.compare_exchange_weak(b, b - 1, std::memory_order_relaxed)) return true;
    }
    return true;
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st) {
    if (!alloc_allowed()) {
        *p = nullptr;
        return (cudaError_t)g_alloc_error.load(std::memory_order_relaxed);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool_ok[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&g_pools[dev], &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
            g_pool_ok[dev] = true;
        }
    }
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 1, g_pools[dev], st);
}

void dev_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PSPC_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return PSPC_E_NOMEM;
    }
    return PSPC_E_CUDA;
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 (tile per block, recursive over tile sums).

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int64_t* a, int64_t n, int64_t* tile_sums) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? a[base + i] : 0;
        s += v[i];
    }
    int64_t incl = warp_incl_scan(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
        t = warp_incl_scan(t);
        if (lane < kScanThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t run = incl - s + (warp ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) a[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == kScanThreads - 1 && tile_sums) tile_sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int64_t* a, int64_t n, const int64_t* tile_offs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += tile_offs[i / kScanTile];
}

int64_t scan_scratch_entries(int64_t n) {
    int64_t total = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        total += n;
    }
    return total;
}

static int scan_rec(int64_t* a, int64_t n, cudaStream_t st, int64_t* launches, int64_t* scratch) {
    if (n <= 0) return PSPC_OK;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_tiles<<<1, kScanThreads, 0, st>>>(a, n, nullptr);
        if (launches) *launches += 1;
        return cuda_status(cudaGetLastError());
    }
    int64_t* sums = scratch;
    if (!sums) PSPC_TRY_CUDA(dev_alloc((void**)&sums, (size_t)tiles * sizeof(int64_t), st));
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(a, n, sums);
    int rc = cuda_status(cudaGetLastError());
    if (rc == PSPC_OK) rc = scan_rec(sums, tiles, st, launches, scratch ? scratch + tiles : nullptr);
    if (rc == PSPC_OK) {
        k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, sums);
        rc = cuda_status(cudaGetLastError());
    }
    if (launches) *launches += 2;
    if (!scratch) dev_free(sums, st);
    return rc;
}

int exclusive_scan_i64(int64_t* a, int64_t n, cudaStream_t st, int64_t* launches, int64_t* scratch) {
    PSPC_TRY_CUDA(cudaMemsetAsync(a + n, 0, sizeof(int64_t), st));
    return scan_rec(a, n + 1, st, launches, scratch);
}

}  // namespace pspc

using namespace pspc;

extern "C" int pspc_inject_alloc_failure(int64_t after, int32_t status) {
    if (status != PSPC_E_NOMEM && status != PSPC_E_CUDA) return PSPC_E_INVAL;
    g_alloc_error.store(status == PSPC_E_NOMEM ? (int)cudaErrorMemoryAllocation : (int)cudaErrorInvalidValue,
                        std::memory_order_relaxed);
    g_alloc_budget.store(after < 0 ? -1 : after, std::memory_order_relaxed);
    return PSPC_OK;
}

extern "C" const char* pspc_strerror(int code) {
    switch (code) {
        case PSPC_OK: return "ok";
        case PSPC_E_INVAL: return "invalid argument (graph, rank, pair or option)";
        case PSPC_E_NOMEM: return "out of memory";
        case PSPC_E_CUDA: return "CUDA error";
        case PSPC_E_DIST: return "distance limit exceeded";
        default: return "unknown status";
    }
}

extern "C" void pspc_free(pspc_index* h) {
    if (!h) return;
    Index& ix = h->ix;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix.device);
    // The index is only freed once no work on it is pending (every call
    // that uses it returns after its stream has drained).
    dev_free(ix.rank, 0);
    dev_free(ix.order, 0);
    dev_free(ix.off, 0);
    dev_free(ix.hub, 0);
    dev_free(ix.dist, 0);
    dev_free(ix.cnt, 0);
    dev_free(ix.lmk, 0);
    dev_free(ix.sh_core, 0);
    dev_free(ix.sh_root, 0);
    dev_free(ix.sh_depth, 0);
    dev_free(ix.sh_parent, 0);
    cudaStreamSynchronize(0);
    if (ix.core) pspc_free(ix.core);
    cudaSetDevice(prev);
    delete h;
}

extern "C" int pspc_stats(const pspc_index* h, pspc_stats_t* s) {
    if (!h || !s) return PSPC_E_INVAL;
    const Index& ix = h->ix;
    memset(s, 0, sizeof(*s));
    s->n = ix.n;
    s->arcs = ix.arcs;
    s->entries = ix.entries;
    s->levels = ix.levels;
    s->device = ix.device;
    s->index_bytes = (ix.n * 2 + (ix.n + 1) * 2) * 4 + ix.entries * (4 + 2 + 8);
    s->overflow_entries = ix.overflow_entries;
    s->kernel_launches = ix.launches;
    s->query_kernel_launches = ix.query_launches;
    s->graphs = ix.graphs;
    s->build_ms = ix.build_ms;
    s->landmarks = ix.lmk ? ix.lmk_k : 0;
    s->landmark_ms = ix.lmk_ms;
    if (ix.core) {  // labels, landmarks and their sizes are the core's
        pspc_stats_t c;
        pspc_stats(ix.core, &c);
        s->index_bytes = c.index_bytes + ix.n * 16;
        s->landmarks = c.landmarks;
        s->query_kernel_launches += c.query_kernel_launches;
        s->shell_vertices = ix.shell_vertices;
    }
    return PSPC_OK;
}

extern "C" int pspc_landmarks(const pspc_index* h, int32_t* k, uint16_t* dist, int32_t* vertex) {
    if (!h || !k || h->ix.core || (vertex && h->ix.graphs != 1)) return PSPC_E_INVAL;
    const Index& ix = h->ix;
    *k = ix.lmk ? ix.lmk_k : 0;
    if ((!dist && !vertex) || !ix.lmk) return PSPC_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix.device);
    const size_t S = (size_t)ix.lmk_stride, K = (size_t)ix.lmk_k;
    std::vector<uint8_t> rows;
    std::vector<int32_t> rank;
    int rc = PSPC_OK;
    try {
        rows.resize((size_t)ix.n * S);
        rank.resize((size_t)ix.n);
    } catch (...) {
        rc = PSPC_E_NOMEM;
    }
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaMemcpy(rows.data(), ix.lmk, rows.size(), cudaMemcpyDeviceToHost);
    if (!rc && e == cudaSuccess) e = cudaMemcpy(rank.data(), ix.rank, (size_t)ix.n * 4, cudaMemcpyDeviceToHost);
    if (!rc && e != cudaSuccess) rc = cuda_status(e);
    if (!rc && dist)
        for (int64_t v = 0; v < ix.n; ++v) memcpy(dist + (size_t)v * K, rows.data() + (size_t)rank[v] * S, 2 * K);
    if (!rc && vertex) {
        for (size_t j = 0; j < K; ++j) vertex[j] = -1;
        for (int64_t v = 0; v < ix.n; ++v)  // caller id of each landmark's rank
            for (size_t j = 0; j < K; ++j)
                if (ix.lmk_ids[j] == rank[v]) vertex[j] = (int32_t)v;
    }
    cudaSetDevice(prev);
    return rc;
}

extern "C" int pspc_level_stats(const pspc_index* h, pspc_level_stat_t* out, int32_t cap,
                                int32_t* levels) {
    if (!h || cap < 0 || (cap > 0 && !out)) return PSPC_E_INVAL;
    const Index& ix = h->ix;
    const int32_t L = (int32_t)ix.lstats.size();
    if (levels) *levels = L;
    for (int32_t i = 0; i < std::min(cap, L); ++i) out[i] = ix.lstats[i];
    return PSPC_OK;
}

extern "C" int pspc_export(const pspc_index* h, int64_t* off, int32_t* hub, uint16_t* dist,
                           uint64_t* cnt, uint8_t* ovf) {
    if (!h || h->ix.core || !off || (h->ix.entries > 0 && (!hub || !dist || !cnt || !ovf))) return PSPC_E_INVAL;
    const Index& ix = h->ix;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix.device);
    const int64_t n = ix.n, E = ix.entries;
    std::vector<int64_t> roff(n + 1);
    std::vector<int32_t> rank(n), order(n), rhub(E);
    std::vector<uint16_t> rdist(E);
    std::vector<uint64_t> rcnt(E);
    int rc = PSPC_OK;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(roff.data(), ix.off, (n + 1) * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(rank.data(), ix.rank, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(order.data(), ix.order, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && E) e = cudaMemcpy(rhub.data(), ix.hub, E * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && E) e = cudaMemcpy(rdist.data(), ix.dist, E * 2, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && E) e = cudaMemcpy(rcnt.data(), ix.cnt, E * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_status(e);
    if (rc == PSPC_OK) {
        int64_t p = 0;
        for (int64_t v = 0; v < n; ++v) {
            off[v] = p;
            const int32_t r = rank[v];
            for (int64_t i = roff[r]; i < roff[r + 1]; ++i, ++p) {
                hub[p] = order[rhub[i]];
                dist[p] = (uint16_t)(rdist[i] & 0x7FFF);
                ovf[p] = (uint8_t)(rdist[i] >> 15);
                cnt[p] = rcnt[i];
            }
        }
        off[n] = p;
    }
    cudaSetDevice(prev);
    return rc;
}

// ---------------------------------------------------------------------------
// Partial extraction on the device: one hub's column, or selected labels.

namespace pspc {

// Thread per (rank-space) vertex: binary search of the hub in its sorted label.
__global__ void k_hub_column(int64_t n, int32_t rw, const int32_t* __restrict__ order, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ hub, const uint16_t* __restrict__ dist,
                             const uint64_t* __restrict__ cnt, uint16_t* out_dist, uint64_t* out_cnt,
                             uint8_t* out_ovf) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t lo = off[r], hi = off[r + 1];
    const int64_t e = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (hub[mid] < rw) lo = mid + 1; else hi = mid;
    }
    const int32_t v = order[r];
    if (lo < e && hub[lo] == rw) {
        out_dist[v] = (uint16_t)(dist[lo] & 0x7FFF);
        out_cnt[v] = cnt[lo];
        out_ovf[v] = (uint8_t)(dist[lo] >> 15);
    } else {
        out_dist[v] = PSPC_UNREACHED;
        out_cnt[v] = 0;
        out_ovf[v] = 0;
    }
}

__global__ void k_vert_sizes(int64_t k, const int32_t* __restrict__ verts, int64_t n, const int32_t* __restrict__ rank,
                             const int64_t* __restrict__ off, int64_t* __restrict__ sizes, int* err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const int32_t v = verts[i];
    if (v < 0 || v >= n) {
        atomicOr(err, 1);
        sizes[i] = 0;
        return;
    }
    const int32_t r = rank[v];
    sizes[i] = off[r + 1] - off[r];
}

// Warp per selected vertex: its label with hubs as caller ids.
__global__ void k_vert_gather(int64_t k, const int32_t* __restrict__ verts, int64_t n, const int32_t* __restrict__ rank,
                              const int32_t* __restrict__ order, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ hub, const uint16_t* __restrict__ dist,
                              const uint64_t* __restrict__ cnt, const int64_t* __restrict__ pos, int32_t* o_hub,
                              uint16_t* o_dist, uint64_t* o_cnt, uint8_t* o_ovf) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= k) return;
    const int32_t v = verts[i];
    if (v < 0 || v >= n) return;
    const int32_t r = rank[v];
    const int64_t a0 = off[r], len = off[r + 1] - a0, p0 = pos[i];
    for (int64_t j = lane; j < len; j += 32) {
        o_hub[p0 + j] = order[hub[a0 + j]];
        o_dist[p0 + j] = (uint16_t)(dist[a0 + j] & 0x7FFF);
        o_ovf[p0 + j] = (uint8_t)(dist[a0 + j] >> 15);
        o_cnt[p0 + j] = cnt[a0 + j];
    }
}

}  // namespace pspc

extern "C" int pspc_hub_column(const pspc_index* h, int32_t w, uint16_t* dist, uint64_t* cnt, uint8_t* ovf) {
    if (!h || h->ix.core || !dist || !cnt || !ovf) return PSPC_E_INVAL;
    const Index& ix = h->ix;
    if (w < 0 || w >= ix.n) return PSPC_E_INVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix.device);
    const cudaStream_t st = 0;
    int32_t rw = 0;
    uint16_t* d_dist = nullptr;
    uint64_t* d_cnt = nullptr;
    uint8_t* d_ovf = nullptr;
    cudaError_t e = cudaMemcpy(&rw, ix.rank + w, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = dev_alloc((void**)&d_dist, ix.n * 2, st);
    if (e == cudaSuccess) e = dev_alloc((void**)&d_cnt, ix.n * 8, st);
    if (e == cudaSuccess) e = dev_alloc((void**)&d_ovf, ix.n, st);
    if (e == cudaSuccess) {
        k_hub_column<<<(unsigned)((ix.n + 255) / 256), 256, 0, st>>>(ix.n, rw, ix.order, ix.off, ix.hub, ix.dist,
                                                                      ix.cnt, d_dist, d_cnt, d_ovf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(dist, d_dist, ix.n * 2, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, d_cnt, ix.n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ovf, d_ovf, ix.n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(d_dist, st);
    dev_free(d_cnt, st);
    dev_free(d_ovf, st);
    cudaStreamSynchronize(st);
    cudaSetDevice(prev);
    return cuda_status(e);
}

extern "C" int pspc_export_vertices(const pspc_index* h, const int32_t* verts, int64_t k, int64_t* off, int32_t* hub,
                                    uint16_t* dist, uint64_t* cnt, uint8_t* ovf) {
    if (!h || h->ix.core || k < 0 || (k > 0 && !verts) || !off) return PSPC_E_INVAL;
    const Index& ix = h->ix;
    if (k == 0) {
        off[0] = 0;
        return PSPC_OK;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ix.device);
    const cudaStream_t st = 0;
    int32_t* d_verts = nullptr;
    int64_t* d_pos = nullptr;
    int* d_err = nullptr;
    int32_t* d_hub = nullptr;
    uint16_t* d_dist = nullptr;
    uint64_t* d_cnt = nullptr;
    uint8_t* d_ovf = nullptr;
    int herr = 0;
    int rc = PSPC_OK;
    cudaError_t e = dev_alloc((void**)&d_verts, k * 4, st);
    if (e == cudaSuccess) e = dev_alloc((void**)&d_pos, (k + 1) * 8, st);
    if (e == cudaSuccess) e = dev_alloc((void**)&d_err, 4, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_verts, verts, k * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, 4, st);
    if (e == cudaSuccess) {
        k_vert_sizes<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(k, d_verts, ix.n, ix.rank, ix.off, d_pos, d_err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) rc = exclusive_scan_i64(d_pos, k, st);
    if (e == cudaSuccess && rc == PSPC_OK) e = cudaMemcpyAsync(off, d_pos, (k + 1) * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rc == PSPC_OK) e = cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && rc == PSPC_OK && herr) rc = PSPC_E_INVAL;
    // hub == NULL: only the offsets (label sizes) were asked for
    if (e == cudaSuccess && rc == PSPC_OK && hub) {
        if (!dist || !cnt || !ovf) {
            rc = PSPC_E_INVAL;
        } else {
            const int64_t E = off[k];
            e = dev_alloc((void**)&d_hub, E * 4, st);
            if (e == cudaSuccess) e = dev_alloc((void**)&d_dist, E * 2, st);
            if (e == cudaSuccess) e = dev_alloc((void**)&d_cnt, E * 8, st);
            if (e == cudaSuccess) e = dev_alloc((void**)&d_ovf, E, st);
            if (e == cudaSuccess) {
                k_vert_gather<<<(unsigned)((k * 32 + 255) / 256), 256, 0, st>>>(
                    k, d_verts, ix.n, ix.rank, ix.order, ix.off, ix.hub, ix.dist, ix.cnt, d_pos, d_hub, d_dist, d_cnt,
                    d_ovf);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess && E) e = cudaMemcpyAsync(hub, d_hub, E * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && E) e = cudaMemcpyAsync(dist, d_dist, E * 2, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && E) e = cudaMemcpyAsync(cnt, d_cnt, E * 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && E) e = cudaMemcpyAsync(ovf, d_ovf, E, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    dev_free(d_verts, st);
    dev_free(d_pos, st);
    dev_free(d_err, st);
    dev_free(d_hub, st);
    dev_free(d_dist, st);
    dev_free(d_cnt, st);
    dev_free(d_ovf, st);
    cudaStreamSynchronize(st);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_status(e);
    return rc;
}
