// Internal definitions shared by the CUDA translation units of the SPC
// hub-label library (index layout, level-segment encoding, small device
// helpers). Not part of the public ABI (include/pspc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pspc.h"

struct pspc_index;

namespace pspc {

// Vertex and hub ids are rank positions (0 = highest rank) inside the
// library; n < 2^24, so an id fits in 24 bits.
constexpr uint32_t kHubMask = 0x00FFFFFFu;
constexpr uint32_t kOvfBit = 0x80000000u;   // overflow flag carried with a hub word
constexpr uint32_t kMarkBit = 0x40000000u;  // survivor mark inside candidate tables
constexpr uint32_t kEmpty = 0xFFFFFFFFu;    // empty hash slot
constexpr int kLmkMax = 128;               // landmarks per graph at most (64 in a batch of graphs)
constexpr int64_t kMaxVertices = (1 << 24) - 1;
constexpr int kMaxDist = 32767;

// A level segment of one vertex: the entries of L_d(u) live at
// [start, start + len) of the label arena. start < 2^40, len < 2^24.
__host__ __device__ inline uint64_t seg_pack(uint64_t start, uint32_t len) {
    return (start << 24) | (uint64_t)len;
}
__host__ __device__ inline uint64_t seg_start(uint64_t s) { return s >> 24; }
__host__ __device__ inline uint32_t seg_len(uint64_t s) { return (uint32_t)(s & 0xFFFFFFu); }

__host__ __device__ inline uint32_t hash_hub(uint32_t h) { return h * 0x9E3779B1u; }

__host__ __device__ inline uint32_t pow2_ceil(uint64_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Finished index (all device memory, ids in rank space).
struct Index {
    int device = 0;
    int64_t n = 0, arcs = 0;
    int32_t* rank = nullptr;   // caller id -> rank id
    int32_t* order = nullptr;  // rank id -> caller id
    int64_t* off = nullptr;    // [n+1]
    int32_t* hub = nullptr;    // hub rank ids
    uint16_t* dist = nullptr;  // distance | overflow << 15
    uint64_t* cnt = nullptr;   // trough path count mod 2^64
    int64_t entries = 0;
    int64_t max_label = 0;     // entries of the largest label
    int32_t levels = 0;
    int64_t overflow_entries = 0;
    float build_ms = 0.f;
    int64_t launches = 0;
    int64_t query_launches = 0;  // kernels launched by pspc_query on this index
    int32_t query_group = 0;  // lanes per query pair; 0 = chosen from label sizes
    int32_t graphs = 1;       // graphs in the batch the index was built from
    uint8_t* lmk = nullptr;   // [n][lmk_stride] bytes: uint16 landmark distances (rank ids), or NULL
    int32_t lmk_k = 0;        // landmarks per graph
    int32_t lmk_stride = 0;   // bytes per row (2 * lmk_k rounded up to 16)
    int32_t lmk_ids[kLmkMax] = {};  // id (rank) of landmark j of a one-graph index, -1 for none
    float lmk_ms = 0.f;       // device time of the landmark BFS
    // 1-shell reduction: when `core` is set, the labels are those of the
    // 2-core, held by `core` (an index over core ids), and every vertex of G
    // (caller ids) has its core id (-1 if peeled), its root in the core, its
    // depth below the root and its parent towards it (-1 in the core).
    pspc_index* core = nullptr;
    int32_t* sh_core = nullptr;
    int32_t* sh_root = nullptr;
    int32_t* sh_depth = nullptr;
    int32_t* sh_parent = nullptr;
    int64_t shell_vertices = 0;
    std::vector<pspc_level_stat_t> lstats;
};

// Host-side helpers (pspc_util.cu).
bool is_device_ptr(const void* p);
int cuda_status(cudaError_t e);

// Device memory of the library comes from one stream-ordered pool per
// device, created on first use with an unbounded release threshold so that
// memory freed by one build or query is reused by the next without going
// back to the driver. dev_alloc / dev_free are stream-ordered.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);

// Exclusive prefix sum of int64 values in place: a[0..n) -> exclusive
// scan, a[n] = total (a must hold n+1 values). Device memory.
// *launches (if not NULL) is increased by the kernels launched. The tile
// partial sums go to `scratch` when it is given (device memory of at least
// scan_scratch_entries(n + 1) values), else to memory from the pool.
int exclusive_scan_i64(int64_t* a, int64_t n, cudaStream_t st, int64_t* launches = nullptr,
                       int64_t* scratch = nullptr);
// Partial-sum values the scan of m values needs (0 when one tile holds them).
int64_t scan_scratch_entries(int64_t m);

}  // namespace pspc

struct pspc_index {
    pspc::Index ix;
};

#define PSPC_TRY_CUDA(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return pspc::cuda_status(_e);  \
    } while (0)
