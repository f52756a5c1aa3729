// Interface of the 1-shell reduction (pspc_shell.cu) for the build and query
// entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pspc_internal.cuh"

namespace pspc {

// Result of peeling G: per vertex (caller ids) its parent towards the core
// (-1 in the core), its root in the core and depth below it, its core id
// (-1 for a removed vertex); and the core graph in core ids (symmetric CSR,
// ascending rows) with G's order restricted to it. Device memory from the
// library pool; rp/col/rank are released by shell_free once the core index
// is built, the per-vertex arrays move to the index.
struct ShellParts {
    int32_t* parent = nullptr;
    int32_t* root = nullptr;
    int32_t* depth = nullptr;
    int32_t* core_id = nullptr;
    int64_t removed = 0;
    int64_t n_core = 0, arcs = 0;
    int64_t* rp = nullptr;
    int32_t* col = nullptr;
    int32_t* rank = nullptr;
};

int shell_reduce(int64_t n, const int64_t* rp, const int32_t* col, const int32_t* rank, ShellParts& P,
                 cudaStream_t st, int64_t* launches);
void shell_free(ShellParts& P, cudaStream_t st);

cudaError_t launch_shell_pairs(const Index& ix, const int32_t* pairs, int64_t q, int32_t* cpairs, int32_t* extra,
                               uint16_t* dist, uint64_t* cnt, uint8_t* ovf, int* err, cudaStream_t st);
cudaError_t launch_shell_combine(int64_t q, const int32_t* extra, const uint16_t* cd, const uint64_t* cc,
                                 const uint8_t* co, uint16_t* dist, uint64_t* cnt, uint8_t* ovf, int* err,
                                 cudaStream_t st);

}  // namespace pspc
