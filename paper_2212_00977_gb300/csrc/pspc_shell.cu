// Reduction by 1-shell (Section "Index Size Reduction", Reduction by
// 1-Shell). Repeatedly removing vertices of degree 1 strips the trees that
// hang off the rest of the graph. The index is built on what remains (the
// core), and a removed vertex is answered through the core vertex its tree
// hangs from (its root) and its distance to it. A tree meets the rest of
// the graph in its root only, so no shortest path between two core
// vertices enters a tree, and a shortest path from a tree vertex leaves its
// tree through the root. Peeling removes degree-1 vertices only; a vertex
// left with no neighbour (an isolated vertex, the last vertex of a tree
// component) stays in the core, so every tree has a core root.
//
// Queries (s, t), d_s = depth of s, r_s = root of s:
//   same root: the path inside the tree, count 1, length d_s + d_t - 2 d_a
//              with a the lowest common ancestor (walked up the parents);
//   otherwise: (sd(r_s, r_t) + d_s + d_t, SPC(r_s, r_t)) from the core index.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pspc_internal.cuh"
#include "pspc_shell.cuh"

namespace pspc {

constexpr int kShellThreads = 256;

static unsigned blocks_for(int64_t n) { return (unsigned)((n + kShellThreads - 1) / kShellThreads); }

__global__ void k_peel_init(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ deg,
                            uint8_t* __restrict__ alive, int32_t* __restrict__ parent) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    deg[v] = (int32_t)(rp[v + 1] - rp[v]);
    alive[v] = 1;
    parent[v] = -1;
}

// Marks the degree-1 vertices to remove this round and their parents (the
// one neighbour left). Of two adjacent degree-1 vertices (a component that
// is down to one edge) only the smaller id goes; the other stays, isolated.
__global__ void k_peel_mark(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ deg, const uint8_t* __restrict__ alive,
                            uint8_t* __restrict__ mark, int32_t* __restrict__ parent) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || !alive[v] || deg[v] != 1) return;
    int32_t p = -1;
    for (int64_t a = rp[v]; a < rp[v + 1]; ++a)
        if (alive[col[a]]) {
            p = col[a];
            break;
        }
    if (p < 0 || (deg[p] == 1 && p < v)) return;
    mark[v] = 1;
    parent[v] = p;
}

__global__ void k_peel_apply(int64_t n, uint8_t* __restrict__ mark, uint8_t* __restrict__ alive,
                             int32_t* __restrict__ deg, const int32_t* __restrict__ parent,
                             unsigned long long* __restrict__ removed) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || !mark[v]) return;
    mark[v] = 0;
    alive[v] = 0;
    atomicSub(&deg[parent[v]], 1);
    atomicAdd(removed, 1ull);
}

// Root and depth by pointer jumping: anc = next vertex up (itself in the
// core), dd = edges to it; each pass doubles the jump.
__global__ void k_shell_jump_init(int64_t n, const uint8_t* __restrict__ alive, const int32_t* __restrict__ parent,
                                  int32_t* __restrict__ anc, int32_t* __restrict__ dd) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    anc[v] = alive[v] ? (int32_t)v : parent[v];
    dd[v] = alive[v] ? 0 : 1;
}

__global__ void k_shell_jump(int64_t n, const int32_t* __restrict__ anc, const int32_t* __restrict__ dd,
                             int32_t* __restrict__ anc2, int32_t* __restrict__ dd2, int* __restrict__ moved) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t a = anc[v];
    const int32_t aa = anc[a];
    anc2[v] = aa;
    dd2[v] = dd[v] + dd[a];
    if (aa != a) *moved = 1;
}

__global__ void k_core_flags(int64_t n, const uint8_t* __restrict__ alive, int64_t* __restrict__ flag) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    flag[v] = alive[v];
}

// core_id from the scanned flags; degree of each core vertex in the core.
__global__ void k_core_rows(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const uint8_t* __restrict__ alive, const int64_t* __restrict__ scan,
                            int32_t* __restrict__ core_id, int64_t* __restrict__ cdeg) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (!alive[v]) {
        core_id[v] = -1;
        return;
    }
    core_id[v] = (int32_t)scan[v];
    int64_t c = 0;
    for (int64_t a = rp[v]; a < rp[v + 1]; ++a) c += alive[col[a]];
    cdeg[scan[v]] = c;
}

// Rows of the core in core ids; core ids keep the order of caller ids, so
// the rows stay ascending.
__global__ void k_core_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ core_id, const int64_t* __restrict__ crp,
                            int32_t* __restrict__ ccol) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || core_id[v] < 0) return;
    int64_t o = crp[core_id[v]];
    for (int64_t a = rp[v]; a < rp[v + 1]; ++a) {
        const int32_t c = core_id[col[a]];
        if (c >= 0) ccol[o++] = c;
    }
}

// The core keeps G's order: flag[r] = 1 when the vertex of rank r is in the
// core; after a scan, its position among core vertices is its core rank.
__global__ void k_rank_flags(int64_t n, const int32_t* __restrict__ rank, const uint8_t* __restrict__ alive,
                             int64_t* __restrict__ flag) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    flag[rank[v]] = alive[v];
}

__global__ void k_core_rank(int64_t n, const int32_t* __restrict__ rank, const int32_t* __restrict__ core_id,
                            const int64_t* __restrict__ scan, int32_t* __restrict__ crank) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || core_id[v] < 0) return;
    crank[core_id[v]] = (int32_t)scan[rank[v]];
}

int shell_reduce(int64_t n, const int64_t* rp, const int32_t* col, const int32_t* rank, ShellParts& P,
                 cudaStream_t st, int64_t* launches) {
    uint8_t* alive = nullptr;
    uint8_t* mark = nullptr;
    int32_t* deg = nullptr;
    int32_t *anc2 = nullptr, *dd2 = nullptr;
    int64_t* flag = nullptr;
    unsigned long long* cnt = nullptr;
    int* moved = nullptr;
    int rc = PSPC_OK;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = dev_alloc(p, bytes, st);
    };
    alloc((void**)&alive, n);
    alloc((void**)&mark, n);
    alloc((void**)&deg, n * 4);
    alloc((void**)&anc2, n * 4);
    alloc((void**)&dd2, n * 4);
    alloc((void**)&flag, (n + 1) * 8);
    alloc((void**)&cnt, 8);
    alloc((void**)&moved, 4);
    alloc((void**)&P.parent, n * 4);
    alloc((void**)&P.root, n * 4);
    alloc((void**)&P.depth, n * 4);
    alloc((void**)&P.core_id, n * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(mark, 0, n, st);
    int64_t nl = 0;
    if (e == cudaSuccess) {
        k_peel_init<<<blocks_for(n), kShellThreads, 0, st>>>(n, rp, deg, alive, P.parent);
        ++nl;
    }
    // peel rounds until none is removed
    P.removed = 0;
    for (int round = 0; e == cudaSuccess; ++round) {
        unsigned long long h = 0;
        e = cudaMemsetAsync(cnt, 0, 8, st);
        if (e != cudaSuccess) break;
        k_peel_mark<<<blocks_for(n), kShellThreads, 0, st>>>(n, rp, col, deg, alive, mark, P.parent);
        k_peel_apply<<<blocks_for(n), kShellThreads, 0, st>>>(n, mark, alive, deg, P.parent, cnt);
        nl += 2;
        if ((e = cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        if (!h) break;
        P.removed += (int64_t)h;
    }
    // roots and depths
    if (e == cudaSuccess) {
        k_shell_jump_init<<<blocks_for(n), kShellThreads, 0, st>>>(n, alive, P.parent, P.root, P.depth);
        ++nl;
        int32_t *a = P.root, *d = P.depth, *a2 = anc2, *d2 = dd2;
        for (;;) {
            int h = 0;
            if ((e = cudaMemsetAsync(moved, 0, 4, st)) != cudaSuccess) break;
            k_shell_jump<<<blocks_for(n), kShellThreads, 0, st>>>(n, a, d, a2, d2, moved);
            ++nl;
            std::swap(a, a2);
            std::swap(d, d2);
            if ((e = cudaMemcpyAsync(&h, moved, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
            if (!h) break;
        }
        if (e == cudaSuccess && a != P.root) {
            e = cudaMemcpyAsync(P.root, a, n * 4, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(P.depth, d, n * 4, cudaMemcpyDeviceToDevice, st);
        }
    }
    // core ids, rows and order
    if (e == cudaSuccess) {
        k_core_flags<<<blocks_for(n), kShellThreads, 0, st>>>(n, alive, flag);
        ++nl;
        rc = exclusive_scan_i64(flag, n, st, &nl);
    }
    if (e == cudaSuccess && rc == PSPC_OK) e = cudaMemcpyAsync(&P.n_core, flag + n, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rc == PSPC_OK) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && rc == PSPC_OK) {
        alloc((void**)&P.rp, (P.n_core + 1) * 8);
        if (e == cudaSuccess) {
            k_core_rows<<<blocks_for(n), kShellThreads, 0, st>>>(n, rp, col, alive, flag, P.core_id, P.rp);
            ++nl;
            rc = exclusive_scan_i64(P.rp, P.n_core, st, &nl);
        }
    }
    if (e == cudaSuccess && rc == PSPC_OK) e = cudaMemcpyAsync(&P.arcs, P.rp + P.n_core, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rc == PSPC_OK) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && rc == PSPC_OK) {
        alloc((void**)&P.col, (P.arcs > 0 ? P.arcs : 1) * 4);
        alloc((void**)&P.rank, P.n_core * 4);
        if (e == cudaSuccess) {
            k_core_fill<<<blocks_for(n), kShellThreads, 0, st>>>(n, rp, col, P.core_id, P.rp, P.col);
            k_rank_flags<<<blocks_for(n), kShellThreads, 0, st>>>(n, rank, alive, flag);
            nl += 2;
            rc = exclusive_scan_i64(flag, n, st, &nl);
        }
        if (e == cudaSuccess && rc == PSPC_OK) {
            k_core_rank<<<blocks_for(n), kShellThreads, 0, st>>>(n, rank, P.core_id, flag, P.rank);
            ++nl;
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_status(e);
    dev_free(alive, st);
    dev_free(mark, st);
    dev_free(deg, st);
    dev_free(anc2, st);
    dev_free(dd2, st);
    dev_free(flag, st);
    dev_free(cnt, st);
    dev_free(moved, st);
    if (launches) *launches += nl;
    return rc;
}

void shell_free(ShellParts& P, cudaStream_t st) {
    dev_free(P.rp, st);
    dev_free(P.col, st);
    dev_free(P.rank, st);
    P.rp = nullptr;
    P.col = nullptr;
    P.rank = nullptr;
}

// ---------------------------------------------------------------------------
// Queries on a reduced index.

// Per pair: answers s = t and same-root pairs (the tree path, count 1) at
// once and marks them (extra = -1); the others get the pair of their roots
// in core ids and extra = d_s + d_t.
__global__ void k_shell_pairs(const int32_t* __restrict__ pairs, int64_t q, int64_t n,
                              const int32_t* __restrict__ root, const int32_t* __restrict__ depth,
                              const int32_t* __restrict__ parent, const int32_t* __restrict__ core_id,
                              int32_t* __restrict__ cpairs, int32_t* __restrict__ extra, uint16_t* __restrict__ dist,
                              uint64_t* __restrict__ cnt, uint8_t* __restrict__ ovf, int* __restrict__ err) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= q) return;
    int32_t s = pairs[2 * p], t = pairs[2 * p + 1];
    cpairs[2 * p] = 0;
    cpairs[2 * p + 1] = 0;
    extra[p] = -1;
    if (s < 0 || s >= n || t < 0 || t >= n) {
        atomicOr(err, 1);
        dist[p] = PSPC_UNREACHED;
        cnt[p] = 0;
        if (ovf) ovf[p] = 0;
        return;
    }
    const int32_t rs = root[s], rt = root[t];
    if (rs != rt) {
        cpairs[2 * p] = core_id[rs];
        cpairs[2 * p + 1] = core_id[rt];
        extra[p] = depth[s] + depth[t];
        return;
    }
    // the tree path: walk the deeper end up to the other's depth, then both
    int32_t ds = depth[s], dt = depth[t];
    const int32_t total = ds + dt;
    while (ds > dt) {
        s = parent[s];
        --ds;
    }
    while (dt > ds) {
        t = parent[t];
        --dt;
    }
    while (s != t) {
        s = parent[s];
        t = parent[t];
        --ds;
    }
    const int32_t d = total - 2 * ds;
    if (d > kMaxDist) atomicOr(err, 2);
    dist[p] = (uint16_t)(d > kMaxDist ? kMaxDist : d);
    cnt[p] = 1;
    if (ovf) ovf[p] = 0;
}

__global__ void k_shell_combine(int64_t q, const int32_t* __restrict__ extra, const uint16_t* __restrict__ cd,
                                const uint64_t* __restrict__ cc, const uint8_t* __restrict__ co,
                                uint16_t* __restrict__ dist, uint64_t* __restrict__ cnt, uint8_t* __restrict__ ovf,
                                int* __restrict__ err) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= q || extra[p] < 0) return;
    if (cd[p] == PSPC_UNREACHED) {
        dist[p] = PSPC_UNREACHED;
        cnt[p] = 0;
        if (ovf) ovf[p] = 0;
        return;
    }
    const int32_t d = (int32_t)cd[p] + extra[p];
    if (d > kMaxDist) atomicOr(err, 2);
    dist[p] = (uint16_t)(d > kMaxDist ? kMaxDist : d);
    cnt[p] = cc[p];
    if (ovf) ovf[p] = co[p];
}

cudaError_t launch_shell_pairs(const Index& ix, const int32_t* pairs, int64_t q, int32_t* cpairs, int32_t* extra,
                               uint16_t* dist, uint64_t* cnt, uint8_t* ovf, int* err, cudaStream_t st) {
    k_shell_pairs<<<blocks_for(q), kShellThreads, 0, st>>>(pairs, q, ix.n, ix.sh_root, ix.sh_depth, ix.sh_parent,
                                                           ix.sh_core, cpairs, extra, dist, cnt, ovf, err);
    return cudaGetLastError();
}

cudaError_t launch_shell_combine(int64_t q, const int32_t* extra, const uint16_t* cd, const uint64_t* cc,
                                 const uint8_t* co, uint16_t* dist, uint64_t* cnt, uint8_t* ovf, int* err,
                                 cudaStream_t st) {
    k_shell_combine<<<blocks_for(q), kShellThreads, 0, st>>>(q, extra, cd, cc, co, dist, cnt, ovf, err);
    return cudaGetLastError();
}

}  // namespace pspc
