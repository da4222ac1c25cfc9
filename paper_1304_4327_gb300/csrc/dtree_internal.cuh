// dtree_internal.cuh -- types and helpers shared by the library's CUDA sources.
//
// Layout of a tree in HBM (all arrays device-resident, owned by the handle):
//   pts    n x DP float32, rows in tree order, dimensions d..DP-1 zero-padded
//          (DP = 4, 8, 16, 32 or 64: the smallest bucket >= d)
//   idx    n int32, tree position -> row of the build input
//   box    nodes x 2 x DP float32, tight bounding box (lo row then hi row)
//   lam    nodes float32, upper bound on lambda (max distance from the node's
//          centre -- the box centre in float32 -- to a descendant point)
//   nbeg / ncnt  nodes int32, each node's range of tree positions
// Nodes are numbered in heap order (children of i are 2i+1, 2i+2); all leaves
// sit at depth `height`, so leaves are nodes [2^h - 1, 2^(h+1) - 1) and leaf
// l covers the l-th contiguous run of tree positions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>

#include "dtree.h"

struct dtree {
    int64_t n = 0;
    int32_t d = 0, dp = 0, leaf_size = 0, height = 0;
    int64_t nnodes = 0, nleaves = 0;
    float* pts = nullptr;
    int32_t* idx = nullptr;
    float* box = nullptr;
    float* lam = nullptr;
    int32_t* nbeg = nullptr;
    int32_t* ncnt = nullptr;
    int device = 0;
    // frontier capacity that sufficed for the last traversal against this
    // reference tree (a sizing hint only; results never depend on it)
    int64_t cap_hint = 0;
    // learned proposal attached to this reference tree (not owned), or null
    const dtree_model* proposal = nullptr;
    // tensor-core operand rows of the points (TF32, split BF16), made by the
    // first search that needs them and owned by the handle
    void* tc_ops[2] = {nullptr, nullptr};
};

namespace dt {

extern std::atomic<int64_t> g_launches;
extern std::atomic<int64_t> g_allocs;  // device allocations made by the library

// A fixed device range that stands in for the stream-ordered pool (the
// no-allocation entry point), or null.
struct ScratchArena {
    unsigned char* base;
    size_t bytes;
};

// Top-M proposed cells of `n` points (row-major n x d, device), for the seed.
int proposal_cells(const dtree_model* md, const float* pts, int64_t n, int M, int32_t* out,
                   cudaStream_t s);
// Box centres (n x d) of `count` consecutive nodes of a tree.
int box_centres(const dtree_t* t, int64_t node0, int64_t count, float* out, cudaStream_t s);
int model_level(const dtree_model* md);

// dtree_knn's checks and dispatch, with its scratch from the pool (arena
// null) or from a fixed range.
int knn_entry(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
              float* out_dist, const dtree_opts* o, void* stream, dtree_stats* st,
              const ScratchArena* arena);

// Status of the last failing CUDA call, mapped to dtree_status.
int cuda_status(cudaError_t e);

#define DT_CHECK(call)                                       \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ::dt::cuda_status(e_); \
    } while (0)

// Launch, count, and check the launch.
#define DT_LAUNCH(kern, grid, block, smem, stream, ...)                  \
    do {                                                                 \
        kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);        \
        ::dt::g_launches.fetch_add(1, std::memory_order_relaxed);        \
        cudaError_t e_ = cudaGetLastError();                             \
        if (e_ != cudaSuccess) return ::dt::cuda_status(e_);             \
    } while (0)

inline int dp_bucket(int d) {
    return d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : d <= 32 ? 32 : 64;
}

inline int level_of_count(int64_t n, int64_t cap) {
    // smallest L with ceil(n / 2^L) <= cap
    int L = 0;
    while (((n + (int64_t(1) << L) - 1) >> L) > cap) ++L;
    return L;
}

// Order-preserving map float -> uint32 (for radix keys and atomic min/max).
__host__ __device__ inline uint32_t f2o(float f) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ inline float o2f(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}

__device__ inline int level_of_node(int64_t i) { return 63 - __clzll(i + 1); }

// Relative error allowance of a float32 computation over DP terms (a
// generous multiple of the unit roundoff 2^-24).
template <int DP>
__host__ __device__ constexpr float rel_eps() {
    return float(DP + 8) * 5.9604645e-08f;
}

// Scratch from the device's stream-ordered pool.
template <class T>
inline int scratch(T** p, size_t count, cudaStream_t s) {
    *p = nullptr;
    if (count == 0) return DTREE_OK;
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DTREE_ERR_OOM;
    }
    return DTREE_OK;
}

void prepare_pool(int device);

}  // namespace dt
