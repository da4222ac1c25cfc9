// knn_common.cuh -- shared declarations of the kNN kernels (dtree_knn).
#pragma once

#include "dtree_internal.cuh"

namespace dt {

// Counters gathered on the device (dtree_stats order).
enum StatSlot {
    ST_SCORED = 0,
    ST_PRUNED,
    ST_EMITTED,
    ST_SKIPPED,
    ST_EVALUATED,
    ST_POINT_PAIRS,
    ST_RERANK,
    ST_FALLBACK,
    ST_SEED_PAIRS,
    ST_NSTAT
};

// What a BaseCase tile pass starts from and what it leaves behind.
enum TileMode {
    MODE_SEED = 0,  // seed leaves only, empty lists in, approximate lists out
    MODE_MAIN = 1   // traversal candidates, lists in, exact re-rank + output out
};

constexpr int kQB = 128;           // queries of one work item (one thread each)
constexpr int kEmptyIdx = 0x7fffffff;

// One kNN problem of a batch, as the kernels see it.  Blocks (query-tree
// nodes at the block level) are numbered across the batch: the problem's
// blocks are [block0, block0 + nblocks).  Its queries occupy rows
// [q0, q0 + n_query) of the per-query arrays (candidate lists, bounds), in
// query-tree order, and its query nodes of levels 0..Lb occupy entries
// [node0, node0 + 2^(Lb+1) - 1) of the per-node bound arrays.
struct ProbDev {
    // query tree
    const float* qpts;
    const int32_t* qidx;
    const int32_t* qbeg;
    const int32_t* qcnt;
    const float* qlam;
    const float* qbox;  // nodes x 2 x DP
    // reference tree
    const float* rpts;
    const int32_t* ridx;
    const int32_t* rbeg;
    const int32_t* rcnt;
    const float* rbox;  // nodes x 2 x DP; the root box's centre is the tensor-core centring point
    const float* rlam;  // nodes: lambda (largest distance from the box centre to a point)
    const void* rops;   // tensor-core operand rows of the reference points (or null)
    int64_t rls8;       // 8-row groups per leaf in rops
    // outputs, rows in the caller's query order
    int64_t* out_idx;
    float* out_dist;
    int64_t qblock0;  // heap id of the first query block in the query tree
    int64_t rleaf0;   // heap id of reference leaf 0
    int64_t q0;       // first row of the problem in the per-query arrays
    int64_t node0;    // first entry of the problem in the per-node arrays
    int32_t block0;   // first block of the problem
    int32_t nblocks;
    int32_t cpb;      // work items (chunks of <= 128 queries) per block
    int32_t k;
    int32_t mono;
    int32_t Lb;       // level of the query blocks
    int32_t hr;       // height of the reference tree
    int32_t Ls;       // level of the greedy seed subtree in the reference tree
    int32_t Lp;       // level of the learned proposal's cells (the proposed seed subtrees)
    int32_t item0;    // first work item of the problem
    int32_t bound;    // dtree_bound of the node and point lower bounds
};

// ---- lower bounds on distances to a node (Section 3: d_min), rounded down
// so that float32 rounding can only keep what the exact rule would prune.
// A node's centre is its box centre 0.5 (lo + hi) (in float32 exactly as the
// build computed lambda around it: halving is exact); lambda bounds the
// distance from it to every point of the node.

// The box-centre distance |C_a - C_b| of two nodes, rounded down.
template <int DP>
__device__ __forceinline__ float centre_dist_down(const float* a, const float* b) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        const float t = 0.5f * (a[j] + a[DP + j]) - 0.5f * (b[j] + b[DP + j]);
        s = fmaf(t, t, s);
    }
    return __fmul_rd(__fsqrt_rd(s), 1.f - rel_eps<DP>());
}

// Ball bound between two nodes: |C_a - C_b| - lambda_a - lambda_b (>= 0).
template <int DP>
__device__ __forceinline__ float ball_dmin_down(const float* a, float la, const float* b, float lb) {
    return fmaxf(__fsub_rd(__fsub_rd(centre_dist_down<DP>(a, b), la), lb), 0.f);
}

// Point-to-box distance (the box's nearest point), rounded down.
template <int DP>
__device__ __forceinline__ float point_box_dmin_down(const float* q, const float* bx) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        float g = fmaxf(fmaxf(bx[j] - q[j], q[j] - bx[DP + j]), 0.f);
        s = fmaf(g, g, s);
    }
    return __fmul_rd(__fsqrt_rd(s), 1.f - rel_eps<DP>());
}

// Point-to-ball distance |q - C| - lambda (>= 0), rounded down.
template <int DP>
__device__ __forceinline__ float point_ball_dmin_down(const float* q, const float* bx, float lam) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        const float t = q[j] - 0.5f * (bx[j] + bx[DP + j]);
        s = fmaf(t, t, s);
    }
    return fmaxf(__fsub_rd(__fmul_rd(__fsqrt_rd(s), 1.f - rel_eps<DP>()), lam), 0.f);
}

// A point's lower bound against a node under the search's dtree_bound.
template <int DP>
__device__ __forceinline__ float point_dmin_down(int bound, const float* q, const float* bx, float lam) {
    if (bound == DTREE_BOUND_BOX) return point_box_dmin_down<DP>(q, bx);
    const float b = point_ball_dmin_down<DP>(q, bx, lam);
    return bound == DTREE_BOUND_BALL ? b : fmaxf(b, point_box_dmin_down<DP>(q, bx));
}

struct TileArgs {
    const ProbDev* probs;       // the batch's problems
    const int32_t* blk_prob;    // per block: its problem
    const int2* items;          // per work item: (block, chunk of 128 queries)
    int nitems;
    int64_t nq_all;             // rows of the per-query arrays (all problems' queries)
    // candidates
    const int32_t* seed_leaf0;  // per block and seed slot: first leaf of the slot's subtree
    const int32_t* seed_nleaf;  // per block and seed slot: its leaves (0: an unused slot)
    int seed_slots;             // seed slots per block (the greedy subtree, proposed cells)
    int seed_eval_slots;        // of those, the first this many are evaluated by the seed pass;
                                //   the tensor-core main pass evaluates the rest first
    const int64_t* csr_off;     // per block: [off[b], off[b+1]) in csr_leaf / csr_dmin, in
                                //   evaluation order (windows sorted by box-centre distance)
    const int32_t* csr_leaf;
    const float* csr_dmin;
    const float* Bn;            // per query node: B from the bounds pass (or null)
    // approximate candidate lists, [kc_rows][nq_all] layout
    int kc_rows;
    float* cand_d;
    int32_t* cand_i;
    float* qub;                 // per query: upper bound on its true k-th distance (seed pass)
    const float* qcap;          // per query: the cap pass's upper bound on it (or null)
    int* work_ctr;
    int4* fbq_list;    // queries whose error band overflowed: (tree position, block, ub bits, 0)
    int* fbq_count;
    int4* fbq2_list;   // of those, queries whose float32 band overflowed too
    int* fbq2_count;
    // the recomputation's slices per query (1: one CTA per query) and, for
    // more, their lists: queries x slices x KC keys (float64), then as many
    // indices
    int fb_slices;
    void* fb_part;
    unsigned long long* stats;
};

template <int DP>
int launch_tile_cc(const TileArgs& a, int kc, int mode, int items, cudaStream_t s);

// Per-query caps on the k-th distance: a best-first search of up to `budget`
// reference leaves per query, merged into its candidate list of kc (=
// a.kc_rows) entries; writes qcap and lowers qub.
template <int DP>
int launch_query_cap(const TileArgs& a, int kc, int budget, float* qcap, cudaStream_t s);

template <int DP>
int launch_query_fb(const TileArgs& a, int kc, int nfbq, bool exact, cudaStream_t s);

// The tensor-core BaseCase pass (main mode): fmt 1 = BF16 (split), 2 = TF32.
template <int DP>
int launch_tile_tc(const TileArgs& a, int fmt, int kc, int items, int* err, int spin,
                   cudaStream_t s);

// Bytes per operand row, and the fill of a reference tree's operand array
// (nleaves x ls rows, ls a multiple of 8) for the tensor-core pass.
template <int DP>
size_t tc_ops_row_bytes(int fmt);
template <int DP>
int launch_tc_ops(const dtree_t* t, int fmt, int ls, void* out, cudaStream_t s);

// A block's seed: up to `slots` disjoint subtrees of the reference tree,
// slot s covering leaves [leaf0[s], leaf0[s] + nleaf[s]).
__device__ __forceinline__ int seed_count(const int32_t* sn, int slots, int blk) {
    int t = 0;
    for (int s = 0; s < slots; ++s) t += sn[blk * slots + s];
    return t;
}

// Leaves of a block's first n seed slots.
__device__ __forceinline__ int seed_count_n(const int32_t* sn, int slots, int n, int blk) {
    int t = 0;
    for (int s = 0; s < n; ++s) t += sn[blk * slots + s];
    return t;
}

// The ci-th seed leaf of a block (slots in order).
__device__ __forceinline__ int seed_leaf(const int32_t* sl0, const int32_t* sn, int slots, int blk,
                                         int ci) {
    for (int s = 0; s < slots; ++s) {
        const int n = sn[blk * slots + s];
        if (ci < n) return sl0[blk * slots + s] + ci;
        ci -= n;
    }
    return -1;
}

__device__ __forceinline__ bool in_seed(const int32_t* sl0, const int32_t* sn, int slots, int blk,
                                        int leaf) {
    for (int s = 0; s < slots; ++s) {
        const int l0 = sl0[blk * slots + s];
        if (leaf >= l0 && leaf < l0 + sn[blk * slots + s]) return true;
    }
    return false;
}

// The traversal's frontier holds (global query node, reference node) pairs;
// node_prob gives each global query node's problem.
template <int DP>
int launch_expand(const ProbDev* probs, const int32_t* node_prob, const float* Bn, const int2* fin,
                  const int* nin, int2* fout, int* nout, int64_t cap, int4* outp, int* nout_p,
                  int64_t cap_p, int* bcount, const int32_t* seed_leaf0,
                  const int32_t* seed_nleaf, int seed_slots, int* overflow,
                  unsigned long long* stats, int np, int grid, cudaStream_t s);

template <int DP>
int launch_seed(const ProbDev* probs, const int32_t* blk_prob, int nblocks, int seed_slots,
                int32_t* seed_leaf0, int32_t* seed_nleaf, cudaStream_t s);

int occupancy_grid(const void* kernel, int threads, size_t smem);

}  // namespace dt
