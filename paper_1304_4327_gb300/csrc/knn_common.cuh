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

struct TileArgs {
    // query tree
    const float* qpts;
    const int32_t* qidx;
    const int32_t* qbeg;
    const int32_t* qcnt;
    const float* qlam;
    const float* qbox;  // nodes x 2 x DP (the block's box gives the tensor-core centring point)
    int64_t qblock0;  // heap id of the first query block
    int64_t nq;       // queries (rows of the candidate lists)
    int cpb;          // work items (chunks of <= 128 queries) per block
    // reference tree
    const float* rpts;
    const int32_t* ridx;
    const int32_t* rbeg;
    const int32_t* rcnt;
    const float* rbox;  // nodes x 2 x DP
    int64_t rleaf0;   // heap id of reference leaf 0
    int32_t k;
    int32_t mono;
    // candidates
    const int32_t* seed_leaf0;  // per block: first seed leaf
    const int32_t* seed_nleaf;  // per block: seed leaves
    const int64_t* csr_off;     // per block: [off[b], off[b+1]) in csr_leaf / csr_dmin
    const int32_t* csr_leaf;
    const float* csr_dmin;
    const float* csr_key;       // evaluation order: distance between block and leaf box centres
    const float* Bq;            // per block: B of the block from the traversal (or null)
    // approximate candidate lists, [kc_rows][nq] layout
    int kc_rows;
    float* cand_d;
    int32_t* cand_i;
    float* qub;                 // per query: upper bound on its true k-th distance (seed pass)
    // work: blocks to process (null = all nblocks)
    const int32_t* work_blocks;
    int nwork;
    int* work_ctr;
    // outputs
    int64_t* out_idx;
    float* out_dist;
    int4* fbq_list;    // queries whose error band overflowed: (tree position, block, ub bits, 0)
    int* fbq_count;
    int4* fbq2_list;   // of those, queries whose float32 band overflowed too
    int* fbq2_count;
    unsigned long long* stats;
};

template <int DP>
int launch_tile_cc(const TileArgs& a, int kc, int mode, int items, cudaStream_t s);

template <int DP>
int launch_query_fb(const TileArgs& a, int kc, int nfbq, bool exact, cudaStream_t s);

template <int DP>
int launch_tile_tc(const TileArgs& a, int fmt, int kc, int mode, int items, int* err, int spin,
                   cudaStream_t s);

template <int DP>
int launch_expand(const float* qbox, const float* rbox, const float* Bq, const int2* fin,
                  const int* nin, int2* fout, int* nout, int64_t cap, int4* outp, int* nout_p,
                  int64_t cap_p, int* bcount, int Lb, int hr, int64_t qblock0, int64_t rleaf0,
                  const int32_t* seed_leaf0, const int32_t* seed_nleaf, int* overflow,
                  unsigned long long* stats, int grid, cudaStream_t s);

template <int DP>
int launch_seed(const float* qbox, const float* rbox, int64_t qblock0, int nblocks, int Ls, int hr,
                int32_t* seed_leaf0, int32_t* seed_nleaf, cudaStream_t s);

int occupancy_grid(const void* kernel, int threads, size_t smem);

}  // namespace dt
