// range.cuh -- exact range search (dtree_range_count, dtree_range_fill).
//
// Section 6 ("Range Search"): for every query all reference points with
// d_lo <= ||q - r|| <= d_hi, both ends inclusive; the lists are sets (this
// search writes them in its visit order).  The distance that decides is the
// float64 one of the oracle: the correctly rounded square root of the
// float64 sum of (q_j - r_j)^2, left to right, compared with d_lo and d_hi.
//
// One warp serves one query (a query node of one point: Algorithm 1's
// depth-first recursion on the reference tree), as in kfn.cuh:
//   * Score: a child node is kept unless its box is wholly outside the
//     range -- d_min > d_hi or d_max < d_lo (squared, rounded outwards).
//     The printed Score keeps a pair only when d_lo <= d_min <= d_hi, which
//     also drops nodes with d_min < d_lo <= d_max whose points can lie in
//     the range; the rule here is the sound one.
//   * BaseCase: a leaf's points, one per lane.  A float32 key (relative
//     error <= rel_eps) settles a point that is clearly outside or, when no
//     distance is written, clearly inside: the float bounds around d_lo^2 and
//     d_hi^2 carry a relative margin of 1e-12, far above any float64
//     rounding, so such a decision is the float64 one.  Every other point is
//     decided on its float64 distance.
// Counting and filling take the same decisions, so a query's count is the
// length of its filled segment.
#pragma once

#include "knn_tile.cuh"

namespace dt {

struct RangeArgs {
    // query points in query-tree order and their caller rows
    const float* qpts;
    const int32_t* qidx;
    int64_t nq;
    // reference tree
    const float* rpts;
    const int32_t* ridx;
    const int32_t* rbeg;
    const int32_t* rcnt;
    const float* rbox;
    int hr;
    int mono;
    double d_lo, d_hi;            // the range
    float lo2_dn, lo2_up;         // floats below and above d_lo^2 (margin 1e-12)
    float hi2_dn, hi2_up;         // floats below and above d_hi^2
    int64_t* counts;              // count pass: one per caller row
    const int64_t* offsets;       // fill pass: the start of each caller row's segment
    int64_t* out_idx;
    float* out_dist;
    unsigned long long* stats;    // [0] distances, [1] leaves, [2] nodes pruned, [3] float64 decisions
};

template <int DP, bool FILL>
__global__ void __launch_bounds__(128) k_range(const RangeArgs a) {
    constexpr int NT = (2 * DP + 31) / 32;  // box elements per lane
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool mono = a.mono != 0;
    const float eps = rel_eps<DP>();
    const float box_dn = 1.f - (DP + 4) * 1.2e-7f, box_up = 1.f + (DP + 4) * 1.2e-7f;
    unsigned long long n_pts = 0, n_leaves = 0, n_pruned = 0, n_exact = 0;

    for (int64_t qpos = w0; qpos < a.nq; qpos += nw) {
        const float* qp = a.qpts + qpos * DP;
        float q[DP];
#pragma unroll
        for (int j = 0; j < DP / 4; ++j) {
            const float4 v = reinterpret_cast<const float4*>(qp)[j];
            q[4 * j] = v.x;
            q[4 * j + 1] = v.y;
            q[4 * j + 2] = v.z;
            q[4 * j + 3] = v.w;
        }
        float qd[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int e = lane + 32 * t;
            qd[t] = e < 2 * DP ? qp[e % DP] : 0.f;
        }
        const int64_t row = a.qidx[qpos];
        const int64_t base = FILL ? a.offsets[row] : 0;
        int64_t found = 0;
        // the stack: entry `lane` (at most one more entry than the tree has levels)
        int32_t sn = 0;
        int sp = 1;
        while (sp > 0) {
            --sp;
            const int32_t n = __shfl_sync(0xffffffffu, sn, sp);
            if (level_of_node(n) == a.hr) {
                ++n_leaves;
                const int rb = a.rbeg[n], rc = a.rcnt[n];
                n_pts += rc;
                for (int r0 = 0; r0 < rc; r0 += 32) {
                    const int r = rb + r0 + lane;
                    const bool valid = r0 + lane < rc && !(mono && r == qpos);
                    bool in = false, exact = false;
                    double d = 0.0;
                    if (valid) {
                        const float* rp = a.rpts + (int64_t)r * DP;
                        const float kf = approx_d2<DP>(q, rp);
                        const float k_dn = __fmul_rd(kf, 1.f - 2.f * eps), k_up = __fmul_ru(kf, 1.f + 2.f * eps);
                        if (k_up < a.lo2_dn || k_dn > a.hi2_up) {
                            in = false;
                        } else if (!FILL && k_dn >= a.lo2_up && k_up <= a.hi2_dn) {
                            in = true;
                        } else {
                            exact = true;
                            d = sqrt(exact_d2<DP>(q, rp));
                            in = d >= a.d_lo && d <= a.d_hi;
                        }
                    }
                    n_exact += __popc(__ballot_sync(0xffffffffu, exact));
                    const uint32_t m = __ballot_sync(0xffffffffu, in);
                    if (FILL && in) {
                        const int64_t pos = base + found + __popc(m & ((1u << lane) - 1u));
                        a.out_idx[pos] = a.ridx[r];
                        a.out_dist[pos] = (float)d;
                    }
                    found += __popc(m);
                }
                continue;
            }
            // the two children: squared d_min and d_max from the query to each box
            const int64_t l = 2 * (int64_t)n + 1;
            const float* bx = a.rbox + l * 2 * DP;
            float mn0 = 0.f, mn1 = 0.f, mx0 = 0.f, mx1 = 0.f;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int e = lane + 32 * t;
                if (e < 2 * DP) {
                    const int c = e / DP, dd = e % DP;
                    const float lo = bx[c * 2 * DP + dd], hi = bx[c * 2 * DP + DP + dd];
                    const float gn = fmaxf(fmaxf(lo - qd[t], qd[t] - hi), 0.f);
                    const float gx = fmaxf(fabsf(qd[t] - lo), fabsf(hi - qd[t]));
                    if (c == 0) {
                        mn0 = fmaf(gn, gn, mn0);
                        mx0 = fmaf(gx, gx, mx0);
                    } else {
                        mn1 = fmaf(gn, gn, mn1);
                        mx1 = fmaf(gx, gx, mx1);
                    }
                }
            }
            float dmin[2], dmax[2];
            if (2 * DP <= 32) {
                float sn_ = mn0 + mn1, sx_ = mx0 + mx1;
#pragma unroll
                for (int off = DP / 2; off > 0; off >>= 1) {
                    sn_ += __shfl_xor_sync(0xffffffffu, sn_, off);
                    sx_ += __shfl_xor_sync(0xffffffffu, sx_, off);
                }
                dmin[0] = __shfl_sync(0xffffffffu, sn_, 0);
                dmin[1] = __shfl_sync(0xffffffffu, sn_, DP);
                dmax[0] = __shfl_sync(0xffffffffu, sx_, 0);
                dmax[1] = __shfl_sync(0xffffffffu, sx_, DP);
            } else {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    mn0 += __shfl_xor_sync(0xffffffffu, mn0, off);
                    mn1 += __shfl_xor_sync(0xffffffffu, mn1, off);
                    mx0 += __shfl_xor_sync(0xffffffffu, mx0, off);
                    mx1 += __shfl_xor_sync(0xffffffffu, mx1, off);
                }
                dmin[0] = mn0;
                dmin[1] = mn1;
                dmax[0] = mx0;
                dmax[1] = mx1;
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const bool keep = !(__fmul_rd(dmin[c], box_dn) > a.hi2_up) &&
                                  !(__fmul_ru(dmax[c], box_up) < a.lo2_dn);
                if (keep) {
                    if (lane == sp) sn = (int32_t)(l + c);
                    ++sp;
                } else {
                    ++n_pruned;
                }
            }
        }
        if (!FILL && lane == 0) a.counts[row] = found;
    }
    if (a.stats) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            n_pts += __shfl_xor_sync(0xffffffffu, n_pts, off);
            n_leaves += __shfl_xor_sync(0xffffffffu, n_leaves, off);
            n_pruned += __shfl_xor_sync(0xffffffffu, n_pruned, off);
        }
        if (lane == 0) {
            // (n_exact is already a warp total: every lane holds it)
            atomicAdd(&a.stats[0], n_pts / 32);
            atomicAdd(&a.stats[1], n_leaves / 32);
            atomicAdd(&a.stats[2], n_pruned / 32);
            atomicAdd(&a.stats[3], n_exact);
        }
    }
}

template <int DP>
int launch_range(const RangeArgs& a, bool fill, int grid, cudaStream_t s) {
    if (fill) {
        auto kern = k_range<DP, true>;
        DT_LAUNCH(kern, grid, 128, 0, s, a);
    } else {
        auto kern = k_range<DP, false>;
        DT_LAUNCH(kern, grid, 128, 0, s, a);
    }
    return DTREE_OK;
}

}  // namespace dt
