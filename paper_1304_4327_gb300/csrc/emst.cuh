// emst.cuh -- the Euclidean minimum spanning tree by Boruvka rounds (dtree_emst).
//
// Section 7 ("Boruvka's Algorithm"): every component finds the shortest edge
// from one of its points to a point outside it, the components joined by
// those edges merge, and the rounds repeat until one component is left.
// Edges are ranked by (float64 squared length, lower original index, higher
// original index): every edge has its own rank, so the tree is unique and
// the components' chosen edges can only form trees and two-cycles (a pair of
// components choosing the same edge).
//
// One round on the GPU, all in kernels:
//   1. node labels: a node's component when all its points share one, else
//      -1 (leaves first, then each level up);
//   2. for every point, its nearest point outside its component (one warp
//      per point, a depth-first walk of the tree nearer child first, the
//      same walk as kfn.cuh): Algorithm 3's Score with the pruning of the
//      Boruvka Score -- a node is pruned when its d_min exceeds the point's
//      best so far (strictly: an equal length may still have a lower rank)
//      or when all its points lie in the point's own component; BaseCase
//      distances in float64, the oracle's arithmetic;
//   3. every component's shortest edge: an atomicMin over the squared
//      lengths (kept up to date during step 2, whose walks prune with it),
//      then over the endpoint pairs among the points that reach it;
//   4. hooks: each component points to the component across its edge (a
//      two-cycle keeps the lower id as the root), and each edge is written
//      once, in component-id order after an in-kernel scan; then pointer
//      jumping to the roots and relabelling of the points.
#pragma once

#include "knn_tile.cuh"

namespace dt {

struct EmstArgs {
    const float* pts;       // tree order, DP floats each
    const int32_t* idx;     // tree position -> original index
    const int32_t* nbeg;
    const int32_t* ncnt;
    const float* box;
    int64_t n;
    int hr;
    int32_t* comp;          // per point: its component (a root point's tree position)
    const int32_t* nlab;    // per node: its component if all its points share one, else -1
    double* bd;             // per point: the squared length of its best edge out (inf: none)
    int32_t* br;            // per point: the other end of that edge (tree position), or -1
    unsigned long long* ck1;    // per component: the key of its shortest edge found so far
    unsigned long long* stats;  // [0] point distances, [1] leaves visited
};

// Order-preserving key of a non-negative double (inf included).
__device__ __forceinline__ unsigned long long dkey(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

template <int DP>
__global__ void __launch_bounds__(128) k_emst_nn(const EmstArgs a) {
    constexpr int NT = (2 * DP + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double shrink = 1.0 - (DP + 4) * 2.3e-16;  // d_min^2 rounded down
    unsigned long long n_pts = 0, n_leaves = 0;
    for (int64_t pos = w0; pos < a.n; pos += nw) {
        const int32_t mine = a.comp[pos];
        const int32_t op = a.idx[pos];
        const float* qp = a.pts + pos * DP;
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
        // the best edge out: (bd2, blo, bhi) ranks by length, then endpoints
        double bd2 = INFINITY;
        uint32_t blo = 0xffffffffu, bhi = 0xffffffffu;
        int32_t bestr = -1;
        auto better = [](double d1, uint32_t l1, uint32_t h1, double d2, uint32_t l2, uint32_t h2) {
            return d1 < d2 || (d1 == d2 && (l1 < l2 || (l1 == l2 && h1 < h2)));
        };
        // the stack: entry `lane` in (sn, sd = d_min^2 rounded down)
        int32_t sn = 0;
        double sd = 0.0;
        // the pruning bound: the shortest edge out of this point's component
        // found so far by any of its points (the point that holds the
        // component's shortest edge never prunes that edge's other end)
        volatile unsigned long long* cbest = a.ck1 + mine;
        double bound = bd2;
        int sp = a.nlab[0] == mine ? 0 : 1;
        while (sp > 0) {
            --sp;
            const int32_t n = __shfl_sync(0xffffffffu, sn, sp);
            const double dm = __shfl_sync(0xffffffffu, sd, sp);
            bound = fmin(bd2, __longlong_as_double((long long)*cbest));  // (fmin skips the NaN of "none")
            bound = __shfl_sync(0xffffffffu, bound, 0);
            if (dm > bound) continue;
            if (level_of_node(n) == a.hr) {
                ++n_leaves;
                const int rb = a.nbeg[n], rc = a.ncnt[n];
                n_pts += rc;
                for (int r0 = 0; r0 < rc; r0 += 32) {
                    const int r = rb + r0 + lane;
                    bool valid = r0 + lane < rc;
                    double d2 = INFINITY;
                    uint32_t lo = 0xffffffffu, hi = 0xffffffffu;
                    if (valid && a.comp[r] != mine) {
                        d2 = exact_d2<DP>(q, a.pts + (int64_t)r * DP);
                        const uint32_t o = (uint32_t)a.idx[r];
                        lo = min((uint32_t)op, o);
                        hi = max((uint32_t)op, o);
                    } else {
                        valid = false;
                    }
                    // the warp's best candidate
                    int cr = valid ? r : -1;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const double od = __shfl_xor_sync(0xffffffffu, d2, off);
                        const uint32_t ol = __shfl_xor_sync(0xffffffffu, lo, off);
                        const uint32_t oh = __shfl_xor_sync(0xffffffffu, hi, off);
                        const int orr = __shfl_xor_sync(0xffffffffu, cr, off);
                        if (better(od, ol, oh, d2, lo, hi)) {
                            d2 = od;
                            lo = ol;
                            hi = oh;
                            cr = orr;
                        }
                    }
                    if (cr >= 0 && better(d2, lo, hi, bd2, blo, bhi)) {
                        bd2 = d2;
                        blo = lo;
                        bhi = hi;
                        bestr = cr;
                        if (lane == 0) atomicMin(a.ck1 + mine, dkey(bd2));
                        bound = fmin(bound, bd2);
                    }
                }
                continue;
            }
            // the two children: squared d_min from the point to each box
            const int64_t l = 2 * (int64_t)n + 1;
            const float* bx = a.box + l * 2 * DP;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int e = lane + 32 * t;
                if (e < 2 * DP) {
                    const int c = e / DP, dd = e % DP;
                    const double qv = qd[t], lo = bx[c * 2 * DP + dd], hi = bx[c * 2 * DP + DP + dd];
                    const double g = fmax(fmax(lo - qv, qv - hi), 0.0);
                    if (c == 0) s0 += g * g;
                    else s1 += g * g;
                }
            }
            double d0, d1;
            if (2 * DP <= 32) {
                double sv = s0 + s1;
#pragma unroll
                for (int off = DP / 2; off > 0; off >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
                d0 = __shfl_sync(0xffffffffu, sv, 0);
                d1 = __shfl_sync(0xffffffffu, sv, DP);
            } else {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                }
                d0 = s0;
                d1 = s1;
            }
            d0 *= shrink;
            d1 *= shrink;
            // push the farther child first, so that the nearer one is taken next
            const bool right_near = d1 < d0;
            const int32_t cf = (int32_t)(right_near ? l : l + 1), cn = (int32_t)(right_near ? l + 1 : l);
            const double df = right_near ? d0 : d1, dn = right_near ? d1 : d0;
            if (a.nlab[cf] != mine && !(df > bound)) {
                if (lane == sp) {
                    sn = cf;
                    sd = df;
                }
                ++sp;
            }
            if (a.nlab[cn] != mine && !(dn > bound)) {
                if (lane == sp) {
                    sn = cn;
                    sd = dn;
                }
                ++sp;
            }
        }
        if (lane == 0) {
            a.bd[pos] = bd2;
            a.br[pos] = bestr;
        }
    }
    if (a.stats) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            n_pts += __shfl_xor_sync(0xffffffffu, n_pts, off);
            n_leaves += __shfl_xor_sync(0xffffffffu, n_leaves, off);
        }
        if (lane == 0) {
            atomicAdd(&a.stats[0], n_pts / 32);
            atomicAdd(&a.stats[1], n_leaves / 32);
        }
    }
}

template <int DP>
int launch_emst_nn(const EmstArgs& a, int grid, cudaStream_t s) {
    auto kern = k_emst_nn<DP>;
    DT_LAUNCH(kern, grid, 128, 0, s, a);
    return DTREE_OK;
}

}  // namespace dt
