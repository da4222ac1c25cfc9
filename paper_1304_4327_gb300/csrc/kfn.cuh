// kfn.cuh -- exact k-furthest-neighbour search (dtree_kfn).
//
// The extension of Section 5 (the paragraph on k-furthest neighbour search
// after Algorithm 4): the kNN rules inverted -- lists sorted by descending
// distance and initialised to 0 (here: empty), a candidate kept when it is
// farther than the k-th, and a reference node pruned when even its farthest
// possible point is nearer than the query's k-th furthest distance so far.
// Ties are broken by the lower original reference index, so the result is
// unique: the first k of the list sorted by (distance descending, index
// ascending).
//
// One warp serves one query (a query node of one point, so the traversal is
// Algorithm 1's depth-first recursion on the reference tree alone):
//
//   * the stack of reference nodes to visit, with the squared d_max from the
//     query to each node's box, rounded up, holds one entry per lane; a node
//     is visited farther child first;
//   * a node is pruned when its d_max is below the query's k-th furthest
//     squared distance so far, rounded down by the keys' error: every point
//     in it is then strictly nearer than the query's true k-th furthest point
//     (Algorithm 3's Score, inverted; strict, so no tie is lost);
//   * a leaf's points are evaluated one per lane and offered to the list
//     (KC entries, one per lane and slot), the warp inserting them one at a
//     time in ballot order.
//
// Two passes, as in the kNN path's exactness scheme:
//   float    keys are float32 sums of (q_j - r_j)^2 (relative error <= rel_eps).
//            Every true k-furthest point has a key >= band_lo = (k-th key)
//            (1 - 4 rel_eps); if the list also holds every candidate with a
//            key >= band_lo (its KC-th entry is below band_lo), those are
//            recomputed in float64, ranked by (distance descending, index
//            ascending), and the first k are written.  Otherwise the query
//            goes to the second pass.
//   double   keys are the float64 squared distances themselves (the oracle's
//            arithmetic: differences of float32 inputs, squared and summed
//            left to right): the list is the result.
#pragma once

#include <type_traits>

#include "knn_tile.cuh"

namespace dt {

struct KfnArgs {
    // query points in query-tree order (DP floats each) and their caller rows
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
    int k;
    int mono;
    int64_t* out_idx;   // (rows in the caller's query order) x k
    float* out_dist;
    int* fb_list;       // float pass: appends queries whose band overflowed; double pass: its input
    int* fb_count;
    unsigned long long* stats;  // [0] point distances, [1] leaves visited, [2] nodes pruned
};

constexpr int kKfnEmpty = 0x7fffffff;  // the index of an empty list entry

template <int DP, int KC, typename T>
__global__ void __launch_bounds__(128) k_kfn(const KfnArgs a) {
    constexpr bool EXACT = std::is_same<T, double>::value;
    constexpr int NE = (KC + 31) / 32;      // list entries per lane
    constexpr int NT = (2 * DP + 31) / 32;  // box elements per lane
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = EXACT ? (int64_t)*a.fb_count : a.nq;
    const int k = a.k;
    const bool mono = a.mono != 0;
    // squared-distance rounding: d_max up, list keys down (float keys only)
    const T up = EXACT ? (T)(1.0 + (DP + 4) * 2.3e-16) : (T)(1.f + (DP + 4) * 1.2e-7f);
    const float eps = rel_eps<DP>();
    unsigned long long n_pts = 0, n_leaves = 0, n_pruned = 0;

    for (int64_t wi = w0; wi < count; wi += nw) {
        const int64_t qpos = EXACT ? (int64_t)a.fb_list[wi] : wi;
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
        float qd[NT];  // the query coordinate of each of this lane's box elements
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int e = lane + 32 * t;
            qd[t] = e < 2 * DP ? qp[e % DP] : 0.f;
        }
        // the list: entry 32 s + lane in (ld, li = original index, lp = tree position)
        T ld[NE];
        int li[NE], lp[NE];
#pragma unroll
        for (int s = 0; s < NE; ++s) {
            ld[s] = (T)-1;
            li[s] = kKfnEmpty;
            lp[s] = 0;
        }
        // (d1, i1) ranks before (d2, i2): farther, or as far with a lower index
        auto before = [](T d1, int i1, T d2, int i2) { return d1 > d2 || (d1 == d2 && i1 < i2); };
        auto entry_d = [&](int e) {
            T v = ld[0];
#pragma unroll
            for (int s = 1; s < NE; ++s)
                if ((e >> 5) == s) v = ld[s];
            return __shfl_sync(0xffffffffu, v, e & 31);
        };
        auto entry_i = [&](int e) {
            int v = li[0];
#pragma unroll
            for (int s = 1; s < NE; ++s)
                if ((e >> 5) == s) v = li[s];
            return __shfl_sync(0xffffffffu, v, e & 31);
        };
        // the stack: entry `lane` in (sn, sd); a depth-first walk keeps at
        // most one more entry than the tree has levels (the host checks <= 31)
        int32_t sn = 0;
        T sd = (T)INFINITY;
        int sp = 1;
        while (sp > 0) {
            --sp;
            const int32_t n = __shfl_sync(0xffffffffu, sn, sp);
            const T dm = __shfl_sync(0xffffffffu, sd, sp);
            // a lower bound on the query's true k-th furthest squared distance
            const T kth = entry_d(k - 1);
            const T L = kth < (T)0 ? (T)-1 : (EXACT ? kth : (T)__fmul_rd((float)kth, 1.f - 2.f * eps));
            if (dm < L) {
                ++n_pruned;
                continue;
            }
            if (level_of_node(n) == a.hr) {
                // a leaf: its points, one per lane
                ++n_leaves;
                const int rb = a.rbeg[n], rc = a.rcnt[n];
                n_pts += rc;
                for (int r0 = 0; r0 < rc; r0 += 32) {
                    const int r = rb + r0 + lane;
                    const bool valid = r0 + lane < rc && !(mono && r == qpos);
                    T d = (T)-1;
                    int oi = kKfnEmpty;
                    if (valid) {
                        const float* rp = a.rpts + (int64_t)r * DP;
                        d = EXACT ? (T)exact_d2<DP>(q, rp) : (T)approx_d2<DP>(q, rp);
                        oi = a.ridx[r];
                    }
                    T td = entry_d(KC - 1);
                    int ti = entry_i(KC - 1);
                    uint32_t m = __ballot_sync(0xffffffffu, valid && before(d, oi, td, ti));
                    while (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        const T cd = __shfl_sync(0xffffffffu, d, src);
                        const int ci = __shfl_sync(0xffffffffu, oi, src);
                        const int cp = __shfl_sync(0xffffffffu, r, src);
                        if (!before(cd, ci, td, ti)) continue;
                        // insert: entries from its position on move down one place
                        int pos = 0;
#pragma unroll
                        for (int s = 0; s < NE; ++s)
                            pos += __popc(__ballot_sync(0xffffffffu, before(ld[s], li[s], cd, ci)));
#pragma unroll
                        for (int s = NE - 1; s >= 0; --s) {
                            T pv = __shfl_up_sync(0xffffffffu, ld[s], 1);
                            int pi = __shfl_up_sync(0xffffffffu, li[s], 1);
                            int pp = __shfl_up_sync(0xffffffffu, lp[s], 1);
                            if (s > 0) {
                                const T cv = __shfl_sync(0xffffffffu, ld[s > 0 ? s - 1 : 0], 31);
                                const int cix = __shfl_sync(0xffffffffu, li[s > 0 ? s - 1 : 0], 31);
                                const int cpx = __shfl_sync(0xffffffffu, lp[s > 0 ? s - 1 : 0], 31);
                                if (lane == 0) {
                                    pv = cv;
                                    pi = cix;
                                    pp = cpx;
                                }
                            }
                            const int e = 32 * s + lane;
                            if (e < KC) {
                                if (e > pos) {
                                    ld[s] = pv;
                                    li[s] = pi;
                                    lp[s] = pp;
                                } else if (e == pos) {
                                    ld[s] = cd;
                                    li[s] = ci;
                                    lp[s] = cp;
                                }
                            }
                        }
                        td = entry_d(KC - 1);
                        ti = entry_i(KC - 1);
                    }
                }
                continue;
            }
            // the two children: squared d_max from the query to each box
            const int64_t l = 2 * (int64_t)n + 1;
            const float* bx = a.rbox + l * 2 * DP;
            T s0 = 0, s1 = 0;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int e = lane + 32 * t;
                if (e < 2 * DP) {
                    const int c = e / DP, d = e % DP;
                    // (in T: float64 differences of float32 values are exact)
                    const T qv = (T)qd[t], lo = (T)bx[c * 2 * DP + d], hi = (T)bx[c * 2 * DP + DP + d];
                    const T g = fmax(fabs(qv - lo), fabs(hi - qv));
                    if (c == 0) s0 += g * g;
                    else s1 += g * g;
                }
            }
            T dl, dr;
            if (2 * DP <= 32) {
                T sv = s0 + s1;
#pragma unroll
                for (int off = DP / 2; off > 0; off >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
                dl = __shfl_sync(0xffffffffu, sv, 0);
                dr = __shfl_sync(0xffffffffu, sv, DP);
            } else {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                }
                dl = s0;
                dr = s1;
            }
            dl *= up;
            dr *= up;
            // push the nearer child first, so that the farther one is taken next
            const bool right_far = dr > dl;
            const int32_t n_near = (int32_t)(right_far ? l : l + 1), n_far = (int32_t)(right_far ? l + 1 : l);
            const T d_near = right_far ? dl : dr, d_far = right_far ? dr : dl;
            if (!(d_near < L)) {
                if (lane == sp) {
                    sn = n_near;
                    sd = d_near;
                }
                ++sp;
            } else {
                ++n_pruned;
            }
            if (!(d_far < L)) {
                if (lane == sp) {
                    sn = n_far;
                    sd = d_far;
                }
                ++sp;
            } else {
                ++n_pruned;
            }
        }
        const int64_t row = a.qidx[qpos];
        if (EXACT) {
            // exact keys: the list's first k entries are the result
#pragma unroll
            for (int s = 0; s < NE; ++s) {
                const int e = 32 * s + lane;
                if (e < k) {
                    a.out_idx[row * k + e] = li[s];
                    a.out_dist[row * k + e] = (float)sqrt((double)ld[s]);
                }
            }
            continue;
        }
        const float band_lo = __fmul_rd((float)entry_d(k - 1), 1.f - 4.f * eps);
        const bool full = entry_i(KC - 1) != kKfnEmpty;
        if (full && !((float)entry_d(KC - 1) < band_lo)) {
            if (lane == 0) a.fb_list[atomicAdd(a.fb_count, 1)] = (int)qpos;
            continue;
        }
        // float64 re-rank of the band's members
        double dd[NE];
        bool in[NE];
#pragma unroll
        for (int s = 0; s < NE; ++s) {
            in[s] = li[s] != kKfnEmpty && !((float)ld[s] < band_lo);
            dd[s] = in[s] ? exact_d2<DP>(q, a.rpts + (int64_t)lp[s] * DP) : -1.0;
        }
        int rank[NE];
#pragma unroll
        for (int s = 0; s < NE; ++s) rank[s] = 0;
#pragma unroll
        for (int s2 = 0; s2 < NE; ++s2)
            for (int src = 0; src < 32; ++src) {
                const double od = __shfl_sync(0xffffffffu, dd[s2], src);
                const int oi = __shfl_sync(0xffffffffu, li[s2], src);
                const bool oin = __shfl_sync(0xffffffffu, in[s2] ? 1 : 0, src) != 0;
#pragma unroll
                for (int s = 0; s < NE; ++s)
                    rank[s] += oin && (od > dd[s] || (od == dd[s] && oi < li[s]));
            }
#pragma unroll
        for (int s = 0; s < NE; ++s)
            if (in[s] && rank[s] < k) {
                a.out_idx[row * k + rank[s]] = li[s];
                a.out_dist[row * k + rank[s]] = (float)sqrt(dd[s]);
            }
    }
    if (a.stats) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            n_pts += __shfl_xor_sync(0xffffffffu, n_pts, off);
            n_leaves += __shfl_xor_sync(0xffffffffu, n_leaves, off);
            n_pruned += __shfl_xor_sync(0xffffffffu, n_pruned, off);
        }
        if (lane == 0) {
            // every lane counted the same warp-uniform events
            atomicAdd(&a.stats[0], n_pts / 32);
            atomicAdd(&a.stats[1], n_leaves / 32);
            atomicAdd(&a.stats[2], n_pruned / 32);
        }
    }
}

template <int DP>
int launch_kfn(const KfnArgs& a, int kc, bool exact, int grid, cudaStream_t s) {
#define DT_KFN_CASE(KCV)                                                        \
    case KCV:                                                                   \
        if (exact) {                                                            \
            auto kern = k_kfn<DP, KCV, double>;                                 \
            DT_LAUNCH(kern, grid, 128, 0, s, a);                                \
        } else {                                                                \
            auto kern = k_kfn<DP, KCV, float>;                                  \
            DT_LAUNCH(kern, grid, 128, 0, s, a);                                \
        }                                                                       \
        return DTREE_OK;
    switch (kc) {
        DT_KFN_CASE(16)
        DT_KFN_CASE(32)
        DT_KFN_CASE(64)
        default:
            return DTREE_ERR_UNSUPPORTED;
    }
#undef DT_KFN_CASE
}

}  // namespace dt
