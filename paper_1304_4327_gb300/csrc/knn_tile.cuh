// knn_tile.cuh -- the kNN BaseCase (Algorithm 2 of Curtin et al.) on CUDA
// cores, one CTA per work item of <= 128 queries, one thread per query.
//
// For a query block and a list of reference leaves the CTA streams the
// leaves' points through shared memory and each thread keeps its query's
// candidate list (distance key, index) sorted in registers: a reference
// point enters when its key beats the list's last entry, the "d < D[k]"
// test of Algorithm 2 with ties broken by the lower index.
//
// Lists hold KC > k entries.  In float32 the squared distance carries a
// relative error of at most eps = (DP + 8) 2^-24, so
//   - an upper bound on the true k-th distance is sqrt(kth * (1 + 2 eps)),
//     which feeds B_1 and B_2 (Section 5) and the Score test (Algorithm 3)
//     that skips a leaf whose d_min exceeds the block's bound;
//   - every true k-nearest neighbour has a float32 key within
//     band = kth * (1 + 4 eps); at the end those candidates are re-ranked
//     with the exact float64 distance (the same left-to-right sum as the
//     definition) and ordered by (distance, reference index).
// If more than KC - k keys fall inside the band (near-ties or duplicates) the
// list may have dropped a true neighbour: that query is listed and
// recomputed in float64 (k_query_fb), where keys are exact.
#pragma once

#include <type_traits>

#include "knn_common.cuh"

namespace dt {

template <typename T>
__device__ __forceinline__ bool key_less(T d, int i, T e, int j) {
    return d < e || (d == e && i < j);
}

// Insert (d, i) into the ascending list (bubble through; the last entry falls off).
template <typename T, int KC>
__device__ __forceinline__ void list_insert(T (&ld)[KC], int (&li)[KC], T d, int i) {
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        if (key_less(d, i, ld[j], li[j])) {
            T td = ld[j];
            int ti = li[j];
            ld[j] = d;
            li[j] = i;
            d = td;
            i = ti;
        }
    }
}

// The same insertion without a serial chain: every comparison against the
// new key is independent (the list is sorted, so the smaller entries form a
// prefix), then each slot either keeps its entry, takes the new one or takes
// its predecessor.  Descending order reads each predecessor before it moves.
template <typename T, int KC>
__device__ __forceinline__ void list_insert_par(T (&ld)[KC], int (&li)[KC], T d, int i) {
    bool lt[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) lt[j] = key_less(ld[j], li[j], d, i);
#pragma unroll
    for (int j = KC - 1; j >= 0; --j) {
        if (!lt[j]) {
            if (j == 0 || lt[j - 1]) {
                ld[j] = d;
                li[j] = i;
            } else {
                ld[j] = ld[j - 1];
                li[j] = li[j - 1];
            }
        }
    }
}

// Is i among the list's indices?
template <int KC>
__device__ __forceinline__ bool listed(const int (&li)[KC], int i) {
    bool in = false;
#pragma unroll
    for (int j = 0; j < KC; ++j) in |= li[j] == i;
    return in;
}

template <typename T, int KC>
__device__ __forceinline__ T list_at(const T (&ld)[KC], int j) {
    T v = ld[0];
#pragma unroll
    for (int q = 1; q < KC; ++q)
        if (q == j) v = ld[q];
    return v;
}

// Exact squared distance: sum over j of (q_j - r_j)^2 in float64, left to
// right, one rounding per operation (padded dimensions add +0 exactly).
template <int DP>
__device__ __forceinline__ double exact_d2(const float* q, const float* r) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        double t = __dsub_rn((double)q[j], (double)r[j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

template <typename T, int DP>
__device__ __forceinline__ float ub_of(T kth) {
    if (sizeof(T) == 8) return __double2float_ru(__dsqrt_ru((double)kth));
    if (!(kth < INFINITY)) return INFINITY;
    return __fsqrt_ru(__fmul_ru((float)kth, 1.f + 2.f * rel_eps<DP>()));
}

// Warp 0 of a tile CTA: take candidate leaves from the current window, in
// order, skip those whose d_min exceeds the block's bound (Algorithm 3:
// Score = infinity), and pack the rows of the rest (whole leaves, or the
// part of a leaf that fits) into a stage of at most TN points.  stab gets one
// (first row, rows, stage offset) entry per run of rows.
template <int TN, int MODE>
__device__ __forceinline__ void stage_fill(const TileArgs& a, const ProbDev& P, int64_t w0,
                                           int wn, int nseed, int blk, int64_t c0, int3* stab,
                                           unsigned long long& n_skip, unsigned long long& n_eval,
                                           int& s_cur, int& s_part, int& s_nst, int& s_ntab,
                                           const float Bc) {
    const int lane = threadIdx.x & 31;
    int cur = s_cur, part = s_part, nst = 0, ntab = 0;
    while (cur < wn && nst < TN) {
        int c = cur + lane;
        bool valid = c < wn;
        int leaf = 0;
        float dmin = 0.f;
        if (valid) {
            if (MODE == MODE_MAIN) {  // the block's candidates, sorted nearest-first
                const int64_t ci = c0 + w0 + c;
                leaf = a.csr_leaf[ci];
                dmin = a.csr_dmin[ci];
            } else {
                int64_t ci = w0 + c;
                if (ci < nseed) {
                    leaf = seed_leaf(a.seed_leaf0, a.seed_nleaf, a.seed_slots, blk, (int)ci);
                } else {
                    leaf = a.csr_leaf[c0 + ci - nseed];
                    dmin = a.csr_dmin[c0 + ci - nseed];
                }
            }
        }
        bool keep = valid && !(dmin > Bc);
        int lb = 0, lc = 0;
        if (keep) {
            int64_t ln = P.rleaf0 + leaf;
            lb = P.rbeg[ln];
            lc = P.rcnt[ln];
        }
        if (lane == 0 && part > 0 && keep) {  // rest of a split leaf
            lb += part;
            lc -= part;
        }
        int incl = lc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        int excl = incl - lc;
        int take = min(max(TN - nst - excl, 0), lc);
        bool full = valid && take == lc;
        unsigned fm = __ballot_sync(0xffffffffu, full);
        int nlead = fm == 0xffffffffu ? 32 : __ffs(~fm) - 1;
        bool put = take > 0 && lane <= nlead;
        unsigned tm = __ballot_sync(0xffffffffu, put);
        if (put) stab[ntab + __popc(tm & ((1u << lane) - 1u))] = make_int3(lb, take, nst + excl);
        unsigned sk = __ballot_sync(0xffffffffu, valid && !keep && lane < nlead);
        unsigned ev = __ballot_sync(0xffffffffu, keep && lane < nlead);
        if (lane == 0) {
            n_skip += __popc(sk);
            n_eval += __popc(ev);
        }
        int taken = put ? take : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) taken += __shfl_xor_sync(0xffffffffu, taken, off);
        int pn = __shfl_sync(0xffffffffu, take, nlead & 31);
        nst += taken;
        ntab += __popc(tm);
        if (nlead < 32) {
            part = (nlead == 0 ? part : 0) + pn;
            cur += nlead;
            if (!(cur < wn)) part = 0;
            break;  // stage full, or the window is exhausted
        }
        cur += 32;
        part = 0;
    }
    if (lane == 0) {
        s_cur = cur;
        s_part = part;
        s_nst = nst;
        s_ntab = ntab;
    }
}

template <typename T, int DP, int KC, int MODE>
__global__ void __launch_bounds__(kQB) k_tile(const TileArgs a) {
    constexpr int TN = 4096 / DP;       // staged reference points (16 KB)
    constexpr int WINDOW = 2048;        // candidates per window of the main pass
    __shared__ __align__(16) float rs[TN * DP];
    __shared__ int32_t spos[TN];
    __shared__ int3 stab[TN];
    __shared__ int s_item, s_ntab, s_nst, s_cur, s_part;
    __shared__ float s_B;
    __shared__ float s_rmax[kQB / 32], s_rmin[kQB / 32];
    __shared__ ProbDev s_prob;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nitems = a.nitems;
    unsigned long long n_skip = 0, n_eval = 0, n_pp = 0, n_re = 0;
    const ProbDev& P = s_prob;

    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(a.work_ctr, 1);
            if (s_item < nitems) s_prob = a.probs[a.blk_prob[a.items[s_item].x]];
        }
        __syncthreads();
        const int item = s_item;
        if (item >= nitems) break;
        const int2 wi = a.items[item];
        const int blk = wi.x, chunk = wi.y;  // global block, chunk of its queries
        const int64_t qnode = P.qblock0 + (blk - P.block0);
        const int nq = min(kQB, P.qcnt[qnode] - chunk * kQB);
        if (nq > 0) {
            const bool act = tid < nq;
            const int myq = P.qbeg[qnode] + chunk * kQB + tid;
            const int64_t row = P.q0 + myq;  // the query's row in the per-query arrays
            const int kq = P.k;                // read once: stores below could alias P
            const bool mono = P.mono != 0;
            float q[DP];
            {
                const float4* q4 = reinterpret_cast<const float4*>(P.qpts + (int64_t)myq * DP);
#pragma unroll
                for (int j = 0; j < DP / 4; ++j) {
                    float4 v = act ? q4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                    q[4 * j] = v.x;
                    q[4 * j + 1] = v.y;
                    q[4 * j + 2] = v.z;
                    q[4 * j + 3] = v.w;
                }
            }
            T ld[KC];
            int li[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) {
                ld[j] = (T)INFINITY;
                li[j] = kEmptyIdx;
                if (MODE == MODE_MAIN && act) {
                    ld[j] = (T)a.cand_d[(int64_t)j * a.nq_all + row];
                    li[j] = a.cand_i[(int64_t)j * a.nq_all + row];
                }
            }
            const float lam2 = 2.f * P.qlam[qnode];
            const float Bq = a.Bn ? a.Bn[P.node0 + qnode] : INFINITY;
            // the cap pass's bound on the query's k-th distance (main pass only)
            const float qc = MODE == MODE_MAIN && act && a.qcap ? a.qcap[row] : INFINITY;

            // the block's live bound: min(B from the traversal, B_1, B_2)
            auto refresh_bound = [&]() {
                float ub = fminf(ub_of<T, DP>(list_at(ld, kq - 1)), qc);
                float vmax = act ? ub : -INFINITY, vmin = act ? ub : INFINITY;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
                    vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
                }
                if (lane == 0) {
                    s_rmax[warp] = vmax;
                    s_rmin[warp] = vmin;
                }
                __syncthreads();
                if (tid == 0) {
                    for (int w = 1; w < kQB / 32; ++w) {
                        vmax = fmaxf(vmax, s_rmax[w]);
                        vmin = fminf(vmin, s_rmin[w]);
                    }
                    float b2 = __fadd_ru(vmin, lam2);
                    s_B = fminf(Bq, fminf(vmax, b2));
                }
                __syncthreads();
            };
            refresh_bound();

            const int nseed = MODE == MODE_MAIN ? 0 : seed_count_n(a.seed_nleaf, a.seed_slots, a.seed_eval_slots, blk);
            const int64_t c0 = MODE == MODE_SEED ? 0 : a.csr_off[blk];
            const int64_t c1 = MODE == MODE_SEED ? 0 : a.csr_off[blk + 1];
            const int64_t ntot = nseed + (c1 - c0);
            const int64_t win = MODE == MODE_MAIN ? WINDOW : (ntot > 0 ? ntot : 1);

            for (int64_t w0 = 0; w0 < ntot; w0 += win) {
                const int wn = (int)(ntot - w0 < win ? ntot - w0 : win);
                if (tid == 0) {
                    s_cur = 0;
                    s_part = 0;
                }
                __syncthreads();
                while (s_cur < wn) {
                    // ---- warp 0 fills the stage with whole or partial leaves
                    if (warp == 0)
                        stage_fill<TN, MODE>(a, P, w0, wn, nseed, blk, c0, stab, n_skip,
                                             n_eval, s_cur, s_part, s_nst, s_ntab, s_B);
                    __syncthreads();
                    // ---- all warps copy the staged rows
                    const int ntab = s_ntab, nst = s_nst;
                    for (int t = warp; t < ntab; t += kQB / 32) {
                        int3 e = stab[t];
                        const float4* src = reinterpret_cast<const float4*>(P.rpts) + (int64_t)e.x * (DP / 4);
                        float4* dst = reinterpret_cast<float4*>(rs) + e.z * (DP / 4);
                        for (int f = lane; f < e.y * (DP / 4); f += 32) dst[f] = src[f];
                        for (int i = lane; i < e.y; i += 32) {
                            spos[e.z + i] = e.x + i;
                        }
                    }
                    __syncthreads();
                    // ---- BaseCase over the stage
                    if (act) {
#pragma unroll 2
                        for (int e = 0; e < nst; ++e) {
                            const float4* r4 = reinterpret_cast<const float4*>(rs + e * DP);
                            T acc = 0;
#pragma unroll
                            for (int j = 0; j < DP / 4; ++j) {
                                float4 v = r4[j];
                                if (sizeof(T) == 4) {
                                    float t0 = q[4 * j] - v.x, t1 = q[4 * j + 1] - v.y;
                                    float t2 = q[4 * j + 2] - v.z, t3 = q[4 * j + 3] - v.w;
                                    float f = (float)acc;
                                    f = fmaf(t0, t0, f);
                                    f = fmaf(t1, t1, f);
                                    f = fmaf(t2, t2, f);
                                    f = fmaf(t3, t3, f);
                                    acc = (T)f;
                                } else {
                                    double s = (double)acc;
                                    const float rv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        double t = __dsub_rn((double)q[4 * j + u], (double)rv[u]);
                                        s = __dadd_rn(s, __dmul_rn(t, t));
                                    }
                                    acc = (T)s;
                                }
                            }
                            const int rp = spos[e];
                            const int tie = rp;
                            // (the cap pass may have listed this point already)
                            if (key_less(acc, tie, ld[KC - 1], li[KC - 1]) && !(mono && rp == myq) &&
                                !(MODE == MODE_MAIN && listed(li, tie)))
                                list_insert(ld, li, acc, tie);
                        }
                    }
                    if (tid == 0) n_pp += (unsigned long long)nst * nq;
                    refresh_bound();
                }
                __syncthreads();
            }

            // ---- finish the work item
            if (MODE == MODE_SEED) {
                if (act) {
#pragma unroll
                    for (int j = 0; j < KC; ++j) {
                        a.cand_d[(int64_t)j * a.nq_all + row] = (float)ld[j];
                        a.cand_i[(int64_t)j * a.nq_all + row] = li[j];
                    }
                    // the main pass may keep longer lists: their other rows start empty
                    for (int j = KC; j < a.kc_rows; ++j) {
                        a.cand_d[(int64_t)j * a.nq_all + row] = INFINITY;
                        a.cand_i[(int64_t)j * a.nq_all + row] = kEmptyIdx;
                    }
                    a.qub[row] = ub_of<T, DP>(list_at(ld, kq - 1));
                }
            } else {
                const float kth = (float)list_at(ld, kq - 1);
                const float band = __fmul_ru(kth, 1.f + 4.f * rel_eps<DP>());
                const bool ovf = act && li[KC - 1] != kEmptyIdx && !((float)ld[KC - 1] > band);
                if (ovf) {
                    a.fbq_list[atomicAdd(a.fbq_count, 1)] =
                        make_int4(myq, blk, __float_as_int(ub_of<T, DP>(list_at(ld, kq - 1))), 0);
                } else if (act) {
                    double rd[KC];
                    int ri[KC];
#pragma unroll
                    for (int j = 0; j < KC; ++j) {
                        rd[j] = (double)INFINITY;
                        ri[j] = kEmptyIdx;
                    }
#pragma unroll
                    for (int j = 0; j < KC; ++j) {
                        if (li[j] != kEmptyIdx && !((float)ld[j] > band)) {
                            float r[DP];
                            const float4* r4 = reinterpret_cast<const float4*>(P.rpts + (int64_t)li[j] * DP);
#pragma unroll
                            for (int u = 0; u < DP / 4; ++u) {
                                float4 v = r4[u];
                                r[4 * u] = v.x;
                                r[4 * u + 1] = v.y;
                                r[4 * u + 2] = v.z;
                                r[4 * u + 3] = v.w;
                            }
                            list_insert(rd, ri, exact_d2<DP>(q, r), P.ridx[li[j]]);
                            ++n_re;
                        }
                    }
                    int64_t base = (int64_t)P.qidx[myq] * kq;
#pragma unroll
                    for (int j = 0; j < KC; ++j)
                        if (j < kq) {
                            P.out_idx[base + j] = ri[j];
                            P.out_dist[base + j] = (float)sqrt(rd[j]);
                        }
                }
            }
        }
        __syncthreads();
    }
    // counters: one atomic per thread that holds any
    if (n_skip) atomicAdd(&a.stats[ST_SKIPPED], n_skip);
    if (n_eval) atomicAdd(&a.stats[ST_EVALUATED], n_eval);
    if (n_pp) atomicAdd(&a.stats[MODE == MODE_SEED ? ST_SEED_PAIRS : ST_POINT_PAIRS], n_pp);
    if (n_re) atomicAdd(&a.stats[ST_RERANK], n_re);
}

// Recomputation of one query whose error band overflowed its list, one CTA
// per query.  The candidate leaves are its block's seed leaves and traversal
// candidates; each is kept only if the distance from the query to the leaf's
// box (rounded down) does not exceed the query's upper bound on its k-th
// distance (the single-tree form of Algorithm 3's Score), so the work follows
// the query's own ball, not its block's.  Kept leaves gather in a shared
// buffer; when it fills, the 128 threads evaluate its points, one point each
// in turn, each keeping a candidate list, and the lists are merged.
//   EXACT = false  float32 keys (relative error <= rel_eps): the merged KC
//                  best keys give a band of possible k-th neighbours; if the
//                  band fits the list, its members are re-ranked in float64
//                  and written, else the query goes on to the exact pass.
//   EXACT = true   float64 (distance, index) keys, the result itself.
constexpr int kFbLeafBuf = 512;

template <int DP>
__device__ __forceinline__ float approx_d2(const float* q, const float* r) {
    const float4* r4 = reinterpret_cast<const float4*>(r);
    float f = 0.f;
#pragma unroll
    for (int j = 0; j < DP / 4; ++j) {
        const float4 v = r4[j];
        const float t0 = q[4 * j] - v.x, t1 = q[4 * j + 1] - v.y;
        const float t2 = q[4 * j + 2] - v.z, t3 = q[4 * j + 3] - v.w;
        f = fmaf(t0, t0, f);
        f = fmaf(t1, t1, f);
        f = fmaf(t2, t2, f);
        f = fmaf(t3, t3, f);
    }
    return f;
}

//   stage 0  one CTA per query over all of its candidate leaves (many queries)
//   stage 1  S CTAs per query, each over 1/S of the candidates, each writing
//            the KC best keys of its slice to part (few queries: the scan of
//            one query's candidates then spreads over the GPU)
//   stage 2  one CTA per query merges its S slices' lists and finishes as
//            stage 0 does
template <int DP, int KC, bool EXACT>
__global__ void __launch_bounds__(kQB) k_query_fb(const TileArgs a, int stage, int S, void* part) {
    using T = typename std::conditional<EXACT, double, float>::type;
    extern __shared__ __align__(16) unsigned char fsm[];
    T* md = reinterpret_cast<T*>(fsm);                           // KC x 128
    int32_t* mi = reinterpret_cast<int32_t*>(md + KC * kQB);     // KC x 128
    __shared__ int s_lb[kFbLeafBuf], s_pre[kFbLeafBuf + 1];
    __shared__ int s_n, s_nb;
    __shared__ float s_fd[KC];
    __shared__ int s_fi[KC];
    __shared__ double s_rd[KC];
    __shared__ int s_ri[KC];
    const int fq = stage == 1 ? blockIdx.x / S : blockIdx.x;  // the query's slot in its list
    const int sl = stage == 1 ? blockIdx.x % S : 0;           // stage 1: the CTA's slice
    T* part_d = reinterpret_cast<T*>(part);                   // [query][slice][KC]
    int32_t* part_i = reinterpret_cast<int32_t*>(part_d + (size_t)gridDim.x * (stage == 1 ? 1 : S) * KC);
    const int4 e = (EXACT ? a.fbq2_list : a.fbq_list)[fq];
    const int myq = e.x, blk = e.y;  // query (tree position in its problem), global block
    const ProbDev& P = a.probs[a.blk_prob[blk]];
    const int kq = P.k;  // read once: stores below could alias P
    const bool mono = P.mono != 0;
    const float ub = __int_as_float(e.z);
    const int tid = threadIdx.x;
    float q[DP];
    {
        const float4* q4 = reinterpret_cast<const float4*>(P.qpts + (int64_t)myq * DP);
#pragma unroll
        for (int j = 0; j < DP / 4; ++j) {
            float4 v = q4[j];
            q[4 * j] = v.x;
            q[4 * j + 1] = v.y;
            q[4 * j + 2] = v.z;
            q[4 * j + 3] = v.w;
        }
    }
    T ld[KC];
    int li[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        ld[j] = (T)INFINITY;
        li[j] = kEmptyIdx;
    }
    if (stage != 2) {
        const int nseed = seed_count(a.seed_nleaf, a.seed_slots, blk);
        const int bound = P.bound;  // read once
        const int64_t c0 = a.csr_off[blk], c1 = a.csr_off[blk + 1];
        const int64_t ntot = nseed + (c1 - c0);
        // this CTA's candidates: all of them, or slice sl of S
        const int64_t c_lo = stage == 1 ? ntot * sl / S : 0, c_hi = stage == 1 ? ntot * (sl + 1) / S : ntot;
        if (tid == 0) s_n = 0;
        __syncthreads();
        for (int64_t base = c_lo; base < c_hi; base += kQB) {
            // 1. test one candidate leaf per thread against the query's ball
            const int64_t c = base + tid;
            int leaf = -1;
            if (c < c_hi) {
                if (c < nseed) {
                    leaf = seed_leaf(a.seed_leaf0, a.seed_nleaf, a.seed_slots, blk, (int)c);
                } else if (!(a.csr_dmin[c0 + c - nseed] > ub)) {
                    leaf = a.csr_leaf[c0 + c - nseed];
                }
                if (leaf >= 0) {
                    const float* bx = P.rbox + (P.rleaf0 + leaf) * 2 * DP;
                    const float dl = bound == DTREE_BOUND_BOX
                                         ? point_box_dmin_down<DP>(q, bx)
                                         : point_dmin_down<DP>(bound, q, bx, P.rlam[P.rleaf0 + leaf]);
                    if (dl > ub) leaf = -1;
                }
            }
            if (leaf >= 0) s_lb[atomicAdd(&s_n, 1)] = leaf;
            __syncthreads();
            // 2. evaluate the buffered leaves once the next round might not fit
            const int nb = s_n;
            const bool flush = nb > 0 && (base + kQB >= c_hi || nb + kQB > kFbLeafBuf);
            __syncthreads();  // every thread has read s_n before the next round adds to it
            if (flush) {
                if (tid == 0) {
                    int acc = 0;
                    for (int i = 0; i < nb; ++i) {
                        s_pre[i] = acc;
                        acc += P.rcnt[P.rleaf0 + s_lb[i]];
                    }
                    s_pre[nb] = acc;
                }
                __syncthreads();
                const int npts = s_pre[nb];
                for (int p = tid; p < npts; p += kQB) {
                    int lo = 0, hi = nb - 1;  // the buffered leaf holding point p
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_pre[mid] <= p) lo = mid;
                        else hi = mid - 1;
                    }
                    const int r = P.rbeg[P.rleaf0 + s_lb[lo]] + (p - s_pre[lo]);
                    if (mono && r == myq) continue;
                    if constexpr (EXACT) {
                        const double d2 = exact_d2<DP>(q, P.rpts + (int64_t)r * DP);
                        const int orig = P.ridx[r];
                        if (key_less(d2, orig, ld[KC - 1], li[KC - 1])) list_insert(ld, li, d2, orig);
                    } else {
                        const float d2 = approx_d2<DP>(q, P.rpts + (int64_t)r * DP);
                        if (key_less(d2, r, ld[KC - 1], li[KC - 1])) list_insert(ld, li, d2, r);
                    }
                }
                __syncthreads();
                if (tid == 0) s_n = 0;
                __syncthreads();
            }
        }
    }
    if (stage == 2) {
        // the S slices' lists are the columns to merge (the rest are empty)
        for (int j = 0; j < KC; ++j) {
            md[j * kQB + tid] = tid < S ? part_d[((size_t)fq * S + tid) * KC + j] : (T)INFINITY;
            mi[j * kQB + tid] = tid < S ? part_i[((size_t)fq * S + tid) * KC + j] : kEmptyIdx;
        }
    } else {
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            md[j * kQB + tid] = ld[j];
            mi[j * kQB + tid] = li[j];
        }
    }
    __syncthreads();
    if (stage == 1) {
        // the slice's KC best keys (a merge of the 128 sorted thread lists)
        if (tid == 0) {
            int head[kQB];
            for (int t = 0; t < kQB; ++t) head[t] = 0;
            for (int j = 0; j < KC; ++j) {
                int best = -1;
                T bd = (T)INFINITY;
                int bi = kEmptyIdx;
                for (int t = 0; t < kQB; ++t) {
                    if (head[t] >= KC) continue;
                    const T d = md[head[t] * kQB + t];
                    const int i = mi[head[t] * kQB + t];
                    if (best < 0 || key_less(d, i, bd, bi)) {
                        best = t;
                        bd = d;
                        bi = i;
                    }
                }
                head[best]++;
                part_d[(size_t)blockIdx.x * KC + j] = bd;
                part_i[(size_t)blockIdx.x * KC + j] = bi;
            }
        }
        return;
    }
    const int64_t obase = (int64_t)P.qidx[myq] * kq;
    const int nout = EXACT ? kq : KC;
    if (tid == 0) {
        // merge the 128 sorted lists: the first nout keys overall
        int head[kQB];
        for (int t = 0; t < kQB; ++t) head[t] = 0;
        for (int j = 0; j < nout; ++j) {
            int best = -1;
            T bd = (T)INFINITY;
            int bi = kEmptyIdx;
            for (int t = 0; t < kQB; ++t) {
                if (head[t] >= KC) continue;
                const T d = md[head[t] * kQB + t];
                const int i = mi[head[t] * kQB + t];
                if (best < 0 || key_less(d, i, bd, bi)) {
                    best = t;
                    bd = d;
                    bi = i;
                }
            }
            head[best]++;
            if constexpr (EXACT) {
                P.out_idx[obase + j] = bi;
                P.out_dist[obase + j] = (float)sqrt(bd);
            } else {
                s_fd[j] = bd;
                s_fi[j] = bi;
            }
        }
        if constexpr (!EXACT) {
            // every true k-nearest neighbour has a key <= band; the band must
            // end inside the list, else the float64 pass takes the query
            const float band = __fmul_ru(s_fd[kq - 1], 1.f + 4.f * rel_eps<DP>());
            int n = 0;
            while (n < KC && s_fi[n] != kEmptyIdx && !(s_fd[n] > band)) ++n;
            if (n == KC) {
                a.fbq2_list[atomicAdd(a.fbq2_count, 1)] = e;
                n = -1;
            }
            s_nb = n;
        }
    }
    if constexpr (!EXACT) {
        __syncthreads();
        const int n = s_nb;
        if (n < 0) return;  // uniform: the float64 pass recomputes this query
        if (tid < n) {
            s_rd[tid] = exact_d2<DP>(q, P.rpts + (int64_t)s_fi[tid] * DP);
            s_ri[tid] = P.ridx[s_fi[tid]];
        }
        __syncthreads();
        if (tid == 0) {
            double rd[KC];
            int ri[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) {
                rd[j] = (double)INFINITY;
                ri[j] = kEmptyIdx;
            }
            for (int j = 0; j < n; ++j) list_insert(rd, ri, s_rd[j], s_ri[j]);
            for (int j = 0; j < kq; ++j) {
                P.out_idx[obase + j] = ri[j];
                P.out_dist[obase + j] = (float)sqrt(rd[j]);
            }
        }
        if (tid == 0) atomicAdd(&a.stats[ST_RERANK], (unsigned long long)n);
    }
}

template <int DP>
int launch_query_fb(const TileArgs& a, int kc, int nfbq, bool exact, cudaStream_t s) {
#define DT_FB_CASE(KCV)                                                                       \
    case KCV: {                                                                               \
        auto kern = exact ? k_query_fb<DP, KCV, true> : k_query_fb<DP, KCV, false>;           \
        const size_t smem = (size_t)KCV * kQB * ((exact ? 8 : 4) + 4);                      \
        DT_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                      (int)smem));                                            \
        const int S = a.fb_slices > 1 ? a.fb_slices : 1;                                       \
        if (S > 1) {                                                                          \
            DT_LAUNCH(kern, nfbq * S, kQB, smem, s, a, 1, S, a.fb_part);                      \
            DT_LAUNCH(kern, nfbq, kQB, smem, s, a, 2, S, a.fb_part);                          \
        } else {                                                                              \
            DT_LAUNCH(kern, nfbq, kQB, smem, s, a, 0, 1, a.fb_part);                          \
        }                                                                                     \
        return DTREE_OK;                                                                      \
    }
    switch (kc) {
        DT_FB_CASE(4)
        DT_FB_CASE(8)
        DT_FB_CASE(16)
        DT_FB_CASE(24)
        DT_FB_CASE(32)
        DT_FB_CASE(48)
        DT_FB_CASE(64)
        default:
            return DTREE_ERR_UNSUPPORTED;
    }
#undef DT_FB_CASE
}

template <class K>
inline int tile_grid(K kern, int items) {
    int g = occupancy_grid((const void*)kern, kQB, 0);
    return items < g ? (items > 0 ? items : 1) : g;
}

// The cap pass: a budgeted best-first search of the reference tree for every
// query, merged into the query's candidate list.  One warp serves one query
// at a time.  The list starts as the seed pass left it.  From the root the
// search walks down to a leaf, always into the child whose box is nearer
// (the left one on a tie), queueing the farther child with its box
// distance; it offers the leaf's points (itself excluded in a monochromatic
// search) to the list with their float32 keys, the seed pass's keys, then
// resumes from the nearest queued node, until it has evaluated `budget`
// leaves or no queued box is nearer than the list's k-th key.  The block's
// seed leaves are skipped (the seed pass offered their points already), and
// no leaf is reached twice, so no point enters the list twice.  The list
// goes back to cand_d / cand_i, and ub_of of its k-th key, a valid bound on
// the true k-th distance, lowers the query's qub (so B of Section 5 shrinks
// before the traversal) and caps the BaseCase's thresholds.  The BaseCase
// still evaluates every candidate leaf, these included: its insertions skip
// points already listed.
//
// Lane layout: list entry 32 s + lane in (ld[s], li[s]); queue entry `lane`
// in (pd, pn), ascending (32 entries, more than a budget can reach); box
// element e = lane + 32 t of the two children (child e / DP, coordinate
// e % DP), whose query coordinate is qd[t]; point rb + lane (+ 32 u) of a leaf.
constexpr int kCapMaxLeaves = 17;

template <int DP, int KC>
__global__ void __launch_bounds__(kQB) k_query_cap(const TileArgs a, float* qcap, int budget) {
    constexpr int NE = (KC + 31) / 32;      // list entries per lane
    constexpr int NT = (2 * DP + 31) / 32;  // box elements per lane
    const int item = blockIdx.x;
    if (item >= a.nitems) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 wi = a.items[item];
    const int blk = wi.x;
    const ProbDev& P = a.probs[a.blk_prob[blk]];
    const int64_t qnode = P.qblock0 + (blk - P.block0);
    const int nq = min(kQB, P.qcnt[qnode] - wi.y * kQB);
    const int kq = P.k, hr = P.hr;
    const bool mono = P.mono != 0;
    for (int qi = warp; qi < nq; qi += kQB / 32) {
        const int myq = P.qbeg[qnode] + wi.y * kQB + qi;
        const int64_t row = P.q0 + myq;
        const float* qp = P.qpts + (int64_t)myq * DP;
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
        float ld[NE];
        int li[NE];
#pragma unroll
        for (int s = 0; s < NE; ++s) {
            const int e = 32 * s + lane;
            ld[s] = e < KC ? a.cand_d[(int64_t)e * a.nq_all + row] : INFINITY;
            li[s] = e < KC ? a.cand_i[(int64_t)e * a.nq_all + row] : kEmptyIdx;
        }
        // list entry e (uniform e), broadcast to the warp
        auto entry_d = [&](int e) {
            float v = ld[0];
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
        float pd = INFINITY;
        int32_t pn = 0;
        int64_t n = 0;
        int lev = 0;
        float kth = entry_d(kq - 1);
        for (int used = 0;;) {
            for (; lev < hr; ++lev) {
                const int64_t l = 2 * n + 1;
                const float* bx = P.rbox + l * 2 * DP;  // the boxes of children l and l + 1
                // per child: squared distance to its box (s) and to its box
                // centre (u, for the ball bound)
                float s0 = 0.f, s1 = 0.f, u0 = 0.f, u1 = 0.f;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const int e = lane + 32 * t;
                    if (e < 2 * DP) {
                        const int c = e / DP, d = e % DP;
                        const float lo = bx[c * 2 * DP + d], hi = bx[c * 2 * DP + DP + d];
                        const float g = fmaxf(fmaxf(lo - qd[t], qd[t] - hi), 0.f);
                        const float w = qd[t] - 0.5f * (lo + hi);
                        if (c == 0) {
                            s0 = fmaf(g, g, s0);
                            u0 = fmaf(w, w, u0);
                        } else {
                            s1 = fmaf(g, g, s1);
                            u1 = fmaf(w, w, u1);
                        }
                    }
                }
                const bool ball = P.bound != DTREE_BOUND_BOX;  // uniform over the warp
                float dl, dr;
                if (2 * DP <= 32) {
                    // child c's coordinates sit in lanes [c DP, c DP + DP)
                    float sv = s0 + s1, uv = u0 + u1;
#pragma unroll
                    for (int off = DP / 2; off > 0; off >>= 1) {
                        sv += __shfl_xor_sync(0xffffffffu, sv, off);
                        if (ball) uv += __shfl_xor_sync(0xffffffffu, uv, off);
                    }
                    dl = __shfl_sync(0xffffffffu, sv, 0);
                    dr = __shfl_sync(0xffffffffu, sv, DP);
                    u0 = __shfl_sync(0xffffffffu, uv, 0);
                    u1 = __shfl_sync(0xffffffffu, uv, DP);
                } else {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                        if (ball) {
                            u0 += __shfl_xor_sync(0xffffffffu, u0, off);
                            u1 += __shfl_xor_sync(0xffffffffu, u1, off);
                        }
                    }
                    dl = s0;
                    dr = s1;
                }
                if (ball) {
                    // squared ball distances max(0, |q - C| - lambda)^2 (an
                    // order and a stopping rule only: any choice is exact)
                    const float gl = fmaxf(sqrtf(u0) - P.rlam[l], 0.f), gr = fmaxf(sqrtf(u1) - P.rlam[l + 1], 0.f);
                    const bool both = P.bound == DTREE_BOUND_BOTH;
                    dl = both ? fmaxf(dl, gl * gl) : gl * gl;
                    dr = both ? fmaxf(dr, gr * gr) : gr * gr;
                }
                const bool right = dr < dl;
                const float df = right ? dl : dr;
                if (df < kth) {
                    // sorted insertion of the farther child (the last entry drops)
                    const int32_t nf = (int32_t)(right ? l : l + 1);
                    const int pos = __popc(__ballot_sync(0xffffffffu, pd <= df));
                    const float upd = __shfl_up_sync(0xffffffffu, pd, 1);
                    const int32_t upn = __shfl_up_sync(0xffffffffu, pn, 1);
                    if (lane > pos) {
                        pd = upd;
                        pn = upn;
                    } else if (lane == pos) {
                        pd = df;
                        pn = nf;
                    }
                }
                n = right ? l + 1 : l;
            }
            if (!in_seed(a.seed_leaf0, a.seed_nleaf, a.seed_slots, blk, (int)(n - P.rleaf0))) {
                const int rb = P.rbeg[n], rc = P.rcnt[n];
                float td = entry_d(KC - 1);
                int ti = entry_i(KC - 1);
                for (int r0 = 0; r0 < rc; r0 += 32) {
                    const int r = rb + r0 + lane;
                    float d = INFINITY;
                    if (r0 + lane < rc && !(mono && r == myq)) d = approx_d2<DP>(q, P.rpts + (int64_t)r * DP);
                    uint32_t m = __ballot_sync(0xffffffffu, d < INFINITY && key_less(d, r, td, ti));
                    while (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        const float cd = __shfl_sync(0xffffffffu, d, src);
                        const int ci = __shfl_sync(0xffffffffu, r, src);
                        if (!key_less(cd, ci, td, ti)) continue;
                        // insert (cd, ci): entries from its position on move up one
                        int pos = 0;
#pragma unroll
                        for (int s = 0; s < NE; ++s)
                            pos += __popc(__ballot_sync(0xffffffffu, key_less(ld[s], li[s], cd, ci)));
#pragma unroll
                        for (int s = NE - 1; s >= 0; --s) {
                            float pv = __shfl_up_sync(0xffffffffu, ld[s], 1);
                            int pi = __shfl_up_sync(0xffffffffu, li[s], 1);
                            if (s > 0) {
                                const float cv = __shfl_sync(0xffffffffu, ld[s > 0 ? s - 1 : 0], 31);
                                const int cix = __shfl_sync(0xffffffffu, li[s > 0 ? s - 1 : 0], 31);
                                if (lane == 0) {
                                    pv = cv;
                                    pi = cix;
                                }
                            }
                            const int e = 32 * s + lane;
                            if (e < KC) {
                                if (e > pos) {
                                    ld[s] = pv;
                                    li[s] = pi;
                                } else if (e == pos) {
                                    ld[s] = cd;
                                    li[s] = ci;
                                }
                            }
                        }
                        td = entry_d(KC - 1);
                        ti = entry_i(KC - 1);
                    }
                }
            }
            kth = entry_d(kq - 1);
            const float head = __shfl_sync(0xffffffffu, pd, 0);
            if (++used >= budget || !(head < kth)) break;
            // resume from the nearest queued node
            n = __shfl_sync(0xffffffffu, pn, 0);
            lev = 63 - __clzll((long long)n + 1);
            pd = __shfl_down_sync(0xffffffffu, pd, 1);
            pn = __shfl_down_sync(0xffffffffu, pn, 1);
            if (lane == 31) pd = INFINITY;
        }
#pragma unroll
        for (int s = 0; s < NE; ++s) {
            const int e = 32 * s + lane;
            if (e < KC) {
                a.cand_d[(int64_t)e * a.nq_all + row] = ld[s];
                a.cand_i[(int64_t)e * a.nq_all + row] = li[s];
            }
        }
        if (lane == 0) {
            const float cap = ub_of<float, DP>(kth);
            qcap[row] = cap;
            a.qub[row] = fminf(a.qub[row], cap);
        }
    }
}

template <int DP>
int launch_query_cap(const TileArgs& a, int kc, int budget, float* qcap, cudaStream_t s) {
    if (a.nitems <= 0) return DTREE_OK;
    if (budget < 1 || kc != a.kc_rows) return DTREE_ERR_UNSUPPORTED;
    budget = std::min(budget, kCapMaxLeaves);
#define DT_CAP_CASE(KCV)                                                   \
    case KCV: {                                                            \
        auto kern = k_query_cap<DP, KCV>;                                  \
        DT_LAUNCH(kern, a.nitems, kQB, 0, s, a, qcap, budget);             \
        return DTREE_OK;                                                   \
    }
    switch (kc) {
        DT_CAP_CASE(4)
        DT_CAP_CASE(8)
        DT_CAP_CASE(16)
        DT_CAP_CASE(24)
        DT_CAP_CASE(32)
        DT_CAP_CASE(48)
        DT_CAP_CASE(64)
        default:
            return DTREE_ERR_UNSUPPORTED;
    }
#undef DT_CAP_CASE
}

template <int DP>
int launch_tile_cc(const TileArgs& a, int kc, int mode, int items, cudaStream_t s) {
#define DT_TILE_CASE(KCV)                                                                 \
    case KCV:                                                                             \
        if (mode == MODE_SEED) {                                                          \
            auto kern = k_tile<float, DP, KCV, MODE_SEED>;                                \
            DT_LAUNCH(kern, tile_grid(kern, items), kQB, 0, s, a);                        \
        } else if (mode == MODE_MAIN) {                                                   \
            auto kern = k_tile<float, DP, KCV, MODE_MAIN>;                                \
            DT_LAUNCH(kern, tile_grid(kern, items), kQB, 0, s, a);                        \
        }                                                                                 \
        return DTREE_OK;
    switch (kc) {
        DT_TILE_CASE(4)
        DT_TILE_CASE(8)
        DT_TILE_CASE(16)
        DT_TILE_CASE(24)
        DT_TILE_CASE(32)
        DT_TILE_CASE(48)
        DT_TILE_CASE(64)
        default:
            return DTREE_ERR_UNSUPPORTED;
    }
#undef DT_TILE_CASE
}

}  // namespace dt
