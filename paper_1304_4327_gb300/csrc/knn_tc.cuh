// knn_tc.cuh -- the kNN BaseCase (Algorithm 2) on the tensor cores.
//
// A work item is a query block of <= 128 queries (one TMEM lane and one
// thread each).  Points are centred on the block's box centre c; queries and
// staged reference points are rounded to BF16 (or TF32) into shared memory
// and tcgen05.mma forms Q R^T in TMEM with FP32 accumulation.  The epilogue
// reads each thread's TMEM lane and forms
//     s = |q~|^2 + (|r~|^2 - 2 q~.r~),
// the squared distance of the rounded, centred points, then runs the
// Algorithm 2 insertion on (s, index) exactly as the CUDA-core tile does.
//
// Exactness.  With a = |q - c|, b = |r - c|, u_p the input unit roundoff
// (2^-8 for BF16, 2^-11 for TF32) and u = 2^-24, the true distance
// D = |q - r| and the computed s satisfy
//     |D~ - D| <= e1 (a + b),            e1 = u_p + 2u,  D~ = |q~ - r~|
//     |s - D~^2| <= alpha (a^2 + b^2),   alpha = (4 K + 16) u,
// (K = MMA depth; the alpha term covers the two norms, the accumulation
// and the epilogue's two roundings).  Hence, per query with k-th key S,
//     ub = sqrt(S + alpha' (a^2 + bb^2)) + e1 (a + bb),  bb = 1.03 (a + sqrt S)
// bounds the true k-th distance (it feeds B_1, B_2 and Score), and every
// true k-nearest neighbour has s <= T = (ub + e1 (a + bu))^2 + alpha' (a^2 + bu^2),
// bu = 1.01 (a + ub).  Candidates with s <= T are re-ranked in float64; a
// list too short to hold them all sends the block to the float64 pass.
#pragma once

#include <cuda_bf16.h>

#include "knn_tile.cuh"
#include "tc_ptx.cuh"

namespace dt {

// Operand formats.  hw is the MMA's input type (1 = BF16 with .kind::f16,
// 2 = TF32 with .kind::tf32); split is how many copies of the d coordinates a
// row carries; u bounds the relative error of a centred coordinate as the
// MMA sees it; cross bounds, relative to a^2 + b^2, what the norm columns'
// hi/lo split and any dropped product add to the key.
template <int FMT>
struct TcFmt;
template <>
struct TcFmt<1> {  // BF16: 8 significant bits
    static constexpr int esize = 2, kstep = 16, hw = 1, split = 1;
    static constexpr float u = 0.00390625f;  // 2^-8
    static constexpr float cross = u * u;
};
template <>
struct TcFmt<2> {  // TF32 (round to nearest): 11 significant bits
    static constexpr int esize = 4, kstep = 8, hw = 2, split = 1;
    static constexpr float u = 0.00048828125f;  // 2^-11
    static constexpr float cross = u * u;
};
// Split BF16: a centred coordinate x is carried as hi = bf16(x) and
// lo = bf16(x - hi), so |x - (hi + lo)| <= 2^-8 |x - hi| <= 2^-16 |x|; three
// BF16 products per coordinate (hi.hi + lo.hi + hi.lo) leave out lo.lo, whose
// size in the key is at most 2 (1 + 2^-8)^2 2^-16 |q||r|.
template <>
struct TcFmt<3> {
    static constexpr int esize = 2, kstep = 16, hw = 1, split = 3;
    static constexpr float u = 1.5411377e-05f;   // 2^-16 (1 + 2^-8)
    // 2^-16 (norm split) + 1.01 x 2^-16 (lo.lo, as 2 |q||r| <= a^2 + b^2): 3.1e-5, rounded up
    static constexpr float cross = 4.6e-05f;
};

// Operand rows carry the centred coordinates plus two augmented columns:
//   BF16 / TF32 (split 1)
//     A row (query):     -2 q~_1 .. -2 q~_d, 1, 1
//     B row (reference):    r~_1 ..    r~_d, hi(|r~|^2), lo(|r~|^2)
//   split BF16 (split 3), with q^ = q_hi + q_lo and r^ likewise
//     A row: -2 q_hi, -2 q_lo, -2 q_hi, 1, 1
//     B row:    r_hi,    r_hi,    r_lo, hi(|r^|^2), lo(|r^|^2)
// so the accumulator holds w = |r~|^2 - 2 q~.r~ directly (hi + lo carries the
// float32 norm to about twice the input precision); K is padded to the MMA step.
template <int FMT, int DP>
struct TcShape {
    static constexpr int KD = DP * TcFmt<FMT>::split;  // coordinate columns
    static constexpr int KP = (KD + 2 + TcFmt<FMT>::kstep - 1) / TcFmt<FMT>::kstep * TcFmt<FMT>::kstep;
    static constexpr int RB = KP * TcFmt<FMT>::esize;  // bytes per operand row
    static constexpr int NCH = RB / 16;                // 16-byte chunks per row
    static constexpr int SBO = NCH * 128;
    // reference points per tile: 256 (the MMA's widest N) where the operand
    // slots fit shared memory, so per-tile hand-overs are paid per 256 points
    static constexpr int TN = DP <= 16 ? 256 : 128;
    // TMEM accumulators: one per epilogue group (2 x TN <= 512 columns)
    static constexpr int NS = 2;
    // operand slots in shared memory: the converters fill ahead of the groups
    // (each group issues its own MMAs from them)
    static constexpr int NB = RB >= 160 ? 2 : (TN == 256 ? 3 : 4);
    static constexpr int NK = KP / TcFmt<FMT>::kstep;  // MMAs per tile
    static constexpr int SORTCAP = (DP >= 64 || TN == 256) ? 512 : 1024;  // candidates per window
    static constexpr int CB = (DP >= 32 || TN == 256) ? 8 : 16;           // deferred insertions per thread
    static constexpr int RAWB = TN * DP * 4;                     // raw float32 rows of a stage
    static constexpr int RINGB = (DP >= 32 || RB >= 128) ? 32768 : 65536;  // raw ring budget
    static constexpr int NR = RINGB / RAWB > 8 ? 8 : (RINGB / RAWB < 2 ? 2 : RINGB / RAWB);
};

// Shared memory of the pipelined kernel (bytes), lists of KC entries.
template <int FMT, int DP, int KC>
struct TcSmem {
    using S = TcShape<FMT, DP>;
    static constexpr int MERGE = kQB * KC * 8;                       // lists / re-rank at block end
    static constexpr int RING = S::NR * S::RAWB;
    static constexpr int OFF_A = 0;                                  // 128 x RB
    static constexpr int OFF_B = OFF_A + kQB * S::RB;                // NB x TN x RB
    static constexpr int OFF_RAW = OFF_B + S::NB * S::TN * S::RB;    // NR x TN x DP float (or merge)
    static constexpr int OFF_POS = OFF_RAW + (RING > MERGE ? RING : MERGE);  // (NB + NS) x TN int
    static constexpr int OFF_RPOS = OFF_POS + (S::NB + S::NS) * S::TN * 4;  // NR x TN int
    static constexpr int OFF_KEY = OFF_RPOS + S::NR * S::TN * 4;     // SORTCAP uint64
    static constexpr int OFF_ROW = OFF_KEY + S::SORTCAP * 8;         // SORTCAP int4
    static constexpr int OFF_SCR = OFF_ROW + S::SORTCAP * 16;        // 2 x 32 x 128 float
    static constexpr int OFF_BUF = OFF_SCR + 2 * 32 * kQB * 4;       // 2 x CB x 128 (float, int)
    static constexpr int OFF_CEN = OFF_BUF + 2 * S::CB * kQB * 8;    // DP float
    static constexpr int BYTES = OFF_CEN + DP * 4;
    static_assert(BYTES <= 225 * 1024, "tensor-core tile shared memory over budget");
};

template <int FMT, int DP>
struct TcBound {
    static constexpr float u = 5.9604645e-08f;
    static constexpr float e1 = TcFmt<FMT>::u + 2.f * u;
    // accumulation over K terms, the norms and the epilogue add, plus the
    // hi/lo split of |r~|^2 (relative residual u_p^2)
    static constexpr float alpha =
        ((4.f * TcShape<FMT, DP>::KP + 16.f) * u + TcFmt<FMT>::cross) * 1.01f;
    // upper bound on the true k-th distance of a query with k-th key S
    __device__ static float ub(float S, float a) {
        if (!(S < INFINITY)) return INFINITY;
        float sq = __fsqrt_ru(fmaxf(S, 0.f));
        float bb = __fmul_ru(1.03f, __fadd_ru(a, sq));
        float n2 = __fmaf_ru(a, a, __fmul_ru(bb, bb));
        float r = __fsqrt_ru(__fmaf_ru(alpha, n2, S));
        return __fmaf_ru(e1, __fadd_ru(a, bb), r);
    }
    // band: every true k-nearest neighbour has a key <= band(ub, a)
    __device__ static float band(float ubk, float a) {
        if (!(ubk < INFINITY)) return INFINITY;
        float bu = __fmul_ru(1.01f, __fadd_ru(a, ubk));
        float x = __fmaf_ru(e1, __fadd_ru(a, bu), ubk);
        float n2 = __fmaf_ru(a, a, __fmul_ru(bu, bu));
        return __fmaf_ru(alpha, n2, __fmul_ru(x, x));
    }
};

// A centred coordinate rounded to the operand type.
template <int FMT>
__device__ __forceinline__ float tc_round(float h) {
    return TcFmt<FMT>::hw == 2 ? tc::to_tf32(h) : __bfloat162float(__float2bfloat16_rn(h));
}

// Rounds the centred coordinates h[0..DP): xh gets x~ (split 1) or hi (split
// 3), xl gets lo (split 3); returns the sum of squares of the represented
// values (x~ or hi + lo, both exact in float32).
template <int FMT, int DP>
__device__ __forceinline__ float tc_round_row(const float* h, float* xh, float* xl) {
    float n = 0.f;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        const float hi = tc_round<FMT>(h[j]);
        float r = hi;
        if (TcFmt<FMT>::split == 3) {
            const float lo = tc_round<FMT>(h[j] - hi);
            xl[j] = lo;
            r = hi + lo;
        }
        xh[j] = hi;
        n = fmaf(r, r, n);
    }
    return n;
}

// Element e of an operand row (A: query, scaled by -2 and ending 1, 1;
// B: reference, ending with the norm's hi and lo), laid out as above.
template <int FMT, int DP, bool AROW>
__device__ __forceinline__ float tc_row_elem(int e, const float* xh, const float* xl, float nhi,
                                             float nlo) {
    const float sc = AROW ? -2.f : 1.f;
    if (TcFmt<FMT>::split == 3) {
        if (e < DP) return sc * xh[e];
        if (e < 2 * DP) return sc * (AROW ? xl[e - DP] : xh[e - DP]);
        if (e < 3 * DP) return sc * (AROW ? xh[e - 2 * DP] : xl[e - 2 * DP]);
        e -= 2 * DP;
    } else if (e < DP) {
        return sc * xh[e];
    }
    if (e == DP) return AROW ? 1.f : nhi;
    if (e == DP + 1) return AROW ? 1.f : nlo;
    return 0.f;
}

// The 16 bytes of chunk c of an operand row.
template <int FMT, int DP, bool AROW>
__device__ __forceinline__ uint4 tc_row_chunk(int c, const float* xh, const float* xl, float nhi,
                                              float nlo) {
    uint4 w;
    uint32_t* p = reinterpret_cast<uint32_t*>(&w);
    if (TcFmt<FMT>::esize == 2) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 b = __floats2bfloat162_rn(
                tc_row_elem<FMT, DP, AROW>(8 * c + 2 * i, xh, xl, nhi, nlo),
                tc_row_elem<FMT, DP, AROW>(8 * c + 2 * i + 1, xh, xl, nhi, nlo));
            p[i] = *reinterpret_cast<uint32_t*>(&b);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            p[i] = __float_as_uint(tc_row_elem<FMT, DP, AROW>(4 * c + i, xh, xl, nhi, nlo));
    }
    return w;
}

struct TcExtra {
    int* err;          // device status word: 1 = a bounded wait gave up
    int spin_budget;
    unsigned long long* timers;  // optional per-role cycle counters (diagnostics), or null
};

// Diagnostic cycle counters of the pipelined kernel (summed over CTAs).
enum TcTimer {
    TT_PLAN_WINDOW = 0,  // planner: loading and sorting candidate windows
    TT_PLAN_WAIT,        // planner: waiting for a free raw stage
    TT_PLAN_STAGE,       // planner: filling stages and issuing copies
    TT_CONV_WAIT_RAW,    // converters: waiting for copied rows
    TT_CONV_WAIT_SLOT,   // converters: waiting for a free operand slot
    TT_CONV_WORK,        // converters: conversion + MMA issue
    TT_EPI_WAIT,         // epilogue (warp 0): waiting for an accumulator
    TT_EPI_WORK,         // epilogue (warp 0): reading TMEM, keys, insertion
    TT_EPI_RARE,         // epilogue (all threads): chunks that took the insertion path
    TT_EPI_FINISH,       // epilogue group 0: merge, re-rank, output
    TT_ITEM_SETUP,       // all: query load, list init
    TT_EPI_TMEM,         // epilogue (warp 0): TMEM load + wait
    TT_EPI_HOT,          // epilogue (warp 0): minimum over the columns
    TT_EPI_RAREC,        // epilogue (warp 0): rare path cycles
    TT_EPI_TAIL,         // epilogue (warp 0): bound update after a tile
    TT_EPI_FLUSH,        // epilogue (warp 0): the end-of-tile insertion of buffered candidates
    TT_TILES,            // converters: tiles produced
    TT_ITEMS,            // items processed
    TT_INSERTS,          // epilogue (all threads): candidate-list insertions
    TT_EPI_WAIT_OP,      // epilogue (warp 0): of TT_EPI_WAIT, waiting for the operand slot
    TT_EPI_WAIT_BAR,     // epilogue (warp 0): of TT_EPI_WAIT, the group barrier before the MMA
    TT_N
};
static_assert(TT_N <= 32, "the diagnostic timer buffer holds 32 counters");

// Named barriers of the pipelined kernel (0 is __syncthreads).
enum { BAR_EPI = 1, BAR_CONV = 2, BAR_G0 = 3, BAR_G1 = 4 };

// The planner warp: read the window's candidates (row range and d_min) into
// shared memory, in list order (a block's list is sorted nearest-first).
template <int NC, int MODE>
__device__ __forceinline__ void load_window(const TileArgs& a, const ProbDev& P, int64_t w0,
                                            int wn, int nseed, int blk, int64_t c0,
                                            uint64_t* skey, int4* srow) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < wn; i += 32) {
        const int64_t ci = w0 + i;
        int leaf;
        float dmin = 0.f;
        if (ci < nseed) {
            leaf = seed_leaf(a.seed_leaf0, a.seed_nleaf, a.seed_slots, blk, (int)ci);
        } else {
            leaf = a.csr_leaf[c0 + ci - nseed];
            dmin = a.csr_dmin[c0 + ci - nseed];
        }
        const int64_t ln = P.rleaf0 + leaf;
        srow[i] = make_int4(P.rbeg[ln], P.rcnt[ln], __float_as_int(dmin), 0);
        skey[i] = (uint64_t)i;
    }
    __syncwarp();
}

// One CTA per SM, 12 warps:
//   warps 0-3  epilogue group 0: query rows 0..127 (TMEM lanes), slot uses 0, 2, 4, ...
//   warps 4-7  epilogue group 1: the same rows, slot uses 1, 3, 5, ...
//   warp  8    planner: walks the block's candidate leaves nearest-first,
//              skips those whose d_min exceeds the block's bound (Algorithm 3)
//              and bulk-copies the rows of the rest (TMA) into a ring of NR
//              raw stages;
//   warps 9-11 converters: centre and round a raw stage into one of NS operand
//              slots; one thread issues the MMAs into that slot's TMEM
//              accumulator.
// Hand-over by mbarriers: raw_full/raw_empty (planner <-> converters, with the
// copies' byte count), full/empty (converters <-> epilogue groups).  Each
// epilogue group keeps its own candidate list per query; the two are merged
// when the block is done.  Every mbarrier wait is bounded, and a group decides
// a failed wait together before its next named barrier.
template <int FMT, int DP, int KC, int MODE>
__global__ void __launch_bounds__(384, 1) k_tile_tc(const TileArgs a, const TcExtra x) {
    using S = TcShape<FMT, DP>;
    using L = TcSmem<FMT, DP, KC>;
    using Bd = TcBound<FMT, DP>;
    constexpr int TN = S::TN, NS = S::NS, NB = S::NB, NR = S::NR;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem + L::OFF_A;
    unsigned char* sB = smem + L::OFF_B;
    float* sraw = reinterpret_cast<float*>(smem + L::OFF_RAW);
    int32_t* spos = reinterpret_cast<int32_t*>(smem + L::OFF_POS);
    int32_t* srpos = reinterpret_cast<int32_t*>(smem + L::OFF_RPOS);
    uint64_t* skey = reinterpret_cast<uint64_t*>(smem + L::OFF_KEY);
    int4* srow = reinterpret_cast<int4*>(smem + L::OFF_ROW);
    float* sscr = reinterpret_cast<float*>(smem + L::OFF_SCR);
    float* sbuf = reinterpret_cast<float*>(smem + L::OFF_BUF);
    float* scen = reinterpret_cast<float*>(smem + L::OFF_CEN);
    __shared__ uint64_t acc_full[NS], raw_full[NR], raw_empty[NR], op_full[NB], op_empty[NB];
    __shared__ int ometa[NB], srmeta[NR];
    __shared__ volatile int s_gfail[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_item;
    __shared__ ProbDev s_prob;
    __shared__ volatile int s_fail, s_cmeta, s_cok;
    __shared__ volatile float s_wmax[8], s_wmin[8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int role = warp < 4 ? 0 : warp < 8 ? 1 : warp == 8 ? 2 : 3;
    const int qt = tid & 127;  // query row of an epilogue thread
    const int nitems = a.nitems;
    unsigned long long n_skip = 0, n_eval = 0, n_pp = 0, n_re = 0, n_ins = 0;

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) tc::mbar_init(&acc_full[i], 1);  // tcgen05.commit
        for (int i = 0; i < NR; ++i) {
            tc::mbar_init(&raw_full[i], 1);   // the planner's arrival (+ copied bytes)
            tc::mbar_init(&raw_empty[i], 1);  // the converters' release
        }
        for (int i = 0; i < NB; ++i) {
            tc::mbar_init(&op_full[i], 1);   // the converters' release
            tc::mbar_init(&op_empty[i], 2);  // tcgen05.commit + the consuming group's release
        }
        s_gfail[0] = 0;
        s_gfail[1] = 0;
        tc::fence_mbar_init();
        s_fail = 0;
    }
    if (warp == 8) tc::tmem_alloc(&s_tmem, TN * NS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc::idesc(TcFmt<FMT>::hw, kQB, TN);
    uint32_t rtile = 0;     // planner / converters: next raw stage
    uint32_t otile = 0;     // converters: next operand slot use (the barriers' phases
                            // carry over from item to item, so the counters do too)
    uint32_t ctile = role;  // epilogue group: next operand slot use of this group
    uint32_t acnt = 0;      // epilogue group: MMAs issued into its accumulator
    bool pend = false;      // epilogue group leader: an MMA whose completion was not seen

    const ProbDev& P = s_prob;
    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(a.work_ctr, 1);
            if (s_item < nitems) s_prob = a.probs[a.blk_prob[a.items[s_item].x]];
        }
        __syncthreads();
        const int item = s_item;
        if (item >= nitems || s_fail) break;
        const int2 wi = a.items[item];
        const int blk = wi.x, chunk = wi.y;  // global block, chunk of its queries
        const int64_t qnode = P.qblock0 + (blk - P.block0);
        const int nq = min(kQB, P.qcnt[qnode] - chunk * kQB);
        if (nq <= 0) {
            __syncthreads();
            continue;
        }
        long long tm0 = clock64();
        const float* bx = P.qbox + qnode * 2 * DP;
        if (tid < DP) scen[tid] = 0.5f * (bx[tid] + bx[DP + tid]);
        __syncthreads();
        const bool act = role < 2 && qt < nq;
        const int myq = P.qbeg[qnode] + chunk * kQB + qt;
        const int kq = P.k;  // read once: stores below could alias P
        const bool mono = P.mono != 0;
        const float lam2 = 2.f * P.qlam[qnode];
        float qa = 0.f, qn = 0.f;
        // the cap pass's bound on the query's k-th distance (main pass only)
        const float qc = MODE == MODE_MAIN && act && a.qcap ? a.qcap[P.q0 + myq] : INFINITY;
        float ld[KC];
        int li[KC];
        if (role < 2) {
            // the query, centred and rounded (group 0 writes row qt of the A tile)
            float qa2 = 0.f;
            float h[DP], xh[DP], xl[DP];
            const float4* q4 = reinterpret_cast<const float4*>(P.qpts + (int64_t)myq * DP);
#pragma unroll
            for (int j = 0; j < DP / 4; ++j) {
                float4 v = act ? q4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                h[4 * j] = v.x;
                h[4 * j + 1] = v.y;
                h[4 * j + 2] = v.z;
                h[4 * j + 3] = v.w;
            }
#pragma unroll
            for (int j = 0; j < DP; ++j) {
                h[j] = act ? h[j] - scen[j] : 0.f;
                qa2 = __fmaf_ru(h[j], h[j], qa2);
            }
            qn = tc_round_row<FMT, DP>(h, xh, xl);
            if (role == 0) {
#pragma unroll
                for (int c = 0; c < S::NCH; ++c)
                    *reinterpret_cast<uint4*>(sA + tc::core_offset(qt, c, S::SBO)) =
                        tc_row_chunk<FMT, DP, true>(c, xh, xl, 1.f, 1.f);
            }
            qa = __fsqrt_ru(qa2);
#pragma unroll
            for (int j = 0; j < KC; ++j) {
                ld[j] = INFINITY;
                li[j] = kEmptyIdx;
                if (MODE == MODE_MAIN && act) {
                    ld[j] = a.cand_d[(int64_t)j * a.nq_all + (P.q0 + myq)];
                    li[j] = a.cand_i[(int64_t)j * a.nq_all + (P.q0 + myq)];
                }
            }
            float ub = fminf(Bd::ub(list_at(ld, kq - 1), qa), qc);
            float vmax = act ? ub : -INFINITY, vmin = act ? ub : INFINITY;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
                vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
            }
            if (lane == 0) {
                s_wmax[warp] = vmax;
                s_wmin[warp] = vmin;
            }
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (x.timers && tid == 0) {
            atomicAdd(&x.timers[TT_ITEM_SETUP], (unsigned long long)(clock64() - tm0));
            atomicAdd(&x.timers[TT_ITEMS], 1ull);
        }

        if (role == 2) {
            // ================= planner (warp 8) =================
            const float Bq = a.Bn ? a.Bn[P.node0 + qnode] : INFINITY;
            const int nseed = MODE == MODE_MAIN ? 0 : seed_count(a.seed_nleaf, a.seed_slots, blk);
            const int64_t c0 = MODE == MODE_SEED ? 0 : a.csr_off[blk];
            const int64_t c1 = MODE == MODE_SEED ? 0 : a.csr_off[blk + 1];
            const int64_t ntot = nseed + (c1 - c0);
            bool fail = false;
            for (int64_t w0 = 0; w0 < ntot && !fail; w0 += S::SORTCAP) {
                const int wn = (int)(ntot - w0 < S::SORTCAP ? ntot - w0 : S::SORTCAP);
                long long t0 = clock64();
                load_window<S::SORTCAP, MODE>(a, P, w0, wn, nseed, blk, c0, skey, srow);
                if (x.timers && lane == 0)
                    atomicAdd(&x.timers[TT_PLAN_WINDOW], (unsigned long long)(clock64() - t0));
                int cur = 0, part = 0;
                bool have_slot = false;
                int r = 0;
                while (cur < wn) {
                    if (!have_slot) {
                        r = rtile % NR;
                        const uint32_t use = rtile / NR;
                        long long t1 = clock64();
                        bool ok = lane == 0 ? tc::mbar_wait(&raw_empty[r], (use & 1u) ^ 1u, x.spin_budget) : true;
                        if (!__all_sync(0xffffffffu, ok)) {
                            fail = true;
                            break;
                        }
                        if (x.timers && lane == 0)
                            atomicAdd(&x.timers[TT_PLAN_WAIT], (unsigned long long)(clock64() - t1));
                        have_slot = true;
                    }
                    long long t2 = clock64();
                    // the block's bound from both epilogue groups' published values
                    float b = Bq;
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        float mx = -INFINITY, mn = INFINITY;
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            mx = fmaxf(mx, s_wmax[4 * g + w]);
                            mn = fminf(mn, s_wmin[4 * g + w]);
                        }
                        b = fminf(b, fminf(mx, __fadd_ru(mn, lam2)));
                    }
                    float* raw = sraw + r * TN * DP;
                    int32_t* rpos = srpos + r * TN;
                    int nst = 0;
                    // rounds of 32 candidates until the stage is full or the window ends
                    while (cur < wn && nst < TN) {
                        const int c = cur + lane;
                        const bool valid = c < wn;
                        int lb = 0, lc = 0;
                        bool keep = false;
                        if (valid) {
                            const int4 rr = srow[(uint32_t)skey[c]];
                            keep = !(__int_as_float(rr.z) > b);
                            if (keep) {
                                lb = rr.x;
                                lc = rr.y;
                            }
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
                        const int excl = incl - lc;
                        const int take = min(max(TN - nst - excl, 0), lc);
                        const bool fullc = valid && take == lc;
                        const unsigned fm = __ballot_sync(0xffffffffu, fullc);
                        const int nlead = fm == 0xffffffffu ? 32 : __ffs(~fm) - 1;
                        const bool put = take > 0 && lane <= nlead;
                        const unsigned sk = __ballot_sync(0xffffffffu, valid && !keep && lane < nlead);
                        const unsigned ev = __ballot_sync(0xffffffffu, keep && lane < nlead);
                        int taken = put ? take : 0;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) taken += __shfl_xor_sync(0xffffffffu, taken, off);
                        if (lane == 0) {
                            n_skip += __popc(sk);
                            n_eval += __popc(ev);
                            if (taken) tc::mbar_expect_tx(&raw_full[r], (uint32_t)taken * DP * 4);
                        }
                        __syncwarp();
                        if (put) {
                            tc::bulk_g2s(raw + (nst + excl) * DP, P.rpts + (int64_t)lb * DP,
                                         (uint32_t)take * DP * 4, &raw_full[r]);
                            for (int i = 0; i < take; ++i) rpos[nst + excl + i] = lb + i;
                        }
                        nst += taken;
                        const int pn = __shfl_sync(0xffffffffu, take, nlead & 31);
                        if (nlead < 32) {
                            part = (nlead == 0 ? part : 0) + pn;
                            cur += nlead;
                            if (!(cur < wn)) part = 0;
                            break;
                        }
                        cur += 32;
                        part = 0;
                    }
                    if (nst > 0) {
                        if (lane == 0) srmeta[r] = nst;
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&raw_full[r], 1);
                        ++rtile;
                        have_slot = false;
                    }
                    if (x.timers && lane == 0)
                        atomicAdd(&x.timers[TT_PLAN_STAGE], (unsigned long long)(clock64() - t2));
                }
                if (fail) break;
            }
            // end of the block for the converters
            {
                const int r = rtile % NR;
                const uint32_t use = rtile / NR;
                bool ok = lane == 0 ? tc::mbar_wait(&raw_empty[r], (use & 1u) ^ 1u, x.spin_budget) : true;
                ok = __all_sync(0xffffffffu, ok);
                if (fail || !ok) {
                    if (lane == 0) s_fail = 1;
                } else {
                    if (lane == 0) {
                        srmeta[r] = -1;
                        tc::mbar_arrive(&raw_full[r], 1);
                    }
                    ++rtile;
                }
            }
        } else if (role == 3) {
            // ================= converters (warps 9-11) =================
            const int ctid = tid - 288;
            int32_t* opos_all = spos;  // NB x TN: the operand slots' column positions
            for (;;) {
                const int r = rtile % NR;
                const uint32_t ruse = rtile / NR;
                const int op = otile % NB;
                const uint32_t ouse = otile / NB;
                long long tc0 = clock64();
                if (ctid == 0) {
                    int m = -2;
                    if (tc::mbar_wait(&raw_full[r], ruse & 1u, x.spin_budget)) {
                        long long tc1 = clock64();
                        if (x.timers) atomicAdd(&x.timers[TT_CONV_WAIT_RAW], (unsigned long long)(tc1 - tc0));
                        m = srmeta[r];
                        // the operand slot is free once its MMA has read it and its
                        // group has copied its column positions
                        if (m >= 0 && !tc::mbar_wait(&op_empty[op], (ouse & 1u) ^ 1u, x.spin_budget))
                            m = -2;
                        if (x.timers) atomicAdd(&x.timers[TT_CONV_WAIT_SLOT], (unsigned long long)(clock64() - tc1));
                    }
                    s_cmeta = m;
                }
                tc::named_sync(BAR_CONV, 96);
                const int m = s_cmeta;
                if (m == -2) {
                    if (ctid == 0) s_fail = 1;
                    break;
                }
                if (m == -1) {
                    // release the stage, then one end marker for each epilogue group
                    // (tiles alternate between the groups)
                    if (ctid == 0) {
                        tc::mbar_arrive(&raw_empty[r], 1);
                        for (int e = 0; e < 2; ++e) {
                            const int sl = (otile + e) % NB;
                            const uint32_t su = (otile + e) / NB;
                            // (on a timeout the groups' own bounded waits end them)
                            if (!tc::mbar_wait(&op_empty[sl], (su & 1u) ^ 1u, x.spin_budget)) s_fail = 1;
                            ometa[sl] = -1;
                            tc::mbar_arrive(&op_full[sl], 1);
                        }
                    }
                    ++rtile;
                    otile += 2;
                    break;
                }
                // every converter thread observes the stage's completion itself
                // (acquire of the bulk-copied rows); it completed already
                tc::mbar_try_wait(&raw_full[r], ruse & 1u);
                long long tc2 = clock64();
                // centre and round the stage's rows into the operand slot
                const float* raw = sraw + r * TN * DP;
                const int32_t* rpos = srpos + r * TN;
                unsigned char* sBs = sB + op * TN * S::RB;
                int32_t* opos = opos_all + op * TN;
                for (int row = ctid; row < TN; row += 96) {
                    if (row < m) {
                        const float4* r4 = reinterpret_cast<const float4*>(raw + row * DP);
                        float h[DP], xh[DP], xl[DP];
#pragma unroll
                        for (int j4 = 0; j4 < DP / 4; ++j4) {
                            float4 v = r4[j4];
                            h[4 * j4] = v.x - scen[4 * j4];
                            h[4 * j4 + 1] = v.y - scen[4 * j4 + 1];
                            h[4 * j4 + 2] = v.z - scen[4 * j4 + 2];
                            h[4 * j4 + 3] = v.w - scen[4 * j4 + 3];
                        }
                        const float rn = tc_round_row<FMT, DP>(h, xh, xl);
                        const float nhi = tc_round<FMT>(rn);
                        const float nlo = tc_round<FMT>(rn - nhi);
#pragma unroll
                        for (int c = 0; c < S::NCH; ++c)
                            *reinterpret_cast<uint4*>(sBs + tc::core_offset(row, c, S::SBO)) =
                                tc_row_chunk<FMT, DP, false>(c, xh, xl, nhi, nlo);
                        opos[row] = rpos[row];
                    } else {
                        // an empty column: w = +inf never qualifies
#pragma unroll
                        for (int c = 0; c < S::NCH; ++c) {
                            uint4 w = make_uint4(0u, 0u, 0u, 0u);
                            const int el = (S::KD * TcFmt<FMT>::esize) / 16 == c ? S::KD % (16 / TcFmt<FMT>::esize) : -1;
                            if (el >= 0) {
                                // place +inf in the hi(|r~|^2) element of this chunk
                                if (TcFmt<FMT>::esize == 2) {
                                    uint32_t inf16 = 0x7f80u;
                                    uint32_t* wp = reinterpret_cast<uint32_t*>(&w);
                                    wp[el >> 1] = (el & 1) ? (inf16 << 16) : inf16;
                                } else {
                                    uint32_t* wp = reinterpret_cast<uint32_t*>(&w);
                                    wp[el] = 0x7f800000u;
                                }
                            }
                            *reinterpret_cast<uint4*>(sBs + tc::core_offset(row, c, S::SBO)) = w;
                        }
                        opos[row] = kEmptyIdx;
                    }
                }
                tc::fence_proxy_async_smem();
                tc::named_sync(BAR_CONV, 96);
                if (ctid == 0) {
                    tc::mbar_arrive(&raw_empty[r], 1);
                    ometa[op] = m;
                    n_pp += (unsigned long long)m * nq;
                    tc::mbar_arrive(&op_full[op], 1);
                    if (x.timers) {
                        atomicAdd(&x.timers[TT_CONV_WORK], (unsigned long long)(clock64() - tc2));
                        atomicAdd(&x.timers[TT_TILES], 1ull);
                    }
                }
                ++rtile;
                ++otile;
            }
        } else {
            // ================= epilogue group `role` =================
            const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
            const int slot = role;  // this group's accumulator
            const int gbar = role == 0 ? BAR_G0 : BAR_G1;
            int32_t* sposs = spos + (NB + slot) * TN;  // its column positions
            for (;;) {
                // this group's next tile: operand slot op (or an end marker)
                const int op = ctile % NB;
                const uint32_t ouse = ctile / NB;
                long long te0 = clock64();
                bool ok = tc::mbar_wait(&op_full[op], ouse & 1u, x.spin_budget);
                if (!__all_sync(0xffffffffu, ok) && lane == 0) s_gfail[role] = 1;
                const int nst = ok ? ometa[op] : -1;
                long long tw1 = clock64();
                // every warp of the group is done with the last tile (its TMEM
                // reads and its column positions) before either is replaced
                tc::fence_before_sync();
                tc::named_sync(gbar, 128);
                tc::fence_after_sync();
                if (x.timers && (warp & 3) == 0 && lane == 0) {
                    const long long tw2 = clock64();
                    atomicAdd(&x.timers[TT_EPI_WAIT_OP], (unsigned long long)(tw1 - te0));
                    atomicAdd(&x.timers[TT_EPI_WAIT_BAR], (unsigned long long)(tw2 - tw1));
                }
                if (s_gfail[role]) {
                    s_fail = 1;
                    break;
                }
                if (qt == 0) {
                    if (nst >= 0) {
                        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB + op * TN * S::RB);
#pragma unroll
                        for (int kk = 0; kk < S::NK; ++kk)
                            tc::mma<TcFmt<FMT>::hw>(tmem + (uint32_t)(slot * TN),
                                                    tc::sdesc(a0 + 256u * kk, 128u, S::SBO),
                                                    tc::sdesc(b0 + 256u * kk, 128u, S::SBO), idesc,
                                                    kk > 0 ? 1u : 0u);
                        tc::mma_commit(&acc_full[slot]);
                        tc::mma_commit(&op_empty[op]);
                        pend = true;
                    } else {
                        tc::mbar_arrive(&op_empty[op], 2);  // an end marker: nothing reads the slot
                    }
                }
                ctile += 2;
                if (nst < 0) break;
                // the operand's column positions move to the accumulator's, so the
                // operand slot can be refilled while this group works
                for (int i = qt; i < TN; i += kQB) sposs[i] = spos[op * TN + i];
                // the accumulator of this tile
                ok = tc::mbar_wait(&acc_full[slot], acnt & 1u, x.spin_budget);
                ++acnt;
                if (!__all_sync(0xffffffffu, ok) && lane == 0) s_gfail[role] = 1;
                tc::named_sync(gbar, 128);  // also: every position is copied
                if (s_gfail[role]) {
                    s_fail = 1;
                    break;
                }
                if (qt == 0) {
                    pend = false;
                    tc::mbar_arrive(&op_empty[op], 1);  // the slot's positions are copied
                }
                long long te1 = clock64();
                if (x.timers && (warp & 3) == 0 && lane == 0)
                    atomicAdd(&x.timers[TT_EPI_WAIT], (unsigned long long)(te1 - te0));
                tc::fence_after_sync();
                bool changed = false;
                {
                    float* scr = sscr + role * 32 * kQB + qt;
                    // insertion threshold in w units: below the list's last key and
                    // inside the error band of the current k-th key (a key above
                    // the band can never be a true k-nearest neighbour)
                    auto threshold = [&]() {
                        const float bnd = Bd::band(fminf(Bd::ub(list_at(ld, kq - 1), qa), qc), qa);
                        return __fsub_ru(fminf(ld[KC - 1], bnd), qn);
                    };
                    float t = threshold();
                    // 64 columns per TMEM read: w = |r~|^2 - 2 q~.r~ straight from the accumulator
                    // candidates under the threshold are buffered per thread and
                    // inserted together by the whole warp at the end of the tile
                    float* bw = sbuf + role * S::CB * kQB + qt;
                    int32_t* bi = reinterpret_cast<int32_t*>(sbuf + 2 * S::CB * kQB) + role * S::CB * kQB + qt;
                    int nb = 0;
                    auto flush = [&]() {
                        for (int e = 0; e < nb; ++e) {
                            const float sv = qn + bw[e * kQB];
                            const int rp = bi[e * kQB];
                            // (the cap pass may have listed this point already)
                            if (key_less(sv, rp, ld[KC - 1], li[KC - 1]) && !(mono && rp == myq) &&
                                !(MODE == MODE_MAIN && listed(li, rp))) {
                                // the band moves only when the k-th key does
                                const bool kth_moves = key_less(sv, rp, list_at(ld, kq - 1),
                                                                list_at(li, kq - 1));
                                list_insert_par(ld, li, sv, rp);
                                t = kth_moves ? threshold() : fminf(t, __fsub_ru(ld[KC - 1], qn));
                                changed = true;
                                ++n_ins;
                            }
                        }
                        nb = 0;
                    };
                    const int nch = (nst + 63) >> 6;
                    const uint32_t tcol = tl + (uint32_t)(slot * TN);
                    for (int cc = 0; cc < nch; ++cc) {
                        uint32_t v[64];
                        long long tt0 = clock64();
                        tc::tmem_ld64(tcol + (uint32_t)(cc * 64), v);
                        tc::tmem_ld_wait_dep64(v);
                        if (x.timers && (warp & 3) == 0 && lane == 0)
                            atomicAdd(&x.timers[TT_EPI_TMEM], (unsigned long long)(clock64() - tt0));
                        long long th0 = clock64();
                        if (!act) continue;
                        // hot path: the minimum over the 64 columns, branch-free
                        float m16[16];
#pragma unroll
                        for (int i4 = 0; i4 < 16; ++i4)
                            m16[i4] = fminf(fminf(__uint_as_float(v[4 * i4]), __uint_as_float(v[4 * i4 + 1])),
                                            fminf(__uint_as_float(v[4 * i4 + 2]), __uint_as_float(v[4 * i4 + 3])));
#pragma unroll
                        for (int h = 8; h > 0; h >>= 1)
#pragma unroll
                            for (int i = 0; i < h; ++i) m16[i] = fminf(m16[i], m16[i + h]);
                        const bool rare = m16[0] <= t;
                        long long th1 = clock64();
                        if (x.timers && (warp & 3) == 0 && lane == 0)
                            atomicAdd(&x.timers[TT_EPI_HOT], (unsigned long long)(th1 - th0));
                        if (!rare) continue;  // per-lane control flow only: no warp collective below
                        if (x.timers) atomicAdd(&x.timers[TT_EPI_RARE], 1ull);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            uint32_t m = 0;
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                m |= (__uint_as_float(v[32 * h + i]) <= t ? 1u : 0u) << i;
                            if (!m) continue;
#pragma unroll
                            for (int i = 0; i < 32; ++i) scr[i * kQB] = __uint_as_float(v[32 * h + i]);
                            while (m) {
                                const int i = __ffs(m) - 1;
                                m &= m - 1;
                                const float w = scr[i * kQB];
                                if (!(w <= t)) continue;
                                if (nb == S::CB) {
                                    flush();
                                    if (!(w <= t)) continue;
                                }
                                bw[nb * kQB] = w;
                                bi[nb * kQB] = sposs[cc * 64 + 32 * h + i];
                                ++nb;
                            }
                        }
                        if (x.timers && (warp & 3) == 0 && lane == 0)
                            atomicAdd(&x.timers[TT_EPI_RAREC], (unsigned long long)(clock64() - th1));
                    }
                    // the whole warp inserts its buffered candidates together
                    long long tf1 = clock64();
                    const int mx = __reduce_max_sync(0xffffffffu, nb);
                    if (mx > 0) flush();
                    if (x.timers && (warp & 3) == 0 && lane == 0)
                        atomicAdd(&x.timers[TT_EPI_FLUSH], (unsigned long long)(clock64() - tf1));
                }
                if (x.timers && (warp & 3) == 0 && lane == 0)
                    atomicAdd(&x.timers[TT_EPI_WORK], (unsigned long long)(clock64() - te1));
                if (!__any_sync(0xffffffffu, changed)) continue;  // the published bound stands
                long long tb0 = clock64();
                float ub = fminf(Bd::ub(list_at(ld, kq - 1), qa), qc);
                float vmax = act ? ub : -INFINITY, vmin = act ? ub : INFINITY;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
                    vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
                }
                if (lane == 0) {
                    s_wmax[warp] = vmax;
                    s_wmin[warp] = vmin;
                }
                if (x.timers && (warp & 3) == 0 && lane == 0)
                    atomicAdd(&x.timers[TT_EPI_TAIL], (unsigned long long)(clock64() - tb0));
            }
            // ---- merge group 1's lists into group 0's (the raw ring is idle now)
            long long tf0 = clock64();
            float* smd = reinterpret_cast<float*>(smem + L::OFF_RAW);
            int32_t* smi = reinterpret_cast<int32_t*>(smem + L::OFF_RAW + kQB * KC * 4);
            tc::named_sync(BAR_EPI, 256);
            if (role == 1) {
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    smd[j * kQB + qt] = ld[j];
                    smi[j * kQB + qt] = li[j];
                }
            }
            tc::named_sync(BAR_EPI, 256);
            if (role == 0) {
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    float d = smd[j * kQB + qt];
                    int i = smi[j * kQB + qt];
                    bool dup = false;
#pragma unroll
                    for (int q = 0; q < KC; ++q) dup |= li[q] == i;
                    if (!dup && key_less(d, i, ld[KC - 1], li[KC - 1])) list_insert(ld, li, d, i);
                }
                // ---- finish the work item
                if (MODE == MODE_SEED) {
                    if (act) {
#pragma unroll
                        for (int j = 0; j < KC; ++j) {
                            a.cand_d[(int64_t)j * a.nq_all + (P.q0 + myq)] = ld[j];
                            a.cand_i[(int64_t)j * a.nq_all + (P.q0 + myq)] = li[j];
                        }
                        a.qub[P.q0 + myq] = Bd::ub(list_at(ld, kq - 1), qa);
                    }
                } else {
                    const float ubk = fminf(Bd::ub(list_at(ld, kq - 1), qa), qc);
                    const float band = Bd::band(ubk, qa);
                    const bool ovf = act && li[KC - 1] != kEmptyIdx && !(ld[KC - 1] > band);
                    // the re-rank below reuses the merge buffers: all of group 0 has read them
                    tc::named_sync(BAR_G0, 128);
                    if (ovf) {
                        a.fbq_list[atomicAdd(a.fbq_count, 1)] =
                            make_int4(myq, blk, __float_as_int(ubk), 0);
                    } else if (act) {
                        // float64 re-rank of the band candidates in shared memory
                        double* rd = reinterpret_cast<double*>(smem + L::OFF_RAW);
                        int32_t* ri = reinterpret_cast<int32_t*>(smem + L::OFF_KEY);
                        const float* qp = P.qpts + (int64_t)myq * DP;
                        int nb = 0;
#pragma unroll
                        for (int j = 0; j < KC; ++j) {
                            if (li[j] != kEmptyIdx && !(ld[j] > band)) {
                                rd[nb * kQB + qt] = exact_d2<DP>(qp, P.rpts + (int64_t)li[j] * DP);
                                ri[nb * kQB + qt] = P.ridx[li[j]];
                                ++nb;
                            }
                        }
                        n_re += nb;
                        const int64_t base = (int64_t)P.qidx[myq] * kq;
                        for (int j = 0; j < kq; ++j) {
                            int best = j;
                            for (int c = j + 1; c < nb; ++c)
                                if (key_less(rd[c * kQB + qt], ri[c * kQB + qt], rd[best * kQB + qt],
                                             ri[best * kQB + qt]))
                                    best = c;
                            const double bd = rd[best * kQB + qt];
                            const int bi = ri[best * kQB + qt];
                            rd[best * kQB + qt] = rd[j * kQB + qt];
                            ri[best * kQB + qt] = ri[j * kQB + qt];
                            P.out_idx[base + j] = bi;
                            P.out_dist[base + j] = (float)sqrt(bd);
                        }
                    }
                }
                if (x.timers && qt == 0)
                    atomicAdd(&x.timers[TT_EPI_FINISH], (unsigned long long)(clock64() - tf0));
            }
        }
        __syncthreads();
    }
    // a failed wait may leave an MMA in flight: its group's leader waits for it
    // (bounded) before the accumulators are released
    if (s_fail && pend) {
        atomicExch(x.err, 1);
        tc::mbar_wait(&acc_full[role], (acnt - 1) & 1u, x.spin_budget);
    }
    if (s_fail && tid == 0) atomicExch(x.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 8) tc::tmem_dealloc(tmem, TN * NS);
    if (n_skip) atomicAdd(&a.stats[ST_SKIPPED], n_skip);
    if (n_eval) atomicAdd(&a.stats[ST_EVALUATED], n_eval);
    if (n_pp) atomicAdd(&a.stats[ST_POINT_PAIRS], n_pp);
    if (n_re) atomicAdd(&a.stats[ST_RERANK], n_re);
    if (x.timers && n_ins) atomicAdd(&x.timers[TT_INSERTS], n_ins);
}

// The kernel allocates all 512 TMEM columns, so at most one CTA may be
// resident per SM: the request is raised above half the SM's shared memory.
template <int FMT, int DP, int KC>
inline size_t tc_smem_bytes() {
    int dev = 0, sm_total = 233472;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaGetLastError();
    size_t guard = (size_t)sm_total / 2 + 1024;
    size_t need = (size_t)TcSmem<FMT, DP, KC>::BYTES;
    return need > guard ? need : guard;
}

// Diagnostic timers for the next tensor-core launches (null = off).
extern unsigned long long* g_tc_timers;

template <int DP>
int launch_tile_tc(const TileArgs& a, int fmt, int kc, int mode, int items, int* err, int spin,
                   cudaStream_t s) {
    // counters 0..31 for the main pass, 32..63 for the seed pass
    // the seed pass runs on the CUDA cores (launch_tile_cc)
    if (mode != MODE_MAIN) return DTREE_ERR_UNSUPPORTED;
    TcExtra x{err, spin, g_tc_timers};
    // TF32 operand rows of 64 dimensions do not fit the pipeline's shared
    // memory; BF16 serves that width (where the MMA cost matters most)
    if (DP > 32 && fmt == 2) return DTREE_ERR_UNSUPPORTED;
    // BF16 requests: split BF16 (hi + lo per coordinate) up to 32 dimensions,
    // single BF16 beyond (whose operand rows would not fit shared memory split)
    if (fmt == 1 && DP <= 32) fmt = 3;
#define DT_TC_CASE(FMTV, KCV)                                                              \
    if constexpr (!(DP > 32 && FMTV != 1) && !(DP <= 32 && FMTV == 1))                     \
    if (fmt == FMTV && kc == KCV) {                                                        \
        auto kern = k_tile_tc<FMTV, DP, KCV, MODE_MAIN>;                                   \
        size_t smem = tc_smem_bytes<FMTV, DP, KCV>();                                      \
        DT_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                      (int)smem));                                         \
        int g = occupancy_grid((const void*)kern, 384, smem);                              \
        if (items < g) g = items > 0 ? items : 1;                                          \
        DT_LAUNCH(kern, g, 384, smem, s, a, x);                                            \
        return DTREE_OK;                                                                   \
    }
    DT_TC_CASE(1, 4)
    DT_TC_CASE(1, 8)
    DT_TC_CASE(1, 16)
    DT_TC_CASE(1, 24)
    DT_TC_CASE(1, 32)
    DT_TC_CASE(2, 4)
    DT_TC_CASE(2, 8)
    DT_TC_CASE(2, 16)
    DT_TC_CASE(2, 24)
    DT_TC_CASE(2, 32)
    DT_TC_CASE(3, 4)
    DT_TC_CASE(3, 8)
    DT_TC_CASE(3, 16)
    DT_TC_CASE(3, 24)
    DT_TC_CASE(3, 32)
#undef DT_TC_CASE
    return DTREE_ERR_UNSUPPORTED;
}

}  // namespace dt
