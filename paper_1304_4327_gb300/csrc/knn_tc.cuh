// knn_tc.cuh -- the kNN BaseCase (Algorithm 2) on the tensor cores.
//
// A work item is a chunk of <= 128 queries of a query block (one TMEM lane
// and one epilogue thread each); the chunks of a block share its candidate
// leaves.  Every point is centred on one point c, the centre
// of the reference tree's root box, and rounded to the MMA's input type:
//   - reference points once per tree and format (k_tc_ops), into an operand
//     array laid out exactly as the tiles sit in shared memory (8-row groups
//     of 16-byte core matrices, every leaf padded to a whole number of
//     groups), so a tile is filled by bulk copies (TMA) of whole leaves with
//     no per-tile conversion;
//   - queries once per work item, by the epilogue threads themselves.
// tcgen05.mma forms Q R^T in TMEM with FP32 accumulation, and the epilogue
// reads each thread's TMEM lane and forms
//     s = |q~|^2 + (|r~|^2 - 2 q~.r~),
// the squared distance of the rounded, centred points, then runs the
// Algorithm 2 insertion on (s, index) exactly as the CUDA-core tile does.
//
// Exactness.  With a = |q - c|, b = |r - c|, u_p the operand's relative
// error (2^-11 for TF32, about 2^-16 for split BF16) and u = 2^-24, the true
// distance D = |q - r| and the computed s satisfy
//     |D~ - D| <= e1 (a + b),            e1 = u_p + 2u,  D~ = |q~ - r~|
//     |s - D~^2| <= alpha (a^2 + b^2),   alpha = (4 K + 16) u + cross,
// (K = MMA depth; the alpha term covers the two norms, the accumulation and
// the epilogue's two roundings; cross the norm's hi/lo split and, for split
// BF16, the dropped lo.lo product).  Hence, per query with k-th key S,
//     ub = sqrt(S + alpha' (a^2 + bb^2)) + e1 (a + bb),  bb = 1.03 (a + sqrt S)
// bounds the true k-th distance (it feeds B_1, B_2 and Score), and every
// true k-nearest neighbour has s <= T = (ub + e1 (a + bu))^2 + alpha' (a^2 + bu^2),
// bu = 1.01 (a + ub).  Candidates with s <= T are re-ranked in float64; a
// list too short to hold them all sends the query to the float64 pass.  The
// bounds hold for any centring point; the root centre trades a wider band
// (larger a, b) for converting each reference point once instead of once
// per tile.
#pragma once

#include <cuda_bf16.h>

#include <algorithm>

#include "knn_tile.cuh"
#include "tc_ptx.cuh"

namespace dt {

// Operand formats.  hw is the MMA's input type (1 = BF16 with .kind::f16,
// 2 = TF32 with .kind::tf32); split is 3 when a coordinate x is carried as
// hi = bf16(x) and lo = bf16(x - hi) (|x - (hi + lo)| <= 2^-16 |x|), whose
// three products hi.hi + lo.hi + hi.lo leave out lo.lo; u bounds the
// relative error of a centred coordinate as the MMA sees it; cross bounds,
// relative to a^2 + b^2, what the norm columns' hi/lo split and any dropped
// product add to the key.
template <int FMT>
struct TcFmt;
template <>
struct TcFmt<2> {  // TF32 (round to nearest): 11 significant bits
    static constexpr int esize = 4, kstep = 8, hw = 2, split = 1;
    static constexpr float u = 0.00048828125f;  // 2^-11
    static constexpr float cross = u * u;
};
template <>
struct TcFmt<3> {  // split BF16
    static constexpr int esize = 2, kstep = 16, hw = 1, split = 3;
    static constexpr float u = 1.5411377e-05f;   // 2^-16 (1 + 2^-8)
    // 2^-16 (norm split) + 1.01 x 2^-16 (lo.lo, as 2 |q||r| <= a^2 + b^2): 3.1e-5, rounded up
    static constexpr float cross = 4.6e-05f;
};

// Operand rows.  A row (query) carries -2 x the centred coordinates and two
// ones; a B row (reference) carries the centred coordinates and the float32
// norm of its represented values split as hi + lo, so the accumulator holds
// w = |r~|^2 - 2 q~.r~ directly.  Rows are NKS K steps of 32 bytes; MMA m
// reads A step astep(m) and B step bstep(m).
//   TF32:                     A: -2x, 1, 1      B: x, nhi, nlo          (one pass)
//   split BF16, DP <= 8:      A: -2hi, -2lo, -2hi, 1, 1
//                             B:  hi,   hi,   lo, nhi, nlo              (one pass)
//   split BF16, DP >= 16:     A: [-2hi] [-2lo] [1, 1]  B: [hi] [lo] [nhi, nlo]
//     (each bracket padded to whole K steps; the MMAs pair A hi/B hi,
//      A lo/B hi, A hi/B lo and the norm steps, so a row stores each copy
//      of the coordinates once)
template <int FMT, int DP>
struct TcShape {
    static constexpr int kstep = TcFmt<FMT>::kstep;  // elements per 32-byte K step
    static constexpr bool REUSE = FMT == 3 && DP >= 16;
    static constexpr int H = (DP + kstep - 1) / kstep;  // K steps of one copy of the coordinates
    static constexpr int NKS = REUSE ? 2 * H + 1 : (DP * TcFmt<FMT>::split + 2 + kstep - 1) / kstep;
    static constexpr int NK = REUSE ? 3 * H + 1 : NKS;  // MMAs per tile
    static constexpr int RB = NKS * 32;                 // bytes per operand row
    static constexpr int NCH = RB / 16;                 // 16-byte chunks per row
    static constexpr int GB = 8 * RB;                   // bytes per 8-row group (the SBO)
    static constexpr int KP = NK * kstep;               // MMA depth
    static constexpr int EPC = 16 / TcFmt<FMT>::esize;  // elements per chunk
    // reference points per tile: 256 (the MMA's widest N) where the operand
    // slots fit shared memory
    static constexpr int TN = DP <= 16 ? 256 : 128;
    static constexpr int TN8 = TN / 8;
    __host__ __device__ static constexpr int astep(int m) {
        return !REUSE ? m : m < 2 * H ? m : m < 3 * H ? m - 2 * H : 2 * H;
    }
    __host__ __device__ static constexpr int bstep(int m) {
        return !REUSE ? m : m < H ? m : m < 3 * H ? m - H : 2 * H;
    }
};

// Shared memory of the tile kernel (bytes): NG epilogue groups, lists of KC.
template <int FMT, int DP, int KC, int NG>
struct TcSmem {
    using S = TcShape<FMT, DP>;
    static constexpr int NB = 4;                                     // operand slots
    static constexpr int GR = 8;                                     // row-group tables (a ring)
    static constexpr int WIN = 256;                                  // candidates per window
    static constexpr int CB = 8;                                     // deferred insertions per thread
    static constexpr int OFF_A = 0;                                  // 128 x RB
    static constexpr int OFF_B = OFF_A + kQB * S::RB;                // NB x TN x RB
    static constexpr int OFF_GRP = OFF_B + NB * S::TN * S::RB;       // GR x TN8 int2 (row groups)
    static constexpr int OFF_WIN = OFF_GRP + GR * S::TN8 * 8;        // 2 x WIN (leaf int, d_min float)
    static constexpr int OFF_WENT = OFF_WIN + 2 * WIN * 8;           // WIN int4 (begin, count, leaf, group0)
    static constexpr int OFF_SCR = OFF_WENT + WIN * 16;              // NG x 32 x 128 float
    static constexpr int OFF_BUF = OFF_SCR + NG * 32 * kQB * 4;      // NG x CB x 128 (float, int)
    static constexpr int OFF_CEN = OFF_BUF + NG * CB * kQB * 8;      // DP float
    static constexpr int END = OFF_CEN + DP * 4;
    // at a block's end everything above is idle: the merge of two groups'
    // lists (float + int per entry) and the float64 re-rank (double + int per
    // entry) reuse it from offset 0
    static constexpr int FIN = kQB * KC * 12;
    static constexpr int BYTES = END > FIN ? END : FIN;
    static_assert(BYTES <= 225 * 1024, "tensor-core tile shared memory over budget");
    static_assert(S::TN8 * 8 == S::TN && S::TN8 <= 32, "tiles hold whole 8-row groups, one per lane");
};

template <int FMT, int DP>
struct TcBound {
    static constexpr float u = 5.9604645e-08f;
    static constexpr float e1 = TcFmt<FMT>::u + 2.f * u;
    // accumulation over K terms, the norms and the epilogue add, plus the
    // hi/lo split of |r~|^2 (and the dropped product of split BF16)
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

// A centred coordinate rounded to the operand type (the hi part of split BF16).
template <int FMT>
__device__ __forceinline__ float tc_round(float h) {
    return FMT == 2 ? tc::to_tf32(h) : __bfloat162float(__float2bfloat16_rn(h));
}

// The lo part of split BF16.
__device__ __forceinline__ float tc_lo(float h) {
    const float hi = __bfloat162float(__float2bfloat16_rn(h));
    return __bfloat162float(__float2bfloat16_rn(h - hi));
}

// Sum of squares of the represented values (x~, or hi + lo, both exact in
// float32), coordinate by coordinate.
template <int FMT, int DP>
__device__ __forceinline__ float tc_norm(const float (&h)[DP]) {
    float n = 0.f;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        const float hi = tc_round<FMT>(h[j]);
        const float r = FMT == 3 ? hi + tc_lo(h[j]) : hi;
        n = fmaf(r, r, n);
    }
    return n;
}

// Element e of an operand row built from the centred coordinates h (A rows:
// the query side, scaled by -2, with ones in the norm columns).
template <int FMT, int DP, bool AROW>
__device__ __forceinline__ float tc_elem(int e, const float (&h)[DP], float nhi, float nlo) {
    using S = TcShape<FMT, DP>;
    const float sc = AROW ? -2.f : 1.f;
    if constexpr (S::REUSE) {
        constexpr int W = S::H * S::kstep;
        if (e < W) return e < DP ? sc * tc_round<FMT>(h[e < DP ? e : 0]) : 0.f;
        if (e < 2 * W) {
            const int j = e - W;
            return j < DP ? sc * tc_lo(h[j < DP ? j : 0]) : 0.f;
        }
        e -= 2 * W;
    } else if constexpr (FMT == 3) {
        if (e < DP) return sc * tc_round<FMT>(h[e]);
        if (e < 2 * DP) return sc * (AROW ? tc_lo(h[e - DP]) : tc_round<FMT>(h[e - DP]));
        if (e < 3 * DP) return sc * (AROW ? tc_round<FMT>(h[e - 2 * DP]) : tc_lo(h[e - 2 * DP]));
        e -= 3 * DP;
    } else {
        if (e < DP) return sc * tc_round<FMT>(h[e]);
        e -= DP;
    }
    if (e == 0) return AROW ? 1.f : nhi;
    if (e == 1) return AROW ? 1.f : nlo;
    return 0.f;
}

// The 16 bytes of chunk c of an operand row.
template <int FMT, int DP, bool AROW>
__device__ __forceinline__ uint4 tc_row_chunk(int c, const float (&h)[DP], float nhi, float nlo) {
    uint4 w;
    uint32_t* p = reinterpret_cast<uint32_t*>(&w);
    if (TcFmt<FMT>::esize == 2) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 b = __floats2bfloat162_rn(tc_elem<FMT, DP, AROW>(8 * c + 2 * i, h, nhi, nlo),
                                                     tc_elem<FMT, DP, AROW>(8 * c + 2 * i + 1, h, nhi, nlo));
            p[i] = *reinterpret_cast<uint32_t*>(&b);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) p[i] = __float_as_uint(tc_elem<FMT, DP, AROW>(4 * c + i, h, nhi, nlo));
    }
    return w;
}

// The reference operand array of a tree: leaf l occupies rows [l ls, (l + 1) ls)
// (ls a multiple of 8); row i < count(l) is the leaf's i-th point centred on
// the root box centre, the rest are padding rows (zero coordinates, norm
// +inf, so that their key is +inf).  Row r sits at byte (r / 8) GB +
// (r % 8) 16 + chunk 128, the shared-memory layout of a tile.
template <int FMT, int DP>
__global__ void __launch_bounds__(128) k_tc_ops(const float* __restrict__ pts,
                                                const int32_t* __restrict__ nbeg,
                                                const int32_t* __restrict__ ncnt,
                                                const float* __restrict__ rootbox, int64_t leaf0,
                                                int64_t nleaves, int ls,
                                                unsigned char* __restrict__ out) {
    using S = TcShape<FMT, DP>;
    const int64_t rows = nleaves * ls;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = r / ls;
        const int i = (int)(r - l * ls);
        const int cnt = ncnt[leaf0 + l];
        float h[DP];
        float nhi = INFINITY, nlo = 0.f;
        if (i < cnt) {
            const float4* p4 = reinterpret_cast<const float4*>(pts + ((int64_t)nbeg[leaf0 + l] + i) * DP);
#pragma unroll
            for (int j4 = 0; j4 < DP / 4; ++j4) {
                const float4 v = p4[j4];
                h[4 * j4] = v.x - 0.5f * (rootbox[4 * j4] + rootbox[DP + 4 * j4]);
                h[4 * j4 + 1] = v.y - 0.5f * (rootbox[4 * j4 + 1] + rootbox[DP + 4 * j4 + 1]);
                h[4 * j4 + 2] = v.z - 0.5f * (rootbox[4 * j4 + 2] + rootbox[DP + 4 * j4 + 2]);
                h[4 * j4 + 3] = v.w - 0.5f * (rootbox[4 * j4 + 3] + rootbox[DP + 4 * j4 + 3]);
            }
            const float rn = tc_norm<FMT, DP>(h);
            nhi = tc_round<FMT>(rn);
            nlo = tc_round<FMT>(rn - nhi);
        } else {
#pragma unroll
            for (int j = 0; j < DP; ++j) h[j] = 0.f;
        }
        unsigned char* base = out + (r >> 3) * S::GB + (r & 7) * 16;
#pragma unroll
        for (int c = 0; c < S::NCH; ++c)
            *reinterpret_cast<uint4*>(base + c * 128) = tc_row_chunk<FMT, DP, false>(c, h, nhi, nlo);
    }
}

struct TcExtra {
    int* err;          // device status word: 1 = a bounded wait gave up
    int spin_budget;
    unsigned long long* timers;  // optional per-role cycle counters (diagnostics), or null
    int stall;         // diagnostics: the planner waits on a barrier nothing completes
};

// Which bounded wait gave up (diagnostics, TT_FAIL_SITES).
enum TcFailSite {
    FS_PLAN_SLOT = 1,   // planner: a free operand slot or row-group table
    FS_PLAN_END = 2,    // planner: the slot for the block's end marker
    FS_MMA_OP = 4,      // MMA warp: a filled slot
    FS_MMA_ACC = 8,     // MMA warp: a free accumulator
    FS_MMA_END = 16,    // MMA warp: an accumulator for the end marker
    FS_EPI_ACC = 32,    // epilogue: a full accumulator
    FS_STALL = 64       // the stall diagnostic
};

#define TC_FAIL_SITE(site) \
    do { if (x.timers) atomicOr(&x.timers[TT_FAIL_SITES], (unsigned long long)(site)); } while (0)

// Polls of the waits that drain a failed item's own copies and MMAs before
// the kernel releases TMEM and exits.  They finish on their own (nothing
// else has to run for a bulk copy or an issued MMA to complete), so the limit
// is fixed and far above their duration, independent of the caller's
// spin_budget.
constexpr int kDrainPolls = 1 << 22;
// End-of-tile insertion policy of the tile kernel's epilogue warps: insert
// when at least flush_lanes(KC) lanes hold buffered candidates, or after
// flush_tiles(KC) tiles with some pending.  A pass of the insertion code
// costs in proportion to the list length, so long lists wait for more lanes
// (2M x 2M, d = 64, lists of 64: 1.84 -> 1.79 s), while short ones insert
// early and keep their threshold tight (gmm16, lists of 24: 32 lanes would
// cost 5%).
__host__ __device__ constexpr int flush_lanes(int kc) { return kc >= 48 ? 32 : 8; }
__host__ __device__ constexpr int flush_tiles(int kc) { return kc >= 48 ? 64 : 16; }

// Diagnostic cycle counters of the tile kernel (summed over CTAs; read only
// when timers are attached).  The per-role cycle counts are compiled in only
// with DTREE_TC_TIMERS=1: their clock reads and registers cost the hot loops
// about a sixth of their speed even when no counters are attached.  The
// failure-site mask (TT_FAIL_SITES) is always kept: it sits on failure paths.
#ifndef DTREE_TC_TIMERS
#define DTREE_TC_TIMERS 0
#endif
#define TC_TIMED (DTREE_TC_TIMERS && x.timers)
enum TcTimer {
    TT_PLAN_WINDOW = 0,  // planner: loading and preparing candidate windows
    TT_PLAN_WAIT,        // planner: waiting for a free operand slot
    TT_PLAN_STAGE,       // planner: filling slots and issuing copies
    TT_MMA_WAIT,         // MMA warp: waiting for a filled slot or a free accumulator
    TT_EPI_WAIT,         // epilogue (warp 0): waiting for an accumulator
    TT_EPI_WORK,         // epilogue (warp 0): reading TMEM, keys, insertion
    TT_EPI_RARE,         // epilogue (all threads): chunks that took the insertion path
    TT_EPI_FINISH,       // epilogue: re-rank, output
    TT_ITEM_SETUP,       // all: query conversion, list init
    TT_TILES,            // planner: tiles produced
    TT_ITEMS,            // items processed
    TT_INSERTS,          // epilogue (all threads): candidate-list insertions
    TT_EPI_LD,           // epilogue (warp 0): TMEM reads, issue to completion
    TT_EPI_LOOP,         // epilogue (warp 0): the column loop (reads, thresholds, buffering)
    TT_EPI_FLUSH,        // epilogue (warp 0): the release and the end-of-tile insertions
    TT_MMA_WAIT_ACC,     // MMA warp: the part of TT_MMA_WAIT spent waiting for an accumulator
    TT_FAIL_SITES,       // bit mask of the waits that gave up (TcFailSite)
    TT_EPI_WORK_W2,      // epilogue (warp 2, alone on its sub-partition): as TT_EPI_WORK
    TT_PLAN_COPY,        // planner (lane 0's view): issuing the tile's bulk copies
    TT_COPY_LAND,        // MMA warp: from the planner's hand-off of a slot to its wait passing
    TT_N
};
static_assert(TT_N <= 32, "the diagnostic timer buffer holds 32 counters");

// One persistent CTA per SM, 4 NG + 2 warps:
//   warps 0 .. 4 NG - 1  NG epilogue groups of four warps: one query row (TMEM
//              lane) per thread; each warp reads its own 32 lanes of an
//              accumulator, examines the keys and keeps its queries' lists,
//              and hands the accumulator and the tile's row-group table back
//              by mbarrier arrivals, independently of the other warps.  Tiles alternate
//              between two accumulators: with NG = 1 the group reads both in
//              turn; with NG = 2 group g reads accumulator g and keeps its own
//              lists, which are merged when the block is done
//   warp 4 NG  planner: prepares a window of the block's candidate leaves at
//              a time (Algorithm 3's test against the block's bound, each
//              kept leaf's range and its place in the window's run of 8-row
//              groups), then fills operand slots with whole 8-row groups by
//              bulk copies (TMA) of the leaves' operand rows, and a table of
//              the groups' first rows (a ring of GR tables, deeper than the
//              slots: a slot is free again once its MMAs are done)
//   warp 4 NG + 1  MMA issuer: one thread turns a filled slot into an
//              accumulator (two in turn) with tcgen05.mma
// Hand-over by mbarriers: op_full (planner -> MMA: its arrival plus the
// copied bytes), acc_full (MMA -> epilogue: the MMA's commit plus the
// issuer's arrival with the tile's row-group table and columns), acc_empty (epilogue ->
// MMA: one arrival per warp once its lanes are read), op_empty (MMA commit
// -> planner), gr_empty (the four epilogue warps -> planner: the tile's
// row-group table is read).  Every wait is bounded; after a
// failed wait the item's work is abandoned, the kernel drains its own copies
// and MMAs, releases TMEM and reports through x.err.
template <int FMT, int DP, int KC, int NG>
__global__ void __launch_bounds__(32 * (4 * NG + 2), 1) k_tile_tc(const TileArgs a, const TcExtra x) {
    using S = TcShape<FMT, DP>;
    using L = TcSmem<FMT, DP, KC, NG>;
    using Bd = TcBound<FMT, DP>;
    constexpr int TN = S::TN, TN8 = S::TN8, NB = L::NB, GR = L::GR, CB = L::CB, WIN = L::WIN;
    constexpr int PW = 4 * NG, MW = 4 * NG + 1;  // the planner's and the MMA issuer's warps
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem + L::OFF_A;
    unsigned char* sB = smem + L::OFF_B;
    int2* sgrp = reinterpret_cast<int2*>(smem + L::OFF_GRP);   // GR x TN8
    int32_t* swleaf = reinterpret_cast<int32_t*>(smem + L::OFF_WIN);
    float* swdmin = reinterpret_cast<float*>(smem + L::OFF_WIN + 2 * WIN * 4);
    int4* went = reinterpret_cast<int4*>(smem + L::OFF_WENT);
    float* sscr = reinterpret_cast<float*>(smem + L::OFF_SCR);
    float* sbuf = reinterpret_cast<float*>(smem + L::OFF_BUF);
    float* scen = reinterpret_cast<float*>(smem + L::OFF_CEN);
    __shared__ uint64_t op_full[NB], op_empty[NB], gr_empty[GR], acc_full[2], acc_empty[2], never;
    __shared__ int ometa[NB];
    __shared__ long long s_handoff[NB];  // diagnostics: when the planner handed each slot over
    __shared__ int2 amet[2];  // the tile in each accumulator: (table, columns), columns < 0 ends the block
    __shared__ uint32_t s_tmem;
    __shared__ int s_item;
    __shared__ ProbDev s_prob;
    __shared__ volatile int s_fail;
    __shared__ volatile float s_wmax[4 * NG], s_wmin[4 * NG];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool epi = warp < 4 * NG;
    const int grp_id = warp >> 2;  // an epilogue thread's group
    const int qt = tid & 127;  // query row of an epilogue thread
    const int nitems = a.nitems;
    unsigned long long n_skip = 0, n_eval = 0, n_pp = 0, n_re = 0, n_ins = 0;

    if (tid == 0) {
        for (int i = 0; i < NB; ++i) {
            tc::mbar_init(&op_full[i], 1);   // the planner's arrival (+ copied bytes)
            tc::mbar_init(&op_empty[i], 1);  // tcgen05.commit
        }
        for (int i = 0; i < GR; ++i) tc::mbar_init(&gr_empty[i], 4);  // the four epilogue warps
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 2);   // tcgen05.commit + the issuer's arrival
            tc::mbar_init(&acc_empty[i], 4);  // the four epilogue warps
        }
        tc::mbar_init(&never, 1);  // nothing arrives on it (the stall diagnostic)
        tc::fence_mbar_init();
        s_fail = 0;
    }
    if (warp == MW) tc::tmem_alloc(&s_tmem, 2 * TN);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc::idesc(TcFmt<FMT>::hw, kQB, TN);
    // the barriers' phases carry over from item to item, so the counters do too
    uint32_t otile = 0;                  // planner / MMA issuer: operand slot uses
    uint32_t gtile = 0;                  // planner / MMA issuer: tiles (row-group table uses)
    // MMA issuer / each epilogue warp: bit b of aph is the parity of the uses
    // of accumulator b, bit b of aused whether it was used (bit masks, not an
    // array: a dynamically indexed array would live in local memory)
    uint32_t aph = 0u, aused = 0u;
    uint32_t acur = 0;                   // MMA issuer / each epilogue warp: the next accumulator

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
        long long tm0 = TC_TIMED ? clock64() : 0;
        // the centring point: the reference root box's centre, as k_tc_ops used it
        if (tid < DP) scen[tid] = 0.5f * (P.rbox[tid] + P.rbox[DP + tid]);
        __syncthreads();
        const bool act = epi && qt < nq;
        const int myq = P.qbeg[qnode] + chunk * kQB + qt;
        const int kq = P.k;  // read once: stores below could alias P
        const bool mono = P.mono != 0;
        const float lam2 = 2.f * P.qlam[qnode];
        float qa = 0.f, qn = 0.f;
        // the cap pass's bound on the query's k-th distance
        const float qc = act && a.qcap ? a.qcap[P.q0 + myq] : INFINITY;
        float ld[KC];
        int li[KC];
        if (epi) {
            // the query, centred and rounded, as row qt of the A tile
            float h[DP];
            float qa2 = 0.f;
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
            qn = tc_norm<FMT, DP>(h);
            if (grp_id == 0) {
#pragma unroll
                for (int c = 0; c < S::NCH; ++c)
                    *reinterpret_cast<uint4*>(sA + tc::core_offset(qt, c, S::GB)) =
                        tc_row_chunk<FMT, DP, true>(c, h, 1.f, 1.f);
            }
            qa = __fsqrt_ru(qa2);
#pragma unroll
            for (int j = 0; j < KC; ++j) {
                ld[j] = act ? a.cand_d[(int64_t)j * a.nq_all + (P.q0 + myq)] : INFINITY;
                li[j] = act ? a.cand_i[(int64_t)j * a.nq_all + (P.q0 + myq)] : kEmptyIdx;
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
        if (TC_TIMED && tid == 0) {
            atomicAdd(&x.timers[TT_ITEM_SETUP], (unsigned long long)(clock64() - tm0));
            atomicAdd(&x.timers[TT_ITEMS], 1ull);
        }

        if (warp == PW) {
            // ================= planner =================
            const float Bq = a.Bn ? a.Bn[P.node0 + qnode] : INFINITY;
            const int64_t c0 = a.csr_off[blk], c1 = a.csr_off[blk + 1];
            // the candidates: the block's proposed cells the seed pass left
            // (first, for a tight bound early), then the traversal's list
            const int sn0 = seed_count_n(a.seed_nleaf, a.seed_slots, a.seed_eval_slots, blk);
            const int npro = seed_count(a.seed_nleaf, a.seed_slots, blk) - sn0;
            const int64_t ntot = npro + (c1 - c0);
            const unsigned char* rops = static_cast<const unsigned char*>(P.rops);
            const int64_t ls8 = P.rls8;
            bool fail = false;
            // window w's leaves and d_min land in buffer w & 1 by cp.async,
            // issued while the previous window is processed
            auto fetch = [&](int64_t w0, int buf) {
                const int wn = (int)(ntot - w0 < WIN ? ntot - w0 : WIN);
                for (int i = lane; i < wn; i += 32) {
                    const int64_t ci = w0 + i - npro;  // entry of the traversal's list
                    if (ci >= 0) {
                        tc::cp_async4(swleaf + buf * WIN + i, a.csr_leaf + c0 + ci);
                        tc::cp_async4(swdmin + buf * WIN + i, a.csr_dmin + c0 + ci);
                    }
                }
                tc::cp_async_commit();
            };
            if (ntot > 0) fetch(0, 0);
            int wbuf = 0;
            for (int64_t w0 = 0; w0 < ntot && !fail; w0 += WIN, wbuf ^= 1) {
                const int wn = (int)(ntot - w0 < WIN ? ntot - w0 : WIN);
                long long t0 = TC_TIMED ? clock64() : 0;
                tc::cp_async_wait_all();
                __syncwarp();
                if (w0 + WIN < ntot) fetch(w0 + WIN, wbuf ^ 1);
                // the block's bound from the epilogue warps' published values
                float b = Bq;
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    float mx = -INFINITY, mn = INFINITY;
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        mx = fmaxf(mx, s_wmax[4 * g + w]);
                        mn = fminf(mn, s_wmin[4 * g + w]);
                    }
                    b = fminf(b, fminf(mx, __fadd_ru(mn, lam2)));
                }
                // the window's kept leaves (Algorithm 3: a leaf whose d_min
                // exceeds the bound is pruned), their ranges, and where each
                // starts in the window's run of 8-row groups
                // (every entry's range is read first, so the loads overlap)
                constexpr int NR = WIN / 32;
                int eleaf[NR], ebeg[NR], ecnt[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int i = r * 32 + lane;
                    const bool pro = w0 + i < npro;  // a proposed cell's leaf (never pruned)
                    const bool keep = i < wn && (pro || !(swdmin[wbuf * WIN + i] > b));
                    eleaf[r] = !keep ? -1
                               : pro ? seed_leaf(a.seed_leaf0, a.seed_nleaf, a.seed_slots, blk, sn0 + (int)(w0 + i))
                                     : swleaf[wbuf * WIN + i];
                    ebeg[r] = keep ? P.rbeg[P.rleaf0 + eleaf[r]] : 0;
                    ecnt[r] = keep ? P.rcnt[P.rleaf0 + eleaf[r]] : 0;
                }
                int G = 0;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int i = r * 32 + lane;
                    const bool valid = i < wn;
                    const int g = (ecnt[r] + 7) >> 3;
                    int4 e = make_int4(ebeg[r], ecnt[r], eleaf[r], 0);
                    int incl = g;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, incl, off);
                        if (lane >= off) incl += v;
                    }
                    e.w = G + incl - g;
                    if (valid) went[i] = e;
                    const unsigned kept = __ballot_sync(0xffffffffu, valid && g > 0);
                    const unsigned all = __ballot_sync(0xffffffffu, valid);
                    if (lane == 0) {
                        n_eval += __popc(kept);
                        n_skip += __popc(all & ~kept);
                    }
                    G += __shfl_sync(0xffffffffu, incl, 31);
                }
                __syncwarp();
                if (TC_TIMED && lane == 0)
                    atomicAdd(&x.timers[TT_PLAN_WINDOW], (unsigned long long)(clock64() - t0));
                // tiles of TN8 groups; the entries overlapping a tile are consecutive
                int cur = 0;
                for (int g0 = 0; g0 < G; g0 += TN8) {
                    const int g1 = min(g0 + TN8, G);
                    const int op = (int)(otile % NB);
                    const uint32_t use = otile / NB;
                    long long t1 = TC_TIMED ? clock64() : 0;
                    const int gi = (int)(gtile % GR);
                    const uint32_t guse = gtile / GR;
                    const bool ok = lane == 0 ? tc::mbar_wait(&op_empty[op], (use & 1u) ^ 1u, x.spin_budget) &&
                                                    tc::mbar_wait(&gr_empty[gi], (guse & 1u) ^ 1u, x.spin_budget)
                                              : true;
                    if (!__all_sync(0xffffffffu, ok)) {
                        if (lane == 0) TC_FAIL_SITE(FS_PLAN_SLOT);
                        fail = true;
                        break;
                    }
                    long long t2 = TC_TIMED ? clock64() : 0;
                    if (lane == 0) tc::mbar_expect_tx(&op_full[op], (uint32_t)(g1 - g0) * S::GB);
                    __syncwarp();
                    unsigned char* slot = sB + op * TN * S::RB;
                    int2* grp = sgrp + gi * TN8;
                    for (;;) {
                        const int i = cur + lane;
                        const bool valid = i < wn;
                        const int4 e = valid ? went[i] : make_int4(0, 0, 0, 0x7fffffff);
                        const int gs = e.w, gg = (e.y + 7) >> 3;
                        const int lo = max(gs, g0), hi = min(gs + gg, g1);
                        int real = 0;
                        const long long tcp = TC_TIMED ? clock64() : 0;
                        if (valid && hi > lo)
                            tc::bulk_g2s(slot + (lo - g0) * S::GB,
                                         rops + ((int64_t)e.z * ls8 + (lo - gs)) * S::GB,
                                         (uint32_t)(hi - lo) * S::GB, &op_full[op]);
                        if (TC_TIMED) {
                            __syncwarp();
                            if (lane == 0) atomicAdd(&x.timers[TT_PLAN_COPY], (unsigned long long)(clock64() - tcp));
                        }
                        if (valid && hi > lo) {
                            for (int q = lo; q < hi; ++q) {
                                const int r0 = 8 * (q - gs);
                                grp[q - g0] = make_int2(e.x + r0, min(8, e.y - r0));
                            }
                            real = min(e.y, 8 * (hi - gs)) - 8 * (lo - gs);
                        }
                        real = __reduce_add_sync(0xffffffffu, real);
                        if (lane == 0) n_pp += (unsigned long long)real * nq;
                        // entries that end within this tile are done; they form a prefix
                        const unsigned fin = __ballot_sync(0xffffffffu, valid && gs + gg <= g1);
                        const int adv = fin == 0xffffffffu ? 32 : __ffs(~fin) - 1;
                        cur += adv;
                        if (adv < 32) break;
                    }
                    if (lane == 0) ometa[op] = (g1 - g0) * 8;
                    __syncwarp();
                    if (lane == 0) {
                        if (TC_TIMED) s_handoff[op] = clock64();
                        tc::mbar_arrive(&op_full[op], 1);
                        if (TC_TIMED) {
                            atomicAdd(&x.timers[TT_TILES], 1ull);
                            atomicAdd(&x.timers[TT_PLAN_WAIT], (unsigned long long)(t2 - t1));
                            atomicAdd(&x.timers[TT_PLAN_STAGE], (unsigned long long)(clock64() - t2));
                        }
                    }
                    ++otile;
                    ++gtile;
                }
            }
            // a window fetch still in flight (after a failure) lands before the
            // buffers can be reused
            tc::cp_async_wait_all();
            __syncwarp();
            if (x.stall && !fail) {
                // diagnostics: a wait that nothing ends, which must give up
                // after spin_budget polls and fail the call
                const bool ok = lane == 0 ? tc::mbar_wait(&never, 0u, x.spin_budget) : true;
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) TC_FAIL_SITE(FS_STALL);
                    fail = true;
                }
            }
            // the end of the block
            if (!fail) {
                const int op = (int)(otile % NB);
                const uint32_t use = otile / NB;
                const bool ok = lane == 0 ? tc::mbar_wait(&op_empty[op], (use & 1u) ^ 1u, x.spin_budget) : true;
                if (__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) {
                        ometa[op] = -1;
                        tc::mbar_arrive(&op_full[op], 1);
                    }
                    ++otile;
                } else {
                    if (lane == 0) TC_FAIL_SITE(FS_PLAN_END);
                    fail = true;
                }
            }
            if (fail && lane == 0) s_fail = 1;
        } else if (warp == MW) {
            // ================= MMA issuer (one thread) =================
            if (lane == 0) {
                for (;;) {
                    const int op = (int)(otile % NB);
                    const uint32_t use = otile / NB;
                    long long t0 = TC_TIMED ? clock64() : 0;
                    if (!tc::mbar_wait(&op_full[op], use & 1u, x.spin_budget)) {
                        TC_FAIL_SITE(FS_MMA_OP);
                        s_fail = 1;
                        break;
                    }
                    if (TC_TIMED && ometa[op] >= 0)
                        atomicAdd(&x.timers[TT_COPY_LAND], (unsigned long long)(clock64() - s_handoff[op]));
                    const int nst = ometa[op];
                    ++otile;
                    if (nst < 0) {
                        // the end of the block: nothing reads the slot; the
                        // accumulators carry the marker to each epilogue group
                        tc::mbar_arrive(&op_empty[op], 1);
                        bool ok = true;
                        for (int e = 0; e < NG && ok; ++e) {
                            const int b = (int)acur;
                            ok = tc::mbar_wait(&acc_empty[b], ((aph >> b) & 1u) ^ 1u, x.spin_budget);
                            if (ok) {
                                amet[b] = make_int2(op, -1);
                                tc::mbar_arrive(&acc_full[b], 2);
                                aph ^= 1u << b;
                                aused |= 1u << b;
                                acur ^= 1u;
                            }
                        }
                        if (!ok) {
                            TC_FAIL_SITE(FS_MMA_END);
                            s_fail = 1;
                        }
                        break;
                    }
                    const int b = (int)acur;
                    const long long ta = TC_TIMED ? clock64() : 0;
                    if (!tc::mbar_wait(&acc_empty[b], ((aph >> b) & 1u) ^ 1u, x.spin_budget)) {
                        TC_FAIL_SITE(FS_MMA_ACC);
                        s_fail = 1;
                        break;
                    }
                    if (TC_TIMED) {
                        const long long tb = clock64();
                        atomicAdd(&x.timers[TT_MMA_WAIT], (unsigned long long)(tb - t0));
                        atomicAdd(&x.timers[TT_MMA_WAIT_ACC], (unsigned long long)(tb - ta));
                    }
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB + op * TN * S::RB);
#pragma unroll
                    for (int m = 0; m < S::NK; ++m)
                        tc::mma<TcFmt<FMT>::hw>(tmem + (uint32_t)(b * TN),
                                                tc::sdesc(a0 + 256u * S::astep(m), 128u, S::GB),
                                                tc::sdesc(b0 + 256u * S::bstep(m), 128u, S::GB), idesc,
                                                m > 0 ? 1u : 0u);
                    tc::mma_commit(&acc_full[b]);
                    tc::mma_commit(&op_empty[op]);  // the slot is free once the MMAs are done
                    amet[b] = make_int2((int)(gtile % GR), nst);
                    ++gtile;
                    tc::mbar_arrive(&acc_full[b], 1);
                    aph ^= 1u << b;
                    aused |= 1u << b;
                    acur ^= 1u;
                }
            }
            __syncwarp();
        } else {
            // ================= epilogue warp =================
            const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lanes
            float* scr = sscr + grp_id * 32 * kQB + qt;
            float* bw = sbuf + grp_id * CB * kQB + qt;
            int32_t* bi = reinterpret_cast<int32_t*>(sbuf + NG * CB * kQB) + grp_id * CB * kQB + qt;
            if (NG == 2) acur = (uint32_t)grp_id;  // group g reads accumulator g
            // insertion threshold in w units: below the list's last key and
            // inside the error band of the current k-th key (a key above the
            // band can never be a true k-nearest neighbour); it changes only
            // when the list does
            // the list's k-th entry, kept at hand: it changes only when an
            // insertion lands before it
            float kd = list_at(ld, kq - 1);
            int ki = list_at(li, kq - 1);
            auto threshold = [&]() {
                const float bnd = Bd::band(fminf(Bd::ub(kd, qa), qc), qa);
                return __fsub_ru(fminf(ld[KC - 1], bnd), qn);
            };
            float t = threshold();
            int nb = 0;
            bool changed = false;
            // candidates under the threshold are buffered per thread and
            // inserted together by the whole warp at the end of the tile
            auto flush = [&]() {
                for (int e = 0; e < nb; ++e) {
                    const float sv = qn + bw[e * kQB];
                    const int rp = bi[e * kQB];
                    // (the cap pass may have listed this point already)
                    if (key_less(sv, rp, ld[KC - 1], li[KC - 1]) && !(mono && rp == myq) && !listed(li, rp)) {
                        // the band moves only when the k-th key does
                        const bool kth_moves = key_less(sv, rp, kd, ki);
                        list_insert_par(ld, li, sv, rp);
                        if (kth_moves) {
                            kd = list_at(ld, kq - 1);
                            ki = list_at(li, kq - 1);
                            t = threshold();
                        } else {
                            t = fminf(t, __fsub_ru(ld[KC - 1], qn));
                        }
                        changed = true;
                        ++n_ins;
                    }
                }
                nb = 0;
            };
            // the minimum of 32 keys, computed (a tree of fminf; NaN ignored)
            auto chunk_min = [](const uint32_t (&v)[32]) {
                float m8[8];
#pragma unroll
                for (int i4 = 0; i4 < 8; ++i4)
                    m8[i4] = fminf(fminf(__uint_as_float(v[4 * i4]), __uint_as_float(v[4 * i4 + 1])),
                                   fminf(__uint_as_float(v[4 * i4 + 2]), __uint_as_float(v[4 * i4 + 3])));
                return fminf(fminf(fminf(m8[0], m8[1]), fminf(m8[2], m8[3])),
                             fminf(fminf(m8[4], m8[5]), fminf(m8[6], m8[7])));
            };
            // examine 32 keys from columns cb.. (rem of them belong to the
            // tile) whose minimum the load reduced to mm
            auto examine = [&](uint32_t (&v)[32], float mm, const int2* grp, int cb, int rem) {
                // columns past the tile's rows hold an earlier tile's values,
                // which the load's minimum includes: NaN never passes a
                // comparison, and the minimum is taken again without them
                if (rem < 32) {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (i >= rem) v[i] = 0x7fc00000u;
                    mm = chunk_min(v);
                }
                if (!(mm <= t)) return;  // per-lane control flow only: no warp collective inside
                if (TC_TIMED) atomicAdd(&x.timers[TT_EPI_RARE], 1ull);
                uint32_t m = 0;
#pragma unroll
                for (int i = 0; i < 32; ++i) m |= (__uint_as_float(v[i]) <= t ? 1u : 0u) << i;
#pragma unroll
                for (int i = 0; i < 32; ++i) scr[i * kQB] = __uint_as_float(v[i]);
                while (m) {
                    const int i = __ffs(m) - 1;
                    m &= m - 1;
                    const float w = scr[i * kQB];
                    if (!(w <= t)) continue;
                    if (nb == CB) {
                        flush();
                        if (!(w <= t)) continue;
                    }
                    const int cidx = cb + i;
                    const int2 gq = grp[cidx >> 3];
                    const int r = cidx & 7;
                    bw[nb * kQB] = w;
                    bi[nb * kQB] = r < gq.y ? gq.x + r : kEmptyIdx;
                    ++nb;
                }
            };
            int since_pub = 0;
            uint32_t ntile = 0;  // tiles this warp has examined (diagnostics)
            int since_flush = 0;  // tiles with buffered candidates since the last insertion
            bool dirty = false;
            for (;;) {
                const int b = (int)acur;
                long long te0 = (TC_TIMED && warp == 0 && lane == 0) ? clock64() : 0;
                const bool ok = tc::mbar_wait(&acc_full[b], (aph >> b) & 1u, x.spin_budget);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) {
                        TC_FAIL_SITE(FS_EPI_ACC);
                        s_fail = 1;
                    }
                    break;
                }
                tc::fence_after_sync();
                const int2 am = amet[b];
                aph ^= 1u << b;
                aused |= 1u << b;
                if (NG == 1) acur ^= 1u;
                if (am.y < 0) {  // the end of the block
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&acc_empty[b], 1);
                    // candidates still buffered go into the lists
                    if (__any_sync(0xffffffffu, nb > 0)) flush();
                    break;
                }
                long long te1 = (TC_TIMED && (warp & 3) != 1 && lane == 0) ? clock64() : 0;
                const int nst = am.y;
                const int2* grp = sgrp + am.x * TN8;  // the tile's row-group table
                const uint32_t tcol = tl + (uint32_t)(b * TN);
                const int nch = (nst + 31) >> 5;
                changed = false;
                long long ld_cyc = 0;
                // the columns 64 at a time: the load's minimum decides whether
                // any lane needs them, and only then are they read again 32 at
                // a time and examined (loops, not unrolled: one copy of the
                // examine path keeps the kernel's code within the instruction
                // cache).  A 64-column read past the tile's columns stays
                // within the accumulator (TN is a multiple of 64); its stale
                // columns only lower the minimum.  With two epilogue groups
                // (registers capped lower) the columns are read 32 at a time;
                // every 8th tile of a warp checks the load's minimum against
                // the computed one (diagnostics).
                if constexpr (NG == 1) {
#pragma unroll 1
                    for (int c2 = 0; c2 < nch; c2 += 2) {
                        const long long l0 = TC_TIMED ? clock64() : 0;
                        const float m2 = tc::tmem_min64_wait(tcol + (uint32_t)(c2 * 32));
                        if (TC_TIMED) ld_cyc += clock64() - l0;
                        const bool need = act && (nst - c2 * 32 < 64 || m2 <= t);
                        if (!__any_sync(0xffffffffu, need)) continue;
                        const int ce = min(c2 + 2, nch);
#pragma unroll 1
                        for (int cc = c2; cc < ce; ++cc) {
                            uint32_t v[32];
                            const float mm = tc::tmem_ld32_min_wait(tcol + (uint32_t)(cc * 32), v);
                            if (act) examine(v, mm, grp, cc * 32, nst - cc * 32);
                        }
                    }
                } else {
#pragma unroll 1
                    for (int cc = 0; cc < nch; ++cc) {
                        uint32_t v[32];
                        const long long l0 = TC_TIMED ? clock64() : 0;
                        const float mm = tc::tmem_ld32_min_wait(tcol + (uint32_t)(cc * 32), v);
                        if (TC_TIMED) ld_cyc += clock64() - l0;
                        if (act) examine(v, mm, grp, cc * 32, nst - cc * 32);
                    }
                }
                ++ntile;
                const long long te2 = (TC_TIMED && warp == 0 && lane == 0) ? clock64() : 0;
                // every lane's TMEM reads are done and its candidates' points
                // are resolved: the accumulator and the row-group table go back
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) {
                    tc::mbar_arrive(&acc_empty[b], 1);
                    tc::mbar_arrive(&gr_empty[am.x], 1);
                }
                // the whole warp inserts its buffered candidates together, once
                // enough lanes hold some (one pass of the insertion code then
                // serves them all), a buffer is nearly full, or a few tiles have
                // passed; the insertion threshold only loosens meanwhile
                {
                    const unsigned pend = __ballot_sync(0xffffffffu, nb > 0);
                    if (pend) ++since_flush;
                    if (__popc(pend) >= flush_lanes(KC) || since_flush >= flush_tiles(KC) ||
                        __any_sync(0xffffffffu, nb >= CB - 2)) {
                        flush();
                        since_flush = 0;
                    }
                }
                const long long te3 = (TC_TIMED && warp == 0 && lane == 0) ? clock64() : 0;
                // publish this warp's bounds for the planner's next window (a
                // later publication only prunes later; any is valid)
                dirty |= __any_sync(0xffffffffu, changed);
                if (dirty && ++since_pub >= 4) {
                    float ub = fminf(Bd::ub(kd, qa), qc);
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
                    dirty = false;
                    since_pub = 0;
                }
                if (TC_TIMED && warp == 2 && lane == 0)
                    atomicAdd(&x.timers[TT_EPI_WORK_W2], (unsigned long long)(clock64() - te1));
                if (TC_TIMED && warp == 0 && lane == 0) {
                    atomicAdd(&x.timers[TT_EPI_WAIT], (unsigned long long)(te1 - te0));
                    atomicAdd(&x.timers[TT_EPI_WORK], (unsigned long long)(clock64() - te1));
                    atomicAdd(&x.timers[TT_EPI_LD], (unsigned long long)ld_cyc);
                    atomicAdd(&x.timers[TT_EPI_LOOP], (unsigned long long)(te2 - te1));
                    atomicAdd(&x.timers[TT_EPI_FLUSH], (unsigned long long)(te3 - te2));
                }
            }
        }
        // every role is done with the item or gave up; a failed item writes
        // nothing (its lists may be incomplete, and copies may still land in
        // the buffers the re-rank would reuse)
        __syncthreads();
        if (s_fail) break;
        if (epi && NG == 2) {
            // merge group 1's lists into group 0's
            float* smd = reinterpret_cast<float*>(smem);
            int32_t* smi = reinterpret_cast<int32_t*>(smem + kQB * KC * 4);
            if (grp_id == 1) {
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    smd[j * kQB + qt] = ld[j];
                    smi[j * kQB + qt] = li[j];
                }
            }
            tc::named_sync(1, 256);
            if (grp_id == 0) {
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    const float d = smd[j * kQB + qt];
                    const int i = smi[j * kQB + qt];
                    if (!listed(li, i) && key_less(d, i, ld[KC - 1], li[KC - 1])) list_insert(ld, li, d, i);
                }
            }
            // the re-rank below reuses the merge buffers: group 0 has read them
            tc::named_sync(1, 256);
        }
        if (epi && grp_id == 0) {
            // ---- finish the work item
            long long tf0 = TC_TIMED ? clock64() : 0;
            const float ubk = fminf(Bd::ub(list_at(ld, kq - 1), qa), qc);
            const float band = Bd::band(ubk, qa);
            const bool ovf = act && li[KC - 1] != kEmptyIdx && !(ld[KC - 1] > band);
            if (ovf) {
                a.fbq_list[atomicAdd(a.fbq_count, 1)] = make_int4(myq, blk, __float_as_int(ubk), 0);
            } else if (act) {
                // float64 re-rank of the band candidates in shared memory
                double* rd = reinterpret_cast<double*>(smem);
                int32_t* ri = reinterpret_cast<int32_t*>(smem + kQB * KC * 8);
                const float* qp = P.qpts + (int64_t)myq * DP;
                int nr = 0;
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    if (li[j] != kEmptyIdx && !(ld[j] > band)) {
                        rd[nr * kQB + qt] = exact_d2<DP>(qp, P.rpts + (int64_t)li[j] * DP);
                        ri[nr * kQB + qt] = P.ridx[li[j]];
                        ++nr;
                    }
                }
                n_re += nr;
                const int64_t base = (int64_t)P.qidx[myq] * kq;
                for (int j = 0; j < kq; ++j) {
                    int best = j;
                    for (int c = j + 1; c < nr; ++c)
                        if (key_less(rd[c * kQB + qt], ri[c * kQB + qt], rd[best * kQB + qt], ri[best * kQB + qt]))
                            best = c;
                    const double bd = rd[best * kQB + qt];
                    const int bix = ri[best * kQB + qt];
                    rd[best * kQB + qt] = rd[j * kQB + qt];
                    ri[best * kQB + qt] = ri[j * kQB + qt];
                    P.out_idx[base + j] = bix;
                    P.out_dist[base + j] = (float)sqrt(bd);
                }
            }
            if (TC_TIMED && qt == 0)
                atomicAdd(&x.timers[TT_EPI_FINISH], (unsigned long long)(clock64() - tf0));
        }
        __syncthreads();
    }
    if (s_fail) {
        // drain this CTA's own asynchronous work before TMEM and shared
        // memory are released: the planner's last NB slot fills (their bulk
        // copies) and the issuer's MMAs
        if (warp == PW && lane == 0) {
            const uint32_t i0 = otile > (uint32_t)NB ? otile - NB : 0u;
            for (uint32_t i = i0; i < otile; ++i) tc::mbar_wait(&op_full[i % NB], (i / NB) & 1u, kDrainPolls);
        }
        if (warp == MW && lane == 0)
            for (int b = 0; b < 2; ++b)
                if ((aused >> b) & 1u) tc::mbar_wait(&acc_full[b], ((aph >> b) & 1u) ^ 1u, kDrainPolls);
        if (tid == 0) atomicExch(x.err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == MW) tc::tmem_dealloc(tmem, 2 * TN);
    if (n_skip) atomicAdd(&a.stats[ST_SKIPPED], n_skip);
    if (n_eval) atomicAdd(&a.stats[ST_EVALUATED], n_eval);
    if (n_pp) atomicAdd(&a.stats[ST_POINT_PAIRS], n_pp);
    if (n_re) atomicAdd(&a.stats[ST_RERANK], n_re);
    if (TC_TIMED && n_ins) atomicAdd(&x.timers[TT_INSERTS], n_ins);
}

// The kernel allocates 2 TN TMEM columns; at most one CTA may be resident per
// SM: the request is raised above half the SM's shared memory.
template <int FMT, int DP, int KC, int NG>
inline size_t tc_smem_bytes() {
    int dev = 0, sm_total = 233472;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaGetLastError();
    size_t guard = (size_t)sm_total / 2 + 1024;
    size_t need = (size_t)TcSmem<FMT, DP, KC, NG>::BYTES;
    return need > guard ? need : guard;
}

// Diagnostic timers for the next tensor-core launches (null = off), and the
// stall diagnostic (non-zero: every block's planner waits on a barrier that
// nothing completes before its end markers).
extern unsigned long long* g_tc_timers;
extern int g_tc_stall;

// Operand formats a precision maps to (1 = BF16 request -> split BF16, 2 = TF32).
inline int tc_format(int fmt) { return fmt == 2 ? 2 : 3; }

template <int DP>
size_t tc_ops_row_bytes(int fmt) {
    return tc_format(fmt) == 2 ? (size_t)TcShape<2, DP>::RB : (size_t)TcShape<3, DP>::RB;
}

// Fill a reference tree's operand array (see k_tc_ops).
template <int DP>
int launch_tc_ops(const dtree_t* t, int fmt, int ls, void* out, cudaStream_t s) {
    const int64_t leaf0 = t->nleaves - 1;
    const int64_t rows = t->nleaves * ls;
    const int grid = (int)std::min<int64_t>((rows + 127) / 128, 152 * 16);
    auto kern = tc_format(fmt) == 2 ? k_tc_ops<2, DP> : k_tc_ops<3, DP>;
    DT_LAUNCH(kern, grid, 128, 0, s, t->pts, t->nbeg, t->ncnt, t->box, leaf0, t->nleaves, ls,
              static_cast<unsigned char*>(out));
    return DTREE_OK;
}

template <int DP>
int launch_tile_tc(const TileArgs& a, int fmt, int kc, int items, int* err, int spin, cudaStream_t s) {
    TcExtra x{err, spin, g_tc_timers, g_tc_stall};
    const int F = tc_format(fmt);
    // two epilogue groups where their lists leave room for a second group's
    // registers (ten warps put three on a sub-partition: 168 registers a
    // thread) and their scratch fits shared memory; else one group
#define DT_TC_CASE(FMTV, KCV)                                                              \
    if (F == FMTV && kc == KCV) {                                                          \
        constexpr int NGV = (KCV <= 32 && DP <= 32) ? 2 : 1;                               \
        auto kern = k_tile_tc<FMTV, DP, KCV, NGV>;                                         \
        size_t smem = tc_smem_bytes<FMTV, DP, KCV, NGV>();                                 \
        DT_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                      (int)smem));                                         \
        const int nt = 32 * (4 * NGV + 2);                                                 \
        int g = occupancy_grid((const void*)kern, nt, smem);                               \
        if (items < g) g = items > 0 ? items : 1;                                          \
        DT_LAUNCH(kern, g, nt, smem, s, a, x);                                             \
        return DTREE_OK;                                                                   \
    }
    DT_TC_CASE(2, 16)
    DT_TC_CASE(2, 24)
    DT_TC_CASE(2, 32)
    DT_TC_CASE(2, 48)
    DT_TC_CASE(2, 64)
    DT_TC_CASE(3, 16)
    DT_TC_CASE(3, 24)
    DT_TC_CASE(3, 32)
    DT_TC_CASE(3, 48)
    DT_TC_CASE(3, 64)
#undef DT_TC_CASE
    return DTREE_ERR_UNSUPPORTED;
}

}  // namespace dt
