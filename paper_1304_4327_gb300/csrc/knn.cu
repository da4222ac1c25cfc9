// knn.cu -- exact k-nearest-neighbour search (dtree_knn).
//
// The meta-algorithm of Curtin et al. (Section 2) with a kd-tree, a pruning
// dual-tree traversal, the kNN BaseCase (Algorithm 2) and the kNN Score
// (Algorithm 3), arranged for one GPU:
//
//   1. seed      every query block (the query-tree node at the level where
//                nodes hold <= query_block points) evaluates the reference
//                subtree its box centre falls into (greedy descent), so that
//                every query has k finite candidates before the traversal;
//   2. bounds    B_1(N) = max and A(N) = min of the blocks' k-th-distance
//                upper bounds over descendant blocks; B(N) = min over N and its
//                ancestors a of min(B_1(a), A(a) + 2 lambda(a)) -- the B of
//                Section 5 with B_2 = A + 2 lambda (kd internal nodes hold no
//                points, leaves have rho = lambda);
//   3. traverse  a level-synchronous pruning dual-tree traversal: every
//                frontier pair (N_q, N_r) is split into its child pairs
//                (a node at the bottom stands in for itself), each child pair
//                is scored with the box distance d_min and pruned when
//                d_min > B(N_q); surviving (block, reference leaf) pairs form
//                each block's candidate list;
//   4. basecase  one CTA per block streams its candidate leaves nearest-first,
//                keeps each query's candidate list, tightens the block's B as
//                the lists improve and skips leaves whose d_min exceeds it,
//                then re-ranks the candidates near the k-th distance in float64
//                and writes the outputs;
//   5. fallback  a query whose band of near-k-th candidates overflowed its
//                list is recomputed exactly in float64 over its block's
//                candidate leaves (one CTA per such query).
#include <algorithm>
#include <vector>

#include "knn_common.cuh"

namespace dt {

int occupancy_grid(const void* kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess)
        per = 1;
    cudaGetLastError();
    if (per < 1) per = 1;
    return sms * per;
}

namespace {

template <int DP>
__device__ __forceinline__ float point_box_d2(const float* c, const float* bx) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        float g = fmaxf(fmaxf(bx[j] - c[j], c[j] - bx[DP + j]), 0.f);
        s = fmaf(g, g, s);
    }
    return s;
}

// Box distance d_min(N_q, N_r) (kd-tree bound of Section 3), rounded down so
// that float32 rounding can only keep a pair the exact rule would prune.
template <int DP>
__device__ __forceinline__ float box_dmin_down(const float* a, const float* b) {
    const float4* al = reinterpret_cast<const float4*>(a);
    const float4* ah = reinterpret_cast<const float4*>(a + DP);
    const float4* bl = reinterpret_cast<const float4*>(b);
    const float4* bh = reinterpret_cast<const float4*>(b + DP);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < DP / 4; ++j) {
        float4 x = al[j], y = ah[j], u = bl[j], v = bh[j];
        float g0 = fmaxf(fmaxf(x.x - v.x, u.x - y.x), 0.f);
        float g1 = fmaxf(fmaxf(x.y - v.y, u.y - y.y), 0.f);
        float g2 = fmaxf(fmaxf(x.z - v.z, u.z - y.z), 0.f);
        float g3 = fmaxf(fmaxf(x.w - v.w, u.w - y.w), 0.f);
        s = fmaf(g0, g0, s);
        s = fmaf(g1, g1, s);
        s = fmaf(g2, g2, s);
        s = fmaf(g3, g3, s);
    }
    return __fmul_rd(__fsqrt_rd(s), 1.f - rel_eps<DP>());
}

template <int DP>
__global__ void k_seed(const float* qbox, const float* rbox, int64_t qblock0, int nblocks, int Ls,
                       int hr, int32_t* seed_leaf0, int32_t* seed_nleaf) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const float* qb = qbox + (qblock0 + b) * 2 * DP;
    float c[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) c[j] = 0.5f * (qb[j] + qb[DP + j]);
    int64_t n = 0;
    for (int L = 0; L < Ls; ++L) {
        int64_t l = 2 * n + 1, r = l + 1;
        float dl = point_box_d2<DP>(c, rbox + l * 2 * DP);
        float dr = point_box_d2<DP>(c, rbox + r * 2 * DP);
        n = dr < dl ? r : l;
    }
    int span = hr - Ls;
    seed_leaf0[b] = (int32_t)(((n + 1) << span) - 1 - (((int64_t)1 << hr) - 1));
    seed_nleaf[b] = 1 << span;
}

template <int DP>
__global__ void __launch_bounds__(256) k_expand(const float* __restrict__ qbox,
                                                const float* __restrict__ rbox,
                                                const float* __restrict__ Bq, const int2* fin,
                                                const int* nin, int2* fout, int* nout, int64_t cap,
                                                int4* outp, int* noutp, int64_t capp, int* bcount,
                                                int Lb, int hr, int64_t qblock0, int64_t rleaf0,
                                                const int32_t* sl0, const int32_t* sn, int* overflow,
                                                unsigned long long* stats) {
    const int n = (int)min((int64_t)*nin, cap);  // the counter runs past cap on overflow
    unsigned long long sc = 0, pr = 0, em = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int2 p = fin[i];
        int lq = level_of_node(p.x), lr = level_of_node(p.y);
        bool cq = lq < Lb, cr = lr < hr;
        bool qbot = (cq ? lq + 1 : lq) == Lb, rbot = (cr ? lr + 1 : lr) == hr;
        for (int a = 0; a < (cq ? 2 : 1); ++a) {
            int64_t qc = cq ? 2 * (int64_t)p.x + 1 + a : p.x;
            float B = Bq[qc];
            const float* qbx = qbox + qc * 2 * DP;
            for (int b = 0; b < (cr ? 2 : 1); ++b) {
                int64_t rc = cr ? 2 * (int64_t)p.y + 1 + b : p.y;
                float dmin = box_dmin_down<DP>(qbx, rbox + rc * 2 * DP);
                ++sc;
                if (dmin > B) {  // Score() = infinity: prune every descendant pair
                    ++pr;
                    continue;
                }
                if (qbot && rbot) {
                    int blk = (int)(qc - qblock0), leaf = (int)(rc - rleaf0);
                    int s0 = sl0[blk];
                    if (leaf >= s0 && leaf < s0 + sn[blk]) continue;  // evaluated by the seed
                    int pos = atomicAdd(noutp, 1);
                    if (pos < capp) {
                        // evaluation order: squared distance between the box centres
                        const float* rbx = rbox + rc * 2 * DP;
                        float o = 0.f;
#pragma unroll
                        for (int j = 0; j < DP; ++j) {
                            float t = 0.5f * (qbx[j] + qbx[DP + j]) - 0.5f * (rbx[j] + rbx[DP + j]);
                            o = fmaf(t, t, o);
                        }
                        outp[pos] = make_int4(blk, leaf, __float_as_int(dmin), __float_as_int(o));
                        atomicAdd(&bcount[blk], 1);
                        ++em;
                    } else {
                        *overflow = 1;
                    }
                } else {
                    int pos = atomicAdd(nout, 1);
                    if (pos < cap) fout[pos] = make_int2((int)qc, (int)rc);
                    else *overflow = 1;
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, off);
        pr += __shfl_xor_sync(0xffffffffu, pr, off);
        em += __shfl_xor_sync(0xffffffffu, em, off);
    }
    if ((threadIdx.x & 31) == 0 && sc) {
        atomicAdd(&stats[ST_SCORED], sc);
        atomicAdd(&stats[ST_PRUNED], pr);
        atomicAdd(&stats[ST_EMITTED], em);
    }
}

__global__ void k_fill(float* p, int64_t n, float v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// One warp per block: B_1 / A of the block from its queries' k-th keys, then
// pushed to every ancestor with monotone atomics (non-negative floats order
// like their bit patterns).
__global__ void k_block_bounds(const float* qub, const int32_t* qbeg, const int32_t* qcnt,
                               int64_t qblock0, int nblocks, float* B1n, float* An) {
    int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (w >= nblocks) return;
    int64_t node = qblock0 + w;
    int b = qbeg[node], c = qcnt[node];
    float mx = 0.f, mn = INFINITY;
    for (int i = lane; i < c; i += 32) {
        float ub = qub[b + i];
        mx = fmaxf(mx, ub);
        mn = fminf(mn, ub);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    }
    if (lane == 0) {
        B1n[node] = mx;
        An[node] = mn;
        for (int64_t p = node; p > 0;) {
            p = (p - 1) / 2;
            atomicMax(reinterpret_cast<int*>(&B1n[p]), __float_as_int(mx));
            atomicMin(reinterpret_cast<int*>(&An[p]), __float_as_int(mn));
        }
    }
}

__global__ void k_node_bounds(const float* B1n, const float* An, const float* lam, int64_t nn,
                              float* Bn) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    float B = INFINITY;
    for (int64_t a = i;; a = (a - 1) / 2) {
        B = fminf(B, fminf(B1n[a], __fadd_ru(An[a], 2.f * lam[a])));
        if (a == 0) break;
    }
    Bn[i] = B;
}

__global__ void __launch_bounds__(1024) k_scan(const int* cnt, int n, int64_t* off) {
    __shared__ int64_t buf[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        int i = base + threadIdx.x;
        int64_t v = i < n ? cnt[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int64_t t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) off[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void k_csr_fill(const int4* outp, int np, const int64_t* off, int* cur, int32_t* leaf,
                           float* dmin, float* key) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int4 e = outp[i];
    int64_t pos = off[e.x] + atomicAdd(&cur[e.x], 1);
    leaf[pos] = e.y;
    dmin[pos] = __int_as_float(e.z);
    key[pos] = __int_as_float(e.w);
}

}  // namespace

template <int DP>
int launch_expand(const float* qbox, const float* rbox, const float* Bq, const int2* fin,
                  const int* nin, int2* fout, int* nout, int64_t cap, int4* outp, int* noutp,
                  int64_t capp, int* bcount, int Lb, int hr, int64_t qblock0, int64_t rleaf0,
                  const int32_t* sl0, const int32_t* sn, int* overflow, unsigned long long* stats,
                  int grid, cudaStream_t s) {
    DT_LAUNCH(k_expand<DP>, grid, 256, 0, s, qbox, rbox, Bq, fin, nin, fout, nout, cap, outp, noutp,
              capp, bcount, Lb, hr, qblock0, rleaf0, sl0, sn, overflow, stats);
    return DTREE_OK;
}

template <int DP>
int launch_seed(const float* qbox, const float* rbox, int64_t qblock0, int nblocks, int Ls, int hr,
                int32_t* seed_leaf0, int32_t* seed_nleaf, cudaStream_t s) {
    DT_LAUNCH(k_seed<DP>, (nblocks + 127) / 128, 128, 0, s, qbox, rbox, qblock0, nblocks, Ls, hr,
              seed_leaf0, seed_nleaf);
    return DTREE_OK;
}

namespace {

// Phase timer: CUDA events on the call's stream, only when stats are wanted.
struct PhaseTimer {
    cudaStream_t s;
    bool on;
    cudaEvent_t ev[8] = {};
    int n = 0;
    PhaseTimer(cudaStream_t st, bool enabled) : s(st), on(enabled) {}
    void mark() {
        if (!on || n >= 8) return;
        if (cudaEventCreate(&ev[n]) == cudaSuccess && cudaEventRecord(ev[n], s) == cudaSuccess) ++n;
        cudaGetLastError();
    }
    int64_t ns(int a, int b) const {
        float ms = 0.f;
        if (!on || b >= n || cudaEventElapsedTime(&ms, ev[a], ev[b]) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return (int64_t)(ms * 1e6);
    }
    ~PhaseTimer() {
        for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
    }
};

// Per-call scratch: from the device's stream-ordered pool, or (arena set)
// carved from a fixed device range with no allocation at all.  In the range,
// blocks are 256-byte aligned and releasing the most recent block gives its
// bytes back; other releases keep them until the call ends.
struct Pool {
    static constexpr int kMaxBlocks = 64;
    cudaStream_t s;
    const ScratchArena* arena = nullptr;
    size_t top = 0;
    int nblk = 0;
    size_t blk_from[kMaxBlocks];
    void* blk_ptr[kMaxBlocks];
    std::vector<void*> ptrs;

    // bytes still free in the range after alignment (0 without a range)
    size_t left() const {
        if (!arena) return 0;
        const size_t off = (top + 255) & ~(size_t)255;
        return off < arena->bytes ? arena->bytes - off : 0;
    }
    template <class T>
    int get(T** p, size_t count) {
        if (arena) {
            *p = nullptr;
            if (count == 0) return DTREE_OK;
            const size_t off = (top + 255) & ~(size_t)255;
            if (nblk >= kMaxBlocks || off > arena->bytes || count > (arena->bytes - off) / sizeof(T))
                return DTREE_ERR_TOO_LARGE;
            *p = reinterpret_cast<T*>(arena->base + off);
            blk_from[nblk] = top;
            blk_ptr[nblk] = *p;
            ++nblk;
            top = off + count * sizeof(T);
            return DTREE_OK;
        }
        int rc = scratch(p, count, s);
        if (rc == DTREE_OK && *p) ptrs.push_back(*p);
        return rc;
    }
    void release(void* p) {
        if (arena) {
            if (nblk > 0 && blk_ptr[nblk - 1] == p) top = blk_from[--nblk];
            return;
        }
        for (auto& q : ptrs)
            if (q == p) {
                cudaFreeAsync(q, s);
                q = nullptr;
            }
    }
    ~Pool() {
        for (void* p : ptrs)
            if (p) cudaFreeAsync(p, s);
    }
};

#define DT_TRY(x)                        \
    do {                                 \
        int rc_ = (x);                   \
        if (rc_ != DTREE_OK) return rc_; \
    } while (0)

// Candidate-list lengths come in buckets of 4, 8, 16, 24 and 32.
inline int kc_bucket(int need) {
    return need <= 4 ? 4 : need <= 8 ? 8 : need <= 16 ? 16 : need <= 24 ? 24 : 32;
}

template <int DP>
int knn_impl(const dtree_t* tq, const dtree_t* tr, bool mono, int k, int64_t* out_idx,
             float* out_dist, int qb_cap, int seed_pts, int prec, int spin, cudaStream_t s,
             dtree_stats* st, const ScratchArena* arena) {
    const int64_t launches0 = g_launches.load();
    const int64_t nq = tq->n, m = tr->n;
    const int Lb = std::min<int>(tq->height, level_of_count(nq, qb_cap));
    const int nblocks = 1 << Lb;
    const int64_t qblock0 = nblocks - 1;
    const int64_t maxcnt = (nq + nblocks - 1) / nblocks;
    const int cpb = (int)((maxcnt + kQB - 1) / kQB);
    const int hr = tr->height;
    const int64_t rleaf0 = ((int64_t)1 << hr) - 1;
    // list length: room for k plus the candidates inside the error band (the
    // tensor-core band is wider, so its lists are longer)
    const int fmt = prec == DTREE_PREC_BF16 ? 1 : prec == DTREE_PREC_TF32 ? 2 : 0;
    // list length: k plus room for the candidates inside the error band
    // (TF32 and split BF16 bands ~1% of d^2 at d=16, single BF16 ~5%, used
    // beyond 32 dimensions); buckets 4, 8, 16, 24, 32
    const int kc_need = fmt == 1 ? (DP <= 32 ? k + 14 : 2 * k + 12) : fmt == 2 ? k + 14 : k + 1;
    const int KC = kc_bucket(kc_need);
    if (k + 1 > 32) return DTREE_ERR_UNSUPPORTED;
    int Ls = 0;
    while (Ls < hr && (m >> (Ls + 1)) >= seed_pts) ++Ls;

    Pool P;
    P.s = s;
    P.arena = arena;
    int32_t *sl0, *sn, *cand_i, *csr_leaf = nullptr;
    int4 *fbq_list, *fbq2_list;
    float *cand_d, *B1n, *An, *Bn, *csr_dmin = nullptr, *csr_key = nullptr;
    int *ctr, *bcount, *bcur;
    int64_t* off;
    unsigned long long* dstats;
    const int64_t nqn = 2 * (int64_t)nblocks - 1;
    DT_TRY(P.get(&sl0, nblocks));
    DT_TRY(P.get(&sn, nblocks));
    DT_TRY(P.get(&cand_d, (size_t)KC * nq));
    DT_TRY(P.get(&cand_i, (size_t)KC * nq));
    float* qub;
    int* derr;
    DT_TRY(P.get(&qub, nq));
    DT_TRY(P.get(&derr, 1));
    DT_CHECK(cudaMemsetAsync(derr, 0, sizeof(int), s));
    DT_TRY(P.get(&B1n, nqn));
    DT_TRY(P.get(&An, nqn));
    DT_TRY(P.get(&Bn, nqn));
    // 0-2 work counters, 3 fb count, 4 overflow, 5-6 frontier, 7 pairs, 8 fb2 count, 9 work
    DT_TRY(P.get(&ctr, 16));
    DT_TRY(P.get(&bcount, nblocks));
    DT_TRY(P.get(&bcur, nblocks));
    DT_TRY(P.get(&fbq_list, nq));
    DT_TRY(P.get(&fbq2_list, nq));
    DT_TRY(P.get(&off, nblocks + 1));
    DT_TRY(P.get(&dstats, ST_NSTAT));
    DT_CHECK(cudaMemsetAsync(ctr, 0, 16 * sizeof(int), s));

    DT_CHECK(cudaMemsetAsync(dstats, 0, ST_NSTAT * sizeof(unsigned long long), s));
    PhaseTimer tm(s, st != nullptr);
    tm.mark();  // 0

    // 1. seed
    DT_TRY(launch_seed<DP>(tq->box, tr->box, qblock0, nblocks, Ls, hr, sl0, sn, s));
    TileArgs a{};
    a.qpts = tq->pts;
    a.qidx = tq->idx;
    a.qbeg = tq->nbeg;
    a.qcnt = tq->ncnt;
    a.qlam = tq->lam;
    a.qbox = tq->box;
    a.qblock0 = qblock0;
    a.nq = nq;
    a.cpb = cpb;
    a.rpts = tr->pts;
    a.ridx = tr->idx;
    a.rbeg = tr->nbeg;
    a.rcnt = tr->ncnt;
    a.rbox = tr->box;
    a.rleaf0 = rleaf0;
    a.k = k;
    a.mono = mono ? 1 : 0;
    a.seed_leaf0 = sl0;
    a.seed_nleaf = sn;
    a.cand_d = cand_d;
    a.cand_i = cand_i;
    a.qub = qub;
    a.nwork = nblocks;
    a.out_idx = out_idx;
    a.out_dist = out_dist;
    a.fbq_list = fbq_list;
    a.fbq_count = ctr + 3;
    a.fbq2_list = fbq2_list;
    a.fbq2_count = ctr + 8;
    a.stats = dstats;
    a.work_ctr = ctr + 0;
    auto tile = [&](int mode, int items) -> int {
        if (fmt)
            return launch_tile_tc<DP>(a, fmt, KC, mode, items, derr, spin, s);
        return launch_tile_cc<DP>(a, KC, mode, items, s);
    };
    // the seed pass runs on the CUDA cores whatever the precision: its lists
    // start empty, so nearly every early candidate is an insertion, which the
    // float32 tile does cheaply; its keys (relative error <= rel_eps) are
    // tighter than any tensor-core key, so the main pass's bounds hold for them
    // with lists of bucket(k + 1) entries (the float32 band needs no more)
    a.kc_rows = KC;
    DT_TRY(launch_tile_cc<DP>(a, kc_bucket(k + 1), MODE_SEED, nblocks * cpb, s));
    tm.mark();  // 1

    // 2. bounds of every query node down to the blocks
    DT_LAUNCH(k_fill, (int)((nqn + 255) / 256), 256, 0, s, B1n, nqn, 0.f);
    DT_LAUNCH(k_fill, (int)((nqn + 255) / 256), 256, 0, s, An, nqn, INFINITY);
    DT_LAUNCH(k_block_bounds, (nblocks * 32 + 255) / 256, 256, 0, s, qub, tq->nbeg, tq->ncnt,
              qblock0, nblocks, B1n, An);
    DT_LAUNCH(k_node_bounds, (int)((nqn + 255) / 256), 256, 0, s, B1n, An, tq->lam, nqn, Bn);

    // 3. level-synchronous pruning dual-tree traversal
    const int steps = std::max(1, std::max(Lb, hr));
    int64_t cap = std::max<int64_t>(tr->cap_hint, std::max<int64_t>(1 << 20, (int64_t)nblocks * 256));
    if (arena) {
        // a fixed range: the pair buffers take what is left, once (the three
        // blocks' alignment costs at most 3 x 255 bytes)
        const size_t per = sizeof(int4) + 2 * sizeof(int2);
        const size_t room = P.left();
        cap = room > 1024 ? (int64_t)std::min<size_t>((room - 1024) / per, (size_t)1 << 30) : 0;
        if (cap < 1) return DTREE_ERR_TOO_LARGE;
    }
    const int egrid = occupancy_grid((const void*)k_expand<DP>, 256, 0);
    int np = 0;
    int4* outp = nullptr;
    auto finish_csr = [&](int npairs) -> int {
        np = npairs;
        DT_TRY(P.get(&csr_leaf, std::max(np, 1)));
        DT_TRY(P.get(&csr_dmin, std::max(np, 1)));
        DT_TRY(P.get(&csr_key, std::max(np, 1)));
        DT_LAUNCH(k_scan, 1, 1024, 0, s, bcount, nblocks, off);
        DT_CHECK(cudaMemsetAsync(bcur, 0, nblocks * sizeof(int), s));
        if (np > 0)
            DT_LAUNCH(k_csr_fill, (np + 255) / 256, 256, 0, s, outp, np, off, bcur, csr_leaf,
                      csr_dmin, csr_key);
        P.release(outp);
        return DTREE_OK;
    };
    const int2 root = make_int2(0, 0);
    const int one = 1;
    if (!arena) {
        // Buffers sized level by level: a frontier pair has at most four child
        // pairs, so before each level the output frontier and the candidate
        // buffer get room for four times the current frontier (the frontier
        // size is read back after every level).
        int2* F[2];
        int64_t fcap[2] = {cap, cap}, ocap = cap;
        DT_TRY(P.get(&outp, ocap));
        DT_TRY(P.get(&F[0], fcap[0]));
        DT_TRY(P.get(&F[1], fcap[1]));
        DT_CHECK(cudaMemsetAsync(bcount, 0, nblocks * sizeof(int), s));
        DT_CHECK(cudaMemsetAsync(ctr + 4, 0, 4 * sizeof(int), s));
        DT_CHECK(cudaMemcpyAsync(F[0], &root, sizeof(int2), cudaMemcpyHostToDevice, s));
        DT_CHECK(cudaMemcpyAsync(ctr + 5, &one, sizeof(int), cudaMemcpyHostToDevice, s));
        int* nc[2] = {ctr + 5, ctr + 6};
        int cur = 0;
        int64_t nf = 1, used = 0;
        for (int t = 0; t < steps && nf > 0; ++t) {
            const int nx = cur ^ 1;
            const int64_t need = 4 * nf;
            if (need > ((int64_t)1 << 31) - 1 || used + need > ((int64_t)1 << 31) - 1)
                return DTREE_ERR_OOM;  // pair counters are 32-bit
            if (fcap[nx] < need) {
                P.release(F[nx]);
                fcap[nx] = std::max(need, 2 * fcap[nx]);
                DT_TRY(P.get(&F[nx], fcap[nx]));
            }
            if (ocap - used < need) {
                int4* o2;
                const int64_t oc2 = std::max(used + need, 2 * ocap);
                DT_TRY(P.get(&o2, oc2));
                if (used > 0)
                    DT_CHECK(cudaMemcpyAsync(o2, outp, used * sizeof(int4), cudaMemcpyDeviceToDevice, s));
                P.release(outp);
                outp = o2;
                ocap = oc2;
            }
            DT_CHECK(cudaMemsetAsync(nc[nx], 0, sizeof(int), s));
            DT_TRY(launch_expand<DP>(tq->box, tr->box, Bn, F[cur], nc[cur], F[nx], nc[nx], fcap[nx],
                                     outp, ctr + 7, ocap, bcount, Lb, hr, qblock0, rleaf0, sl0, sn,
                                     ctr + 4, dstats, egrid, s));
            int hv[4];
            DT_CHECK(cudaMemcpyAsync(hv, ctr + 4, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
            DT_CHECK(cudaStreamSynchronize(s));
            if (hv[0]) return DTREE_ERR_CUDA;  // cannot happen: the buffers were sized for it
            nf = hv[1 + nx];
            used = hv[3];
            cur = nx;
        }
        P.release(F[1]);
        P.release(F[0]);
        cap = std::max(fcap[0], std::max(fcap[1], ocap));
        DT_TRY(finish_csr((int)used));
    } else {
        // a fixed range: one pass with the capacity it has left
        int2 *F0, *F1;
        // in this order, so that releasing F1 then F0 frees the frontier for
        // the candidate arrays
        DT_TRY(P.get(&outp, cap));
        DT_TRY(P.get(&F0, cap));
        DT_TRY(P.get(&F1, cap));
        DT_CHECK(cudaMemsetAsync(bcount, 0, nblocks * sizeof(int), s));
        DT_CHECK(cudaMemsetAsync(ctr + 4, 0, 4 * sizeof(int), s));
        DT_CHECK(cudaMemcpyAsync(F0, &root, sizeof(int2), cudaMemcpyHostToDevice, s));
        DT_CHECK(cudaMemcpyAsync(ctr + 5, &one, sizeof(int), cudaMemcpyHostToDevice, s));
        int2 *fi = F0, *fo = F1;
        int *ni = ctr + 5, *no = ctr + 6;
        for (int t = 0; t < steps; ++t) {
            DT_CHECK(cudaMemsetAsync(no, 0, sizeof(int), s));
            DT_TRY(launch_expand<DP>(tq->box, tr->box, Bn, fi, ni, fo, no, cap, outp, ctr + 7, cap,
                                     bcount, Lb, hr, qblock0, rleaf0, sl0, sn, ctr + 4, dstats,
                                     egrid, s));
            std::swap(fi, fo);
            std::swap(ni, no);
        }
        int hv[4];
        DT_CHECK(cudaMemcpyAsync(hv, ctr + 4, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        DT_CHECK(cudaStreamSynchronize(s));
        P.release(F1);
        P.release(F0);
        if (hv[0]) return DTREE_ERR_TOO_LARGE;  // the fixed range holds no more pairs
        DT_TRY(finish_csr(hv[3]));
    }
    if (!arena) const_cast<dtree_t*>(tr)->cap_hint = cap;
    tm.mark();  // 2

    // 4. BaseCase over the candidates with the tightening bound, re-rank, output
    a.csr_off = off;
    a.csr_leaf = csr_leaf;
    a.csr_dmin = csr_dmin;
    a.csr_key = csr_key;
    a.Bq = Bn + qblock0;
    a.work_ctr = ctr + 1;
    DT_TRY(tile(MODE_MAIN, nblocks * cpb));
    tm.mark();  // 3
    int nfb = 0, herr = 0;
    DT_CHECK(cudaMemcpyAsync(&nfb, ctr + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    DT_CHECK(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    DT_CHECK(cudaStreamSynchronize(s));
    if (herr) return DTREE_ERR_TIMEOUT;

    // 5. recomputation of the queries whose band overflowed: float32 keys
    //    with a float64 re-rank of their band, and exact float64 for those
    //    whose float32 band overflows too
    int nfb2 = 0;
    if (nfb > 0) {
        DT_TRY(launch_query_fb<DP>(a, KC, nfb, false, s));
        DT_CHECK(cudaMemcpyAsync(&nfb2, ctr + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
        DT_CHECK(cudaStreamSynchronize(s));
        if (nfb2 > 0) DT_TRY(launch_query_fb<DP>(a, KC, nfb2, true, s));
    }
    tm.mark();  // 4
    unsigned long long hs[ST_NSTAT];
    DT_CHECK(cudaMemcpyAsync(hs, dstats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    DT_CHECK(cudaStreamSynchronize(s));
    if (st) {
        memset(st, 0, sizeof(*st));
        st->node_pairs_scored = (int64_t)hs[ST_SCORED];
        st->node_pairs_pruned = (int64_t)hs[ST_PRUNED];
        st->leaf_pairs_emitted = (int64_t)hs[ST_EMITTED];
        st->leaf_pairs_skipped = (int64_t)hs[ST_SKIPPED];
        st->leaf_pairs_evaluated = (int64_t)hs[ST_EVALUATED];
        st->point_pairs = (int64_t)hs[ST_POINT_PAIRS];
        st->seed_point_pairs = (int64_t)hs[ST_SEED_PAIRS];
        st->rerank_candidates = (int64_t)hs[ST_RERANK];
        st->fallback_queries = nfb;
        st->fallback64_queries = nfb2;
        st->query_blocks = nblocks;
        st->kernel_launches = g_launches.load() - launches0;
        st->ns_seed = tm.ns(0, 1);
        st->ns_traverse = tm.ns(1, 2);
        st->ns_basecase = tm.ns(2, 3);
        st->ns_fallback = tm.ns(3, 4);
    }
    return DTREE_OK;
}

}  // namespace

int knn_entry(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
              float* out_dist, const dtree_opts* o, void* stream, dtree_stats* st,
              const ScratchArena* arena) {
    if (st) memset(st, 0, sizeof(*st));
    if (!ref) return DTREE_ERR_INVALID_ARG;
    const bool mono = query == nullptr || query == ref;
    const dtree_t* tq = mono ? ref : query;
    const int64_t m = ref->n;
    if (k <= 0 || (mono ? (int64_t)k > m - 1 : (int64_t)k >= m)) return DTREE_ERR_INVALID_K;
    if (!out_idx || !out_dist || tq->d != ref->d) return DTREE_ERR_INVALID_ARG;
    if (o)
        for (int i = 0; i < 10; ++i)
            if (o->reserved[i]) return DTREE_ERR_INVALID_ARG;
    const int prec = o ? o->precision : DTREE_PREC_FP32;
    if (prec < DTREE_PREC_FP32 || prec > DTREE_PREC_BF16) return DTREE_ERR_INVALID_ARG;
    int qb = (o && o->query_block) ? o->query_block : 128;
    if (qb < 16 || qb > 128) return DTREE_ERR_INVALID_ARG;
    if (o && o->proposal) return DTREE_ERR_NOT_TRAINED;
    int seed = std::max<int>(k + 1, (o && o->seed_points > 0) ? o->seed_points : 512);
    int spin = (o && o->spin_budget > 0) ? o->spin_budget : (1 << 20);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    if (arena) {
        if (ref->device != dev || tq->device != dev) return DTREE_ERR_INVALID_ARG;
    } else {
        prepare_pool(dev);
    }
    if (prec != DTREE_PREC_FP32) {
        // the tensor-core tiles are built for sm_103a (tcgen05)
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (major != 10 || minor != 3) return DTREE_ERR_UNSUPPORTED;
    }
    int rc;
    switch (ref->dp) {
        case 4: rc = knn_impl<4>(tq, ref, mono, k, out_idx, out_dist, qb, seed, prec, spin, s, st, arena); break;
        case 8: rc = knn_impl<8>(tq, ref, mono, k, out_idx, out_dist, qb, seed, prec, spin, s, st, arena); break;
        case 16: rc = knn_impl<16>(tq, ref, mono, k, out_idx, out_dist, qb, seed, prec, spin, s, st, arena); break;
        case 32: rc = knn_impl<32>(tq, ref, mono, k, out_idx, out_dist, qb, seed, prec, spin, s, st, arena); break;
        default: rc = knn_impl<64>(tq, ref, mono, k, out_idx, out_dist, qb, seed, prec, spin, s, st, arena); break;
    }
    if (rc != DTREE_OK) cudaStreamSynchronize(s);
    return rc;
}

}  // namespace dt

extern "C" int dtree_knn(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
                         float* out_dist, const dtree_opts* o, void* stream, dtree_stats* st) {
    return dt::knn_entry(query, ref, k, out_idx, out_dist, o, stream, st, nullptr);
}
