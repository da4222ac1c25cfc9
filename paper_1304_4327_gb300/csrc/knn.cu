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
    // a few float4 groups in flight per thread, not all of them: the
    // registers of a full unroll at d = 64 would leave one CTA per SM
#pragma unroll 4
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

// The same box distance and, from the same loads, the squared distance
// between the two box centres (the candidate order of a leaf pair).
template <int DP>
__device__ __forceinline__ float box_dmin_centre(const float* a, const float* b, float& o) {
    const float4* al = reinterpret_cast<const float4*>(a);
    const float4* ah = reinterpret_cast<const float4*>(a + DP);
    const float4* bl = reinterpret_cast<const float4*>(b);
    const float4* bh = reinterpret_cast<const float4*>(b + DP);
    float s = 0.f, c = 0.f;
#pragma unroll 4
    for (int j = 0; j < DP / 4; ++j) {
        const float4 x = al[j], y = ah[j], u = bl[j], v = bh[j];
        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
        const float us[4] = {u.x, u.y, u.z, u.w}, vs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float g = fmaxf(fmaxf(xs[t] - vs[t], us[t] - ys[t]), 0.f);
            s = fmaf(g, g, s);
            const float w = 0.5f * (xs[t] + ys[t]) - 0.5f * (us[t] + vs[t]);
            c = fmaf(w, w, c);
        }
    }
    o = c;
    return __fmul_rd(__fsqrt_rd(s), 1.f - rel_eps<DP>());
}

template <int DP>
__global__ void k_seed(const ProbDev* probs, const int32_t* blk_prob, int nblocks, int slots,
                       int32_t* seed_leaf0, int32_t* seed_nleaf) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nblocks) return;
    const ProbDev& P = probs[blk_prob[g]];
    const float* qb = P.qbox + (P.qblock0 + (g - P.block0)) * 2 * DP;
    const float* rbox = P.rbox;
    float c[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) c[j] = 0.5f * (qb[j] + qb[DP + j]);
    int64_t n = 0;
    for (int L = 0; L < P.Ls; ++L) {
        int64_t l = 2 * n + 1, r = l + 1;
        float dl, dr;
        if (P.bound == DTREE_BOUND_BOX) {
            dl = point_box_d2<DP>(c, rbox + l * 2 * DP);
            dr = point_box_d2<DP>(c, rbox + r * 2 * DP);
        } else {  // nearer by the search's bound (an order only: any choice is exact)
            dl = point_dmin_down<DP>(P.bound, c, rbox + l * 2 * DP, P.rlam[l]);
            dr = point_dmin_down<DP>(P.bound, c, rbox + r * 2 * DP, P.rlam[r]);
        }
        n = dr < dl ? r : l;
    }
    const int span = P.hr - P.Ls;
    seed_leaf0[g * slots] = (int32_t)(((n + 1) << span) - 1 - P.rleaf0);
    seed_nleaf[g * slots] = 1 << span;
    for (int s = 1; s < slots; ++s) {
        seed_leaf0[g * slots + s] = 0;
        seed_nleaf[g * slots + s] = 0;
    }
}

// Slots 1..M of each block's seed: its proposed cells (subtrees at the
// proposal's cell level), skipping any cell that overlaps the seed so far.
__global__ void k_seed_proposal(const ProbDev* probs, const int32_t* blk_prob, int nblocks,
                                int slots, const int32_t* cells, int M, int32_t* seed_leaf0,
                                int32_t* seed_nleaf) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nblocks) return;
    const ProbDev& P = probs[blk_prob[g]];
    const int span = P.hr - P.Lp;
    int used = 1;
    for (int m = 0; m < M && used < slots; ++m) {
        const int l0 = cells[(int64_t)g * M + m] << span, nl = 1 << span;
        // the slots must stay disjoint (every later pass counts a seed leaf
        // once): a cell that overlaps one already in the seed is skipped
        bool dup = false;
        for (int s = 0; s < used; ++s) {
            const int s0 = seed_leaf0[g * slots + s], sn = seed_nleaf[g * slots + s];
            dup |= l0 < s0 + sn && s0 < l0 + nl;
        }
        if (dup) continue;
        seed_leaf0[g * slots + used] = l0;
        seed_nleaf[g * slots + used] = nl;
        ++used;
    }
}

constexpr int kExpandProbs = 64;

template <int DP>
__global__ void __launch_bounds__(256, 2) k_expand(const ProbDev* __restrict__ probs,
                                                const int32_t* __restrict__ node_prob,
                                                const float* __restrict__ Bn, const int2* fin,
                                                const int* nin, int2* fout, int* nout, int64_t cap,
                                                int4* outp, int* noutp, int64_t capp, int* bcount,
                                                const int32_t* sl0, const int32_t* sn, int slots,
                                                int* overflow, unsigned long long* stats, int np) {
    // the first kExpandProbs problems' descriptors are staged in shared memory
    extern __shared__ ProbDev sprob[];
    __shared__ int s_stop;
    // a fixed-range traversal whose pair storage already overflowed (an
    // earlier level) expands no further: its call returns DTREE_ERR_TOO_LARGE
    if (threadIdx.x == 0) s_stop = *reinterpret_cast<volatile int*>(overflow);
    for (int p = threadIdx.x; p < min(np, kExpandProbs); p += blockDim.x) sprob[p] = probs[p];
    __syncthreads();
    if (s_stop) return;  // uniform over the CTA
    const int n = (int)min((int64_t)*nin, cap);  // the counter runs past cap on overflow
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long sc = 0, pr = 0, em = 0;
    // Warps walk the frontier in step.  Each frontier pair has up to four
    // child pairs (slot s = 2a + b); slot by slot, every lane scores its child
    // and the warp appends the slot's candidates and frontier pairs with one
    // atomic each, in lane order: every lane's first child, then every lane's
    // second child, ...  (the order of per-thread appends, which keeps the
    // traversal's spatial order in the lists).
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int i = base + lane;
        const bool live = i < n;
        int2 pq = make_int2(0, 0);
        const ProbDev* Pp = sprob;
        if (live) {
            pq = fin[i];  // (global query node, reference node)
            const int pi = np == 1 ? 0 : node_prob[pq.x];
            Pp = pi < kExpandProbs ? &sprob[pi] : &probs[pi];
        }
        // the problem's fields, read once
        const int64_t node0 = Pp->node0, qblock0 = Pp->qblock0, rleaf0 = Pp->rleaf0;
        const float* __restrict__ qbox = Pp->qbox;
        const float* __restrict__ rbox = Pp->rbox;
        const float* __restrict__ qlam = Pp->qlam;
        const float* __restrict__ rlam = Pp->rlam;
        const int bound = Pp->bound;
        const int Lb = Pp->Lb, hr = Pp->hr, block0 = Pp->block0;
        const int64_t qloc = pq.x - node0;
        const int lq = level_of_node(qloc), lr = level_of_node(pq.y);
        const bool cq = lq < Lb, cr = lr < hr;
        const bool qbot = (cq ? lq + 1 : lq) == Lb, rbot = (cr ? lr + 1 : lr) == hr;
#pragma unroll 1
        for (int slot = 0; slot < 4; ++slot) {
            const int a = slot >> 1, b = slot & 1;
            bool do_emit = false, do_push = false;
            int4 e4 = make_int4(0, 0, 0, 0);
            int2 f2 = make_int2(0, 0);
            if (live && (a == 0 || cq) && (b == 0 || cr)) {
                const int64_t qc = cq ? 2 * qloc + 1 + a : qloc;
                const int64_t rc = cr ? 2 * (int64_t)pq.y + 1 + b : pq.y;
                const float* qbx = qbox + qc * 2 * DP;
                const float* rbx = rbox + rc * 2 * DP;
                // d_min under the search's bound: box, ball, or the larger;
                // for a leaf pair also the centres' squared distance (its
                // order among the candidates), from the same box loads
                const bool leaves = qbot && rbot;
                float o = -1.f;
                float dmin = bound == DTREE_BOUND_BALL ? 0.f
                             : leaves                  ? box_dmin_centre<DP>(qbx, rbx, o)
                                                       : box_dmin_down<DP>(qbx, rbx);
                if (bound != DTREE_BOUND_BOX)
                    dmin = fmaxf(dmin, ball_dmin_down<DP>(qbx, qlam[qc], rbx, rlam[rc]));
                ++sc;
                if (dmin > Bn[node0 + qc]) {  // Score() = infinity: prune every descendant pair
                    ++pr;
                } else if (leaves) {
                    const int blk = block0 + (int)(qc - qblock0);
                    const int leaf = (int)(rc - rleaf0);
                    if (!in_seed(sl0, sn, slots, blk, leaf)) {  // else evaluated by the seed
                        // evaluation order: squared distance between the box centres
                        if (o < 0.f) {
                            o = 0.f;
#pragma unroll
                            for (int j = 0; j < DP; ++j) {
                                float t = 0.5f * (qbx[j] + qbx[DP + j]) - 0.5f * (rbx[j] + rbx[DP + j]);
                                o = fmaf(t, t, o);
                            }
                        }
                        e4 = make_int4(blk, leaf, __float_as_int(dmin), __float_as_int(o));
                        do_emit = true;
                    }
                } else {
                    f2 = make_int2((int)(node0 + qc), (int)rc);
                    do_push = true;
                }
            }
            const unsigned me = __ballot_sync(0xffffffffu, do_emit);
            const unsigned mf = __ballot_sync(0xffffffffu, do_push);
            int be = 0, bf = 0;
            if (lane == 0) {
                if (me) be = atomicAdd(noutp, __popc(me));
                if (mf) bf = atomicAdd(nout, __popc(mf));
            }
            be = __shfl_sync(0xffffffffu, be, 0) + __popc(me & lt);
            bf = __shfl_sync(0xffffffffu, bf, 0) + __popc(mf & lt);
            const bool stored = do_emit && be < capp;
            const unsigned ms = __ballot_sync(0xffffffffu, stored);
            if (stored) {
                outp[be] = e4;
                ++em;
                // the block's count, one atomic per distinct block among the
                // warp's lanes (a frontier's pairs come grouped by query node)
                const unsigned peers = __match_any_sync(ms, e4.x);
                if (lane == __ffs(peers) - 1) atomicAdd(&bcount[e4.x], __popc(peers));
            } else if (do_emit) {
                *overflow = 1;
            }
            if (do_push) {
                if (bf < cap) fout[bf] = f2;
                else *overflow = 1;
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

// One warp per block: B_1 / A of the block from its queries' upper bounds on
// their k-th distances, then pushed to every ancestor with monotone atomics
// (non-negative floats order like their bit patterns).
__global__ void k_block_bounds(const ProbDev* probs, const int32_t* blk_prob, int nblocks,
                               const float* qub, float* B1n, float* An) {
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= nblocks) return;
    const ProbDev& P = probs[blk_prob[w]];
    const int64_t node = P.qblock0 + (w - P.block0);
    const int b = P.qbeg[node], c = P.qcnt[node];
    float mx = 0.f, mn = INFINITY;
    for (int i = lane; i < c; i += 32) {
        const float ub = qub[P.q0 + b + i];
        mx = fmaxf(mx, ub);
        mn = fminf(mn, ub);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    }
    if (lane == 0) {
        B1n[P.node0 + node] = mx;
        An[P.node0 + node] = mn;
        for (int64_t p = node; p > 0;) {
            p = (p - 1) / 2;
            atomicMax(reinterpret_cast<int*>(&B1n[P.node0 + p]), __float_as_int(mx));
            atomicMin(reinterpret_cast<int*>(&An[P.node0 + p]), __float_as_int(mn));
        }
    }
}

// B(N) = min over N and its ancestors a of min(B_1(a), A(a) + 2 lambda(a)).
__global__ void k_node_bounds(const ProbDev* probs, const int32_t* node_prob, const float* B1n,
                              const float* An, int64_t nn, float* Bn) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const ProbDev& P = probs[node_prob[i]];
    float B = INFINITY;
    for (int64_t a = i - P.node0;; a = (a - 1) / 2) {
        B = fminf(B, fminf(B1n[P.node0 + a], __fadd_ru(An[P.node0 + a], 2.f * P.qlam[a])));
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

// Scatter the candidate pairs into the per-block CSR.
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

// Order each block's candidate leaves for the BaseCase pass: the list keeps
// the traversal's order (leaves of one subtree together) in windows of
// kCsrSortCap, and each window is sorted by its order key (the squared
// distance between the block's and the leaf's box centres).  One CTA per
// block at a time, a bitonic sort per window in shared memory.
constexpr int kCsrSortCap = 1024;  // the window index takes the key's low bits
constexpr size_t kCsrSortSmem = (size_t)kCsrSortCap * (8 + 4 + 4);

__global__ void __launch_bounds__(256) k_csr_sort(const int64_t* off, int nb, int32_t* leaf,
                                                  float* dmin, const float* key) {
    extern __shared__ __align__(16) unsigned char csm[];
    uint64_t* sk = reinterpret_cast<uint64_t*>(csm);
    int32_t* tl = reinterpret_cast<int32_t*>(sk + kCsrSortCap);
    float* td = reinterpret_cast<float*>(tl + kCsrSortCap);
    const int tid = threadIdx.x;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t o0 = off[b], n = off[b + 1] - o0;  // uniform in the CTA
        for (int64_t w0 = 0; w0 + 1 < n; w0 += kCsrSortCap) {
            const int wn = (int)(n - w0 < kCsrSortCap ? n - w0 : kCsrSortCap);
            int np2 = 1;
            while (np2 < wn) np2 <<= 1;
            for (int i = tid; i < np2; i += blockDim.x) {
                uint64_t v = ~0ull;
                if (i < wn) {
                    const int64_t c = o0 + w0 + i;
                    v = ((uint64_t)f2o(key[c]) << 32) | (uint32_t)i;
                    tl[i] = leaf[c];
                    td[i] = dmin[c];
                }
                sk[i] = v;
            }
            __syncthreads();
            for (int kk = 2; kk <= np2; kk <<= 1)
                for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                    for (int t = tid; t < np2 / 2; t += blockDim.x) {
                        const int i = 2 * t - (t & (jj - 1));
                        const int l = i + jj;
                        const bool up = (i & kk) == 0;
                        const uint64_t x = sk[i], y = sk[l];
                        if ((x > y) == up) {
                            sk[i] = y;
                            sk[l] = x;
                        }
                    }
                    __syncthreads();
                }
            for (int i = tid; i < wn; i += blockDim.x) {
                const int j = (int)(uint32_t)sk[i];  // the window index (i < kCsrSortCap)
                const int64_t c = o0 + w0 + i;
                leaf[c] = tl[j];
                dmin[c] = td[j];
            }
            __syncthreads();
        }
    }
}

}  // namespace

template <int DP>
int launch_expand(const ProbDev* probs, const int32_t* node_prob, const float* Bn, const int2* fin,
                  const int* nin, int2* fout, int* nout, int64_t cap, int4* outp, int* noutp,
                  int64_t capp, int* bcount, const int32_t* sl0, const int32_t* sn, int slots,
                  int* overflow, unsigned long long* stats, int np, int grid, cudaStream_t s) {
    const size_t smem = (size_t)std::min(np, kExpandProbs) * sizeof(ProbDev);
    DT_LAUNCH(k_expand<DP>, grid, 256, smem, s, probs, node_prob, Bn, fin, nin, fout, nout, cap,
              outp, noutp, capp, bcount, sl0, sn, slots, overflow, stats, np);
    return DTREE_OK;
}

template <int DP>
int launch_seed(const ProbDev* probs, const int32_t* blk_prob, int nblocks, int slots,
                int32_t* seed_leaf0, int32_t* seed_nleaf, cudaStream_t s) {
    DT_LAUNCH(k_seed<DP>, (nblocks + 127) / 128, 128, 0, s, probs, blk_prob, nblocks, slots,
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


// Per block, query node and work item of a batch: the problem it belongs to
// (problems are laid out in order, so each lookup is a binary search over
// the problems' first entries), plus the traversal's root pairs.
__global__ void k_index(const ProbDev* probs, int np, int nb, int64_t nn, int ni,
                        int32_t* blk_prob, int32_t* node_prob, int2* items, int2* roots) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    auto find = [&](int64_t x, int which) {
        int lo = 0, hi = np - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const int64_t first = which == 0 ? probs[mid].block0 : which == 1 ? probs[mid].node0
                                                                              : probs[mid].item0;
            if (first <= x) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    if (t < nb) blk_prob[t] = find(t, 0);
    if (t < nn) node_prob[t] = find(t, 1);
    if (t < ni) {
        const int p = find(t, 2);
        const int local = (int)(t - probs[p].item0);
        items[t] = make_int2(probs[p].block0 + local / probs[p].cpb, local % probs[p].cpb);
    }
    if (t < np) roots[t] = make_int2((int)probs[t].node0, 0);
}

// One problem of a batch on the host side.
struct HostProb {
    const dtree_t* tq;
    const dtree_t* tr;
    bool mono;
    int k;
    int64_t* out_idx;
    float* out_dist;
    int qb;  // queries per block, or 0 for the call's option
    const dtree_model* prop;  // learned proposal to seed with, or null
};

// Candidate-list lengths come in buckets of 4, 8, 16, 24, 32, 48 and 64.
inline int kc_bucket(int need) {
    return need <= 4 ? 4 : need <= 8 ? 8 : need <= 16 ? 16 : need <= 24 ? 24 : need <= 32 ? 32
           : need <= 48 ? 48 : 64;
}

// The search for a batch of problems whose points share the padded dimension
// DP: every phase is one launch (or one per traversal level) over all the
// problems' blocks, pairs and queries.
template <int DP>
int knn_batch_impl(const HostProb* hp, int np, int qb_cap, int seed_pts, int cap_leaves, int prec, int spin,
                   int nprop, int bound, cudaStream_t s, dtree_stats* st, const ScratchArena* arena) {
    const int64_t launches0 = g_launches.load();
    const int fmt = prec == DTREE_PREC_BF16 ? 1 : prec == DTREE_PREC_TF32 ? 2 : 0;
    // list length: k plus room for the candidates inside the error band
    // (the TF32 and split-BF16 bands hold a few per cent more points than
    // k); buckets 4, 8, 16, 24, 32, 48, 64
    int kmax = 0;
    for (int i = 0; i < np; ++i) kmax = std::max(kmax, hp[i].k);
    const int kc_need = fmt ? kmax + 14 : kmax + 1;
    // lists hold up to 64 entries (k <= 63; a band wider than the list sends
    // its queries to the fallback)
    if (kmax + 1 > 64) return DTREE_ERR_UNSUPPORTED;
    const int KC = std::min(kc_bucket(kc_need), 64);

    // the problems' layout in the batch-wide arrays
    ProbDev one[1];
    std::vector<ProbDev> many;
    ProbDev* pd = one;
    if (np > 1) {
        many.resize(np);
        pd = many.data();
    }
    int64_t NQ = 0, NN = 0;
    int NB = 0, NI = 0, steps = 1;
    for (int i = 0; i < np; ++i) {
        const dtree_t *tq = hp[i].tq, *tr = hp[i].tr;
        ProbDev& P = pd[i];
        memset(&P, 0, sizeof(P));
        const int64_t nq = tq->n, m = tr->n;
        P.Lb = std::min<int>(tq->height, level_of_count(nq, hp[i].qb > 0 ? hp[i].qb : qb_cap));
        P.nblocks = 1 << P.Lb;
        P.qblock0 = P.nblocks - 1;
        const int64_t maxcnt = (nq + P.nblocks - 1) / P.nblocks;
        P.cpb = (int)((maxcnt + kQB - 1) / kQB);
        P.hr = tr->height;
        P.rleaf0 = ((int64_t)1 << P.hr) - 1;
        P.Ls = 0;
        {
            const int seed = std::max(hp[i].k + 1, seed_pts);
            while (P.Ls < P.hr && (m >> (P.Ls + 1)) >= seed) ++P.Ls;
        }
        P.Lp = nprop > 0 ? std::min(model_level(hp[i].prop), P.hr) : P.Ls;
        if (nprop > 0 && !fmt) {
            // the CUDA-core search evaluates the proposed cells in its seed
            // pass: its greedy subtree is a cell too, so that the two are
            // equal or disjoint
            P.Ls = P.Lp;
        }
        P.qpts = tq->pts;
        P.qidx = tq->idx;
        P.qbeg = tq->nbeg;
        P.qcnt = tq->ncnt;
        P.qlam = tq->lam;
        P.qbox = tq->box;
        P.rpts = tr->pts;
        P.ridx = tr->idx;
        P.rbeg = tr->nbeg;
        P.rcnt = tr->ncnt;
        P.rbox = tr->box;
        P.rlam = tr->lam;
        P.bound = bound;
        P.out_idx = hp[i].out_idx;
        P.out_dist = hp[i].out_dist;
        P.k = hp[i].k;
        P.mono = hp[i].mono ? 1 : 0;
        P.q0 = NQ;
        P.node0 = NN;
        P.block0 = NB;
        P.item0 = NI;
        NQ += nq;
        NN += 2 * (int64_t)P.nblocks - 1;
        NB += P.nblocks;
        NI += P.nblocks * P.cpb;
        steps = std::max(steps, std::max(P.Lb, P.hr));
    }
    if (NB > (1 << 30) || NI > (1 << 30) || NN > (1 << 30)) return DTREE_ERR_UNSUPPORTED;

    Pool P;
    P.s = s;
    P.arena = arena;
    if (fmt) {
        // the reference points as tensor-core operand rows (made once per
        // tree and format, or carved from the fixed range for this call)
        for (int i = 0; i < np; ++i) {
            const dtree_t* tr = hp[i].tr;
            const int64_t maxleaf = (tr->n + tr->nleaves - 1) / tr->nleaves;
            const int ls = (int)((maxleaf + 7) / 8 * 8);
            void*& cache = const_cast<dtree_t*>(tr)->tc_ops[fmt == 2 ? 0 : 1];
            void* ops = cache;
            if (!ops) {
                const size_t bytes = (size_t)tr->nleaves * ls * tc_ops_row_bytes<DP>(fmt);
                if (arena) {
                    unsigned char* p = nullptr;
                    DT_TRY(P.get(&p, bytes));
                    ops = p;
                } else {
                    g_allocs.fetch_add(1, std::memory_order_relaxed);
                    if (cudaMalloc(&ops, bytes) != cudaSuccess) {
                        cudaGetLastError();
                        return DTREE_ERR_OOM;
                    }
                    cache = ops;
                }
                DT_TRY(launch_tc_ops<DP>(tr, fmt, ls, ops, s));
            }
            pd[i].rops = ops;
            pd[i].rls8 = ls / 8;
        }
    }
    ProbDev* probs;
    int32_t *blk_prob, *node_prob, *sl0, *sn, *cand_i, *csr_leaf = nullptr;
    int2 *items, *roots;
    int4 *fbq_list, *fbq2_list;
    float *cand_d, *B1n, *An, *Bn, *csr_dmin = nullptr, *csr_key = nullptr, *qub;
    int *ctr, *bcount, *bcur, *derr;
    int64_t* off;
    unsigned long long* dstats;
    DT_TRY(P.get(&probs, np));
    DT_TRY(P.get(&blk_prob, NB));
    DT_TRY(P.get(&node_prob, NN));
    DT_TRY(P.get(&items, NI));
    DT_TRY(P.get(&roots, np));
    const int slots = 1 + nprop;
    DT_TRY(P.get(&sl0, (size_t)NB * slots));
    DT_TRY(P.get(&sn, (size_t)NB * slots));
    DT_TRY(P.get(&cand_d, (size_t)KC * NQ));
    DT_TRY(P.get(&cand_i, (size_t)KC * NQ));
    DT_TRY(P.get(&qub, NQ));
    float* qcap = nullptr;
    if (cap_leaves > 0) DT_TRY(P.get(&qcap, NQ));
    DT_TRY(P.get(&derr, 1));
    DT_TRY(P.get(&B1n, NN));
    DT_TRY(P.get(&An, NN));
    DT_TRY(P.get(&Bn, NN));
    // 0-2 work counters, 3 fallback count, 4 overflow, 5-6 frontier, 7 pairs, 8 fallback-64 count
    DT_TRY(P.get(&ctr, 16));
    DT_TRY(P.get(&bcount, NB));
    DT_TRY(P.get(&bcur, NB));
    DT_TRY(P.get(&fbq_list, NQ));
    DT_TRY(P.get(&fbq2_list, NQ));
    DT_TRY(P.get(&off, NB + 1));
    DT_TRY(P.get(&dstats, ST_NSTAT));
    DT_CHECK(cudaMemsetAsync(derr, 0, sizeof(int), s));
    DT_CHECK(cudaMemsetAsync(ctr, 0, 16 * sizeof(int), s));
    DT_CHECK(cudaMemsetAsync(dstats, 0, ST_NSTAT * sizeof(unsigned long long), s));
    DT_CHECK(cudaMemcpyAsync(probs, pd, np * sizeof(ProbDev), cudaMemcpyHostToDevice, s));
    {
        const int64_t nmax = std::max<int64_t>(std::max<int64_t>(NB, NN), std::max<int64_t>(NI, np));
        DT_LAUNCH(k_index, (int)((nmax + 255) / 256), 256, 0, s, probs, np, NB, NN, NI, blk_prob,
                  node_prob, items, roots);
    }
    PhaseTimer tm(s, st != nullptr);
    tm.mark();  // 0

    // 1. seed: the greedy subtree of each block, plus its proposed cells
    DT_TRY(launch_seed<DP>(probs, blk_prob, NB, slots, sl0, sn, s));
    if (nprop > 0) {
        int32_t* cells;
        float* centres;
        int64_t maxnb = 0;
        for (int i = 0; i < np; ++i) maxnb = std::max<int64_t>(maxnb, pd[i].nblocks);
        DT_TRY(P.get(&cells, (size_t)NB * nprop));
        DT_TRY(P.get(&centres, (size_t)maxnb * hp[0].tq->d));
        for (int i = 0; i < np; ++i) {
            DT_TRY(box_centres(hp[i].tq, pd[i].qblock0, pd[i].nblocks, centres, s));
            DT_TRY(proposal_cells(hp[i].prop, centres, pd[i].nblocks, nprop,
                                  cells + (size_t)pd[i].block0 * nprop, s));
        }
        DT_LAUNCH(k_seed_proposal, (NB + 127) / 128, 128, 0, s, probs, blk_prob, NB, slots, cells,
                  nprop, sl0, sn);
    }
    TileArgs a{};
    a.probs = probs;
    a.blk_prob = blk_prob;
    a.items = items;
    a.nitems = NI;
    a.nq_all = NQ;
    a.seed_leaf0 = sl0;
    a.seed_nleaf = sn;
    a.seed_slots = slots;
    // the seed pass evaluates every seed slot for the CUDA-core main pass; with
    // the tensor cores it evaluates the greedy subtree only, and the main pass
    // evaluates the proposed cells first, at the tensor cores' rate
    a.seed_eval_slots = fmt ? 1 : slots;
    a.cand_d = cand_d;
    a.cand_i = cand_i;
    a.qub = qub;
    a.fbq_list = fbq_list;
    a.fbq_count = ctr + 3;
    a.fbq2_list = fbq2_list;
    a.fbq2_count = ctr + 8;
    a.stats = dstats;
    a.work_ctr = ctr + 0;
    // the seed pass runs on the CUDA cores whatever the precision: its lists
    // start empty, so nearly every early candidate is an insertion, which the
    // float32 tile does cheaply; its keys (relative error <= rel_eps) are
    // tighter than any tensor-core key, so the main pass's bounds hold for
    // them.  It keeps lists of bucket(k + 1) entries (the float32 band needs
    // no more); the main pass's other rows start empty.
    a.kc_rows = KC;
    DT_TRY(launch_tile_cc<DP>(a, kc_bucket(kmax + 1), MODE_SEED, NI, s));
    if (qcap) {
        DT_TRY(launch_query_cap<DP>(a, KC, cap_leaves, qcap, s));
        a.qcap = qcap;
    }
    tm.mark();  // 1

    // 2. bounds of every query node down to the blocks
    DT_LAUNCH(k_fill, (int)((NN + 255) / 256), 256, 0, s, B1n, NN, 0.f);
    DT_LAUNCH(k_fill, (int)((NN + 255) / 256), 256, 0, s, An, NN, INFINITY);
    DT_LAUNCH(k_block_bounds, (NB * 32 + 255) / 256, 256, 0, s, probs, blk_prob, NB, qub, B1n, An);
    DT_LAUNCH(k_node_bounds, (int)((NN + 255) / 256), 256, 0, s, probs, node_prob, B1n, An, NN, Bn);

    // 3. level-synchronous pruning dual-tree traversal
    int64_t cap = std::max<int64_t>(1 << 20, (int64_t)NB * 256);
    if (np == 1) cap = std::max<int64_t>(cap, hp[0].tr->cap_hint);
    if (arena) {
        // a fixed range: the pair buffers take what is left, once (the three
        // blocks' alignment costs at most 3 x 255 bytes)
        const size_t per = sizeof(int4) + 2 * sizeof(int2);
        const size_t room = P.left();
        cap = room > 1024 ? (int64_t)std::min<size_t>((room - 1024) / per, (size_t)1 << 30) : 0;
        if (cap < np) return DTREE_ERR_TOO_LARGE;
    }
    const int egrid = occupancy_grid((const void*)k_expand<DP>, 256,
                                     (size_t)std::min(np, kExpandProbs) * sizeof(ProbDev));
    int npairs = 0;
    int4* outp = nullptr;
    auto finish_csr = [&](int n) -> int {
        npairs = n;
        DT_TRY(P.get(&csr_leaf, std::max(npairs, 1)));
        DT_TRY(P.get(&csr_dmin, std::max(npairs, 1)));
        DT_TRY(P.get(&csr_key, std::max(npairs, 1)));
        DT_LAUNCH(k_scan, 1, 1024, 0, s, bcount, NB, off);
        DT_CHECK(cudaMemsetAsync(bcur, 0, NB * sizeof(int), s));
        if (npairs > 0) {
            DT_LAUNCH(k_csr_fill, (npairs + 255) / 256, 256, 0, s, outp, npairs, off, bcur, csr_leaf,
                      csr_dmin, csr_key);
            DT_CHECK(cudaFuncSetAttribute(k_csr_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kCsrSortSmem));
            const int sgrid = std::min(NB, occupancy_grid((const void*)k_csr_sort, 256, kCsrSortSmem));
            DT_LAUNCH(k_csr_sort, sgrid, 256, kCsrSortSmem, s, off, NB, csr_leaf, csr_dmin, csr_key);
        }
        P.release(csr_key);  // only the order needed it
        P.release(outp);
        return DTREE_OK;
    };
    if (!arena) {
        // Buffers sized level by level: a frontier pair has at most four child
        // pairs, so before each level the output frontier and the candidate
        // buffer get room for four times the current frontier (the frontier
        // size is read back after every level).
        int2* F[2];
        int64_t fcap[2] = {std::max<int64_t>(cap, np), std::max<int64_t>(cap, np)}, ocap = cap;
        DT_TRY(P.get(&outp, ocap));
        DT_TRY(P.get(&F[0], fcap[0]));
        DT_TRY(P.get(&F[1], fcap[1]));
        DT_CHECK(cudaMemsetAsync(bcount, 0, NB * sizeof(int), s));
        DT_CHECK(cudaMemsetAsync(ctr + 4, 0, 4 * sizeof(int), s));
        DT_CHECK(cudaMemcpyAsync(F[0], roots, np * sizeof(int2), cudaMemcpyDeviceToDevice, s));
        DT_CHECK(cudaMemcpyAsync(ctr + 5, &np, sizeof(int), cudaMemcpyHostToDevice, s));
        int* nc[2] = {ctr + 5, ctr + 6};
        int cur = 0;
        int64_t nf = np, used = 0;
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
            DT_TRY(launch_expand<DP>(probs, node_prob, Bn, F[cur], nc[cur], F[nx], nc[nx], fcap[nx],
                                     outp, ctr + 7, ocap, bcount, sl0, sn, slots, ctr + 4, dstats,
                                     np, egrid, s));
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
        if (np == 1)
            const_cast<dtree_t*>(hp[0].tr)->cap_hint = std::max(fcap[0], std::max(fcap[1], ocap));
        DT_TRY(finish_csr((int)used));
    } else {
        // a fixed range: one pass with the capacity it has left
        int2 *F0, *F1;
        // in this order, so that releasing F1 then F0 frees the frontier for
        // the candidate arrays
        DT_TRY(P.get(&outp, cap));
        DT_TRY(P.get(&F0, cap));
        DT_TRY(P.get(&F1, cap));
        DT_CHECK(cudaMemsetAsync(bcount, 0, NB * sizeof(int), s));
        DT_CHECK(cudaMemsetAsync(ctr + 4, 0, 4 * sizeof(int), s));
        DT_CHECK(cudaMemcpyAsync(F0, roots, np * sizeof(int2), cudaMemcpyDeviceToDevice, s));
        DT_CHECK(cudaMemcpyAsync(ctr + 5, &np, sizeof(int), cudaMemcpyHostToDevice, s));
        int2 *fi = F0, *fo = F1;
        int *ni = ctr + 5, *no = ctr + 6;
        for (int t = 0; t < steps; ++t) {
            DT_CHECK(cudaMemsetAsync(no, 0, sizeof(int), s));
            DT_TRY(launch_expand<DP>(probs, node_prob, Bn, fi, ni, fo, no, cap, outp, ctr + 7, cap,
                                     bcount, sl0, sn, slots, ctr + 4, dstats, np, egrid, s));
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
    tm.mark();  // 2

    // 4. BaseCase over the candidates with the tightening bound, re-rank, output
    a.csr_off = off;
    a.csr_leaf = csr_leaf;
    a.csr_dmin = csr_dmin;
    a.Bn = Bn;
    a.work_ctr = ctr + 1;
    if (fmt)
        DT_TRY(launch_tile_tc<DP>(a, fmt, KC, NI, derr, spin, s));
    else
        DT_TRY(launch_tile_cc<DP>(a, KC, MODE_MAIN, NI, s));
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
        // few such queries: each one's candidates are split over up to 64
        // CTAs (about two per SM in all), whose lists are then merged
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        auto slices = [&](int n) {
            int sl = std::min(64, std::max(1, 2 * sms / n));
            if (sl > 1) {
                void* part = nullptr;
                const size_t bytes = (size_t)n * sl * KC * (sizeof(double) + sizeof(int32_t));
                if (P.get(reinterpret_cast<unsigned char**>(&part), bytes) != DTREE_OK) return 1;
                a.fb_part = part;
            }
            return sl;
        };
        a.fb_slices = slices(nfb);
        DT_TRY(launch_query_fb<DP>(a, KC, nfb, false, s));
        DT_CHECK(cudaMemcpyAsync(&nfb2, ctr + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
        DT_CHECK(cudaStreamSynchronize(s));
        if (nfb2 > 0) {
            a.fb_slices = slices(nfb2);
            DT_TRY(launch_query_fb<DP>(a, KC, nfb2, true, s));
        }
    }
    tm.mark();  // 4
    unsigned long long hs[ST_NSTAT];
    DT_CHECK(cudaMemcpyAsync(hs, dstats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    DT_CHECK(cudaStreamSynchronize(s));
    if (st) {
        st->node_pairs_scored += (int64_t)hs[ST_SCORED];
        st->node_pairs_pruned += (int64_t)hs[ST_PRUNED];
        st->leaf_pairs_emitted += (int64_t)hs[ST_EMITTED];
        st->leaf_pairs_skipped += (int64_t)hs[ST_SKIPPED];
        st->leaf_pairs_evaluated += (int64_t)hs[ST_EVALUATED];
        st->point_pairs += (int64_t)hs[ST_POINT_PAIRS];
        st->seed_point_pairs += (int64_t)hs[ST_SEED_PAIRS];
        st->rerank_candidates += (int64_t)hs[ST_RERANK];
        st->fallback_queries += nfb;
        st->fallback64_queries += nfb2;
        st->query_blocks += NB;
        st->kernel_launches += g_launches.load() - launches0;
        st->ns_seed += tm.ns(0, 1);
        st->ns_traverse += tm.ns(1, 2);
        st->ns_basecase += tm.ns(2, 3);
        st->ns_fallback += tm.ns(3, 4);
    }
    return DTREE_OK;
}

// Shared option checks of dtree_knn and dtree_knn_batch.
struct KnnOpts {
    int prec, qb, seed_pts, cap, spin, nprop, bound;
};

int parse_opts(const dtree_opts* o, KnnOpts* ko) {
    if (o)
        for (int i = 0; i < 8; ++i)
            if (o->reserved[i]) return DTREE_ERR_INVALID_ARG;
    ko->bound = o ? o->bound : DTREE_BOUND_BOX;
    if (ko->bound < DTREE_BOUND_BOX || ko->bound > DTREE_BOUND_BOTH) return DTREE_ERR_INVALID_ARG;
    ko->prec = o ? o->precision : DTREE_PREC_FP32;
    if (ko->prec < DTREE_PREC_FP32 || ko->prec > DTREE_PREC_BF16) return DTREE_ERR_INVALID_ARG;
    ko->qb = (o && o->query_block) ? o->query_block : 128;
    if (ko->qb < 16 || ko->qb > 512) return DTREE_ERR_INVALID_ARG;
    ko->nprop = o ? o->proposal : 0;
    if (ko->nprop < 0 || ko->nprop > 8) return DTREE_ERR_INVALID_ARG;
    ko->seed_pts = (o && o->seed_points > 0) ? o->seed_points : 64;
    ko->cap = (o && o->cap_leaves) ? o->cap_leaves : 8;
    if (ko->cap < -1 || ko->cap > 17) return DTREE_ERR_INVALID_ARG;
    if (ko->cap < 0) ko->cap = 0;
    ko->spin = (o && o->spin_budget > 0) ? o->spin_budget : (1 << 20);
    return DTREE_OK;
}

int check_problem(const dtree_t* query, const dtree_t* ref, int32_t k, const int64_t* out_idx,
                  const float* out_dist, HostProb* hp) {
    if (!ref) return DTREE_ERR_INVALID_ARG;
    const bool mono = query == nullptr || query == ref;
    const dtree_t* tq = mono ? ref : query;
    const int64_t m = ref->n;
    if (k <= 0 || (mono ? (int64_t)k > m - 1 : (int64_t)k >= m)) return DTREE_ERR_INVALID_K;
    if (!out_idx || !out_dist || tq->d != ref->d) return DTREE_ERR_INVALID_ARG;
    hp->tq = tq;
    hp->tr = ref;
    hp->mono = mono;
    hp->k = k;
    hp->out_idx = const_cast<int64_t*>(out_idx);
    hp->out_dist = const_cast<float*>(out_dist);
    hp->qb = 0;
    hp->prop = ref->proposal;
    return DTREE_OK;
}

int run_group(int dp, const HostProb* hp, int np, const KnnOpts& ko, cudaStream_t s,
              dtree_stats* st, const ScratchArena* arena) {
    if (ko.nprop > 0) {
        // every problem needs a proposal; the seed's model pass allocates
        if (arena) return DTREE_ERR_UNSUPPORTED;
        for (int i = 0; i < np; ++i)
            if (!hp[i].prop) return DTREE_ERR_NOT_TRAINED;
    }
    switch (dp) {
        case 4: return knn_batch_impl<4>(hp, np, ko.qb, ko.seed_pts, ko.cap, ko.prec, ko.spin, ko.nprop, ko.bound, s, st, arena);
        case 8: return knn_batch_impl<8>(hp, np, ko.qb, ko.seed_pts, ko.cap, ko.prec, ko.spin, ko.nprop, ko.bound, s, st, arena);
        case 16: return knn_batch_impl<16>(hp, np, ko.qb, ko.seed_pts, ko.cap, ko.prec, ko.spin, ko.nprop, ko.bound, s, st, arena);
        case 32: return knn_batch_impl<32>(hp, np, ko.qb, ko.seed_pts, ko.cap, ko.prec, ko.spin, ko.nprop, ko.bound, s, st, arena);
        default: return knn_batch_impl<64>(hp, np, ko.qb, ko.seed_pts, ko.cap, ko.prec, ko.spin, ko.nprop, ko.bound, s, st, arena);
    }
}

int device_checks(int prec, bool arena, const HostProb* hp, int np, int* dev_out) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (arena) {
        for (int i = 0; i < np; ++i)
            if (hp[i].tr->device != dev || hp[i].tq->device != dev) return DTREE_ERR_INVALID_ARG;
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
    *dev_out = dev;
    return DTREE_OK;
}

}  // namespace

int knn_entry(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
              float* out_dist, const dtree_opts* o, void* stream, dtree_stats* st,
              const ScratchArena* arena) {
    if (st) memset(st, 0, sizeof(*st));
    HostProb hp;
    int rc = check_problem(query, ref, k, out_idx, out_dist, &hp);
    if (rc != DTREE_OK) return rc;
    KnnOpts ko;
    rc = parse_opts(o, &ko);
    if (rc != DTREE_OK) return rc;
    int dev = 0;
    rc = device_checks(ko.prec, arena != nullptr, &hp, 1, &dev);
    if (rc != DTREE_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = run_group(ref->dp, &hp, 1, ko, s, st, arena);
    if (rc != DTREE_OK) cudaStreamSynchronize(s);
    return rc;
}

}  // namespace dt

extern "C" int dtree_knn(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
                         float* out_dist, const dtree_opts* o, void* stream, dtree_stats* st) {
    return dt::knn_entry(query, ref, k, out_idx, out_dist, o, stream, st, nullptr);
}

extern "C" int dtree_knn_batch(int32_t nprob, const dtree_problem* probs, const dtree_opts* o,
                               void* stream, dtree_stats* st) {
    if (st) memset(st, 0, sizeof(*st));
    if (nprob < 0 || (nprob > 0 && !probs)) return DTREE_ERR_INVALID_ARG;
    if (nprob == 0) return DTREE_OK;
    dt::KnnOpts ko;
    int rc = dt::parse_opts(o, &ko);
    if (rc != DTREE_OK) return rc;
    std::vector<dt::HostProb> hp(nprob);
    for (int i = 0; i < nprob; ++i) {
        const int qb = probs[i].query_block;
        if (qb != 0 && (qb < 16 || qb > 512)) return DTREE_ERR_INVALID_ARG;
        rc = dt::check_problem(probs[i].query, probs[i].ref, probs[i].k, probs[i].out_idx,
                               probs[i].out_dist, &hp[i]);
        if (rc != DTREE_OK) return rc;
        hp[i].qb = qb;
    }
    int dev = 0;
    rc = dt::device_checks(ko.prec, false, hp.data(), nprob, &dev);
    if (rc != DTREE_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // one batched search per padded dimension (the kernels are built per width)
    for (int dp : {4, 8, 16, 32, 64}) {
        std::vector<dt::HostProb> group;
        for (const auto& h : hp)
            if (h.tr->dp == dp) group.push_back(h);
        if (group.empty()) continue;
        rc = dt::run_group(dp, group.data(), (int)group.size(), ko, s, st, nullptr);
        if (rc != DTREE_OK) {
            cudaStreamSynchronize(s);
            return rc;
        }
    }
    return DTREE_OK;
}
