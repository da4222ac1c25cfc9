// build.cu -- kd-tree construction on the device (dtree_build).
//
// The kd-tree is a space tree (Definition 1 of Curtin et al.): every node's
// convex set is the tight bounding box of its points, and kd-tree nodes hold
// points only in their leaves.  Splits put floor(n/2) points left, chosen as
// the smallest along the widest box dimension; the paper leaves construction
// open, this is the classic median rule.  The tree is balanced so that node
// ranges and the heap numbering follow from n alone.
//
// Two phases:
//   top    levels whose nodes are larger than one CTA's shared memory: per
//          level, a bounding-box pass, an exact radix select of each node's
//          median key (three histogram passes of 11, 11 and 10 bits over
//          order-preserving uint32 keys), and a scatter into the children.
//          Many CTAs work on one node.
//   bottom one CTA per remaining subtree: the subtree's points are staged in
//          shared memory and split level by level with a bitonic sort on
//          (segment, key, slot) composite keys; boxes and the exact lambda of
//          every node of the subtree are written on the way.
// lambda of top-phase nodes is bounded from their children:
//   lambda(N) <= max_c ( |C_N - C_c| + lambda(c) )   (triangle inequality),
// rounded upward, which keeps it a valid bound for the B_2 term of Section 5.
#include <algorithm>
#include <new>

#include "dtree_internal.cuh"

namespace dt {
namespace {

constexpr int kTPB = 256;            // threads of the top-phase kernels
constexpr int kChunk = 4096;         // elements per CTA in a top-phase pass
constexpr int kBottomFloats = 8192;  // floats of points one bottom CTA stages
constexpr int kBottomThreads = 256;

template <int DP>
__host__ __device__ constexpr int bottom_cap() {
    return kBottomFloats / DP < 2048 ? kBottomFloats / DP : 2048;
}

__global__ void k_layout(int64_t n, int64_t nnodes, int32_t* nbeg, int32_t* ncnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nnodes) return;
    int L = level_of_node(i);
    int64_t pos = i - ((int64_t(1) << L) - 1);
    int64_t b = 0, c = n;
    for (int l = L - 1; l >= 0; --l) {
        int64_t nl = c / 2;
        if ((pos >> l) & 1) {
            b += nl;
            c -= nl;
        } else {
            c = nl;
        }
    }
    nbeg[i] = (int32_t)b;
    ncnt[i] = (int32_t)c;
}

__global__ void k_init(const float* in, int64_t n, int d, int dp, float* pts, int32_t* idx,
                       int* bad) {
    int64_t total = n * dp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / dp;
        int j = (int)(t - r * dp);
        float v = 0.f;
        if (j < d) {
            v = in[r * d + j];
            if (!isfinite(v)) *bad = 1;
        }
        pts[t] = v;
        if (j == 0) idx[r] = (int32_t)r;
    }
}

// Per (node, chunk) CTA of level L: min/max of each dimension -> atomics on
// order-preserving encodings.
template <int DP>
__global__ void __launch_bounds__(kTPB) k_bbox(const float* __restrict__ pts, const int32_t* nbeg,
                                               const int32_t* ncnt, int64_t node0, int cpn,
                                               uint32_t* blo, uint32_t* bhi) {
    int64_t nl = blockIdx.x / cpn;
    int c = blockIdx.x % cpn;
    int64_t node = node0 + nl;
    int64_t b = nbeg[node], e = b + ncnt[node];
    int64_t s = b + (int64_t)c * kChunk;
    int64_t t_end = e < s + kChunk ? e : s + kChunk;
    if (s >= t_end) return;
    constexpr int RPI = kTPB / DP;
    int j = threadIdx.x % DP;
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t r = s + threadIdx.x / DP; r < t_end; r += RPI) {
        float v = pts[r * DP + j];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    __shared__ float slo[kTPB], shi[kTPB];
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    if (threadIdx.x < DP) {
        for (int q = 1; q < RPI; ++q) {
            lo = fminf(lo, slo[q * DP + j]);
            hi = fmaxf(hi, shi[q * DP + j]);
        }
        atomicMin(&blo[nl * DP + j], f2o(lo));
        atomicMax(&bhi[nl * DP + j], f2o(hi));
    }
}

// Decode the level's boxes into the tree and pick each node's split dimension
// (widest extent, lowest dimension on ties).
template <int DP>
__global__ void k_box_decode(const uint32_t* blo, const uint32_t* bhi, int64_t node0, int64_t nn,
                             int d, float* box, uint8_t* sdim) {
    int64_t nl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (nl >= nn) return;
    float* bx = box + (node0 + nl) * 2 * DP;
    int best = 0;
    float bext = -1.f;
    for (int j = 0; j < DP; ++j) {
        float lo = j < d ? o2f(blo[nl * DP + j]) : 0.f;
        float hi = j < d ? o2f(bhi[nl * DP + j]) : 0.f;
        bx[j] = lo;
        bx[DP + j] = hi;
        float ext = hi - lo;
        if (j < d && ext > bext) {
            bext = ext;
            best = j;
        }
    }
    sdim[nl] = (uint8_t)best;
}

// Keys of the level (order-preserving uint32 of the split coordinate) and
// the first histogram (top 11 bits).
template <int DP>
__global__ void __launch_bounds__(kTPB) k_keys_hist(const float* __restrict__ pts,
                                                    const int32_t* nbeg, const int32_t* ncnt,
                                                    int64_t node0, int cpn, const uint8_t* sdim,
                                                    uint32_t* keys, uint32_t* ghist) {
    __shared__ uint32_t h[2048];
    for (int i = threadIdx.x; i < 2048; i += kTPB) h[i] = 0;
    __syncthreads();
    int64_t nl = blockIdx.x / cpn;
    int c = blockIdx.x % cpn;
    int64_t node = node0 + nl;
    int64_t b = nbeg[node], e = b + ncnt[node];
    int64_t s = b + (int64_t)c * kChunk;
    int64_t t_end = e < s + kChunk ? e : s + kChunk;
    int dim = sdim[nl];
    for (int64_t i = s + threadIdx.x; i < t_end; i += kTPB) {
        uint32_t key = f2o(pts[i * DP + dim]);
        keys[i] = key;
        atomicAdd(&h[key >> 21], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += kTPB)
        if (h[i]) atomicAdd(&ghist[nl * 2048 + i], h[i]);
}

// Histogram pass 1 (bits 20..10 among keys whose top 11 bits match) or
// pass 2 (bits 9..0 among keys whose top 22 bits match).
__global__ void __launch_bounds__(kTPB) k_hist(const uint32_t* keys, const int32_t* nbeg,
                                               const int32_t* ncnt, int64_t node0, int cpn,
                                               int pass, const uint32_t* prefix,
                                               uint32_t* ghist) {
    __shared__ uint32_t h[2048];
    for (int i = threadIdx.x; i < 2048; i += kTPB) h[i] = 0;
    __syncthreads();
    int64_t nl = blockIdx.x / cpn;
    int c = blockIdx.x % cpn;
    int64_t node = node0 + nl;
    int64_t b = nbeg[node], e = b + ncnt[node];
    int64_t s = b + (int64_t)c * kChunk;
    int64_t t_end = e < s + kChunk ? e : s + kChunk;
    uint32_t pre = prefix[nl];
    int hi_shift = pass == 1 ? 21 : 10;
    int lo_shift = pass == 1 ? 10 : 0;
    uint32_t mask = pass == 1 ? 0x7ffu : 0x3ffu;
    for (int64_t i = s + threadIdx.x; i < t_end; i += kTPB) {
        uint32_t key = keys[i];
        if ((key >> hi_shift) == pre) atomicAdd(&h[(key >> lo_shift) & mask], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += kTPB)
        if (h[i]) atomicAdd(&ghist[nl * 2048 + i], h[i]);
}

// One CTA per node: find the bin holding rank `rank` (0-based), narrow the
// prefix, count what lies below, and clear the histogram for the next pass.
// After pass 2, prefix is the exact key m of rank floor(n/2)-1 and
// eq_left = floor(n/2) - #{key < m} of the keys equal to m go left.
__global__ void __launch_bounds__(kTPB) k_select(const int32_t* ncnt, int64_t node0, int pass,
                                                 uint32_t* ghist, uint32_t* prefix,
                                                 int32_t* rank, int32_t* less, int32_t* eq_left) {
    int64_t nl = blockIdx.x;
    int nbins = pass == 2 ? 1024 : 2048;
    int per = nbins / kTPB;
    uint32_t* h = ghist + nl * 2048;
    __shared__ int32_t ssum[kTPB];
    __shared__ int32_t sres[3];
    if (pass == 0 && threadIdx.x == 0) {
        rank[nl] = ncnt[node0 + nl] / 2 - 1;
        less[nl] = 0;
        prefix[nl] = 0;
    }
    __syncthreads();
    int32_t r = rank[nl];
    int32_t sum = 0;
    for (int q = 0; q < per; ++q) sum += (int32_t)h[threadIdx.x * per + q];
    ssum[threadIdx.x] = sum;
    __syncthreads();
    // exclusive scan (Hillis-Steele over 256 entries)
    for (int off = 1; off < kTPB; off <<= 1) {
        int32_t v = threadIdx.x >= off ? ssum[threadIdx.x - off] : 0;
        __syncthreads();
        ssum[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t incl = ssum[threadIdx.x];
    int32_t excl = incl - sum;
    if (r >= excl && r < incl) {
        int32_t cum = excl;
        int bin = threadIdx.x * per;
        for (int q = 0; q < per; ++q) {
            int32_t v = (int32_t)h[threadIdx.x * per + q];
            if (r < cum + v) {
                bin = threadIdx.x * per + q;
                break;
            }
            cum += v;
        }
        sres[0] = bin;
        sres[1] = cum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += kTPB) h[i] = 0;
    if (threadIdx.x == 0) {
        int bits = pass == 2 ? 10 : 11;
        uint32_t pre = (prefix[nl] << bits) | (uint32_t)sres[0];
        prefix[nl] = pre;
        less[nl] += sres[1];
        rank[nl] = r - sres[1];
        if (pass == 2) eq_left[nl] = ncnt[node0 + nl] / 2 - less[nl];
    }
}

// Move each point to its child: key < m left, key > m right, keys equal to m
// take tickets (the first eq_left go left).  Positions come from one atomic
// per CTA and side plus a CTA-local scan.
template <int DP>
__global__ void __launch_bounds__(kTPB) k_scatter(const float* __restrict__ src,
                                                  const int32_t* __restrict__ isrc,
                                                  float* __restrict__ dst, int32_t* __restrict__ idst,
                                                  const uint32_t* keys, const int32_t* nbeg,
                                                  const int32_t* ncnt, int64_t node0, int cpn,
                                                  const uint32_t* msplit, const int32_t* eq_left,
                                                  int32_t* eq_ctr, int32_t* cursor, int* bad) {
    int64_t nl = blockIdx.x / cpn;
    int c = blockIdx.x % cpn;
    int64_t node = node0 + nl;
    int64_t b = nbeg[node], cnt = ncnt[node], e = b + cnt;
    int64_t s = b + (int64_t)c * kChunk;
    int64_t t_end = e < s + kChunk ? e : s + kChunk;
    int64_t half = cnt / 2;
    uint32_t m = msplit[nl];
    int32_t eql = eq_left[nl];
    __shared__ int32_t wl[kTPB / 32], wr[kTPB / 32];
    __shared__ int64_t baseL, baseR;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned lt = (1u << lane) - 1u;
    for (int64_t base = s; base < t_end; base += kTPB) {
        int64_t i = base + threadIdx.x;
        bool valid = i < t_end;
        int side = 1;
        if (valid) {
            uint32_t key = keys[i];
            if (key < m) side = 0;
            else if (key == m) side = atomicAdd(&eq_ctr[nl], 1) < eql ? 0 : 1;
        }
        unsigned bl = __ballot_sync(0xffffffffu, valid && side == 0);
        unsigned br = __ballot_sync(0xffffffffu, valid && side == 1);
        if (lane == 0) {
            wl[w] = __popc(bl);
            wr[w] = __popc(br);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tl = 0, tr = 0;
            for (int q = 0; q < kTPB / 32; ++q) {
                int32_t a = wl[q], bb = wr[q];
                wl[q] = tl;
                wr[q] = tr;
                tl += a;
                tr += bb;
            }
            baseL = tl ? atomicAdd(&cursor[2 * nl], tl) : 0;
            baseR = tr ? atomicAdd(&cursor[2 * nl + 1], tr) : 0;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = side == 0 ? b + baseL + wl[w] + __popc(bl & lt)
                                    : b + half + baseR + wr[w] + __popc(br & lt);
            bool inside = side == 0 ? pos < b + half : pos < e;
            if (inside) {
                const float4* sr = reinterpret_cast<const float4*>(src + i * DP);
                float4* dr = reinterpret_cast<float4*>(dst + pos * DP);
#pragma unroll
                for (int q = 0; q < DP / 4; ++q) dr[q] = sr[q];
                idst[pos] = isrc[i];
            } else {
                *bad = 2;  // a wrong median would overfill a child: never write past it
            }
        }
        __syncthreads();
    }
}

// Segment statistics of the bottom phase, one warp per segment: box, split
// dimension, exact lambda (rounded up).
template <int DP>
__device__ void seg_stats(const float* sp, const uint64_t* sk, int sb, int cnt, int d,
                          float* box_out, float* lam_out, uint8_t* sdim_out, float* scen) {
    constexpr int NA = DP > 32 ? 2 : 1;
    int lane = threadIdx.x & 31;
    float lo[NA], hi[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
    for (int f = lane; f < cnt * DP; f += 32) {
        int e = f / DP, jj = f % DP;
        int p = (int)(sk[sb + e] & 0xffffu);
        float v = sp[p * DP + jj];
        int a = NA == 2 ? (f >> 5) & 1 : 0;
        lo[a] = fminf(lo[a], v);
        hi[a] = fmaxf(hi[a], v);
    }
    if (DP < 32) {
#pragma unroll
        for (int off = DP; off < 32; off <<= 1) {
            lo[0] = fminf(lo[0], __shfl_xor_sync(0xffffffffu, lo[0], off));
            hi[0] = fmaxf(hi[0], __shfl_xor_sync(0xffffffffu, hi[0], off));
        }
    }
    // lane's dimensions: lane % DP (DP <= 32) or lane + 32a (DP = 64)
    float bext = -1.f;
    int bdim = 0;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        int jj = NA == 2 ? lane + 32 * a : lane % DP;
        float l = jj < d ? lo[a] : 0.f, h = jj < d ? hi[a] : 0.f;
        if (lane < DP || NA == 2) {
            box_out[jj] = l;
            box_out[DP + jj] = h;
            scen[jj] = 0.5f * (l + h);
        }
        float ext = h - l;
        if (jj < d && (ext > bext || (ext == bext && jj < bdim))) {
            bext = ext;
            bdim = jj;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        float oe = __shfl_xor_sync(0xffffffffu, bext, off);
        int od = __shfl_xor_sync(0xffffffffu, bdim, off);
        if (oe > bext || (oe == bext && od < bdim)) {
            bext = oe;
            bdim = od;
        }
    }
    __syncwarp();
    float mx = 0.f;
    for (int e = lane; e < cnt; e += 32) {
        int p = (int)(sk[sb + e] & 0xffffu);
        float acc = 0.f;
#pragma unroll
        for (int jj = 0; jj < DP; ++jj) {
            float t = scen[jj] - sp[p * DP + jj];
            acc = fmaf(t, t, acc);
        }
        mx = fmaxf(mx, acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) {
        *lam_out = __fmul_ru(__fsqrt_ru(mx), 1.f + rel_eps<DP>());
        *sdim_out = (uint8_t)bdim;
    }
    __syncwarp();
}

template <int DP>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(float* pts, int32_t* idx,
                                                           const int32_t* nbeg,
                                                           const int32_t* ncnt, int Ltop, int h,
                                                           int d, float* box, float* lam) {
    constexpr int S = bottom_cap<DP>();
    constexpr int NW = kBottomThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    float* sp = reinterpret_cast<float*>(smem);                // S * DP points
    uint64_t* sk = reinterpret_cast<uint64_t*>(sp + S * DP);   // S composite keys
    float* scen = reinterpret_cast<float*>(sk + S);            // NW * DP centres
    int32_t* so = reinterpret_cast<int32_t*>(scen + NW * DP);  // S input rows
    uint16_t* sseg = reinterpret_cast<uint16_t*>(so + S);      // S + 2 segment begins
    uint8_t* sdim = reinterpret_cast<uint8_t*>(sseg + S + 2);  // S split dimensions

    int64_t root = ((int64_t)1 << Ltop) - 1 + blockIdx.x;
    int rb = nbeg[root], rc = ncnt[root];
    int tid = threadIdx.x, warp = tid >> 5;
    for (int f = tid; f < rc * DP; f += kBottomThreads) sp[f] = pts[(int64_t)rb * DP + f];
    for (int e = tid; e < rc; e += kBottomThreads) so[e] = idx[rb + e];
    for (int e = tid; e < S; e += kBottomThreads) sk[e] = e < rc ? (uint64_t)e : ~0ull;
    __syncthreads();
    int nsub = h - Ltop;
    for (int j = 0; j <= nsub; ++j) {
        int nseg = 1 << j;
        int64_t first = (root + 1) * nseg - 1;
        for (int s = tid; s < nseg; s += kBottomThreads) sseg[s] = (uint16_t)(nbeg[first + s] - rb);
        if (tid == 0) sseg[nseg] = (uint16_t)rc;
        __syncthreads();
        for (int s = warp; s < nseg; s += NW) {
            int sb = sseg[s], cnt = sseg[s + 1] - sb;
            seg_stats<DP>(sp, sk, sb, cnt, d, box + (first + s) * 2 * DP, lam + first + s, sdim + s,
                          scen + warp * DP);
        }
        __syncthreads();
        if (j == nsub) break;
        for (int e = tid; e < rc; e += kBottomThreads) {
            int p = (int)(sk[e] & 0xffffu);
            int lo = 0, hi = nseg - 1;  // last segment whose begin <= e
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (sseg[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            uint32_t key = f2o(sp[p * DP + sdim[lo]]);
            sk[e] = ((uint64_t)lo << 48) | ((uint64_t)key << 16) | (uint64_t)p;
        }
        __syncthreads();
        for (int kk = 2; kk <= S; kk <<= 1) {
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int t = tid; t < S / 2; t += kBottomThreads) {
                    int i = 2 * t - (t & (jj - 1));
                    int l = i + jj;
                    bool up = (i & kk) == 0;
                    uint64_t a = sk[i], bb = sk[l];
                    if ((a > bb) == up) {
                        sk[i] = bb;
                        sk[l] = a;
                    }
                }
                __syncthreads();
            }
        }
    }
    for (int f = tid; f < rc * DP; f += kBottomThreads) {
        int e = f / DP, jj = f % DP;
        int p = (int)(sk[e] & 0xffffu);
        pts[(int64_t)rb * DP + f] = sp[p * DP + jj];
    }
    for (int e = tid; e < rc; e += kBottomThreads) idx[rb + e] = so[sk[e] & 0xffffu];
}

template <int DP>
constexpr size_t bottom_smem() {
    constexpr int S = bottom_cap<DP>();
    return (size_t)S * DP * 4 + (size_t)S * 8 + (kBottomThreads / 32) * DP * 4 + (size_t)S * 4 +
           (size_t)(S + 2) * 2 + (size_t)S;
}

// Leaves too large for the bottom phase: exact lambda from the points.
template <int DP>
__global__ void __launch_bounds__(kTPB) k_leaf_lambda(const float* __restrict__ pts,
                                                      const int32_t* nbeg, const int32_t* ncnt,
                                                      int64_t node0, const float* box, float* lam) {
    int64_t node = node0 + blockIdx.x;
    __shared__ float cen[DP];
    __shared__ float red[kTPB / 32];
    const float* bx = box + node * 2 * DP;
    for (int j = threadIdx.x; j < DP; j += kTPB) cen[j] = 0.5f * (bx[j] + bx[DP + j]);
    __syncthreads();
    int64_t b = nbeg[node], e = b + ncnt[node];
    float mx = 0.f;
    for (int64_t r = b + threadIdx.x; r < e; r += kTPB) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < DP; ++j) {
            float t = cen[j] - pts[r * DP + j];
            acc = fmaf(t, t, acc);
        }
        mx = fmaxf(mx, acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kTPB / 32; ++q) mx = fmaxf(mx, red[q]);
        lam[node] = __fmul_ru(__fsqrt_ru(mx), 1.f + rel_eps<DP>());
    }
}

// lambda of top-phase nodes from their children, levels Ltop-1 .. 0 (one CTA).
template <int DP>
__global__ void __launch_bounds__(1024) k_top_lambda(int Ltop, const float* box, float* lam) {
    for (int L = Ltop - 1; L >= 0; --L) {
        int64_t n0 = ((int64_t)1 << L) - 1, nn = (int64_t)1 << L;
        for (int64_t q = threadIdx.x; q < nn; q += blockDim.x) {
            int64_t node = n0 + q;
            const float* bx = box + node * 2 * DP;
            float best = 0.f;
            for (int ch = 1; ch <= 2; ++ch) {
                int64_t c = 2 * node + ch;
                const float* cb = box + c * 2 * DP;
                float acc = 0.f;
                for (int j = 0; j < DP; ++j) {
                    float t = 0.5f * (bx[j] + bx[DP + j]) - 0.5f * (cb[j] + cb[DP + j]);
                    acc = fmaf(t, t, acc);
                }
                float dist = __fmul_ru(__fsqrt_ru(acc), 1.f + rel_eps<DP>());
                best = fmaxf(best, __fadd_ru(dist, lam[c]));
            }
            lam[node] = best;
        }
        __syncthreads();
    }
}

struct Scratch {
    cudaStream_t s;
    void* p[16] = {};
    int n = 0;
    template <class T>
    int get(T** out, size_t count) {
        int rc = scratch(out, count, s);
        if (rc == DTREE_OK) p[n++] = *out;
        return rc;
    }
    ~Scratch() {
        for (int i = 0; i < n; ++i) cudaFreeAsync(p[i], s);
    }
};

#define DT_TRY(x)                   \
    do {                            \
        int rc_ = (x);              \
        if (rc_ != DTREE_OK) return rc_; \
    } while (0)

inline int grid_for(int64_t work, int tpb, int cap = 1 << 16) {
    int64_t g = (work + tpb - 1) / tpb;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

template <int DP>
int build_impl(dtree_t* t, const float* in, cudaStream_t s) {
    const int64_t n = t->n;
    const int h = t->height;
    Scratch sc{s};
    int* dbad = nullptr;
    DT_TRY(sc.get(&dbad, 1));
    DT_CHECK(cudaMemsetAsync(dbad, 0, sizeof(int), s));
    DT_LAUNCH(k_layout, grid_for(t->nnodes, 256), 256, 0, s, n, t->nnodes, t->nbeg, t->ncnt);
    DT_LAUNCH(k_init, grid_for(n * DP, 256, 8192), 256, 0, s, in, n, t->d, DP, t->pts, t->idx,
              dbad);

    const int Lsmall = level_of_count(n, bottom_cap<DP>());
    const bool bottom = Lsmall <= h;
    const int Ltop = bottom ? Lsmall : h;
    // levels [0, Ltop) are split by the top phase; `statl` is the first level
    // whose boxes come from somewhere else
    int64_t maxnodes = (int64_t)1 << (bottom ? (Ltop > 0 ? Ltop - 1 : 0) : h);
    float* alt = nullptr;
    int32_t* ialt = nullptr;
    uint32_t *keys = nullptr, *blo = nullptr, *bhi = nullptr, *ghist = nullptr, *prefix = nullptr,
             *msplit = nullptr;
    int32_t *rank = nullptr, *less = nullptr, *eql = nullptr, *eqc = nullptr, *cur = nullptr;
    uint8_t* sdim = nullptr;
    if (Ltop > 0 || !bottom) {
        DT_TRY(sc.get(&blo, maxnodes * DP));
        DT_TRY(sc.get(&bhi, maxnodes * DP));
        DT_TRY(sc.get(&sdim, maxnodes));
    }
    struct PingPong {
        float* p = nullptr;
        int32_t* i = nullptr;
        ~PingPong() {
            cudaFree(p);
            cudaFree(i);
        }
    } pp;
    if (Ltop > 0) {
        g_allocs.fetch_add(2, std::memory_order_relaxed);
        if (cudaMalloc((void**)&pp.p, (size_t)n * DP * 4) != cudaSuccess ||
            cudaMalloc((void**)&pp.i, (size_t)n * 4) != cudaSuccess) {
            cudaGetLastError();
            return DTREE_ERR_OOM;
        }
        alt = pp.p;
        ialt = pp.i;
        DT_TRY(sc.get(&keys, (size_t)n));
        DT_TRY(sc.get(&ghist, maxnodes * 2048));
        DT_TRY(sc.get(&prefix, maxnodes));
        DT_TRY(sc.get(&msplit, maxnodes));
        DT_TRY(sc.get(&rank, maxnodes));
        DT_TRY(sc.get(&less, maxnodes));
        DT_TRY(sc.get(&eql, maxnodes));
        DT_TRY(sc.get(&eqc, maxnodes));
        DT_TRY(sc.get(&cur, 2 * maxnodes));
        DT_CHECK(cudaMemsetAsync(ghist, 0, maxnodes * 2048 * 4, s));
    }
    float* src = t->pts;
    int32_t* isrc = t->idx;
    float* dst = alt;
    int32_t* idst = ialt;
    auto level_boxes = [&](int L) -> int {
        int64_t node0 = ((int64_t)1 << L) - 1, nn = (int64_t)1 << L;
        int64_t maxc = (n + nn - 1) / nn;
        int cpn = (int)((maxc + kChunk - 1) / kChunk);
        DT_CHECK(cudaMemsetAsync(blo, 0xff, nn * DP * 4, s));
        DT_CHECK(cudaMemsetAsync(bhi, 0x00, nn * DP * 4, s));
        DT_LAUNCH(k_bbox<DP>, (int)(nn * cpn), kTPB, 0, s, src, t->nbeg, t->ncnt, node0, cpn, blo,
                  bhi);
        DT_LAUNCH(k_box_decode<DP>, grid_for(nn, 256), 256, 0, s, blo, bhi, node0, nn, t->d,
                  t->box, sdim);
        return DTREE_OK;
    };
    for (int L = 0; L < Ltop; ++L) {
        int64_t node0 = ((int64_t)1 << L) - 1, nn = (int64_t)1 << L;
        int64_t maxc = (n + nn - 1) / nn;
        int cpn = (int)((maxc + kChunk - 1) / kChunk);
        int grid = (int)(nn * cpn);
        DT_TRY(level_boxes(L));
        DT_LAUNCH(k_keys_hist<DP>, grid, kTPB, 0, s, src, t->nbeg, t->ncnt, node0, cpn, sdim, keys,
                  ghist);
        DT_LAUNCH(k_select, (int)nn, kTPB, 0, s, t->ncnt, node0, 0, ghist, prefix, rank, less, eql);
        DT_LAUNCH(k_hist, grid, kTPB, 0, s, keys, t->nbeg, t->ncnt, node0, cpn, 1, prefix, ghist);
        DT_LAUNCH(k_select, (int)nn, kTPB, 0, s, t->ncnt, node0, 1, ghist, prefix, rank, less, eql);
        DT_LAUNCH(k_hist, grid, kTPB, 0, s, keys, t->nbeg, t->ncnt, node0, cpn, 2, prefix, ghist);
        DT_LAUNCH(k_select, (int)nn, kTPB, 0, s, t->ncnt, node0, 2, ghist, prefix, rank, less, eql);
        DT_CHECK(cudaMemsetAsync(eqc, 0, nn * 4, s));
        DT_CHECK(cudaMemsetAsync(cur, 0, 2 * nn * 4, s));
        DT_LAUNCH(k_scatter<DP>, grid, kTPB, 0, s, src, isrc, dst, idst, keys, t->nbeg, t->ncnt,
                  node0, cpn, prefix, eql, eqc, cur, dbad);
        std::swap(src, dst);
        std::swap(isrc, idst);
    }
    if (bottom) {
        size_t smem = bottom_smem<DP>();
        DT_CHECK(cudaFuncSetAttribute(k_bottom<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        DT_LAUNCH(k_bottom<DP>, 1 << Ltop, kBottomThreads, smem, s, src, isrc, t->nbeg, t->ncnt,
                  Ltop, h, t->d, t->box, t->lam);
    } else {
        DT_TRY(level_boxes(h));
        DT_LAUNCH(k_leaf_lambda<DP>, 1 << h, kTPB, 0, s, src, t->nbeg, t->ncnt,
                  ((int64_t)1 << h) - 1, t->box, t->lam);
    }
    if (Ltop > 0) DT_LAUNCH(k_top_lambda<DP>, 1, 1024, 0, s, Ltop, t->box, t->lam);
    int bad = 0;
    DT_CHECK(cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s));
    DT_CHECK(cudaStreamSynchronize(s));
    if (src != t->pts) {
        // the final order lives in the second buffer: the tree keeps it and
        // the first one is released with the ping-pong pair
        std::swap(t->pts, pp.p);
        std::swap(t->idx, pp.i);
    }
    if (bad == 2) return DTREE_ERR_CUDA;  // internal consistency check failed
    return bad ? DTREE_ERR_INVALID_ARG : DTREE_OK;
}

}  // namespace
}  // namespace dt

extern "C" int dtree_build(const float* pts, int64_t n, int32_t d, const dtree_opts* o,
                           void* stream, dtree_t** out) {
    if (!out) return DTREE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!pts || n <= 0 || n >= ((int64_t)1 << 31) || d < 1 || d > 64) return DTREE_ERR_INVALID_ARG;
    int leaf = (o && o->leaf_size) ? o->leaf_size : 32;
    if (leaf < 1 || leaf > 1024) return DTREE_ERR_INVALID_ARG;
    if (o)
        for (int i = 0; i < 8; ++i)
            if (o->reserved[i]) return DTREE_ERR_INVALID_ARG;
    // A balanced tree with one-point leaves would leave some leaves empty
    // whenever n is not a power of two; two-point leaves never do.
    if (leaf < 2) leaf = 2;
    cudaStream_t s = (cudaStream_t)stream;
    dtree_t* t = new (std::nothrow) dtree_t();
    if (!t) return DTREE_ERR_OOM;
    cudaGetDevice(&t->device);
    dt::prepare_pool(t->device);
    t->n = n;
    t->d = d;
    t->dp = dt::dp_bucket(d);
    t->leaf_size = leaf;
    t->height = dt::level_of_count(n, leaf);
    t->nleaves = (int64_t)1 << t->height;
    t->nnodes = 2 * t->nleaves - 1;
    int rc = DTREE_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (rc != DTREE_OK) return;
        dt::g_allocs.fetch_add(1, std::memory_order_relaxed);
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = DTREE_ERR_OOM;
        }
    };
    alloc((void**)&t->pts, (size_t)n * t->dp * 4);
    alloc((void**)&t->idx, (size_t)n * 4);
    alloc((void**)&t->box, (size_t)t->nnodes * 2 * t->dp * 4);
    alloc((void**)&t->lam, (size_t)t->nnodes * 4);
    alloc((void**)&t->nbeg, (size_t)t->nnodes * 4);
    alloc((void**)&t->ncnt, (size_t)t->nnodes * 4);
    if (rc == DTREE_OK) {
        switch (t->dp) {
            case 4: rc = dt::build_impl<4>(t, pts, s); break;
            case 8: rc = dt::build_impl<8>(t, pts, s); break;
            case 16: rc = dt::build_impl<16>(t, pts, s); break;
            case 32: rc = dt::build_impl<32>(t, pts, s); break;
            default: rc = dt::build_impl<64>(t, pts, s); break;
        }
    }
    if (rc != DTREE_OK) {
        cudaStreamSynchronize(s);
        dtree_free(t);
        return rc;
    }
    *out = t;
    return DTREE_OK;
}
