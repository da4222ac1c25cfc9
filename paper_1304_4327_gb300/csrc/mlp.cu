// mlp.cu -- the learned leaf proposal: a small MLP (d -> 256 -> 256 -> C)
// that maps a point to the reference-tree cells (subtrees at the seed level)
// most likely to hold its neighbours.  The search evaluates a query block's
// proposed cells in its seed pass, before the traversal, so that B(N_q)
// starts tight; the traversal then finds every neighbour the proposal missed,
// so results never depend on the network (Section 5's bound stays exact).
//
// Everything runs in this file's kernels: an FP16 tensor-core GEMM
// (tcgen05, FP32 accumulation in TMEM), softmax cross-entropy, the backward
// pass, Adam with FP32 master weights, and the top-M selection at search
// time.  Training data is the method's own kNN output: for each node of a
// training query tree (about 16 queries), the input is the node's box centre
// and the target is the distribution of its queries' k nearest neighbours
// over the cells.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "dtree_internal.cuh"
#include "tc_ptx.cuh"

struct dtree_model {
    int32_t d = 0, dpad = 16, H = 256, C = 0, level = 0;
    float mean[64] = {}, scale[64] = {};
    float* p[6] = {};      // W1 [H x dpad], b1 [H], W2 [H x H], b2 [H], W3 [C x H], b3 [C]
    float* m[6] = {};      // Adam moments
    float* v[6] = {};
    __half* wh[3] = {};    // FP16 copies of W1, W2, W3 for the GEMMs
    int64_t t = 0;         // Adam steps taken
    int device = 0;
    uint64_t tree_hash = 0;  // fingerprint of the reference tree's cells (tree_fingerprint)
    int64_t size(int i) const {
        switch (i) {
            case 0: return (int64_t)H * dpad;
            case 1: return H;
            case 2: return (int64_t)H * H;
            case 3: return H;
            case 4: return (int64_t)C * H;
            default: return C;
        }
    }
};

namespace dt {
namespace {

constexpr int kGK = 128;                       // K chunk of the GEMM (halves): 256 B per row
constexpr uint32_t kGSBO = (kGK * 2 / 16) * 128;  // core-matrix group stride
constexpr size_t kGSmem = 2 * 128 * kGK * 2;   // A and B tiles (64 KB: at most 3 CTAs / SM)

// C[m, n] = act(sum_k A[m, k] B[n, k] + bias[n]) for one 128 x 128 tile per
// CTA.  A (M x K) and B (N x K) are FP16, K contiguous; out of range rows and
// K are zero.  C (FP32) and Ch (FP16) are optional.  act: 0 none, 1 ReLU.
__global__ void __launch_bounds__(128) k_gemm_f16(const __half* A, int64_t lda, const __half* B,
                                                  int64_t ldb, int M, int N, int K,
                                                  const float* bias, int act, float* C,
                                                  int64_t ldc, __half* Ch, int64_t ldch, int* err,
                                                  int spin) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    unsigned char* sA = gsm;
    unsigned char* sB = gsm + 128 * kGK * 2;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * 128;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_s, 128);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_s;
    const uint32_t id = tc::idesc(0, 128, 128);  // FP16 A and B, FP32 accumulator
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < K; k0 += kGK) {
        // thread tid stages row tid of the A tile and of the B tile
#pragma unroll
        for (int mtx = 0; mtx < 2; ++mtx) {
            const __half* src = mtx == 0 ? A : B;
            const int64_t ld = mtx == 0 ? lda : ldb;
            const int r = (mtx == 0 ? m0 : n0) + tid;
            const bool rin = r < (mtx == 0 ? M : N);
            unsigned char* dst = mtx == 0 ? sA : sB;
            const __half* row = src + (int64_t)r * ld;
            const bool vec = rin && ((reinterpret_cast<uintptr_t>(row) & 15u) == 0) && (ld % 8 == 0);
#pragma unroll 4
            for (int c = 0; c < kGK / 8; ++c) {
                const int k = k0 + 8 * c;
                uint4 w = make_uint4(0u, 0u, 0u, 0u);
                if (rin && k < K) {
                    if (vec && k + 8 <= K) {
                        w = *reinterpret_cast<const uint4*>(row + k);
                    } else {
                        __half hv[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) hv[j] = k + j < K ? row[k + j] : __float2half(0.f);
                        w = *reinterpret_cast<const uint4*>(hv);
                    }
                }
                *reinterpret_cast<uint4*>(dst + tc::core_offset(tid, c, kGSBO)) = w;
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
            for (int kk = 0; kk < kGK / 16; ++kk)
                tc::mma<1>(tmem, tc::sdesc(a0 + 256u * kk, 128u, kGSBO),
                           tc::sdesc(b0 + 256u * kk, 128u, kGSBO), id,
                           (k0 > 0 || kk > 0) ? 1u : 0u);
            tc::mma_commit(&bar);
        }
        // the tiles may be overwritten only once the MMAs have read them
        ok = tc::mbar_wait(&bar, phase, spin);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        tc::fence_after_sync();
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        tc::mbar_wait(&bar, phase ^ 1u, spin);  // the last commit, before TMEM is released
    } else if (K > 0) {
        const int m = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int cc = 0; cc < 4; ++cc) {
            uint32_t v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
            tc::tmem_ld_wait_dep(v);
            if (m < M) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int n = n0 + cc * 32 + i;
                    if (n < N) {
                        float x = __uint_as_float(v[i]) + (bias ? bias[n] : 0.f);
                        if (act == 1) x = fmaxf(x, 0.f);
                        if (C) C[(int64_t)m * ldc + n] = x;
                        if (Ch) Ch[(int64_t)m * ldch + n] = __float2half_rn(x);
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// out[c, r] = in[r, c] (FP16, R x C -> C x R), 32 x 32 tiles.
__global__ void k_transpose_h(const __half* in, int R, int Cc, __half* out) {
    __shared__ __half t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        t[y][threadIdx.x] = (r < R && c < Cc) ? in[(int64_t)r * Cc + c] : __float2half(0.f);
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (c < Cc && r < R) out[(int64_t)c * R + r] = t[threadIdx.x][y];
    }
}

__global__ void k_f32_to_f16(const float* in, int64_t n, __half* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2half_rn(in[i]);
}

// Softmax cross-entropy per row against a target distribution T (rows sum to
// 1): loss += -sum_c T[r, c] log p[r, c]; dZ = (p - T) / B (FP32 and FP16).
__global__ void __launch_bounds__(256) k_softmax_xent(const float* Z, const float* T, int B, int Cc,
                                                      float* dZ, __half* dZh, float* loss) {
    const int r = blockIdx.x;
    const float* z = Z + (int64_t)r * Cc;
    const float* t = T + (int64_t)r * Cc;
    __shared__ float red[32];
    float mx = -INFINITY;
    for (int c = threadIdx.x; c < Cc; c += blockDim.x) mx = fmaxf(mx, z[c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    __syncthreads();
    float se = 0.f;
    for (int c = threadIdx.x; c < Cc; c += blockDim.x) se += expf(z[c] - mx);
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
    __syncthreads();
    se = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) se += red[w];
    __syncthreads();
    const float lse = mx + logf(se);
    float l = 0.f;
    for (int c = threadIdx.x; c < Cc; c += blockDim.x) {
        const float p = expf(z[c] - lse);
        const float tc_ = t[c];
        if (tc_ > 0.f) l -= tc_ * (z[c] - lse);
        const float g = (p - tc_) / (float)B;
        dZ[(int64_t)r * Cc + c] = g;
        dZh[(int64_t)r * Cc + c] = __float2half_rn(g);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s / (float)B);
    }
}

// g[r, c] *= (h[r, c] > 0) (the ReLU's derivative), also writing an FP16 copy.
__global__ void k_relu_mask(float* g, const float* h, int64_t n, __half* gh) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = h[i] > 0.f ? g[i] : 0.f;
    g[i] = x;
    gh[i] = __float2half_rn(x);
}

// out[c] = sum_r g[r, c] (bias gradients).
__global__ void k_colsum(const float* g, int R, int Cc, float* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Cc) return;
    float s = 0.f;
    for (int r = 0; r < R; ++r) s += g[(int64_t)r * Cc + c];
    out[c] = s;
}

// Adam with bias correction; also refreshes the FP16 copy when given.
__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1,
                       float b2, float c1, float c2, float eps, __half* ph) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float x = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = x;
    if (ph) ph[i] = __float2half_rn(x);
}

// Network inputs: standardised coordinates, FP16, padded to dpad columns.
__global__ void k_inputs(const float* pts, int64_t ld, int d, int64_t n, const float* mean,
                         const float* scale, int dpad, __half* X) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * dpad) return;
    const int64_t r = i / dpad;
    const int j = (int)(i % dpad);
    X[i] = __float2half_rn(j < d ? (pts[r * ld + j] - mean[j]) * scale[j] : 0.f);
}

// Inputs of a training batch: rows ex[0..B) of `pts`, standardised.
__global__ void k_inputs_gather(const float* pts, int d, const int32_t* ex, int B, const float* mean,
                                const float* scale, int dpad, __half* X) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * dpad) return;
    const int r = (int)(i / dpad), j = (int)(i % dpad);
    X[i] = __float2half_rn(j < d ? (pts[(int64_t)ex[r] * d + j] - mean[j]) * scale[j] : 0.f);
}

// Box centres of `count` consecutive tree nodes starting at node0.
__global__ void k_centres(const float* box, int dp, int d, int64_t node0, int64_t count,
                          float* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count * d) return;
    const int64_t r = i / d;
    const int j = (int)(i % d);
    const float* b = box + (node0 + r) * 2 * dp;
    out[r * d + j] = 0.5f * (b[j] + b[dp + j]);
}

// Training targets of one batch: row e gets, for each of its node's queries
// and each of their k neighbours, weight 1 / (queries x k) on the
// neighbour's cell.
__global__ void k_targets(const int64_t* nbr, int k, const int32_t* qbeg, const int32_t* qcnt,
                          const int32_t* qidx, int64_t node0, const int32_t* ex, int nb,
                          const int32_t* cell_of_orig, int Cc, float* T) {
    const int e = blockIdx.x;
    if (e >= nb) return;
    const int64_t node = node0 + ex[e];
    const int b = qbeg[node], c = qcnt[node];
    const float w = 1.f / (float)(c * k);
    for (int i = threadIdx.x; i < c * k; i += blockDim.x) {
        const int q = qidx[b + i / k];
        const int64_t r = nbr[(int64_t)q * k + i % k];
        atomicAdd(&T[(int64_t)e * Cc + cell_of_orig[r]], w);
    }
}

// cell_of_orig[idx[p]] = the level-`level` cell holding tree position p.
__global__ void k_cell_map(const int32_t* nbeg, const int32_t* ncnt, int64_t cell0, int ncell,
                           const int32_t* idx, int32_t* cell_of_orig) {
    const int c = blockIdx.x;
    if (c >= ncell) return;
    const int b = nbeg[cell0 + c], n = ncnt[cell0 + c];
    for (int i = threadIdx.x; i < n; i += blockDim.x) cell_of_orig[idx[b + i]] = c;
}

// Top-M entries of each row of Z (ties by lower column), as cell ids.
__global__ void __launch_bounds__(256) k_topm(const float* Z, int Cc, int M, int32_t* out) {
    const int r = blockIdx.x;
    const float* z = Z + (int64_t)r * Cc;
    __shared__ float sv[8];
    __shared__ int si[8];
    __shared__ int chosen[16];
    for (int t = 0; t < M; ++t) {
        float bv = -INFINITY;
        int bi = 0x7fffffff;
        for (int c = threadIdx.x; c < Cc; c += blockDim.x) {
            bool used = false;
            for (int u = 0; u < t; ++u) used |= chosen[u] == c;
            const float x = z[c];
            if (!used && (x > bv || (x == bv && c < bi))) {
                bv = x;
                bi = c;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            sv[threadIdx.x >> 5] = bv;
            si[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (sv[w] > sv[0] || (sv[w] == sv[0] && si[w] < si[0])) {
                    sv[0] = sv[w];
                    si[0] = si[w];
                }
            chosen[t] = si[0] < Cc ? si[0] : 0;
            out[(int64_t)r * M + t] = chosen[t];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int gemm(cudaStream_t s, const __half* A, int64_t lda, const __half* B, int64_t ldb, int M, int N,
         int K, const float* bias, int act, float* C, int64_t ldc, __half* Ch, int64_t ldch,
         int* err) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(k_gemm_f16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kGSmem);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    if (M <= 0 || N <= 0) return DTREE_OK;
    dim3 grid((N + 127) / 128, (M + 127) / 128);
    DT_LAUNCH(k_gemm_f16, grid, 128, kGSmem, s, A, lda, B, ldb, M, N, K, bias, act, C, ldc, Ch, ldch,
              err, 1 << 20);
    return DTREE_OK;
}

int transpose(cudaStream_t s, const __half* in, int R, int Cc, __half* out) {
    if (R <= 0 || Cc <= 0) return DTREE_OK;
    dim3 grid((Cc + 31) / 32, (R + 31) / 32);
    DT_LAUNCH(k_transpose_h, grid, dim3(32, 8), 0, s, in, R, Cc, out);
    return DTREE_OK;
}

template <class T>
struct DevBuf {
    T* p = nullptr;
    cudaStream_t s = nullptr;
    int get(int64_t n, cudaStream_t st) {
        s = st;
        return scratch(&p, (size_t)std::max<int64_t>(n, 1), st);
    }
    ~DevBuf() {
        if (p) cudaFreeAsync(p, s);
    }
};

#define MT(x)                            \
    do {                                 \
        int rc_ = (x);                   \
        if (rc_ != DTREE_OK) return rc_; \
    } while (0)

// Activations and gradients of one batch of B rows.
struct Work {
    int B = 0;
    DevBuf<__half> X, XT, H1h, H1T, H2h, H2T, dZh, dZT, dH2h, dH2T, dH1h, dH1T, W3T, W2T;
    DevBuf<float> H1, H2, Z, dZ, dH2, dH1, g[6];
    DevBuf<float> loss;
    DevBuf<int> err;
    int alloc(const dtree_model& md, int B_, cudaStream_t s, bool train) {
        B = B_;
        const int H = md.H, C = md.C, dp = md.dpad;
        MT(X.get((int64_t)B * dp, s));
        MT(H1.get((int64_t)B * H, s));
        MT(H1h.get((int64_t)B * H, s));
        MT(H2.get((int64_t)B * H, s));
        MT(H2h.get((int64_t)B * H, s));
        MT(Z.get((int64_t)B * C, s));
        MT(err.get(1, s));
        MT(loss.get(1, s));
        if (!train) return DTREE_OK;
        MT(XT.get((int64_t)dp * B, s));
        MT(H1T.get((int64_t)H * B, s));
        MT(H2T.get((int64_t)H * B, s));
        MT(dZ.get((int64_t)B * C, s));
        MT(dZh.get((int64_t)B * C, s));
        MT(dZT.get((int64_t)C * B, s));
        MT(dH2.get((int64_t)B * H, s));
        MT(dH2h.get((int64_t)B * H, s));
        MT(dH2T.get((int64_t)H * B, s));
        MT(dH1.get((int64_t)B * H, s));
        MT(dH1h.get((int64_t)B * H, s));
        MT(dH1T.get((int64_t)H * B, s));
        MT(W3T.get((int64_t)H * C, s));
        MT(W2T.get((int64_t)H * H, s));
        for (int i = 0; i < 6; ++i) MT(g[i].get(md.size(i), s));
        return DTREE_OK;
    }
};

// Z = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for the B rows of w.X.
int forward(const dtree_model& md, Work& w, int B, cudaStream_t s) {
    const int H = md.H, C = md.C, dp = md.dpad;
    MT(gemm(s, w.X.p, dp, md.wh[0], dp, B, H, dp, md.p[1], 1, w.H1.p, H, w.H1h.p, H, w.err.p));
    MT(gemm(s, w.H1h.p, H, md.wh[1], H, B, H, H, md.p[3], 1, w.H2.p, H, w.H2h.p, H, w.err.p));
    MT(gemm(s, w.H2h.p, H, md.wh[2], H, B, C, H, md.p[5], 0, w.Z.p, C, nullptr, 0, w.err.p));
    return DTREE_OK;
}

// Loss against the targets T (B x C) and every parameter's gradient in w.g.
int backward(const dtree_model& md, Work& w, int B, const float* T, cudaStream_t s) {
    const int H = md.H, C = md.C, dp = md.dpad;
    DT_CHECK(cudaMemsetAsync(w.loss.p, 0, sizeof(float), s));
    DT_LAUNCH(k_softmax_xent, B, 256, 0, s, w.Z.p, T, B, C, w.dZ.p, w.dZh.p, w.loss.p);
    // layer 3: dW3 = dZ^T H2, db3 = colsum dZ, dH2 = dZ W3
    MT(transpose(s, w.dZh.p, B, C, w.dZT.p));
    MT(transpose(s, w.H2h.p, B, H, w.H2T.p));
    MT(gemm(s, w.dZT.p, B, w.H2T.p, B, C, H, B, nullptr, 0, w.g[4].p, H, nullptr, 0, w.err.p));
    DT_LAUNCH(k_colsum, (C + 255) / 256, 256, 0, s, w.dZ.p, B, C, w.g[5].p);
    MT(transpose(s, md.wh[2], C, H, w.W3T.p));
    MT(gemm(s, w.dZh.p, C, w.W3T.p, C, B, H, C, nullptr, 0, w.dH2.p, H, nullptr, 0, w.err.p));
    DT_LAUNCH(k_relu_mask, (int)(((int64_t)B * H + 255) / 256), 256, 0, s, w.dH2.p, w.H2.p,
              (int64_t)B * H, w.dH2h.p);
    // layer 2
    MT(transpose(s, w.dH2h.p, B, H, w.dH2T.p));
    MT(transpose(s, w.H1h.p, B, H, w.H1T.p));
    MT(gemm(s, w.dH2T.p, B, w.H1T.p, B, H, H, B, nullptr, 0, w.g[2].p, H, nullptr, 0, w.err.p));
    DT_LAUNCH(k_colsum, (H + 255) / 256, 256, 0, s, w.dH2.p, B, H, w.g[3].p);
    MT(transpose(s, md.wh[1], H, H, w.W2T.p));
    MT(gemm(s, w.dH2h.p, H, w.W2T.p, H, B, H, H, nullptr, 0, w.dH1.p, H, nullptr, 0, w.err.p));
    DT_LAUNCH(k_relu_mask, (int)(((int64_t)B * H + 255) / 256), 256, 0, s, w.dH1.p, w.H1.p,
              (int64_t)B * H, w.dH1h.p);
    // layer 1
    MT(transpose(s, w.dH1h.p, B, H, w.dH1T.p));
    MT(transpose(s, w.X.p, B, dp, w.XT.p));
    MT(gemm(s, w.dH1T.p, B, w.XT.p, B, H, dp, B, nullptr, 0, w.g[0].p, dp, nullptr, 0, w.err.p));
    DT_LAUNCH(k_colsum, (H + 255) / 256, 256, 0, s, w.dH1.p, B, H, w.g[1].p);
    return DTREE_OK;
}

int refresh_half(dtree_model& md, cudaStream_t s) {
    const int src[3] = {0, 2, 4};
    for (int i = 0; i < 3; ++i) {
        const int64_t n = md.size(src[i]);
        DT_LAUNCH(k_f32_to_f16, (int)((n + 255) / 256), 256, 0, s, md.p[src[i]], n, md.wh[i]);
    }
    return DTREE_OK;
}

int model_alloc(dtree_model* md, cudaStream_t s) {
    for (int i = 0; i < 6; ++i) {
        const size_t n = (size_t)md->size(i);
        g_allocs.fetch_add(3, std::memory_order_relaxed);
        if (cudaMalloc((void**)&md->p[i], n * 4) != cudaSuccess ||
            cudaMalloc((void**)&md->m[i], n * 4) != cudaSuccess ||
            cudaMalloc((void**)&md->v[i], n * 4) != cudaSuccess) {
            cudaGetLastError();
            return DTREE_ERR_OOM;
        }
        DT_CHECK(cudaMemsetAsync(md->m[i], 0, n * 4, s));
        DT_CHECK(cudaMemsetAsync(md->v[i], 0, n * 4, s));
    }
    const int src[3] = {0, 2, 4};
    for (int i = 0; i < 3; ++i) {
        g_allocs.fetch_add(1, std::memory_order_relaxed);
        if (cudaMalloc((void**)&md->wh[i], (size_t)md->size(src[i]) * 2) != cudaSuccess) {
            cudaGetLastError();
            return DTREE_ERR_OOM;
        }
    }
    return DTREE_OK;
}

void model_release(dtree_model* md) {
    if (!md) return;
    for (int i = 0; i < 6; ++i) {
        cudaFree(md->p[i]);
        cudaFree(md->m[i]);
        cudaFree(md->v[i]);
    }
    for (int i = 0; i < 3; ++i) cudaFree(md->wh[i]);
    delete md;
}

// He-uniform initialisation from a counter-based generator (splitmix64).
uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int model_init(dtree_model* md, uint64_t seed, cudaStream_t s) {
    uint64_t st = seed;
    const int fan_in[6] = {md->dpad, 1, md->H, 1, md->H, 1};
    for (int i = 0; i < 6; ++i) {
        const int64_t n = md->size(i);
        std::vector<float> h((size_t)n, 0.f);
        if (i % 2 == 0) {
            const float lim = std::sqrt(6.f / (float)fan_in[i]);
            for (int64_t j = 0; j < n; ++j) {
                const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
                h[(size_t)j] = (float)((2.0 * u - 1.0) * lim);
            }
            if (i == 0)  // padded input columns carry no weight
                for (int64_t r = 0; r < md->H; ++r)
                    for (int j = md->d; j < md->dpad; ++j) h[(size_t)(r * md->dpad + j)] = 0.f;
        }
        DT_CHECK(cudaMemcpyAsync(md->p[i], h.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
        DT_CHECK(cudaStreamSynchronize(s));
    }
    return refresh_half(*md, s);
}

int adam_step(dtree_model& md, Work& w, float lr, cudaStream_t s) {
    md.t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)md.t), c2 = 1.f - std::pow(b2, (float)md.t);
    const int half_of[6] = {0, -1, 1, -1, 2, -1};
    for (int i = 0; i < 6; ++i) {
        const int64_t n = md.size(i);
        DT_LAUNCH(k_adam, (int)((n + 255) / 256), 256, 0, s, md.p[i], w.g[i].p, md.m[i], md.v[i], n,
                  lr, b1, b2, c1, c2, 1e-8f, half_of[i] >= 0 ? md.wh[half_of[i]] : nullptr);
    }
    return DTREE_OK;
}

int check_err(Work& w, cudaStream_t s) {
    int herr = 0;
    DT_CHECK(cudaMemcpyAsync(&herr, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DT_CHECK(cudaStreamSynchronize(s));
    return herr ? DTREE_ERR_TIMEOUT : DTREE_OK;
}

int level_for_cells(const dtree_t* ref, int seed_pts) {
    int L = 0;
    while (L < ref->height && (ref->n >> (L + 1)) >= seed_pts) ++L;
    return L;
}

}  // namespace

// Top-M proposed cells for `n` points (box centres), for the search.
int proposal_cells(const dtree_model* md, const float* pts, int64_t n, int M, int32_t* out,
                   cudaStream_t s) {
    if (n <= 0) return DTREE_OK;
    DevBuf<float> mean, scale;
    MT(mean.get(md->d, s));
    MT(scale.get(md->d, s));
    DT_CHECK(cudaMemcpyAsync(mean.p, md->mean, md->d * 4, cudaMemcpyHostToDevice, s));
    DT_CHECK(cudaMemcpyAsync(scale.p, md->scale, md->d * 4, cudaMemcpyHostToDevice, s));
    const int64_t chunk = 4096;  // rows per forward pass (bounds the logits buffer)
    Work w;
    MT(w.alloc(*md, (int)std::min<int64_t>(chunk, n), s, false));
    DT_CHECK(cudaMemsetAsync(w.err.p, 0, sizeof(int), s));
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int B = (int)std::min<int64_t>(chunk, n - r0);
        DT_LAUNCH(k_inputs, (int)(((int64_t)B * md->dpad + 255) / 256), 256, 0, s, pts + r0 * md->d,
                  (int64_t)md->d, md->d, (int64_t)B, mean.p, scale.p, md->dpad, w.X.p);
        MT(forward(*md, w, B, s));
        DT_LAUNCH(k_topm, B, 256, 0, s, w.Z.p, md->C, M, out + r0 * M);
    }
    return check_err(w, s);
}

int model_level(const dtree_model* md) { return md->level; }

// Fingerprint of the reference tree a model's cells refer to: FNV-1a over
// its size, dimension, height, the cell level and the bounding boxes of the
// cells (the subtrees at that level).  A model only makes sense for a tree
// with the same cells; trees built from the same points with the same leaf
// size agree.
int tree_fingerprint(const dtree_t* t, int level, uint64_t* out, cudaStream_t s) {
    const int64_t cells = (int64_t)1 << level, node0 = cells - 1;
    std::vector<float> box((size_t)(cells * 2 * t->dp));
    DT_CHECK(cudaMemcpyAsync(box.data(), t->box + node0 * 2 * t->dp, box.size() * 4,
                             cudaMemcpyDeviceToHost, s));
    DT_CHECK(cudaStreamSynchronize(s));
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    };
    const int64_t head[4] = {t->n, t->d, t->height, level};
    mix(head, sizeof(head));
    for (int64_t c = 0; c < cells; ++c) {
        mix(box.data() + c * 2 * t->dp, (size_t)t->d * 4);           // lo
        mix(box.data() + c * 2 * t->dp + t->dp, (size_t)t->d * 4);   // hi
    }
    *out = h;
    return DTREE_OK;
}

int box_centres(const dtree_t* t, int64_t node0, int64_t count, float* out, cudaStream_t s) {
    if (count <= 0) return DTREE_OK;
    DT_LAUNCH(k_centres, (int)((count * t->d + 255) / 256), 256, 0, s, t->box, t->dp, t->d, node0,
              count, out);
    return DTREE_OK;
}

}  // namespace dt

using dt::DevBuf;

extern "C" {

int dtree_proposal_train(const dtree_t* ref, const dtree_t* train, int32_t k,
                         const dtree_train_opts* o, void* stream, dtree_model** out) {
    if (!out) return DTREE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ref || !train || train == ref || ref->d != train->d) return DTREE_ERR_INVALID_ARG;
    if (k <= 0 || (int64_t)k >= ref->n) return DTREE_ERR_INVALID_K;
    const int epochs = o && o->epochs > 0 ? o->epochs : 20;
    const int batch = o && o->batch > 0 ? o->batch : 256;
    const float lr = o && o->lr > 0.f ? o->lr : 1e-3f;
    const int ex_size = o && o->example_queries > 0 ? o->example_queries : 16;
    const int seed_pts = o && o->seed_points > 0 ? o->seed_points : 512;
    if (batch > 4096 || ex_size > 1024) return DTREE_ERR_INVALID_ARG;
    if (o)
        for (int i = 0; i < 7; ++i)
            if (o->reserved[i]) return DTREE_ERR_INVALID_ARG;
    if (o && (o->precision < DTREE_PREC_FP32 || o->precision > DTREE_PREC_BF16)) return DTREE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return DTREE_ERR_UNSUPPORTED;
    dt::prepare_pool(dev);

    auto* md = new (std::nothrow) dtree_model;
    if (!md) return DTREE_ERR_OOM;
    md->device = dev;
    md->d = ref->d;
    md->dpad = 16;
    while (md->dpad < md->d) md->dpad *= 2;
    md->level = dt::level_for_cells(ref, std::max(k + 1, seed_pts));
    md->C = 1 << md->level;
    if (md->C < 2) {
        dt::model_release(md);
        return DTREE_ERR_UNSUPPORTED;  // a reference tree of one cell has nothing to propose
    }
    int rc = dt::model_alloc(md, s);
    if (rc != DTREE_OK) {
        dt::model_release(md);
        return rc;
    }
    auto fail = [&](int r) {
        cudaStreamSynchronize(s);
        dt::model_release(md);
        return r;
    };

    // standardisation from the reference points (host copy of a strided sample)
    {
        const int64_t ns = std::min<int64_t>(ref->n, 65536);
        std::vector<float> h((size_t)ns * ref->dp);
        const int64_t step = ref->n / ns;
        for (int64_t i = 0; i < ns; ++i)
            if (cudaMemcpyAsync(h.data() + i * ref->dp, ref->pts + i * step * ref->dp, ref->dp * 4,
                                cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return fail(DTREE_ERR_CUDA);
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(DTREE_ERR_CUDA);
        for (int j = 0; j < md->d; ++j) {
            double a = 0.0, b = 0.0;
            for (int64_t i = 0; i < ns; ++i) {
                const double x = h[(size_t)(i * ref->dp + j)];
                a += x;
                b += x * x;
            }
            const double mu = a / ns, var = std::max(b / ns - mu * mu, 1e-12);
            md->mean[j] = (float)mu;
            md->scale[j] = (float)(1.0 / std::sqrt(var));
        }
    }
    rc = dt::model_init(md, o && o->seed ? (uint64_t)o->seed : 1304432701ull, s);
    if (rc != DTREE_OK) return fail(rc);
    if ((rc = dt::tree_fingerprint(ref, md->level, &md->tree_hash, s)) != DTREE_OK) return fail(rc);

    // the method's own answers for the training queries
    DevBuf<int64_t> nbr;
    DevBuf<float> ndist;
    if ((rc = nbr.get(train->n * k, s)) != DTREE_OK) return fail(rc);
    if ((rc = ndist.get(train->n * k, s)) != DTREE_OK) return fail(rc);
    dtree_opts so{};
    so.precision = o ? o->precision : DTREE_PREC_FP32;
    rc = dt::knn_entry(train, ref, k, nbr.p, ndist.p, &so, s, nullptr, nullptr);
    if (rc != DTREE_OK) return fail(rc);
    // neighbour (original reference row) -> cell
    DevBuf<int32_t> cell_of;
    if ((rc = cell_of.get(ref->n, s)) != DTREE_OK) return fail(rc);
    {
        const int64_t cell0 = ((int64_t)1 << md->level) - 1;
        DT_LAUNCH(dt::k_cell_map, md->C, 256, 0, s, ref->nbeg, ref->ncnt, cell0, md->C, ref->idx,
                  cell_of.p);
    }
    // examples: the training tree's nodes at the level holding ~ex_size queries
    const int Le = std::min<int>(train->height, dt::level_of_count(train->n, ex_size));
    const int nex = 1 << Le;
    const int64_t ex0 = ((int64_t)1 << Le) - 1;
    DevBuf<float> centres, mean, scale;
    if ((rc = centres.get((int64_t)nex * md->d, s)) != DTREE_OK) return fail(rc);
    if ((rc = mean.get(md->d, s)) != DTREE_OK) return fail(rc);
    if ((rc = scale.get(md->d, s)) != DTREE_OK) return fail(rc);
    if ((rc = dt::box_centres(train, ex0, nex, centres.p, s)) != DTREE_OK) return fail(rc);
    if (cudaMemcpyAsync(mean.p, md->mean, md->d * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(scale.p, md->scale, md->d * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(DTREE_ERR_CUDA);
    const int B = std::min(batch, nex);
    dt::Work w;
    if ((rc = w.alloc(*md, B, s, true)) != DTREE_OK) return fail(rc);
    DevBuf<float> T;
    DevBuf<int32_t> exd;
    if ((rc = T.get((int64_t)B * md->C, s)) != DTREE_OK) return fail(rc);
    if ((rc = exd.get(B, s)) != DTREE_OK) return fail(rc);
    if (cudaMemsetAsync(w.err.p, 0, sizeof(int), s) != cudaSuccess) return fail(DTREE_ERR_CUDA);
    std::vector<int32_t> order(nex), hb(B);
    for (int i = 0; i < nex; ++i) order[i] = i;
    uint64_t st = o && o->seed ? (uint64_t)o->seed : 1304432701ull;
    float last = 0.f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = nex - 1; i > 0; --i) std::swap(order[i], order[dt::splitmix(st) % (uint64_t)(i + 1)]);
        double sum = 0.0;
        int nb = 0;
        for (int b0 = 0; b0 + B <= nex; b0 += B) {  // whole batches only
            for (int i = 0; i < B; ++i) hb[i] = order[b0 + i];
            if (cudaMemcpyAsync(exd.p, hb.data(), B * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return fail(DTREE_ERR_CUDA);
            // inputs: the examples' box centres, standardised
            DT_LAUNCH(dt::k_inputs_gather, (int)(((int64_t)B * md->dpad + 255) / 256), 256, 0, s,
                      centres.p, md->d, exd.p, B, mean.p, scale.p, md->dpad, w.X.p);
            if (cudaMemsetAsync(T.p, 0, (size_t)B * md->C * 4, s) != cudaSuccess)
                return fail(DTREE_ERR_CUDA);
            DT_LAUNCH(dt::k_targets, B, 128, 0, s, nbr.p, k, train->nbeg, train->ncnt, train->idx,
                      ex0, exd.p, B, cell_of.p, md->C, T.p);
            if ((rc = dt::forward(*md, w, B, s)) != DTREE_OK) return fail(rc);
            if ((rc = dt::backward(*md, w, B, T.p, s)) != DTREE_OK) return fail(rc);
            if ((rc = dt::adam_step(*md, w, lr, s)) != DTREE_OK) return fail(rc);
            float hl = 0.f;
            if (cudaMemcpyAsync(&hl, w.loss.p, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return fail(DTREE_ERR_CUDA);
            sum += hl;
            ++nb;
        }
        last = nb ? (float)(sum / nb) : 0.f;
        if (o && o->loss_out && ep < o->loss_out_len) o->loss_out[ep] = last;
    }
    if ((rc = dt::check_err(w, s)) != DTREE_OK) return fail(rc);
    (void)last;
    *out = md;
    return DTREE_OK;
}

void dtree_model_free(dtree_model* m) { dt::model_release(m); }

// File layout (little-endian): the 8 magic bytes "DTRMODL1"; int32 d, dpad,
// H, C, level; uint64 the tree fingerprint; int64 Adam steps; float32
// mean[d], scale[d]; the six float32 parameter arrays W1, b1, W2, b2, W3, b3;
// uint64 FNV-1a of every byte before it.
static const char kModelMagic[8] = {'D', 'T', 'R', 'M', 'O', 'D', 'L', '1'};

int dtree_model_save(const dtree_model* m, const char* path, void* stream) {
    if (!m || !path) return DTREE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<unsigned char> buf;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        buf.insert(buf.end(), b, b + n);
    };
    put(kModelMagic, 8);
    const int32_t hdr[5] = {m->d, m->dpad, m->H, m->C, m->level};
    put(hdr, sizeof(hdr));
    put(&m->tree_hash, 8);
    put(&m->t, 8);
    put(m->mean, (size_t)m->d * 4);
    put(m->scale, (size_t)m->d * 4);
    for (int i = 0; i < 6; ++i) {
        std::vector<float> h((size_t)m->size(i));
        DT_CHECK(cudaMemcpyAsync(h.data(), m->p[i], h.size() * 4, cudaMemcpyDeviceToHost, s));
        DT_CHECK(cudaStreamSynchronize(s));
        put(h.data(), h.size() * 4);
    }
    uint64_t sum = 1469598103934665603ull;
    for (unsigned char b : buf) {
        sum ^= b;
        sum *= 1099511628211ull;
    }
    put(&sum, 8);
    FILE* f = std::fopen(path, "wb");
    if (!f) return DTREE_ERR_IO;
    const bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    return (std::fclose(f) == 0 && ok) ? DTREE_OK : DTREE_ERR_IO;
}

int dtree_model_load(const char* path, const dtree_t* ref, void* stream, dtree_model** out) {
    if (!path || !out) return DTREE_ERR_INVALID_ARG;
    *out = nullptr;
    // the whole file, checked before anything touches the device
    std::vector<unsigned char> buf;
    {
        FILE* f = std::fopen(path, "rb");
        if (!f) return DTREE_ERR_IO;
        unsigned char tmp[65536];
        size_t n;
        while ((n = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
        const bool err = std::ferror(f) != 0;
        std::fclose(f);
        if (err) return DTREE_ERR_IO;
    }
    size_t at = 0;
    auto get = [&](void* p, size_t n) {
        if (buf.size() - at < n) return false;
        std::memcpy(p, buf.data() + at, n);
        at += n;
        return true;
    };
    char magic[8];
    int32_t hdr[5];
    uint64_t hash = 0;
    int64_t steps = 0;
    if (buf.size() < 8 + 8 || !get(magic, 8) || std::memcmp(magic, kModelMagic, 8) != 0 ||
        !get(hdr, sizeof(hdr)) || !get(&hash, 8) || !get(&steps, 8))
        return DTREE_ERR_IO;
    const int32_t d = hdr[0], dpad = hdr[1], H = hdr[2], C = hdr[3], level = hdr[4];
    if (d < 1 || d > 64 || dpad < d || dpad > 64 || H != 256 || level < 1 || level > 30 ||
        C != (1 << level))
        return DTREE_ERR_IO;
    {
        uint64_t sum = 1469598103934665603ull, stored = 0;
        std::memcpy(&stored, buf.data() + buf.size() - 8, 8);
        for (size_t i = 0; i + 8 < buf.size(); ++i) {
            sum ^= buf[i];
            sum *= 1099511628211ull;
        }
        if (sum != stored) return DTREE_ERR_IO;
    }
    if (!ref) return DTREE_ERR_INVALID_ARG;
    if (ref->d != d || level > ref->height) return DTREE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t mine = 0;
    int rc = dt::tree_fingerprint(ref, level, &mine, s);
    if (rc != DTREE_OK) return rc;
    if (mine != hash) return DTREE_ERR_INVALID_ARG;  // trained for another tree
    auto* md = new (std::nothrow) dtree_model;
    if (!md) return DTREE_ERR_OOM;
    md->d = d;
    md->dpad = dpad;
    md->H = H;
    md->C = C;
    md->level = level;
    md->t = steps;
    md->tree_hash = hash;
    cudaGetDevice(&md->device);
    if (!get(md->mean, (size_t)d * 4) || !get(md->scale, (size_t)d * 4)) {
        dt::model_release(md);
        return DTREE_ERR_IO;
    }
    rc = dt::model_alloc(md, s);
    for (int i = 0; i < 6 && rc == DTREE_OK; ++i) {
        const size_t n = (size_t)md->size(i) * 4;
        if (buf.size() - 8 < at || buf.size() - 8 - at < n) {
            rc = DTREE_ERR_IO;
            break;
        }
        if (cudaMemcpyAsync(md->p[i], buf.data() + at, n, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = DTREE_ERR_CUDA;
        at += n;
    }
    if (rc == DTREE_OK && at + 8 != buf.size()) rc = DTREE_ERR_IO;
    if (rc == DTREE_OK) rc = dt::refresh_half(*md, s);
    if (rc == DTREE_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = DTREE_ERR_CUDA;
    if (rc != DTREE_OK) {
        cudaStreamSynchronize(s);
        dt::model_release(md);
        return rc;
    }
    *out = md;
    return DTREE_OK;
}

int dtree_model_classes(const dtree_model* m) { return m ? m->C : -1; }

int dtree_attach_proposal(dtree_t* ref, const dtree_model* m) {
    if (!ref) return DTREE_ERR_INVALID_ARG;
    if (m && (m->d != ref->d || m->level > ref->height)) return DTREE_ERR_INVALID_ARG;
    ref->proposal = m;
    return DTREE_OK;
}

int dtree_mlp_loss_grad(int32_t d, int32_t C, const float* const* params, const float* X,
                        const float* T, int32_t n, float* loss, float* const* grads, void* stream) {
    if (d < 1 || d > 64 || C < 1 || n < 1 || n > 4096 || !params || !X || !T || !loss || !grads)
        return DTREE_ERR_INVALID_ARG;
    for (int i = 0; i < 6; ++i)
        if (!params[i] || !grads[i]) return DTREE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return DTREE_ERR_UNSUPPORTED;
    dtree_model md;
    md.d = d;
    md.dpad = 16;
    while (md.dpad < d) md.dpad *= 2;
    md.C = C;
    // the caller's parameters, with W1 padded to dpad columns
    DevBuf<float> w1;
    DevBuf<__half> wh[3];
    int rc;
    if ((rc = w1.get((int64_t)md.H * md.dpad, s)) != DTREE_OK) return rc;
    DT_CHECK(cudaMemsetAsync(w1.p, 0, (size_t)md.H * md.dpad * 4, s));
    DT_CHECK(cudaMemcpy2DAsync(w1.p, md.dpad * 4, params[0], d * 4, d * 4, md.H,
                               cudaMemcpyDeviceToDevice, s));
    md.p[0] = w1.p;
    for (int i = 1; i < 6; ++i) md.p[i] = const_cast<float*>(params[i]);
    const int src[3] = {0, 2, 4};
    for (int i = 0; i < 3; ++i) {
        if ((rc = wh[i].get(md.size(src[i]), s)) != DTREE_OK) return rc;
        md.wh[i] = wh[i].p;
    }
    if ((rc = dt::refresh_half(md, s)) != DTREE_OK) return rc;
    dt::Work w;
    if ((rc = w.alloc(md, n, s, true)) != DTREE_OK) return rc;
    DT_CHECK(cudaMemsetAsync(w.err.p, 0, sizeof(int), s));
    DevBuf<float> zero_mean, one_scale;
    if ((rc = zero_mean.get(d, s)) != DTREE_OK) return rc;
    if ((rc = one_scale.get(d, s)) != DTREE_OK) return rc;
    DT_CHECK(cudaMemsetAsync(zero_mean.p, 0, d * 4, s));
    std::vector<float> ones((size_t)d, 1.f);
    DT_CHECK(cudaMemcpyAsync(one_scale.p, ones.data(), d * 4, cudaMemcpyHostToDevice, s));
    DT_LAUNCH(dt::k_inputs, (int)(((int64_t)n * md.dpad + 255) / 256), 256, 0, s, X, (int64_t)d, d,
              (int64_t)n, zero_mean.p, one_scale.p, md.dpad, w.X.p);
    if ((rc = dt::forward(md, w, n, s)) != DTREE_OK) return rc;
    if ((rc = dt::backward(md, w, n, T, s)) != DTREE_OK) return rc;
    // gradients out (W1 without its padding)
    DT_CHECK(cudaMemcpy2DAsync(grads[0], d * 4, w.g[0].p, md.dpad * 4, d * 4, md.H,
                               cudaMemcpyDeviceToDevice, s));
    for (int i = 1; i < 6; ++i)
        DT_CHECK(cudaMemcpyAsync(grads[i], w.g[i].p, (size_t)md.size(i) * 4,
                                 cudaMemcpyDeviceToDevice, s));
    DT_CHECK(cudaMemcpyAsync(loss, w.loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
    md.p[0] = nullptr;  // not owned
    for (int i = 0; i < 6; ++i) md.p[i] = nullptr;
    for (int i = 0; i < 3; ++i) md.wh[i] = nullptr;
    return dt::check_err(w, s);
}

}  // extern "C"
