// tc_debug.cu -- dtree_debug_mma: one tcgen05 tile through the same operand
// layout, descriptors and TMEM read-out as the BaseCase kernel, for tests;
// with it, the minima tcgen05.ld.red returns for 32 and 64 columns.
#include <cuda_bf16.h>

#include "dtree_internal.cuh"
#include "tc_ptx.cuh"

namespace dt {
unsigned long long* g_tc_timers = nullptr;
int g_tc_stall = 0;
namespace {

template <int FMT, int KP>
__global__ void __launch_bounds__(128) k_debug_mma(const float* A, const float* B, int K,
                                                   float* out, float* min32, float* min64, int* err,
                                                   int spin) {
    constexpr int esize = FMT == 1 ? 2 : 4;
    constexpr int RB = KP * esize, NCH = RB / 16, SBO = NCH * 128;
    constexpr int NK = KP / (FMT == 1 ? 16 : 8);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + 128 * RB;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int m = 0; m < 2; ++m) {
        const float* src = (m == 0 ? A : B) + (int64_t)tid * K;
        unsigned char* dst = m == 0 ? sA : sB;
        float hv[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            float h = j < K ? src[j] : 0.f;
            hv[j] = FMT == 1 ? __bfloat162float(__float2bfloat16_rn(h)) : tc::to_tf32(h);
        }
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            uint4 w;
            if (FMT == 1) {
                __nv_bfloat162 p0 = __floats2bfloat162_rn(hv[8 * c], hv[8 * c + 1]);
                __nv_bfloat162 p1 = __floats2bfloat162_rn(hv[8 * c + 2], hv[8 * c + 3]);
                __nv_bfloat162 p2 = __floats2bfloat162_rn(hv[8 * c + 4], hv[8 * c + 5]);
                __nv_bfloat162 p3 = __floats2bfloat162_rn(hv[8 * c + 6], hv[8 * c + 7]);
                w.x = *reinterpret_cast<uint32_t*>(&p0);
                w.y = *reinterpret_cast<uint32_t*>(&p1);
                w.z = *reinterpret_cast<uint32_t*>(&p2);
                w.w = *reinterpret_cast<uint32_t*>(&p3);
            } else {
                w.x = __float_as_uint(hv[4 * c]);
                w.y = __float_as_uint(hv[4 * c + 1]);
                w.z = __float_as_uint(hv[4 * c + 2]);
                w.w = __float_as_uint(hv[4 * c + 3]);
            }
            *reinterpret_cast<uint4*>(dst + tc::core_offset(tid, c, SBO)) = w;
        }
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_s, 128);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_s;
    if (tid == 0) {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        const uint32_t id = tc::idesc(FMT, 128, 128);
#pragma unroll
        for (int kk = 0; kk < NK; ++kk)
            tc::mma<FMT>(tmem, tc::sdesc(a0 + 256u * kk, 128u, SBO),
                         tc::sdesc(b0 + 256u * kk, 128u, SBO), id, kk > 0 ? 1u : 0u);
        tc::mma_commit(&bar);
    }
    bool ok = tc::mbar_wait(&bar, 0, spin);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) *err = 1;
        tc::mbar_wait(&bar, 0, spin);
    } else {
        tc::fence_after_sync();
        for (int cc = 0; cc < 4; ++cc) {
            uint32_t v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
            tc::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i) out[(warp * 32 + lane) * 128 + cc * 32 + i] = __uint_as_float(v[i]);
        }
        if (min32) {
            // the same accumulator read with the loads' min reduction, as the
            // BaseCase epilogue reads it
            const int row = warp * 32 + lane;
            for (int cc = 0; cc < 4; ++cc) {
                uint32_t v[32];
                min32[row * 4 + cc] = tc::tmem_ld32_min_wait(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
            }
            for (int cc = 0; cc < 2; ++cc)
                min64[row * 2 + cc] = tc::tmem_min64_wait(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 64));
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

template <int FMT, int KP>
int run_debug(const float* A, const float* B, int K, float* out, float* min32, float* min64, int* err,
              cudaStream_t s) {
    constexpr int esize = FMT == 1 ? 2 : 4;
    size_t smem = 2 * 128 * KP * esize;
    DT_CHECK(cudaFuncSetAttribute(k_debug_mma<FMT, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    DT_LAUNCH((k_debug_mma<FMT, KP>), 1, 128, smem, s, A, B, K, out, min32, min64, err, 1 << 20);
    return DTREE_OK;
}

}  // namespace
}  // namespace dt

namespace {
int debug_mma(const float* A, const float* B, int32_t K, int32_t precision, float* out, float* min32,
              float* min64, void* stream) {
    if (!A || !B || !out || K < 1 || K > 64) return DTREE_ERR_INVALID_ARG;
    if (precision != DTREE_PREC_BF16 && precision != DTREE_PREC_TF32) return DTREE_ERR_INVALID_ARG;
    const int fmt = precision == DTREE_PREC_BF16 ? 1 : 2;  // tcgen05 operand format code
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return DTREE_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    int* err = nullptr;
    DT_CHECK(cudaMallocAsync((void**)&err, sizeof(int), s));
    DT_CHECK(cudaMemsetAsync(err, 0, sizeof(int), s));
    int step = fmt == 1 ? 16 : 8;
    int kp = (K + step - 1) / step * step;
    int rc = DTREE_ERR_INVALID_ARG;
    if (fmt == 1) {
        rc = kp <= 16 ? dt::run_debug<1, 16>(A, B, K, out, min32, min64, err, s)
             : kp <= 32 ? dt::run_debug<1, 32>(A, B, K, out, min32, min64, err, s)
                        : dt::run_debug<1, 64>(A, B, K, out, min32, min64, err, s);
    } else {
        rc = kp <= 8 ? dt::run_debug<2, 8>(A, B, K, out, min32, min64, err, s)
             : kp <= 16 ? dt::run_debug<2, 16>(A, B, K, out, min32, min64, err, s)
             : kp <= 32 ? dt::run_debug<2, 32>(A, B, K, out, min32, min64, err, s)
                        : dt::run_debug<2, 64>(A, B, K, out, min32, min64, err, s);
    }
    int herr = 0;
    if (rc == DTREE_OK) {
        DT_CHECK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        DT_CHECK(cudaStreamSynchronize(s));
    }
    cudaFreeAsync(err, s);
    if (rc != DTREE_OK) return rc;
    return herr ? DTREE_ERR_TIMEOUT : DTREE_OK;
}
}  // namespace

extern "C" int dtree_debug_mma(const float* A, const float* B, int32_t K, int32_t precision,
                               float* out, void* stream) {
    return debug_mma(A, B, K, precision, out, nullptr, nullptr, stream);
}

extern "C" int dtree_debug_tmem_min(const float* A, const float* B, int32_t K, int32_t precision,
                                    float* out, float* min32, float* min64, void* stream) {
    if (!min32 || !min64) return DTREE_ERR_INVALID_ARG;
    return debug_mma(A, B, K, precision, out, min32, min64, stream);
}

extern "C" int dtree_debug_tc_timers(unsigned long long* counters) {
    dt::g_tc_timers = counters;
    return DTREE_OK;
}

extern "C" int dtree_debug_tc_stall(int32_t on) {
    dt::g_tc_stall = on ? 1 : 0;
    return DTREE_OK;
}

