// api.cu -- handle lifetime, accessors, status strings and the launch counter.
#include <mutex>

#include "dtree_internal.cuh"

namespace dt {

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_allocs{0};

int cuda_status(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return DTREE_ERR_OOM;
    }
    return DTREE_ERR_CUDA;
}

void prepare_pool(int device) {
    // Keep freed scratch in the stream-ordered pool instead of returning it to
    // the driver after every call.
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> g(mu);
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[device] = true;
}

}  // namespace dt

extern "C" {

void dtree_free(dtree_t* t) {
    if (!t) return;
    cudaFree(t->pts);
    cudaFree(t->idx);
    cudaFree(t->box);
    cudaFree(t->lam);
    cudaFree(t->nbeg);
    cudaFree(t->ncnt);
    cudaFree(t->tc_ops[0]);
    cudaFree(t->tc_ops[1]);
    delete t;
}

int64_t dtree_size(const dtree_t* t) { return t ? t->n : -1; }
int32_t dtree_dim(const dtree_t* t) { return t ? t->d : -1; }
int32_t dtree_depth(const dtree_t* t) { return t ? t->height : -1; }
int64_t dtree_leaf_count(const dtree_t* t) { return t ? t->nleaves : -1; }

int64_t dtree_launch_count(void) { return dt::g_launches.load(); }

int64_t dtree_alloc_count(void) { return dt::g_allocs.load(); }

const char* dtree_error_string(int status) {
    switch (status) {
        case DTREE_OK: return "success";
        case DTREE_ERR_INVALID_ARG: return "invalid argument";
        case DTREE_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of the no-allocation entry point";
        case DTREE_ERR_INVALID_K: return "invalid k (need 0 < k < m, or k <= m - 1 monochromatic)";
        case DTREE_ERR_CUDA: return "CUDA error";
        case DTREE_ERR_OOM: return "out of device memory";
        case DTREE_ERR_TIMEOUT: return "device-side wait timed out";
        case DTREE_ERR_NOT_TRAINED: return "learned proposal requested without a trained model";
        case DTREE_ERR_UNSUPPORTED: return "unsupported on this build or device";
        case DTREE_ERR_IO: return "model file cannot be written or read, or is malformed";
        default: return "unknown status";
    }
}

// Copies one (possibly padded) per-node box row layout into the caller's
// nodes x 2 x d buffer.
static __global__ void k_export_box(const float* box, int64_t nnodes, int d, int dp, float* out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = nnodes * 2 * d;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = t / d;
        int j = (int)(t - row * d);
        out[t] = box[row * dp + j];
    }
}

int dtree_export(const dtree_t* t, int32_t* perm, float* box, float* lambda, int32_t* begin,
                 int32_t* count, void* stream) {
    if (!t) return DTREE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (perm) DT_CHECK(cudaMemcpyAsync(perm, t->idx, t->n * 4, cudaMemcpyDeviceToDevice, s));
    if (lambda) DT_CHECK(cudaMemcpyAsync(lambda, t->lam, t->nnodes * 4, cudaMemcpyDeviceToDevice, s));
    if (begin) DT_CHECK(cudaMemcpyAsync(begin, t->nbeg, t->nnodes * 4, cudaMemcpyDeviceToDevice, s));
    if (count) DT_CHECK(cudaMemcpyAsync(count, t->ncnt, t->nnodes * 4, cudaMemcpyDeviceToDevice, s));
    if (box) {
        int64_t total = t->nnodes * 2 * t->d;
        int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
        DT_LAUNCH(k_export_box, grid, 256, 0, s, t->box, t->nnodes, t->d, t->dp, box);
    }
    DT_CHECK(cudaStreamSynchronize(s));
    return DTREE_OK;
}

}  // extern "C"
