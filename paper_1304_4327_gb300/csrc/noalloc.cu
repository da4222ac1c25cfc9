// noalloc.cu -- dtree_knn_noalloc: dtree_knn with its per-call scratch carved
// from one file-scope static device array instead of the stream-ordered pool,
// so that a call allocates nothing.  The search itself is dtree_knn's (same
// kernels, same results); only where the scratch lives differs.
#include "dtree_internal.cuh"

namespace dt {
namespace {

constexpr size_t kStaticScratchBytes = DTREE_NOALLOC_SCRATCH_BYTES;

// The scratch.  Zero at module load; afterwards it holds whatever the last
// call left, and the call clears what must start at zero itself.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// The array's address on the current device.  It is looked up on every
// call (cudaGetSymbolAddress allocates nothing), so a context that was reset
// and reloaded the module never gets a stale address.
int scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return DTREE_ERR_CUDA;
    }
    *out = p;
    return DTREE_OK;
}

}  // namespace
}  // namespace dt

extern "C" int dtree_knn_noalloc(const dtree_t* query, const dtree_t* ref, int32_t k,
                                 int64_t* out_idx, float* out_dist, const dtree_opts* opts,
                                 void* stream) {
    if (!ref) return DTREE_ERR_INVALID_ARG;
    const dtree_t* tq = (query == nullptr || query == ref) ? ref : query;
    if (tq->n > DTREE_NOALLOC_MAX_QUERIES) return DTREE_ERR_TOO_LARGE;
    void* base = nullptr;
    const int rc = dt::scratch_address(&base);
    if (rc != DTREE_OK) return rc;
    const dt::ScratchArena arena{static_cast<unsigned char*>(base), dt::kStaticScratchBytes};
    return dt::knn_entry(query, ref, k, out_idx, out_dist, opts, stream, nullptr, &arena);
}
