// range.cu -- dtree_range_count / dtree_range_fill: exact range search, host
// side, and the scan that turns per-query counts into segment offsets (the
// kernels and their reading of Section 6 are in range.cuh).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "range.cuh"

namespace dt {
namespace {

// In place: counts c[0..n) -> exclusive prefix sums, and c[n] = the total.
// One CTA; each thread sums a contiguous chunk, the chunk sums are scanned in
// shared memory, then each thread rewrites its chunk.
__global__ void __launch_bounds__(1024) k_range_scan(int64_t* c, int64_t n) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t b0 = t * chunk, b = b0 < n ? b0 : n, e = b + chunk < n ? b + chunk : n;
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += c[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;  // exclusive
    for (int64_t i = b; i < e; ++i) {
        const int64_t v = c[i];
        c[i] = run;
        run += v;
    }
    if (t == 1023) c[n] = part[1023];
}

int range_launch(int dp, const RangeArgs& a, bool fill, int grid, cudaStream_t s) {
    switch (dp) {
        case 4: return launch_range<4>(a, fill, grid, s);
        case 8: return launch_range<8>(a, fill, grid, s);
        case 16: return launch_range<16>(a, fill, grid, s);
        case 32: return launch_range<32>(a, fill, grid, s);
        default: return launch_range<64>(a, fill, grid, s);
    }
}

// Shared argument checks; fills the tree fields and the float bounds.
int range_setup(const dtree_t* query, const dtree_t* ref, double d_lo, double d_hi,
                const dtree_opts* o, RangeArgs* a) {
    if (!ref) return DTREE_ERR_INVALID_ARG;
    const bool mono = query == nullptr || query == ref;
    const dtree_t* tq = mono ? ref : query;
    if (tq->d != ref->d) return DTREE_ERR_INVALID_ARG;
    if (!(d_lo >= 0.0) || !(d_hi >= d_lo)) return DTREE_ERR_INVALID_ARG;  // (NaN fails both)
    if (o) {
        for (int i = 0; i < 8; ++i)
            if (o->reserved[i]) return DTREE_ERR_INVALID_ARG;
        if (o->precision != DTREE_PREC_FP32 || o->bound != DTREE_BOUND_BOX) return DTREE_ERR_UNSUPPORTED;
    }
    if (ref->height > 30) return DTREE_ERR_UNSUPPORTED;  // the depth-first stack: one entry per lane
    int dev = 0;
    cudaGetDevice(&dev);
    if (ref->device != dev || tq->device != dev) return DTREE_ERR_INVALID_ARG;
    memset(a, 0, sizeof(*a));
    a->qpts = tq->pts;
    a->qidx = tq->idx;
    a->nq = tq->n;
    a->rpts = ref->pts;
    a->ridx = ref->idx;
    a->rbeg = ref->nbeg;
    a->rcnt = ref->ncnt;
    a->rbox = ref->box;
    a->hr = ref->height;
    a->mono = mono ? 1 : 0;
    a->d_lo = d_lo;
    a->d_hi = d_hi;
    // floats below and above the squared ends, 1e-12 apart from them
    const double lo2 = d_lo * d_lo, hi2 = d_hi * d_hi;
    a->lo2_dn = std::nextafter((float)(lo2 * (1.0 - 1e-12)), -INFINITY);
    a->lo2_up = std::nextafter((float)(lo2 * (1.0 + 1e-12)), INFINITY);
    a->hi2_dn = std::isinf(hi2) ? INFINITY : std::nextafter((float)(hi2 * (1.0 - 1e-12)), -INFINITY);
    a->hi2_up = std::isinf(hi2) ? INFINITY : std::nextafter((float)(hi2 * (1.0 + 1e-12)), INFINITY);
    if (a->lo2_dn < 0.f) a->lo2_dn = 0.f;
    return DTREE_OK;
}

int range_grid(int64_t nq) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::max<int64_t>(1, std::min<int64_t>((nq + 3) / 4, (int64_t)sms * 16));
}

}  // namespace
}  // namespace dt

extern "C" int dtree_range_count(const dtree_t* query, const dtree_t* ref, double d_lo, double d_hi,
                                 int64_t* offsets, int64_t* total, const dtree_opts* o, void* stream,
                                 dtree_stats* st) {
    using namespace dt;
    if (st) memset(st, 0, sizeof(*st));
    RangeArgs a;
    int rc = range_setup(query, ref, d_lo, d_hi, o, &a);
    if (rc != DTREE_OK) return rc;
    if (!offsets || !total) return DTREE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t launches0 = g_launches.load();
    unsigned long long* cnt = nullptr;
    DT_CHECK(cudaMallocAsync((void**)&cnt, 4 * sizeof(unsigned long long), s));
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    a.counts = offsets;
    a.stats = cnt;
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaEvent_t ev[2] = {};
    const bool timed = st && cudaEventCreate(&ev[0]) == cudaSuccess && cudaEventCreate(&ev[1]) == cudaSuccess;
    cudaGetLastError();
    do {
        if (cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), s) != cudaSuccess) {
            rc = cuda_status(cudaGetLastError());
            break;
        }
        if (timed) cudaEventRecord(ev[0], s);
        rc = range_launch(ref->dp, a, false, range_grid(a.nq), s);
        if (rc != DTREE_OK) break;
        k_range_scan<<<1, 1024, 0, s>>>(offsets, a.nq);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if (cudaGetLastError() != cudaSuccess) {
            rc = DTREE_ERR_CUDA;
            break;
        }
        if (timed) cudaEventRecord(ev[1], s);
        if (cudaMemcpyAsync(total, offsets + a.nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            rc = cuda_status(cudaGetLastError());
            break;
        }
    } while (false);
    cudaFreeAsync(cnt, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == DTREE_OK) rc = cuda_status(cudaGetLastError());
    if (st && rc == DTREE_OK) {
        st->point_pairs = (int64_t)h[0];
        st->leaf_pairs_evaluated = (int64_t)h[1];
        st->node_pairs_pruned = (int64_t)h[2];
        st->rerank_candidates = (int64_t)h[3];
        float ms = 0.f;
        if (timed && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) st->ns_basecase = (int64_t)(ms * 1e6);
        st->kernel_launches = g_launches.load() - launches0;
    }
    if (timed) {
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    cudaGetLastError();
    return rc;
}

extern "C" int dtree_range_fill(const dtree_t* query, const dtree_t* ref, double d_lo, double d_hi,
                                const int64_t* offsets, int64_t* out_idx, float* out_dist,
                                const dtree_opts* o, void* stream) {
    using namespace dt;
    RangeArgs a;
    int rc = range_setup(query, ref, d_lo, d_hi, o, &a);
    if (rc != DTREE_OK) return rc;
    if (!offsets || !out_idx || !out_dist) return DTREE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    a.offsets = offsets;
    a.out_idx = out_idx;
    a.out_dist = out_dist;
    rc = range_launch(ref->dp, a, true, range_grid(a.nq), s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == DTREE_OK) rc = cuda_status(cudaGetLastError());
    return rc;
}
