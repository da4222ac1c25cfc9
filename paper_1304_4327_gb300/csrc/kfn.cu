// kfn.cu -- dtree_kfn: exact k-furthest-neighbour search, host side (the
// kernels and their reading of Section 5 are in kfn.cuh).
#include <algorithm>
#include <cstring>

#include "kfn.cuh"

namespace dt {
namespace {

int kfn_launch(int dp, const KfnArgs& a, int kc, bool exact, int grid, cudaStream_t s) {
    switch (dp) {
        case 4: return launch_kfn<4>(a, kc, exact, grid, s);
        case 8: return launch_kfn<8>(a, kc, exact, grid, s);
        case 16: return launch_kfn<16>(a, kc, exact, grid, s);
        case 32: return launch_kfn<32>(a, kc, exact, grid, s);
        default: return launch_kfn<64>(a, kc, exact, grid, s);
    }
}

}  // namespace
}  // namespace dt

extern "C" int dtree_kfn(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
                         float* out_dist, const dtree_opts* o, void* stream, dtree_stats* st) {
    using namespace dt;
    if (st) memset(st, 0, sizeof(*st));
    if (!ref) return DTREE_ERR_INVALID_ARG;
    const bool mono = query == nullptr || query == ref;
    const dtree_t* tq = mono ? ref : query;
    const int64_t m = ref->n, nq = tq->n;
    if (k <= 0 || (mono ? (int64_t)k > m - 1 : (int64_t)k >= m)) return DTREE_ERR_INVALID_K;
    if (!out_idx || !out_dist || tq->d != ref->d) return DTREE_ERR_INVALID_ARG;
    if (o) {
        for (int i = 0; i < 8; ++i)
            if (o->reserved[i]) return DTREE_ERR_INVALID_ARG;
        if (o->precision != DTREE_PREC_FP32 || o->bound != DTREE_BOUND_BOX) return DTREE_ERR_UNSUPPORTED;
    }
    // lists of up to 64 entries; the depth-first stack holds one entry per lane
    if (k > 63 || ref->height > 30) return DTREE_ERR_UNSUPPORTED;
    int dev = 0;
    cudaGetDevice(&dev);
    if (ref->device != dev || tq->device != dev) return DTREE_ERR_INVALID_ARG;
    const int kc = k + 1 <= 16 ? 16 : k + 1 <= 32 ? 32 : 64;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t launches0 = g_launches.load();

    // scratch: three counters, the fallback count, and the fallback list
    unsigned char* scratch = nullptr;
    const size_t bytes = 32 + 16 + (size_t)nq * sizeof(int);
    DT_CHECK(cudaMallocAsync((void**)&scratch, bytes, s));
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    KfnArgs a{};
    a.qpts = tq->pts;
    a.qidx = tq->idx;
    a.nq = nq;
    a.rpts = ref->pts;
    a.ridx = ref->idx;
    a.rbeg = ref->nbeg;
    a.rcnt = ref->ncnt;
    a.rbox = ref->box;
    a.hr = ref->height;
    a.k = k;
    a.mono = mono ? 1 : 0;
    a.out_idx = out_idx;
    a.out_dist = out_dist;
    a.stats = reinterpret_cast<unsigned long long*>(scratch);
    a.fb_count = reinterpret_cast<int*>(scratch + 32);
    a.fb_list = reinterpret_cast<int*>(scratch + 48);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t ev[2] = {};
    const bool timed = st && cudaEventCreate(&ev[0]) == cudaSuccess && cudaEventCreate(&ev[1]) == cudaSuccess;
    cudaGetLastError();
    int rc = DTREE_OK;
    int nfb = 0;
    unsigned long long cnt[3] = {0, 0, 0};
    do {
        if (cudaMemsetAsync(scratch, 0, 48, s) != cudaSuccess) { rc = cuda_status(cudaGetLastError()); break; }
        if (timed) cudaEventRecord(ev[0], s);
        // one warp per query, four per CTA; a grid of whole waves of CTAs
        const int64_t want = (nq + 3) / 4;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 16));
        rc = kfn_launch(ref->dp, a, kc, false, grid, s);
        if (rc != DTREE_OK) break;
        if (cudaMemcpyAsync(&nfb, a.fb_count, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = cuda_status(cudaGetLastError());
            break;
        }
        if (nfb > 0) {
            const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)nfb + 3) / 4, (int64_t)sms * 16));
            rc = kfn_launch(ref->dp, a, kc, true, g2, s);
            if (rc != DTREE_OK) break;
        }
        if (timed) cudaEventRecord(ev[1], s);
        if (st && cudaMemcpyAsync(cnt, a.stats, sizeof(cnt), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            rc = cuda_status(cudaGetLastError());
            break;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = cuda_status(cudaGetLastError());
    } while (false);
    cudaFreeAsync(scratch, s);
    if (rc == DTREE_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = cuda_status(cudaGetLastError());
    if (st && rc == DTREE_OK) {
        st->point_pairs = (int64_t)cnt[0];
        st->leaf_pairs_evaluated = (int64_t)cnt[1];
        st->node_pairs_pruned = (int64_t)cnt[2];
        st->fallback_queries = nfb;
        st->fallback64_queries = nfb;
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
