// emst.cu -- dtree_emst: the Euclidean minimum spanning tree by Boruvka
// rounds, host side and the round's small kernels (the nearest-edge search
// and the reading of Section 7 are in emst.cuh).
#include <algorithm>
#include <cstring>

#include "emst.cuh"

namespace dt {
namespace {

__global__ void k_emst_iota(int32_t* v, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

// Leaf labels: the leaf's component when all its points share one, else -1.
__global__ void k_emst_leaf_lab(const int32_t* comp, const int32_t* nbeg, const int32_t* ncnt,
                                int64_t leaf0, int64_t nleaves, int32_t* nlab) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nleaves) return;
    const int64_t nd = leaf0 + i;
    const int b = nbeg[nd], c = ncnt[nd];
    int32_t lab = c > 0 ? comp[b] : -1;
    for (int j = 1; j < c && lab >= 0; ++j)
        if (comp[b + j] != lab) lab = -1;
    nlab[nd] = lab;
}

// The nodes of one level from their children's labels.
__global__ void k_emst_up(int64_t first, int64_t count, int32_t* nlab) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t nd = first + i;
    const int32_t a = nlab[2 * nd + 1], b = nlab[2 * nd + 2];
    nlab[nd] = (a == b && a >= 0) ? a : -1;
}

// Every component's shortest edge out, by length ...
__global__ void k_emst_min1(const int32_t* comp, const double* bd, const int32_t* br, int64_t n,
                            unsigned long long* ck1) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && br[i] >= 0) atomicMin(&ck1[comp[i]], dkey(bd[i]));
}

// ... then by endpoints among the points that reach that length ...
__global__ void k_emst_min2(const int32_t* comp, const double* bd, const int32_t* br,
                            const int32_t* idx, int64_t n, const unsigned long long* ck1,
                            unsigned long long* ck2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || br[i] < 0 || dkey(bd[i]) != ck1[comp[i]]) return;
    const uint32_t a = (uint32_t)idx[i], b = (uint32_t)idx[br[i]];
    atomicMin(&ck2[comp[i]], ((unsigned long long)min(a, b) << 32) | max(a, b));
}

// ... and the one point of the component that holds it.
__global__ void k_emst_pick(const int32_t* comp, const double* bd, const int32_t* br,
                            const int32_t* idx, int64_t n, const unsigned long long* ck1,
                            const unsigned long long* ck2, int32_t* pick) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || br[i] < 0) return;
    const int32_t c = comp[i];
    const uint32_t a = (uint32_t)idx[i], b = (uint32_t)idx[br[i]];
    if (dkey(bd[i]) == ck1[c] && (((unsigned long long)min(a, b) << 32) | max(a, b)) == ck2[c])
        pick[c] = (int32_t)i;
}

// Hooks: a component points to the one across its edge; of two components
// that chose the same edge, the lower id stays a root and writes the edge.
__global__ void k_emst_hook(const int32_t* comp, const int32_t* br, const int32_t* pick,
                            const unsigned long long* ck1, const unsigned long long* ck2,
                            int64_t n, int32_t* par, int64_t* adds) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    par[c] = (int32_t)c;
    adds[c] = 0;
    const int32_t p = pick[c];
    if (p < 0) return;
    const int32_t o = comp[br[p]];
    const bool mutual = pick[o] >= 0 && ck1[o] == ck1[c] && ck2[o] == ck2[c];
    par[c] = (mutual && c < o) ? (int32_t)c : o;
    adds[c] = (!mutual || c < o) ? 1 : 0;
}

// In place: a[0..n) -> exclusive prefix sums, a[n] = the total (one CTA).
__global__ void __launch_bounds__(1024) k_emst_scan(int64_t* a, int64_t n) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t b0 = t * chunk, b = b0 < n ? b0 : n, e = b + chunk < n ? b + chunk : n;
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int64_t i = b; i < e; ++i) {
        const int64_t v = a[i];
        a[i] = run;
        run += v;
    }
    if (t == 1023) a[n] = part[1023];
}

// The round's edges, in component-id order after the ones written before.
__global__ void k_emst_emit(const int32_t* pick, const int32_t* br, const double* bd,
                            const int32_t* idx, const int64_t* offs, int64_t n, int64_t base,
                            int64_t* edges, float* dist) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n || offs[c + 1] == offs[c]) return;
    const int32_t p = pick[c];
    const int32_t a = idx[p], b = idx[br[p]];
    const int64_t slot = base + offs[c];
    if (slot >= n - 1) return;  // (cannot happen: the host reports a count other than n - 1)
    edges[2 * slot] = min(a, b);
    edges[2 * slot + 1] = max(a, b);
    dist[slot] = (float)sqrt(bd[p]);
}

__global__ void k_emst_jump(int32_t* par, int64_t n, int* changed) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t p = par[i], pp = par[p];
    if (pp != p) {
        par[i] = pp;
        *changed = 1;
    }
}

__global__ void k_emst_relabel(int32_t* comp, const int32_t* par, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) comp[i] = par[comp[i]];
}

int emst_nn(int dp, const EmstArgs& a, int grid, cudaStream_t s) {
    switch (dp) {
        case 4: return launch_emst_nn<4>(a, grid, s);
        case 8: return launch_emst_nn<8>(a, grid, s);
        case 16: return launch_emst_nn<16>(a, grid, s);
        case 32: return launch_emst_nn<32>(a, grid, s);
        default: return launch_emst_nn<64>(a, grid, s);
    }
}

inline int g256(int64_t n) { return (int)std::max<int64_t>(1, (n + 255) / 256); }

}  // namespace
}  // namespace dt

extern "C" int dtree_emst(const dtree_t* t, int64_t* out_edges, float* out_dist, const dtree_opts* o,
                          void* stream, dtree_stats* st) {
    using namespace dt;
    if (st) memset(st, 0, sizeof(*st));
    if (!t) return DTREE_ERR_INVALID_ARG;
    const int64_t n = t->n;
    if (n > 1 && (!out_edges || !out_dist)) return DTREE_ERR_INVALID_ARG;
    if (o) {
        for (int i = 0; i < 8; ++i)
            if (o->reserved[i]) return DTREE_ERR_INVALID_ARG;
        if (o->precision != DTREE_PREC_FP32 || o->bound != DTREE_BOUND_BOX) return DTREE_ERR_UNSUPPORTED;
    }
    if (t->height > 30) return DTREE_ERR_UNSUPPORTED;  // the depth-first stack: one entry per lane
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (t->device != dev) return DTREE_ERR_INVALID_ARG;
    if (n < 2) return DTREE_OK;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t launches0 = g_launches.load();
    const int64_t nn = t->nnodes;
    // scratch, one block: comp, br, pick, par (int32 n each), nlab (int32
    // nodes), bd (double n), ck1, ck2 (u64 n each), adds (int64 n + 1),
    // counters
    const size_t b_i32 = (size_t)n * 4, b_nl = (size_t)nn * 4, b_d = (size_t)n * 8;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_comp = 0, o_br = al(o_comp + b_i32), o_pick = al(o_br + b_i32),
                 o_par = al(o_pick + b_i32), o_nlab = al(o_par + b_i32), o_bd = al(o_nlab + b_nl),
                 o_ck1 = al(o_bd + b_d), o_ck2 = al(o_ck1 + b_d), o_adds = al(o_ck2 + b_d),
                 o_cnt = al(o_adds + (size_t)(n + 1) * 8), bytes = o_cnt + 64;
    unsigned char* m = nullptr;
    DT_CHECK(cudaMallocAsync((void**)&m, bytes, s));
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    int32_t* comp = reinterpret_cast<int32_t*>(m + o_comp);
    int32_t* br = reinterpret_cast<int32_t*>(m + o_br);
    int32_t* pick = reinterpret_cast<int32_t*>(m + o_pick);
    int32_t* par = reinterpret_cast<int32_t*>(m + o_par);
    int32_t* nlab = reinterpret_cast<int32_t*>(m + o_nlab);
    double* bd = reinterpret_cast<double*>(m + o_bd);
    unsigned long long* ck1 = reinterpret_cast<unsigned long long*>(m + o_ck1);
    unsigned long long* ck2 = reinterpret_cast<unsigned long long*>(m + o_ck2);
    int64_t* adds = reinterpret_cast<int64_t*>(m + o_adds);
    int* changed = reinterpret_cast<int*>(m + o_cnt);
    unsigned long long* cstats = reinterpret_cast<unsigned long long*>(m + o_cnt + 16);
    EmstArgs a{};
    a.pts = t->pts;
    a.idx = t->idx;
    a.nbeg = t->nbeg;
    a.ncnt = t->ncnt;
    a.box = t->box;
    a.n = n;
    a.hr = t->height;
    a.comp = comp;
    a.nlab = nlab;
    a.bd = bd;
    a.br = br;
    a.ck1 = ck1;
    a.stats = cstats;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 3) / 4, (int64_t)sms * 16));
    const int64_t leaf0 = ((int64_t)1 << t->height) - 1, nleaves = (int64_t)1 << t->height;
    cudaEvent_t ev[2] = {};
    const bool timed = st && cudaEventCreate(&ev[0]) == cudaSuccess && cudaEventCreate(&ev[1]) == cudaSuccess;
    cudaGetLastError();
    int rc = DTREE_OK;
    int64_t base = 0;
    unsigned long long hs[2] = {0, 0};
    auto launch_ok = [&]() {
        g_launches.fetch_add(1, std::memory_order_relaxed);
        return cudaGetLastError() == cudaSuccess;
    };
    do {
        if (cudaMemsetAsync(cstats, 0, 16, s) != cudaSuccess) { rc = DTREE_ERR_CUDA; break; }
        if (timed) cudaEventRecord(ev[0], s);
        k_emst_iota<<<g256(n), 256, 0, s>>>(comp, n);
        if (!launch_ok()) { rc = DTREE_ERR_CUDA; break; }
        // each round at least halves the number of components
        for (int round = 0; round < 64 && base < n - 1 && rc == DTREE_OK; ++round) {
            k_emst_leaf_lab<<<g256(nleaves), 256, 0, s>>>(comp, t->nbeg, t->ncnt, leaf0, nleaves, nlab);
            if (!launch_ok()) { rc = DTREE_ERR_CUDA; break; }
            for (int L = t->height - 1; L >= 0; --L) {
                const int64_t cnt = (int64_t)1 << L;
                k_emst_up<<<g256(cnt), 256, 0, s>>>(cnt - 1, cnt, nlab);
                if (!launch_ok()) { rc = DTREE_ERR_CUDA; break; }
            }
            if (rc != DTREE_OK) break;
            if (cudaMemsetAsync(ck1, 0xff, b_d, s) != cudaSuccess ||
                cudaMemsetAsync(ck2, 0xff, b_d, s) != cudaSuccess ||
                cudaMemsetAsync(pick, 0xff, b_i32, s) != cudaSuccess) {
                rc = DTREE_ERR_CUDA;
                break;
            }
            rc = emst_nn(t->dp, a, grid, s);
            if (rc != DTREE_OK) break;
            k_emst_min1<<<g256(n), 256, 0, s>>>(comp, bd, br, n, ck1);
            k_emst_min2<<<g256(n), 256, 0, s>>>(comp, bd, br, t->idx, n, ck1, ck2);
            k_emst_pick<<<g256(n), 256, 0, s>>>(comp, bd, br, t->idx, n, ck1, ck2, pick);
            k_emst_hook<<<g256(n), 256, 0, s>>>(comp, br, pick, ck1, ck2, n, par, adds);
            k_emst_scan<<<1, 1024, 0, s>>>(adds, n);
            k_emst_emit<<<g256(n), 256, 0, s>>>(pick, br, bd, t->idx, adds, n, base, out_edges, out_dist);
            g_launches.fetch_add(5, std::memory_order_relaxed);
            if (!launch_ok()) { rc = DTREE_ERR_CUDA; break; }
            // pointer jumping to the roots
            for (int it = 0; it < 64; ++it) {
                int h = 0;
                if (cudaMemsetAsync(changed, 0, sizeof(int), s) != cudaSuccess) { rc = DTREE_ERR_CUDA; break; }
                k_emst_jump<<<g256(n), 256, 0, s>>>(par, n, changed);
                if (!launch_ok() ||
                    cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) {
                    rc = DTREE_ERR_CUDA;
                    break;
                }
                if (!h) break;
            }
            if (rc != DTREE_OK) break;
            k_emst_relabel<<<g256(n), 256, 0, s>>>(comp, par, n);
            if (!launch_ok()) { rc = DTREE_ERR_CUDA; break; }
            int64_t added = 0;
            if (cudaMemcpyAsync(&added, adds + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = DTREE_ERR_CUDA;
                break;
            }
            if (added <= 0) rc = DTREE_ERR_CUDA;  // no edge left to add: cannot happen with >= 2 components
            base += added;
        }
        if (rc == DTREE_OK && base != n - 1) rc = DTREE_ERR_CUDA;
        if (timed) cudaEventRecord(ev[1], s);
        if (st && cudaMemcpyAsync(hs, cstats, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = DTREE_ERR_CUDA;
    } while (false);
    cudaFreeAsync(m, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == DTREE_OK) rc = cuda_status(cudaGetLastError());
    if (st && rc == DTREE_OK) {
        st->point_pairs = (int64_t)hs[0];
        st->leaf_pairs_evaluated = (int64_t)hs[1];
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
