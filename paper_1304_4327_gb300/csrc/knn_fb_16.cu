// knn_fb_16.cu -- per-query recomputation of band overflows (k_query_fb) for
// dimension bucket DP = 16 (its own translation unit, to compile in parallel).
#include "knn_tile.cuh"

namespace dt {
template int launch_query_fb<16>(const TileArgs&, int, int, bool, cudaStream_t);
}  // namespace dt
