// knn_fb_8.cu -- per-query recomputation of band overflows (k_query_fb) for
// dimension bucket DP = 8 (its own translation unit, to compile in parallel).
#include "knn_tile.cuh"

namespace dt {
template int launch_query_fb<8>(const TileArgs&, int, int, bool, cudaStream_t);
}  // namespace dt
