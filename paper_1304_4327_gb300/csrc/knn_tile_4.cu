// knn_tile_4.cu -- CUDA-core BaseCase tiles for dimension bucket DP = 4.
#include "knn_tile.cuh"

namespace dt {
template int launch_tile_cc<4>(const TileArgs&, int, int, int, cudaStream_t);
template int launch_query_cap<4>(const TileArgs&, int, int, float*, cudaStream_t);
}  // namespace dt
