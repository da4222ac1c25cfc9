// knn_tile_64.cu -- CUDA-core BaseCase tiles for dimension bucket DP = 64.
#include "knn_tile.cuh"

namespace dt {
template int launch_tile_cc<64>(const TileArgs&, int, int, int, cudaStream_t);
template int launch_query_cap<64>(const TileArgs&, int, int, float*, cudaStream_t);
}  // namespace dt
