// knn_tile_16.cu -- CUDA-core BaseCase tiles for dimension bucket DP = 16.
#include "knn_tile.cuh"

namespace dt {
template int launch_tile_cc<16>(const TileArgs&, int, int, int, cudaStream_t);
template int launch_query_cap<16>(const TileArgs&, int, int, float*, cudaStream_t);
}  // namespace dt
