// knn_tile_8.cu -- CUDA-core BaseCase tiles for dimension bucket DP = 8.
#include "knn_tile.cuh"

namespace dt {
template int launch_tile_cc<8>(const TileArgs&, int, int, int, cudaStream_t);
template int launch_query_cap<8>(const TileArgs&, int, int, float*, cudaStream_t);
}  // namespace dt
