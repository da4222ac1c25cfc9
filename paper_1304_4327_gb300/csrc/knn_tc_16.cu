// knn_tc_16.cu -- tensor-core BaseCase tiles for dimension bucket DP = 16.
#include "knn_tc.cuh"

namespace dt {
template int launch_tile_tc<16>(const TileArgs&, int, int, int, int, int*, int, cudaStream_t);
}  // namespace dt
