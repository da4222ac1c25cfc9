// knn_tc_16.cu -- tensor-core BaseCase tiles for dimension bucket DP = 16.
#include "knn_tc.cuh"

namespace dt {
template int launch_tile_tc<16>(const TileArgs&, int, int, int, int*, int, cudaStream_t);
template size_t tc_ops_row_bytes<16>(int);
template int launch_tc_ops<16>(const dtree_t*, int, int, void*, cudaStream_t);
}  // namespace dt
