// range_64.cu -- range search kernels for dimension bucket DP = 64.
#include "range.cuh"

namespace dt {
template int launch_range<64>(const RangeArgs&, bool, int, cudaStream_t);
}  // namespace dt
