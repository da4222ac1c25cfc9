// range_8.cu -- range search kernels for dimension bucket DP = 8.
#include "range.cuh"

namespace dt {
template int launch_range<8>(const RangeArgs&, bool, int, cudaStream_t);
}  // namespace dt
