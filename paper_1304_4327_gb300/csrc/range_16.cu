// range_16.cu -- range search kernels for dimension bucket DP = 16.
#include "range.cuh"

namespace dt {
template int launch_range<16>(const RangeArgs&, bool, int, cudaStream_t);
}  // namespace dt
