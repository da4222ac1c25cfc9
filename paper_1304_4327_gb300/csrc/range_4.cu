// range_4.cu -- range search kernels for dimension bucket DP = 4.
#include "range.cuh"

namespace dt {
template int launch_range<4>(const RangeArgs&, bool, int, cudaStream_t);
}  // namespace dt
