// range_32.cu -- range search kernels for dimension bucket DP = 32.
#include "range.cuh"

namespace dt {
template int launch_range<32>(const RangeArgs&, bool, int, cudaStream_t);
}  // namespace dt
