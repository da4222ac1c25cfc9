// emst_16.cu -- minimum-spanning-tree search kernel for dimension bucket DP = 16.
#include "emst.cuh"

namespace dt {
template int launch_emst_nn<16>(const EmstArgs&, int, cudaStream_t);
}  // namespace dt
