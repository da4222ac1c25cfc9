// emst_64.cu -- minimum-spanning-tree search kernel for dimension bucket DP = 64.
#include "emst.cuh"

namespace dt {
template int launch_emst_nn<64>(const EmstArgs&, int, cudaStream_t);
}  // namespace dt
