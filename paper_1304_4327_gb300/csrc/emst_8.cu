// emst_8.cu -- minimum-spanning-tree search kernel for dimension bucket DP = 8.
#include "emst.cuh"

namespace dt {
template int launch_emst_nn<8>(const EmstArgs&, int, cudaStream_t);
}  // namespace dt
