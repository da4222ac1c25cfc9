// emst_4.cu -- minimum-spanning-tree search kernel for dimension bucket DP = 4.
#include "emst.cuh"

namespace dt {
template int launch_emst_nn<4>(const EmstArgs&, int, cudaStream_t);
}  // namespace dt
