// emst_32.cu -- minimum-spanning-tree search kernel for dimension bucket DP = 32.
#include "emst.cuh"

namespace dt {
template int launch_emst_nn<32>(const EmstArgs&, int, cudaStream_t);
}  // namespace dt
