// kfn_8.cu -- k-furthest-neighbour search kernels for dimension bucket DP = 8.
#include "kfn.cuh"

namespace dt {
template int launch_kfn<8>(const KfnArgs&, int, bool, int, cudaStream_t);
}  // namespace dt
