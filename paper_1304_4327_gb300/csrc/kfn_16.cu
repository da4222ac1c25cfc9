// kfn_16.cu -- k-furthest-neighbour search kernels for dimension bucket DP = 16.
#include "kfn.cuh"

namespace dt {
template int launch_kfn<16>(const KfnArgs&, int, bool, int, cudaStream_t);
}  // namespace dt
