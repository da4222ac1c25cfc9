// kfn_64.cu -- k-furthest-neighbour search kernels for dimension bucket DP = 64.
#include "kfn.cuh"

namespace dt {
template int launch_kfn<64>(const KfnArgs&, int, bool, int, cudaStream_t);
}  // namespace dt
