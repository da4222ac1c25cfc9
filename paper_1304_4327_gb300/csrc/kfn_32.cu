// kfn_32.cu -- k-furthest-neighbour search kernels for dimension bucket DP = 32.
#include "kfn.cuh"

namespace dt {
template int launch_kfn<32>(const KfnArgs&, int, bool, int, cudaStream_t);
}  // namespace dt
