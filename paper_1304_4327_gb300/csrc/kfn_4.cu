// kfn_4.cu -- k-furthest-neighbour search kernels for dimension bucket DP = 4.
#include "kfn.cuh"

namespace dt {
template int launch_kfn<4>(const KfnArgs&, int, bool, int, cudaStream_t);
}  // namespace dt
