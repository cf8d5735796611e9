// FP16 instantiations of the stencil's alternative launch configurations (hop_tuned.cuh).
#include "hop_tuned.cuh"

namespace lq {
template int hop_lin_tuned<16>(int, bool, int, int, dim3, const HopArgs&, cudaStream_t);
template int hop_clinv_tuned<16>(int, bool, int, dim3, const HopArgs&, cudaStream_t);
}  // namespace lq
