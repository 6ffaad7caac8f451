// FP32 forward P2P, packed-pair variant (see fwd_f32_common.cuh).
#include "fwd_f32_common.cuh"

namespace psr {

template int launch_fwd_f32_variant<true>(const FwdArgs&, int, size_t, cudaStream_t);
template const void* fwd_f32_kernel_ptr<true>(int, int, int, int);

}  // namespace psr
