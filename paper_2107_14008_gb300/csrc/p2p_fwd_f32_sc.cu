// FP32 forward P2P, scalar-stream variant (see fwd_f32_common.cuh).
#include "fwd_f32_common.cuh"

namespace psr {

template int launch_fwd_f32_variant<false>(const FwdArgs&, int, size_t, cudaStream_t);
template const void* fwd_f32_kernel_ptr<false>(int, int, int, int);

}  // namespace psr
