// kpp_batched_bf16.cu -- batched-form wave kernels for BF16 points, one per d.
#include "kpp_batched.cuh"

namespace kpp {

BatchFn batched_kernel_bf16(int d) { return batched_kernel_of<KPP_BF16>(d); }

} // namespace kpp
