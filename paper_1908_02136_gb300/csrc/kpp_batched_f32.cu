// kpp_batched_f32.cu -- batched-form kernel for F32 points.
#include "kpp_batched.cuh"

namespace kpp {

BatchFn batched_kernel_f32() { return &batched_kernel<KPP_F32>; }

} // namespace kpp
