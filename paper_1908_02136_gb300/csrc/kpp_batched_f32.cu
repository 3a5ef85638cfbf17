// kpp_batched_f32.cu -- batched-form wave kernels for F32 points, one per d.
#include "kpp_batched.cuh"

namespace kpp {

BatchFn batched_kernel_f32(int d) { return batched_kernel_of<KPP_F32>(d); }

} // namespace kpp
