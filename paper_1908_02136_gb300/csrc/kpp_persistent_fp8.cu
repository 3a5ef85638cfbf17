// kpp_persistent_fp8.cu -- persistent-form kernels for FP8 points.
#include "kpp_persistent.cuh"

namespace kpp {

namespace {
const PSpec kSpecs[] = {
    make_pspec<KPP_FP8_E4M3, 2, 1>(),
    make_pspec<KPP_FP8_E4M3, 4, 1>(),
    make_pspec<KPP_FP8_E4M3, 8, 1>(),
    make_pspec<KPP_FP8_E4M3, 16, 1>(),
    make_pspec<KPP_FP8_E4M3, 32, 2>(),
    make_pspec<KPP_FP8_E4M3, 64, 4>(),
    make_pspec<KPP_FP8_E4M3, 128, 8>(),
};
} // namespace

const PSpec *persistent_specs_fp8(int *n)
{
    *n = (int)(sizeof(kSpecs) / sizeof(kSpecs[0]));
    return kSpecs;
}

} // namespace kpp
