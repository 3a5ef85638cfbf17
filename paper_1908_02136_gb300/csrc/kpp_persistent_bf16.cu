// kpp_persistent_bf16.cu -- persistent-form kernels for BF16 points.
#include "kpp_persistent.cuh"

namespace kpp {

namespace {
const PSpec kSpecs[] = {
    make_pspec<KPP_BF16, 2, 1>(),
    make_pspec<KPP_BF16, 4, 1>(),
    make_pspec<KPP_BF16, 8, 1>(),
    make_pspec<KPP_BF16, 16, 2>(),
    make_pspec<KPP_BF16, 32, 2>(),
    make_pspec<KPP_BF16, 32, 4>(),
    make_pspec<KPP_BF16, 64, 4>(),
    make_pspec<KPP_BF16, 64, 8>(),
    make_pspec<KPP_BF16, 128, 4>(),
    make_pspec<KPP_BF16, 128, 8>(),
};
} // namespace

const PSpec *persistent_specs_bf16(int *n)
{
    *n = (int)(sizeof(kSpecs) / sizeof(kSpecs[0]));
    return kSpecs;
}

} // namespace kpp
