// kpp_persistent_f32.cu -- persistent-form kernels for F32 points.
#include "kpp_persistent.cuh"

namespace kpp {

namespace {
const PSpec kSpecs[] = {
    make_pspec<KPP_F32, 2, 1>(),
    make_pspec<KPP_F32, 4, 1>(),
    make_pspec<KPP_F32, 8, 2>(),
    make_pspec<KPP_F32, 16, 4>(),
    make_pspec<KPP_F32, 32, 2>(),
    make_pspec<KPP_F32, 32, 4>(),
    make_pspec<KPP_F32, 32, 8>(),
    make_pspec<KPP_F32, 64, 4>(),
    make_pspec<KPP_F32, 64, 8>(),
    make_pspec<KPP_F32, 128, 4>(),
    make_pspec<KPP_F32, 128, 8>(),
};
} // namespace

const PSpec *persistent_specs_f32(int *n)
{
    *n = (int)(sizeof(kSpecs) / sizeof(kSpecs[0]));
    return kSpecs;
}

} // namespace kpp
