// Generation kernels with 128 threads per block, for rounds of up to
// 128 x QMAX words (QMAX in {3, 6, 11}), in both tail schedules (the
// interleaved one for launches with fewer work items than SMs).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel gen_kernel_t128(uint32_t qmax)
{
    switch (qmax) {
    case 3: return dev::k_generate<128, 3>;
    case 6: return dev::k_generate<128, 6>;
    case 11: return dev::k_generate<128, 11>;
    default: return nullptr;
    }
}

GenKernel gen_kernel_t128_il(uint32_t qmax)
{
    switch (qmax) {
    case 3: return dev::k_generate<128, 3, true>;
    case 6: return dev::k_generate<128, 6, true>;
    case 11: return dev::k_generate<128, 11, true>;
    default: return nullptr;
    }
}

}  // namespace mtgp
