// Generation kernels with 32 threads per block, for rounds of up to
// 32 x QMAX words (QMAX in {4, 11}).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel gen_kernel_t32(uint32_t qmax)
{
    switch (qmax) {
    case 4: return dev::k_generate<32, 4>;
    case 11: return dev::k_generate<32, 11>;
    default: return nullptr;
    }
}

}  // namespace mtgp
