// Generation kernels with 64 threads per block, for rounds of up to
// 64 x QMAX words (QMAX in {3, 6, 12}).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel gen_kernel_t64(uint32_t qmax)
{
    switch (qmax) {
    case 3: return dev::k_generate<64, 3>;
    case 6: return dev::k_generate<64, 6>;
    case 12: return dev::k_generate<64, 12>;
    default: return nullptr;
    }
}

}  // namespace mtgp
