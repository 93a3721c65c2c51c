// Generation kernels with 256 threads per block, for rounds of up to
// 256 x QMAX words (QMAX in {2, 3, 6}).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel gen_kernel_t256(uint32_t qmax)
{
    switch (qmax) {
    case 2: return dev::k_generate<256, 2>;
    case 3: return dev::k_generate<256, 3>;
    case 6: return dev::k_generate<256, 6>;
    default: return nullptr;
    }
}

}  // namespace mtgp
