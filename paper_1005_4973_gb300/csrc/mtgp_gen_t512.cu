// Generation kernels with 512 threads per block, for rounds of up to
// 512 x QMAX words (QMAX in {2, 4, 8}).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel gen_kernel_t512(uint32_t qmax)
{
    switch (qmax) {
    case 2: return dev::k_generate<512, 2>;
    case 4: return dev::k_generate<512, 4>;
    case 8: return dev::k_generate<512, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
