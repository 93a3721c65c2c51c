// Warp-specialised generation kernels with 128 recursion and 128 output
// threads per block (blocks of 256), for rounds of up to 128 x QMAX words
// (QMAX in {3, 6, 11}).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel split_kernel_rt128(uint32_t qmax)
{
    switch (qmax) {
    case 3: return dev::k_split<128, 3>;
    case 6: return dev::k_split<128, 6>;
    case 11: return dev::k_split<128, 11>;
    default: return nullptr;
    }
}

}  // namespace mtgp
