// Warp-specialised generation kernels with 64 recursion and 64 output
// threads per block (blocks of 128), for rounds of up to 64 x QMAX words
// (QMAX in {6, 12}).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel split_kernel_rt64(uint32_t qmax)
{
    switch (qmax) {
    case 6: return dev::k_split<64, 6>;
    case 12: return dev::k_split<64, 12>;
    default: return nullptr;
    }
}

}  // namespace mtgp
