// Warp-specialised generation kernels with 256 recursion and 256 output
// threads per block (blocks of 512), for rounds of up to 256 x QMAX words
// (QMAX in {3, 6}).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel split_kernel_rt256(uint32_t qmax)
{
    switch (qmax) {
    case 3: return dev::k_split<256, 3>;
    case 6: return dev::k_split<256, 6>;
    default: return nullptr;
    }
}

}  // namespace mtgp
