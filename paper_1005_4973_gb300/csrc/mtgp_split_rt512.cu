// Warp-specialised generation kernels with 512 recursion and 512 output
// threads per block (blocks of 1024), for rounds of up to 512 x QMAX words
// (QMAX in {3}).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel split_kernel_rt512(uint32_t qmax)
{
    switch (qmax) {
    case 3: return dev::k_split<512, 3>;
    default: return nullptr;
    }
}

}  // namespace mtgp
