// Flow-form generation kernels with 16 recursion and 16 output warps per
// block (blocks of 1024), for rounds of up to 512 x CMAX words
// (CMAX in {3, 8} chunks of 32 columns per recursion warp).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel flow_kernel_w16(uint32_t cmax)
{
    switch (cmax) {
    case 3: return dev::k_flow<16, 3>;
    case 8: return dev::k_flow<16, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
