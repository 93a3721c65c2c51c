// Flow-form generation kernels with 4 recursion and 4 output warps per
// block (blocks of 256), for rounds of up to 128 x CMAX words
// (CMAX in {3, 6, 11} chunks of 32 columns per recursion warp).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel flow_kernel_w4(uint32_t cmax)
{
    switch (cmax) {
    case 3: return dev::k_flow<4, 3>;
    case 6: return dev::k_flow<4, 6>;
    case 11: return dev::k_flow<4, 11>;
    default: return nullptr;
    }
}

}  // namespace mtgp
