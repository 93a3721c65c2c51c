// Flow-form generation kernels with 2 recursion and 2 output warps per
// block (blocks of 128), for rounds of up to 64 x CMAX words
// (CMAX in {6, 12} chunks of 32 columns per recursion warp).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel flow_kernel_w2(uint32_t cmax)
{
    switch (cmax) {
    case 6: return dev::k_flow<2, 6>;
    case 12: return dev::k_flow<2, 12>;
    default: return nullptr;
    }
}

}  // namespace mtgp
