// Flow-form generation kernels with 8 recursion and 8 output warps per
// block (blocks of 512), for rounds of up to 256 x CMAX words
// (CMAX in {3, 6} chunks of 32 columns per recursion warp).
#include "mtgp_device.cuh"

namespace mtgp {

GenKernel flow_kernel_w8(uint32_t cmax)
{
    switch (cmax) {
    case 3: return dev::k_flow<8, 3>;
    case 6: return dev::k_flow<8, 6>;
    default: return nullptr;
    }
}

}  // namespace mtgp
