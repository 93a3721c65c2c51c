// Dual-form generation kernel (form 5) with 128 threads per block, two work
// items of rounds of 257 .. 384 words (MTGP 11213) at a time.
#include "mtgp_dual.cuh"

namespace mtgp {

GenKernel dual_kernel_t128_q3() { return dev::k_dual<128, 3>; }

}  // namespace mtgp
