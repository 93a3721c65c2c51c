// Pair-form generation kernel (form 4) with 128 threads per block, for rounds
// of up to 256 x 2 words.
#include "mtgp_pairs.cuh"

namespace mtgp {

GenKernel pair_kernel_t128_q2() { return dev::k_pairs<128, 2>; }

}  // namespace mtgp
