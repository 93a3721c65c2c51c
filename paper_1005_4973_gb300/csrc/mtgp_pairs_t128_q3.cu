// Pair-form generation kernel (form 4) with 128 threads per block, for rounds
// of up to 256 x 3 words.
#include "mtgp_pairs.cuh"

namespace mtgp {

GenKernel pair_kernel_t128_q3() { return dev::k_pairs<128, 3>; }

}  // namespace mtgp
