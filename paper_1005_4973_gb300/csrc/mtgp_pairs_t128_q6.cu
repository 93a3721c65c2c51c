// Pair-form generation kernel (form 4) with 128 threads per block, for rounds
// of up to 256 x 6 words.
#include "mtgp_pairs.cuh"

namespace mtgp {

GenKernel pair_kernel_t128_q6() { return dev::k_pairs<128, 6>; }

}  // namespace mtgp
