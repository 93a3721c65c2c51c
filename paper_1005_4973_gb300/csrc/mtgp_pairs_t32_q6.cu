// Pair-form generation kernel (form 4) with one warp per block, for rounds
// of up to 64 x 6 words (MTGP11213).
#include "mtgp_pairs.cuh"

namespace mtgp {

GenKernel pair_kernel_t32_q6() { return dev::k_pairs<32, 6, 28>; }

}  // namespace mtgp
