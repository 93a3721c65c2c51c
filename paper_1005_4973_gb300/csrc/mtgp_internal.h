// Internal interface between the host library (mtgp_host.cpp) and the CUDA
// kernels (mtgp_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "mtgp_layout.h"

namespace mtgp {

// One job of the jump kernels: walk the recursion (Sec. 3.6) from the state at
// src for nseq words into the sequence scratch at seq, then XOR the states the
// coefficients of g select (Sec. 7) into the destination at dst.
struct alignas(16) DevJump {
    const uint64_t *poly;         // g: bit i of word i/64 = coefficient of x^i
    uint64_t src, dst, seq;       // word offsets: source state, destination, sequence (16-byte aligned)
    uint32_t gen;
    uint32_t nseq;                // sequence words walked (>= N)
    uint32_t ncoef;               // coefficients of g; 0 copies the state
    uint32_t mode;                // kJumpSum or kJumpStep
};
static_assert(sizeof(DevJump) == 48, "DevJump layout");
constexpr uint32_t kJumpSum = 0u;   // destination = sum_i g_i F^i s (first word's r low bits unspecified)
constexpr uint32_t kJumpStep = 1u;  // destination = F(sum_i g_i F^i s): with g = x^(J-1) mod psi, F^J s exactly
constexpr uint32_t kJumpPad = 32u;  // sequence words walked past ncoef + N (window of the sum)

cudaError_t launch_walk(const DevGen *gens, const uint32_t *src_base, uint32_t *seq_base, const DevJump *jobs,
                        uint32_t njobs, uint32_t max_N, cudaStream_t s);
// Walk and sum in one kernel with the sequence in shared memory (no scratch),
// when every job's sequence fits; the two kernels above otherwise.
bool jump_fused_fits(uint32_t max_N, uint32_t max_nseq, uint32_t max_ncoef);
// njobs jobs on `grid` blocks (0: one block per job); with njobs_dev set (a
// captured launch) the job count is read from *njobs_dev, at most njobs.
// prepare_jump_fused raises the kernel's shared-memory limit for these sizes
// (call it before capturing the launch).
cudaError_t launch_jump_fused(const DevGen *gens, const uint32_t *src_base, uint32_t *dst_base, const DevJump *jobs,
                              uint32_t njobs, uint32_t max_N, uint32_t max_nseq, uint32_t max_ncoef, cudaStream_t s,
                              const uint32_t *njobs_dev = nullptr, uint32_t grid = 0);
cudaError_t prepare_jump_fused(uint32_t max_N, uint32_t max_nseq, uint32_t max_ncoef);
cudaError_t launch_jump_sum(const DevGen *gens, const uint32_t *seq_base, uint32_t *dst_base, const DevJump *jobs,
                            uint32_t njobs, uint32_t max_N, cudaStream_t s);

// Generation kernels are compiled per block size T and per maximum slot
// count QMAX: k_generate<T, QMAX> runs generators whose round size S = N - M
// needs ceil(S / T) <= QMAX column slots per thread.  Slot counts compiled:
#define MTGP_QMAX_LIST 2, 3, 4, 6, 8, 11, 12
//   T = 32: 4, 11    T = 64: 3, 6, 12    T = 128: 3, 6, 11    T = 256: 2, 3, 6
//   T = 512: 2, 4, 8
__host__ __device__ constexpr uint32_t max_slots(uint32_t threads)
{
    return threads == 32u ? 11u : threads == 64u ? 12u : threads == 128u ? 11u : threads == 256u ? 6u
         : threads == 512u ? 8u : 0u;
}

typedef void (*GenKernel)(const LaunchArgs);
GenKernel gen_kernel_t32(uint32_t qmax);
GenKernel gen_kernel_t64(uint32_t qmax);
GenKernel gen_kernel_t128(uint32_t qmax);
GenKernel gen_kernel_t128_il(uint32_t qmax);   // interleaved round tails (LaunchArgs::interleave)
GenKernel gen_kernel_t256(uint32_t qmax);
GenKernel gen_kernel_t512(uint32_t qmax);
// Warp-specialised kernels: blocks of 2 RT threads (RT recursion + RT output).
GenKernel split_kernel_rt64(uint32_t qmax);
GenKernel split_kernel_rt128(uint32_t qmax);
GenKernel split_kernel_rt256(uint32_t qmax);
GenKernel split_kernel_rt512(uint32_t qmax);
// Wide-form kernels (form 3): T threads per block, each owning QW groups of 4
// adjacent columns of a round; T in {96, 128, 192}, QW in {1, 2, 4},
// {1, 2, 3}, {1, 2}.  Blocked layouts only.
GenKernel wide_kernel(uint32_t threads, uint32_t qw);
// Pair-form kernels (form 4): 128 threads per block, each owning two adjacent
// columns per slot; QMAX pair slots (rounds of up to 256 QMAX words), QMAX in
// {2, 3, 6}.
GenKernel pair_kernel_t128_q2();
GenKernel pair_kernel_t128_q3();
GenKernel pair_kernel_t128_q6();
GenKernel dual_kernel_t128_q3();   // dual form (two items per block), rounds of 257 .. 384 words
// Flow-form kernels: blocks of 2 W warps (W recursion + W output warps).
GenKernel flow_kernel_w2(uint32_t cmax);
GenKernel flow_kernel_w4(uint32_t cmax);
GenKernel flow_kernel_w8(uint32_t cmax);
GenKernel flow_kernel_w16(uint32_t cmax);

// Berlekamp-Massey on the GPU, one warp per sequence (mtgp_bm.cu): nseq bit
// sequences of n bits, `words` = ceil(n / 32) words apart; writes each
// annihilator (owords words, bit j = coefficient of x^j) and its degree
// (0xFFFFFFFF when above about n / 2 or owords * 32).
cudaError_t launch_bm(const uint32_t *seq, uint32_t nseq, uint32_t n, uint32_t words, uint32_t *out,
                      uint32_t owords, uint32_t *len, cudaStream_t s);

// Irreducibility of polynomials of prime degree p >= 33 on the GPU, one block
// per polynomial (mtgp_irr.cu): count polynomials of `words` 32-bit words
// (bit j = coefficient of x^j), their degrees in deg (nullptr: from the
// words).  Stage 0 (sieve: degree, roots, factors of degree <= K by a gcd)
// sets verdict[j] = 0 (reducible) or 2 (survivor); stage 1 (the p squarings
// of the survivors) turns each 2 into 1 (irreducible) or 0, or into 0 early
// once *abort (mapped host memory, nullptr for none) is nonzero.
cudaError_t launch_irr(const uint32_t *polys, uint32_t count, uint32_t words, const uint32_t *deg, uint32_t p,
                       uint32_t K, uint32_t stage, const uint32_t *abort, uint32_t *verdict, cudaStream_t s);

// Records msg as the calling thread's last error and returns status.
int report_error(int status, const char *msg);

// The runtime keeps one last-error word per host thread, and a clean-up call
// whose status is ignored can leave an error there; the launch wrappers clear
// it first, so that the check after a launch reports that launch alone.
inline void clear_stale_error() { (void)cudaGetLastError(); }

// Raises a kernel's dynamic shared-memory limit to at least dyn_bytes (never
// lowers it: captured launches rely on the limit at replay).
cudaError_t raise_smem_limit(const void *kernel, size_t dyn_bytes);

bool threads_supported(uint32_t threads, uint32_t form);
// Smallest compiled QMAX >= nq for this block size and form, 0 if none.
// In the split and flow forms a thread owns ceil(S / (threads / 2)) columns;
// in the pair form ceil(S / (2 threads)) pairs of columns.
uint32_t kernel_slots(uint32_t threads, uint32_t form, uint32_t nq);
cudaError_t launch_seed(DevGen *gens, uint32_t *state, const uint32_t *gen_ids,
                        const uint64_t *seeds, uint32_t first, uint32_t count, cudaStream_t s);
cudaError_t launch_generate(const LaunchArgs &a, uint32_t threads, uint32_t form, uint32_t qmax, uint32_t grid,
                            cudaStream_t s);
cudaError_t generate_occupancy(uint32_t threads, uint32_t form, uint32_t qmax, uint32_t buf_words,
                               int *blocks_per_sm, bool interleave = false);
cudaError_t launch_fill(uint32_t *buf, uint64_t words, uint32_t pattern, cudaStream_t s);

}  // namespace mtgp
