// Internal interface between the host library (mtgp_host.cpp) and the CUDA
// kernels (mtgp_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace mtgp {

// Device-resident record of one generator.  176 bytes, 16-byte aligned.
struct alignas(16) DevGen {
    uint32_t N, M, mask, sh1;     // recursion parameters (Sec. 3.6)
    uint32_t sh2, mexp, id, rsv;
    uint64_t state_off;           // word offset of x_k .. x_{k+N-1} in the state buffer
    uint64_t count;               // numbers generated so far (stream position k)
    uint32_t rec[16];             // rectbl (Sec. 3.6)
    uint32_t tmp[16];             // tmptbl (Sec. 3.7)
};
static_assert(sizeof(DevGen) == 176, "DevGen layout");

// One output segment of a work item: n numbers of one dtype.
struct alignas(16) DevSeg {
    uint64_t n;
    uint64_t out_off;             // element offset of the segment's first number
    uint64_t stride;              // interleaved: elements between consecutive chunks
    uint32_t dtype;               // 0 u32, 1 f32 [1,2), 2 f32 [0,1)
    uint32_t chunk_log2;          // kBlocked = contiguous
};
static_assert(sizeof(DevSeg) == 32, "DevSeg layout");
constexpr uint32_t kBlocked = 0xFFFFFFFFu;

// One work item: consecutive segments of one generator, run by one block.
struct alignas(16) DevWork {
    uint32_t gen, seg_begin, seg_count, rsv;
    uint64_t total, rsv2;
};
static_assert(sizeof(DevWork) == 32, "DevWork layout");

// Error bits the kernels may set in LaunchArgs::err.
constexpr unsigned kErrRing = 1u;    // a generator did not fit the launch's ring

struct LaunchArgs {
    DevGen *gens;
    uint32_t *state;
    const DevWork *work;
    const DevSeg *segs;
    uint32_t *out;
    unsigned *counter;            // persistent work counter, zero at launch
    unsigned *err;
    uint32_t nwork;
    uint32_t ring_words;          // power of two, >= N + round size of every item
    uint32_t wpr_cap;             // cap on the round size
    uint32_t persistent;
};

constexpr uint32_t kMaxQ = 8;       // rounds may be up to kMaxQ x threads words

// Largest block for a kernel instance that keeps up to q words per thread in
// flight (keeps 4q live words per thread in registers without spilling).
__host__ __device__ constexpr uint32_t max_threads_for_q(uint32_t q)
{
    return q <= 2u ? 1024u : 512u;
}

// Round size of a generator: min(cap, N - M) (Sec. 3.2), rounded down to a
// whole number of warps when at least one warp, and at most qmax x threads.
__host__ __device__ inline uint32_t round_words(uint32_t N, uint32_t M, uint32_t cap, uint32_t threads, uint32_t qmax)
{
    uint32_t w = N - M;
    if (cap && cap < w) w = cap;
    if (w >= 32u) w &= ~31u;
    if (w > qmax * threads) w = qmax * threads;
    return w;
}

cudaError_t launch_seed(DevGen *gens, uint32_t *state, const uint32_t *gen_ids,
                        const uint64_t *seeds, uint32_t first, uint32_t count, cudaStream_t s);
cudaError_t launch_generate(const LaunchArgs &a, uint32_t threads, uint32_t grid, uint32_t qmax,
                            cudaStream_t s);
cudaError_t generate_occupancy(uint32_t threads, uint32_t qmax, uint32_t ring_words, int *blocks_per_sm);
cudaError_t launch_fill(uint32_t *buf, uint64_t words, uint32_t pattern, cudaStream_t s);

}  // namespace mtgp
