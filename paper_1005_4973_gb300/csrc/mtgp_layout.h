// Data layouts the generation kernels read (generator records, work items,
// output segments, launch arguments) and the kernels' error bits.  Shared by
// the host library and the kernels; not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

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
// A piece (flags & kItemPiece) is part of a generator's stream split across
// blocks by jump-ahead (Sec. 7): it starts from the state at LaunchArgs::jstate
// + src and writes the generator's state back only if it is the last piece.
struct alignas(16) DevWork {
    uint32_t gen, seg_begin, seg_count, flags;
    uint64_t total, src;
};
static_assert(sizeof(DevWork) == 32, "DevWork layout");
constexpr uint32_t kItemPiece = 1u;
constexpr uint32_t kItemLast = 2u;

// Error bits the kernels may set in LaunchArgs::err.
constexpr unsigned kErrBuffer = 1u;  // a generator did not fit the launch's shape or buffer
constexpr unsigned kErrTimeout = 2u; // a bounded wait between warps ran out

struct LaunchArgs {
    DevGen *gens;
    uint32_t *state;
    const DevWork *work;
    const DevSeg *segs;
    uint32_t *out;
    unsigned *counter;            // persistent work counter, zero at launch
    unsigned *err;
    uint32_t nwork;
    uint32_t buf_words;
    // Graph form: when set, the work-item count and the output base are read
    // from these device words at launch, so one captured launch can be
    // replayed with a new work list.
    const uint32_t *nwork_dev;
    uint32_t *const *out_dev;           // shared buffer, >= 2N + S + 32 words for every item
    uint32_t persistent;
    const uint32_t *jstate;             // start states of pieces (DevWork::src)
    uint32_t interleave;                // 1: interleaved round tails where compiled (latency-bound launches)
    uint32_t spin_limit;                // flow form: polls per bounded wait, 0 = the default
    uint32_t round_words;               // wide form: words per round if below S (0 = S)
};

}  // namespace mtgp
