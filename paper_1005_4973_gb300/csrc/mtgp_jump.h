// Host side of jump-ahead (Sec. 7): annihilating polynomials of generator
// states and device copies of jump polynomials.  Internal to libmtgp.
#pragma once

#include <cstdint>
#include <unordered_map>
#include <utility>
#include <vector>

#include "mtgp_f2.h"
#include "mtgp_internal.h"

namespace mtgp {

struct JumpPoly {
    const uint64_t *d = nullptr;   // device copy of g = x^(J-1) mod psi
    uint32_t ncoef = 0;            // deg g + 1
};

struct JumpCache {
    // psi of each generator: psi(F) s = 0 for the generator's state s when it
    // was computed, hence for every later state F^k s.  Empty = not known.
    std::vector<f2::Poly> ann;
    struct KeyHash {
        size_t operator()(const std::pair<uint32_t, uint64_t> &k) const
        {
            return (size_t)(k.second * 0x9E3779B97F4A7C15ull) ^ (size_t)k.first;
        }
    };
    std::unordered_map<std::pair<uint32_t, uint64_t>, JumpPoly, KeyHash> polys;
    std::vector<void *> chunks;    // device memory holding the polynomials
    size_t dev_bytes = 0;
};

// Computes psi for every listed generator without one.  Synchronous on s (runs
// after the work already queued there, so it sees the current states).
// Returns an mtgp_status; the error text goes through report_error.
int jump_annihilate(JumpCache &jc, const DevGen *host_gens, const DevGen *d_gens, const uint32_t *d_state,
                    const uint32_t *gens, size_t n, cudaStream_t s);

// Makes device copies of x^(J-1) mod psi_gen for every (gen, J), J >= 1, that
// is not cached yet (psi must be known).  Synchronous.
int jump_polys(JumpCache &jc, const std::vector<std::pair<uint32_t, uint64_t>> &need);

JumpPoly jump_poly(const JumpCache &jc, uint32_t gen, uint64_t J);

// Frees the device polynomials; with all = true also forgets psi (a state was
// replaced).  The caller makes sure no queued work still reads them.
void jump_clear(JumpCache &jc, bool all);

// Sequence words a job of jump J from a generator of N words walks (16-byte
// multiple), given the polynomial's coefficient count.
inline uint32_t jump_seq_words(uint32_t N, uint32_t ncoef)
{
    const uint32_t n = ncoef ? ncoef + N + kJumpPad : N;
    return (n + 3u) & ~3u;
}

}  // namespace mtgp
