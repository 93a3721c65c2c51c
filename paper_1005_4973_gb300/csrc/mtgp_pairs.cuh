// Pair form of the MTGP generation kernel (form 4), included by the
// instantiation units mtgp_pairs_q*.cu.
//
// As in the plain form, one thread block owns one generator at a time and
// computes the sequence in rounds of S = N - M words (Sec. 3.2): round r
// produces x_{N+rS+c} for the columns c = 0 .. S-1.  Here each thread owns two
// ADJACENT columns 2p, 2p+1 (p = qT + tid for slot q), so that
//   - the recursion inputs x_{rS+2p}, x_{rS+2p+1}, x_{rS+2p+2} are three
//     shared loads for two words (x_{i+1} of one column is x_i of the next);
//   - the tempering word of column 2p+1, x_{M-1+rS+2p+1} = x_{N+(r-1)S+2p}, is
//     the thread's own output of column 2p in the previous round (Sec. 3.7),
//     kept in a register like the recursion input x_{M+i} of every column;
//   - the two outputs leave in one 8-byte streaming store when the round's
//     output address is 8-byte aligned.
// The shared buffer is split into an even and an odd half: the word with
// buffer index b lives at E[b/2] (b even) or O[b/2] (b odd), O = E + H.  A
// warp's 32 pairs then read and write consecutive words of each half, free of
// bank conflicts for either parity of the round's start; H = 16 (mod 32) also
// keeps the state load, write-back and compaction copies conflict-free.
//
// The recursion (Sec. 3.6) is u = t ^ (t << sh1) ^ (x_{M+i} >> sh2) with
// t = x_{i+1} ^ (x_i & mask), x_{N+i} = u ^ rec[u & 15]; the tempering and the
// float fill are those of Sec. 3.7 and Sec. 6.  Parameter sets with the shifts
// sh1 = 13, sh2 = 4 of Sec. 5 run a copy with the shifts as constants; others
// run with run-time shifts.  Outputs are bit-identical to the plain form.
#pragma once

#include "mtgp_device.cuh"

namespace mtgp {
namespace dev {

// Parameters of the generator a block is running, with the word offsets (from
// buf + (rel >> 1)) of the buffer words the rounds read and write: for the
// round's start parity rho = rel & 1, offT[rho] locates x_{rS+M-1} (the first
// tempering word), offS0/offS1[rho] x_{rS+N} and x_{rS+N+1} (the first stores).
struct PairCtx {
    uint32_t N, M, mask, sh1, sh2, S, H;
    uint32_t rec_r, tmp_r, tmpf_r;
    uint32_t offT[2], offS0[2], offS1[2];
};

__device__ __forceinline__ uint32_t half_off(uint32_t H, uint32_t rho, uint32_t o)
{
    const uint32_t b = rho + o;
    return (b & 1u) * H + (b >> 1);
}

// Word with buffer index b.
__device__ __forceinline__ uint32_t &bx(uint32_t *buf, uint32_t H, uint32_t b)
{
    return buf[(b & 1u) * H + (b >> 1)];
}

// u of the recursion (Sec. 3.6) from x_i, x_{i+1} and x_{M+i}.
template <bool CS>
__device__ __forceinline__ uint32_t rec_u(const PairCtx &g, uint32_t xi, uint32_t xi1, uint32_t xm)
{
    const uint32_t t = xi1 ^ (xi & g.mask);
    if constexpr (CS)
        return t ^ (t << 13) ^ (xm >> 4);
    else
        return t ^ (t << g.sh1) ^ (xm >> g.sh2);
}

// Tempering index (Sec. 3.7) of the word y: the four low bits of
// y ^ (y >> 8) ^ (y >> 16) ^ (y >> 24); the width-16 shuffle drops the rest.
__device__ __forceinline__ uint32_t fold(uint32_t y)
{
    const uint32_t s = y ^ (y >> 16);
    return s ^ (s >> 8);
}

// Output of dtype DT from the new word x and its entry v of pair_table<DT>
// (Sec. 3.7, 6): x ^ v for integers; (x >> 9) ^ v, the [1,2) bits, for floats,
// minus 1.0f (exact) for [0,1).
template <int DT>
__device__ __forceinline__ uint32_t pair_finish(uint32_t x, uint32_t v)
{
    if constexpr (DT == 0) return x ^ v;
    const uint32_t f12 = (x >> 9) ^ v;
    if constexpr (DT == 1) return f12;
    return __float_as_uint(__fsub_rn(__uint_as_float(f12), 1.0f));
}

template <int DT>
__device__ __forceinline__ uint32_t pair_table(const PairCtx &g)
{
    return DT == 0 ? g.tmp_r : g.tmpf_r;
}

// Shared-memory access at a 32-bit byte address plus a constant offset: the
// round computes one address per stream, and every slot's access adds only an
// immediate.  The "memory" clobber keeps the accesses in program order with
// the barriers and the other memory operations.
template <int OFF>
__device__ __forceinline__ uint32_t lds(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF) : "memory");
    return v;
}

template <int OFF>
__device__ __forceinline__ void sts(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0+%1], %2;" ::"r"(a), "n"(OFF), "r"(v) : "memory");
}

// Byte addresses of this thread's first word of the five word streams of a
// round (slot 0; slot q adds 4 q T bytes): x_{rS+2p} (and x_{rS+2p+2} four
// bytes on), x_{rS+2p+1}, x_{rS+M-1+2p}, x_{rS+N+2p}, x_{rS+N+2p+1}.
struct PairAddr {
    uint32_t a, b, t, s0, s1;
};

// Shared loads of slots Q0 + K .. Q0 + QN - 1 (one slot per recursion step).
template <int T, int Q0, int K, int QN>
__device__ __forceinline__ void pair_loads(const PairAddr &ad, uint32_t *a0, uint32_t *a1, uint32_t *a2,
                                           uint32_t *tw)
{
    if constexpr (K < QN) {
        constexpr int o = 4 * (Q0 + K) * T;
        a0[K] = lds<o>(ad.a);
        a1[K] = lds<o>(ad.b);
        a2[K] = lds<o + 4>(ad.a);
        tw[K] = lds<o>(ad.t);
        pair_loads<T, Q0, K + 1, QN>(ad, a0, a1, a2, tw);
    }
}

// New words x_{N+i} of slots Q0 + K .. Q0 + QN - 1 to the buffer, and their
// outputs: AL = 1, 8-byte stores (the round's outputs are 8-byte aligned);
// AL = 0, 4-byte stores; AL = 2, chosen by `aligned` at run time.
template <int T, int Q0, int K, int QN, int AL>
__device__ __forceinline__ void pair_stores(const PairAddr &ad, const uint32_t *n0, const uint32_t *n1,
                                            const uint32_t *o0, const uint32_t *o1, uint32_t *__restrict__ out,
                                            bool aligned)
{
    if constexpr (K < QN) {
        constexpr int o = (Q0 + K) * T;
        sts<4 * o>(ad.s0, n0[K]);
        sts<4 * o>(ad.s1, n1[K]);
        if (AL == 1 || (AL == 2 && aligned)) {
            __stcs(reinterpret_cast<uint2 *>(out + 2 * o), make_uint2(o0[K], o1[K]));
        } else {
            __stcs(out + 2 * o, o0[K]);
            __stcs(out + 2 * o + 1, o1[K]);
        }
        pair_stores<T, Q0, K + 1, QN, AL>(ad, n0, n1, o0, o1, out, aligned);
    }
}

// Slots Q0 .. Q1-1 of one round whose outputs all belong to one blocked
// segment of dtype DT, processed stage by stage so that the slots' dependency
// chains interleave.  out = the round's first output + 2 tid; AL as for
// pair_stores.  TAIL: the round's last slot (Q1 = Q0 + 1), where this lane's
// columns are valid only as v0 / v1 say.
template <int T, int Q, int Q0, int Q1, int DT, bool CS, int AL, bool TAIL>
__device__ __forceinline__ void pair_slots(const PairCtx &g, const PairAddr &ad, uint32_t (&prev)[2 * Q],
                                           uint32_t *__restrict__ out, bool aligned, bool v0, bool v1)
{
    constexpr int QN = Q1 - Q0;
    if constexpr (QN > 0) {
        uint32_t a0[QN], a1[QN], a2[QN], tw[QN];
        pair_loads<T, Q0, 0, QN>(ad, a0, a1, a2, tw);
        uint32_t u0[QN], u1[QN];
#pragma unroll
        for (int k = 0; k < QN; ++k) {                    // recursion up to the look-up (Sec. 3.6)
            u0[k] = rec_u<CS>(g, a0[k], a1[k], prev[2 * (Q0 + k)]);
            u1[k] = rec_u<CS>(g, a1[k], a2[k], prev[2 * (Q0 + k) + 1]);
        }
#pragma unroll
        for (int k = 0; k < QN; ++k) {                    // tempering indexes (Sec. 3.7)
            tw[k] = fold(tw[k]);                          // column 2p: x_{M-1+i} from shared memory
            a2[k] = fold(prev[2 * (Q0 + k)]);             // column 2p+1: column 2p's previous word
        }
#pragma unroll
        for (int k = 0; k < QN; ++k) {
            a0[k] = __shfl_sync(0xffffffffu, g.rec_r, (int)u0[k], 16);
            a1[k] = __shfl_sync(0xffffffffu, g.rec_r, (int)u1[k], 16);
        }
        const uint32_t tbl = pair_table<DT>(g);
#pragma unroll
        for (int k = 0; k < QN; ++k) {
            tw[k] = __shfl_sync(0xffffffffu, tbl, (int)tw[k], 16);
            a2[k] = __shfl_sync(0xffffffffu, tbl, (int)a2[k], 16);
        }
#pragma unroll
        for (int k = 0; k < QN; ++k) {                    // new words (Sec. 3.6) and outputs (Sec. 3.7, 6)
            uint32_t &n0 = prev[2 * (Q0 + k)], &n1 = prev[2 * (Q0 + k) + 1];
            n0 = u0[k] ^ a0[k];
            n1 = u1[k] ^ a1[k];
            u0[k] = pair_finish<DT>(n0, tw[k]);
            u1[k] = pair_finish<DT>(n1, a2[k]);
        }
        if constexpr (!TAIL) {
            uint32_t n0s[QN], n1s[QN];
#pragma unroll
            for (int k = 0; k < QN; ++k) {
                n0s[k] = prev[2 * (Q0 + k)];
                n1s[k] = prev[2 * (Q0 + k) + 1];
            }
            pair_stores<T, Q0, 0, QN, AL>(ad, n0s, n1s, u0, u1, out, aligned);
        } else {                                          // odd S: the round's last pair is half
            constexpr int o = Q0 * T;
            if (v0) {
                sts<4 * o>(ad.s0, prev[2 * Q0]);
                __stcs(out + 2 * o, u0[0]);
            }
            if (v1) {
                sts<4 * o>(ad.s1, prev[2 * Q0 + 1]);
                __stcs(out + 2 * o + 1, u1[0]);
            }
        }
    }
}

// One full round of S words inside one blocked segment: every warp runs the
// Q-1 full slots, then warps with columns in the tail slot run it.
template <int T, int Q, int DT, bool CS, int AL>
__device__ __forceinline__ void pair_round(const PairCtx &g, const PairAddr &ad, uint32_t (&prev)[2 * Q],
                                           uint32_t *__restrict__ out, bool aligned, bool tail_warp, bool v0,
                                           bool v1)
{
    pair_slots<T, Q, 0, Q - 1, DT, CS, AL, false>(g, ad, prev, out, aligned, true, true);
    if (tail_warp) pair_slots<T, Q, Q - 1, Q, DT, CS, AL, true>(g, ad, prev, out, aligned, v0, v1);
}

// Moves the N live words (buffer indexes rel .. rel+N-1) to the front when a
// round at rel would run past the end (rel >= N then: no overlap).
template <int T>
__device__ __forceinline__ void pair_compact(const PairCtx &g, uint32_t *buf, uint32_t rel)
{
    for (uint32_t j = threadIdx.x; j < g.N; j += T) bx(buf, g.H, j) = bx(buf, g.H, rel + j);
    round_sync<T>();
}

// One full round at buffer index rel, whose parity is RHO: the five stream
// addresses, then the round.  sb = byte address of buf + 4 tid.
template <int T, int Q, int DT, bool CS, int RHO, int AL>
__device__ __forceinline__ void pair_round_at(const PairCtx &g, uint32_t sb, uint32_t rel, uint32_t (&prev)[2 * Q],
                                              uint32_t *__restrict__ out, bool tail_warp, bool v0, bool v1)
{
    const uint32_t base = sb + 2u * rel - 2u * RHO;       // + 4 (rel >> 1)
    PairAddr ad;
    ad.a = base + (RHO ? 4u * g.H : 0u);
    ad.b = base + (RHO ? 4u : 4u * g.H);
    ad.t = base + 4u * g.offT[RHO];
    ad.s0 = base + 4u * g.offS0[RHO];
    ad.s1 = base + 4u * g.offS1[RHO];
    pair_round<T, Q, DT, CS, AL>(g, ad, prev, out, false, tail_warp, v0, v1);
}

// A single round at rel of either parity, outputs of either alignment, with
// the run-time shifts: the stream addresses and the store width are chosen at
// run time (one code path for every case).
template <int T, int Q, int DT>
__device__ __forceinline__ void pair_round_any(const PairCtx &g, uint32_t sb, uint32_t rel, uint32_t (&prev)[2 * Q],
                                               uint32_t *__restrict__ out, bool tail_warp, bool v0, bool v1)
{
    const bool aligned = ((uintptr_t)out & 7u) == 0u;
    const uint32_t rho = rel & 1u;
    const uint32_t base = sb + 2u * (rel - rho);
    PairAddr ad;
    ad.a = base + (rho ? 4u * g.H : 0u);
    ad.b = base + (rho ? 4u : 4u * g.H);
    ad.t = base + 4u * (rho ? g.offT[1] : g.offT[0]);
    ad.s0 = base + 4u * (rho ? g.offS0[1] : g.offS0[0]);
    ad.s1 = base + 4u * (rho ? g.offS1[1] : g.offS1[0]);
    pair_round<T, Q, DT, false, 2>(g, ad, prev, out, aligned, tail_warp, v0, v1);
}

// Pairs of full rounds from an even buffer index: the first round's parity
// is 0 and the second's is S's; 2 S words of output keep the 8-byte alignment
// of each round fixed over the loop (AL0 for the first round; the second has
// AL0 unless S is odd).  One compaction check per pair.
template <int T, int Q, int DT, bool CS, bool ODD, bool AL0>
__device__ __forceinline__ void pair_loop(const PairCtx &g, uint32_t *buf, uint32_t sb, uint32_t &rel,
                                          uint32_t (&prev)[2 * Q], uint32_t npairs, uint32_t *&out, bool tail_warp,
                                          bool v0, bool v1, uint32_t span)
{
    const uint32_t B = 2u * g.H;
    for (uint32_t i = 0; i < npairs; ++i) {
        if (rel + span + g.S > B) {                       // compaction: rel >= N, index 0 is even
            pair_compact<T>(g, buf, rel);
            rel = 0;
        }
        pair_round_at<T, Q, DT, CS, 0, AL0 ? 1 : 0>(g, sb, rel, prev, out, tail_warp, v0, v1);
        round_sync<T>();
        pair_round_at<T, Q, DT, CS, ODD ? 1 : 0, (ODD ? !AL0 : AL0) ? 1 : 0>(g, sb, rel + g.S, prev, out + g.S,
                                                                              tail_warp, v0, v1);
        round_sync<T>();
        rel += 2u * g.S;
        out += 2u * g.S;
    }
}

// `rounds` full rounds inside one blocked segment of dtype DT.  A round moves
// the start parity by S: single rounds until rel is even, then pairs of
// rounds (compaction moves the live words to index 0, which is even).
template <int T, int Q, int DT, bool CS, bool ODD>
__device__ __forceinline__ void pair_run_fast_s(const PairCtx &g, uint32_t *buf, uint32_t &rel,
                                                uint32_t (&prev)[2 * Q], uint32_t rounds, uint32_t *out)
{
    const uint32_t tid = threadIdx.x;
    const uint32_t c0 = 2u * ((uint32_t)(Q - 1) * T + tid);   // this lane's first tail column
    const bool tail_warp = 2u * ((uint32_t)(Q - 1) * T + (tid & ~31u)) < g.S;
    const bool v0 = c0 < g.S, v1 = c0 + 1u < g.S;
    const uint32_t B = 2u * g.H;
    const uint32_t span = g.N + 2u * (uint32_t)(Q * T) + 32u;   // buffer words a round at rel touches
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(buf) + 4u * tid;
    out += 2u * tid;
    uint32_t r = 0;
    // the buffer holds two rounds past the one-round bound: pairs of rounds
    const bool pairs = B >= g.N + span + g.S;
    while (r < rounds && ((rel & 1u) || !pairs)) {
        if (rel + span > B) {
            pair_compact<T>(g, buf, rel);
            rel = 0;
        }
        pair_round_any<T, Q, DT>(g, sb, rel, prev, out, tail_warp, v0, v1);
        round_sync<T>();
        rel += g.S;
        out += g.S;
        ++r;
    }
    const uint32_t npairs = (rounds - r) / 2u;
    if (npairs) {
        if (((uintptr_t)out & 7u) == 0u)
            pair_loop<T, Q, DT, CS, ODD, true>(g, buf, sb, rel, prev, npairs, out, tail_warp, v0, v1, span);
        else
            pair_loop<T, Q, DT, CS, ODD, false>(g, buf, sb, rel, prev, npairs, out, tail_warp, v0, v1, span);
        r += 2u * npairs;
    }
    if (r < rounds) {                                     // the last odd round
        if (rel + span > B) {
            pair_compact<T>(g, buf, rel);
            rel = 0;
        }
        pair_round_any<T, Q, DT>(g, sb, rel, prev, out, tail_warp, v0, v1);
        round_sync<T>();
        rel += g.S;
    }
}

// Slot counts with the specialised paired-round loops (the rounds of
// MTGPs 11213, 23209 and 44497 in 128-thread blocks); other counts, and
// parameter sets with other shifts than sh1 = 13, sh2 = 4, run single rounds
// of the one run-time path (same outputs; it bounds the kernel's code size).
template <int T, int Q>
__host__ __device__ constexpr bool pair_fast_slots()
{
    return T == 128 && (Q == 2 || Q == 3 || Q == 6);
}

// `rounds` full rounds inside one blocked segment of dtype DT, one at a time.
template <int T, int Q, int DT>
__device__ __forceinline__ void pair_run_single(const PairCtx &g, uint32_t *buf, uint32_t &rel,
                                                uint32_t (&prev)[2 * Q], uint32_t rounds, uint32_t *out)
{
    const uint32_t tid = threadIdx.x;
    const uint32_t c0 = 2u * ((uint32_t)(Q - 1) * T + tid);
    const bool tail_warp = 2u * ((uint32_t)(Q - 1) * T + (tid & ~31u)) < g.S;
    const bool v0 = c0 < g.S, v1 = c0 + 1u < g.S;
    const uint32_t B = 2u * g.H;
    const uint32_t span = g.N + 2u * (uint32_t)(Q * T) + 32u;
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(buf) + 4u * tid;
    out += 2u * tid;
    for (uint32_t r = 0; r < rounds; ++r) {
        if (rel + span > B) {
            pair_compact<T>(g, buf, rel);
            rel = 0;
        }
        pair_round_any<T, Q, DT>(g, sb, rel, prev, out, tail_warp, v0, v1);
        round_sync<T>();
        rel += g.S;
        out += g.S;
    }
}

template <int T, int Q, int DT, bool CS>
__device__ __forceinline__ void pair_run_fast(const PairCtx &g, uint32_t *buf, uint32_t &rel,
                                              uint32_t (&prev)[2 * Q], uint32_t rounds, uint32_t *out)
{
    if constexpr (CS && pair_fast_slots<T, Q>()) {
        if (g.S & 1u)
            pair_run_fast_s<T, Q, DT, CS, true>(g, buf, rel, prev, rounds, out);
        else
            pair_run_fast_s<T, Q, DT, CS, false>(g, buf, rel, prev, rounds, out);
    } else {
        pair_run_single<T, Q, DT>(g, buf, rel, prev, rounds, out);
    }
}

// A round that may be partial (S_r < S words) or span several segments of
// any layout and dtype: each output finds its segment on its own.
template <int T, int Q>
__device__ __forceinline__ void pair_round_general(const PairCtx &g, uint32_t *buf, uint32_t rel,
                                                   uint32_t (&prev)[2 * Q], uint32_t S_r, uint64_t k0,
                                                   const DevSeg *segs, uint32_t si, uint64_t seg_start,
                                                   uint32_t *out)
{
    const uint32_t tid = threadIdx.x, wbase = tid & ~31u;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (2u * (q * T + wbase) < S_r) {
            const uint32_t c = 2u * (q * T + tid);
            const uint32_t b = rel + c;
            const uint32_t a0 = bx(buf, g.H, b), a1 = bx(buf, g.H, b + 1u), a2 = bx(buf, g.H, b + 2u);
            const uint32_t t0 = bx(buf, g.H, b + g.M - 1u), t1 = bx(buf, g.H, b + g.M);
            const uint32_t u0 = rec_u<false>(g, a0, a1, prev[2 * q]);
            const uint32_t u1 = rec_u<false>(g, a1, a2, prev[2 * q + 1]);
            const uint32_t n0 = u0 ^ __shfl_sync(0xffffffffu, g.rec_r, (int)u0, 16);
            const uint32_t n1 = u1 ^ __shfl_sync(0xffffffffu, g.rec_r, (int)u1, 16);
            const uint32_t o0 = n0 ^ __shfl_sync(0xffffffffu, g.tmp_r, (int)fold(t0), 16);
            const uint32_t o1 = n1 ^ __shfl_sync(0xffffffffu, g.tmp_r, (int)fold(t1), 16);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (c + j < S_r) {
                    const uint32_t n = j ? n1 : n0;
                    bx(buf, g.H, b + g.N + j) = n;
                    prev[2 * q + j] = n;
                    const uint64_t k = k0 + c + j;
                    uint32_t s = si;
                    uint64_t start = seg_start, end = seg_start + segs[si].n;
                    while (k >= end) {
                        ++s;
                        start = end;
                        end += segs[s].n;
                    }
                    const DevSeg sg = segs[s];
                    const uint64_t kk = k - start;
                    const uint64_t idx = sg.chunk_log2 == kBlocked
                                             ? kk
                                             : (kk >> sg.chunk_log2) * sg.stride +
                                                   (kk & ((1ull << sg.chunk_log2) - 1ull));
                    __stcs(out + sg.out_off + idx, finish(sg.dtype, j ? o1 : o0));
                }
            }
        }
    }
}

// All rounds of one work item (a generator's consecutive segments) with Q pair
// slots per thread, the state already in the buffer at buffer indexes 0 .. N-1.
template <int T, int Q, bool CS>
__device__ __forceinline__ void pair_item(const PairCtx &g, uint32_t *buf, const DevWork &w, const DevSeg *segs,
                                          uint32_t *out_base, uint32_t *st)
{
    const uint32_t tid = threadIdx.x;
    const uint32_t B = 2u * g.H, span = g.N + 2u * (uint32_t)(Q * T) + 32u;
    uint32_t prev[2 * Q];
#pragma unroll
    for (int q = 0; q < Q; ++q)                          // x_{c+M}, c = column
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint32_t c = 2u * (q * T + tid) + j;
            prev[2 * q + j] = c < g.S ? bx(buf, g.H, c + g.M) : 0u;
        }
    uint32_t rel = 0, si = 0;
    uint64_t k0 = 0, seg_start = 0, seg_end = segs[0].n;
    while (k0 < w.total) {
        while (k0 >= seg_end) {                          // skip finished segments
            ++si;
            seg_start = seg_end;
            seg_end += segs[si].n;
        }
        const DevSeg sg = segs[si];
        const uint64_t full = (seg_end - k0) / g.S;      // whole rounds inside this segment
        if (full > 0 && sg.chunk_log2 == kBlocked) {
            uint32_t *out = out_base + sg.out_off + (k0 - seg_start);
            const uint32_t rounds = (uint32_t)min(full, (uint64_t)0x7FFFFFFFu);
            if (sg.dtype == 0u)
                pair_run_fast<T, Q, 0, CS>(g, buf, rel, prev, rounds, out);
            else if (sg.dtype == 1u)
                pair_run_fast<T, Q, 1, CS>(g, buf, rel, prev, rounds, out);
            else
                pair_run_fast<T, Q, 2, CS>(g, buf, rel, prev, rounds, out);
            k0 += (uint64_t)rounds * g.S;
        } else {
            if (rel + span > B) {
                pair_compact<T>(g, buf, rel);
                rel = 0;
            }
            const uint32_t S_r = (uint32_t)min((uint64_t)g.S, w.total - k0);
            pair_round_general<T, Q>(g, buf, rel, prev, S_r, k0, segs, si, seg_start, out_base);
            round_sync<T>();
            rel += S_r;
            k0 += S_r;
        }
    }
    if (st)                                              // state write-back (Sec. 8)
        for (uint32_t j = tid; j < g.N; j += T) st[j] = bx(buf, g.H, rel + j);
}

// Runs the item with the pair-slot count Q = ceil(S / 2T) it needs, searching
// the compiled counts QMAX, QMAX-1, ..., 1.  Returns false if none matches.
template <int T, int QMAX>
__device__ __forceinline__ bool pair_dispatch(uint32_t nq, bool cs, const PairCtx &g, uint32_t *buf,
                                              const DevWork &w, const DevSeg *segs, uint32_t *out, uint32_t *st)
{
    if (nq == (uint32_t)QMAX) {
        if (pair_fast_slots<T, QMAX>() && cs)
            pair_item<T, QMAX, pair_fast_slots<T, QMAX>()>(g, buf, w, segs, out, st);
        else
            pair_item<T, QMAX, false>(g, buf, w, segs, out, st);
        return true;
    }
    if constexpr (QMAX > 1)
        return pair_dispatch<T, QMAX - 1>(nq, cs, g, buf, w, segs, out, st);
    else
        return false;
}

// Pair-form generation kernel: one work item per block at a time (a persistent
// grid pulls items from a device counter).  Shared buffer: a.buf_words words,
// used as two halves of H = a.buf_words / 2 words.  MINB blocks per SM bound
// the registers (1024 threads per SM: 64 registers, no spills for QMAX <= 6).
template <int T, int QMAX, int MINB = 1024 / T>
__global__ void __launch_bounds__(T, MINB) k_pairs(const LaunchArgs a)
{
    extern __shared__ __align__(16) uint32_t buf[];
    __shared__ uint32_t s_item;
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint32_t H = a.buf_words / 2u;
    uint32_t item = blockIdx.x;
    const uint32_t nwork = a.nwork_dev ? *a.nwork_dev : a.nwork;
    uint32_t *const out = a.out_dev ? *a.out_dev : a.out;
    for (;;) {
        if (a.persistent) {
            if (tid == 0) s_item = atomicAdd(a.counter, 1u);
            __syncthreads();
            item = s_item;
        }
        if (item >= nwork) break;
        const DevWork w = a.work[item];
        DevGen &gd = a.gens[w.gen];
        PairCtx g;
        g.N = gd.N;
        g.M = gd.M;
        g.mask = gd.mask;
        g.sh1 = gd.sh1;
        g.sh2 = gd.sh2;
        g.S = g.N - g.M;
        g.H = H;
        g.rec_r = gd.rec[lane & 15u];
        g.tmp_r = gd.tmp[lane & 15u];
        g.tmpf_r = 0x3F800000u | (g.tmp_r >> 9);
#pragma unroll
        for (uint32_t rho = 0; rho < 2u; ++rho) {
            g.offT[rho] = half_off(H, rho, g.M - 1u);
            g.offS0[rho] = half_off(H, rho, g.N);
            g.offS1[rho] = half_off(H, rho, g.N + 1u);
        }
        const uint32_t nq = (g.S + 2u * T - 1u) / (2u * T);
        bool ok = nq <= (uint32_t)QMAX && 2u * g.N + 2u * nq * T + 32u <= 2u * H;
        if (ok) {
            uint32_t *st = a.state + gd.state_off;
            const bool piece = (w.flags & kItemPiece) != 0u;   // jump-ahead piece (Sec. 7)
            const uint32_t *ld = piece ? a.jstate + w.src : st;
            if (piece && !(w.flags & kItemLast)) st = nullptr;
            for (uint32_t j = tid; j < g.N; j += T) bx(buf, H, j) = ld[j];
            __syncthreads();
            const bool cs = g.sh1 == 13u && g.sh2 == 4u;
            ok = pair_dispatch<T, QMAX>(nq, cs, g, buf, w, a.segs + w.seg_begin, out, st);
            if (ok && tid == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&gd.count), (unsigned long long)w.total);
        }
        if (!ok && tid == 0) atomicOr(a.err, kErrBuffer);
        __syncthreads();                                     // buffer and s_item reuse
        if (!a.persistent) break;
    }
}

}  // namespace dev
}  // namespace mtgp
