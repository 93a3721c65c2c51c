// Device code of the MTGP generation kernel, included by the per-block-size
// translation units mtgp_gen_t*.cu (each instantiates k_generate<T, QMAX>).
//
// One thread block owns one generator at a time (Sec. 3.2).  The block keeps
// the generator's recent words in a linear shared-memory buffer X, holding
// x_j at X[j - off], and computes the sequence in rounds of S = N - M words:
// round r produces x_{N+rS+c} for columns c = 0 .. S-1, all independent
// because each reads only x_{rS+c}, x_{rS+c+1} and x_{rS+c+M} (Sec. 3.2).  A
// round needs one block barrier.  When the next round would run past the end
// of X, the N live words are copied back to the front (every ~30 rounds).
//
// Column c is owned by the same thread in every round, so the word
// x_{rS+c+M} = x_{N+(r-1)S+c} that the recursion needs is that thread's own
// output of the previous round and stays in a register; only x_{rS+c},
// x_{rS+c+1} (recursion) and x_{rS+c+M-1} (tempering, Sec. 3.7) are read from
// shared memory, at pointer + immediate addresses.
//
// The 16-entry tables are held one entry per lane and read with a width-16
// warp shuffle, which takes the index modulo 16 in hardware.  Floats are
// filled from the tempered integer o: 0x3F800000 | (o >> 9) is bit for bit
// the paper's (x >> 9) ^ sngltbl[...] of Sec. 6 eq. C, since
// sngltbl = 0x3F800000 | (tmptbl >> 9); [0,1) subtracts 1.0f (exact).
#pragma once

#include "mtgp_internal.h"

namespace mtgp {
namespace dev {

// Output value of dtype dt from the tempered 32-bit integer o (Sec. 3.7, 6).
__device__ __forceinline__ uint32_t finish(uint32_t dt, uint32_t o)
{
    const uint32_t f12 = 0x3F800000u | (o >> 9);
    if (dt == 0u) return o;
    if (dt == 1u) return f12;
    return __float_as_uint(__fsub_rn(__uint_as_float(f12), 1.0f));
}

// Parameters of the generator a block is running.
struct GenCtx {
    uint32_t N, M, mask, sh1, sh2, S;
    uint32_t rec_r, tmp_r;      // this lane's table entries rec[lane & 15], tmp[lane & 15]
    uint32_t tmpf_r;            // 0x3F800000 | (tmp_r >> 9): the single-precision table of Sec. 6
};

// The tempering table that outputs of dtype DT read: tmp for integers, the
// pre-shifted single-precision table for floats (Sec. 6), with which a float
// output is (x >> 9) ^ entry -- the bits of 0x3F800000 | ((x ^ tmp) >> 9),
// since x >> 9 leaves the nine high bits clear.
template <int DT>
__device__ __forceinline__ uint32_t out_table(const GenCtx &g)
{
    return DT == 0 ? g.tmp_r : g.tmpf_r;
}

// Output value of dtype DT from the new word xn and its entry v of out_table<DT>.
template <int DT>
__device__ __forceinline__ uint32_t finish_entry(uint32_t xn, uint32_t v)
{
    if constexpr (DT == 0) return xn ^ v;
    const uint32_t f12 = (xn >> 9) ^ v;
    if constexpr (DT == 1) return f12;
    return __float_as_uint(__fsub_rn(__uint_as_float(f12), 1.0f));
}

// Block-wide barrier between rounds; a one-warp block only needs the warp's.
template <int T>
__device__ __forceinline__ void round_sync()
{
    if (T == 32)
        __syncwarp();
    else
        __syncthreads();
}

// QN slots of a full round, processed stage by stage so that their
// dependency chains interleave: all shared loads, the recursion up to the
// table look-up (Sec. 3.6), the look-ups, the tempering (Sec. 3.7), then the
// stores.  x points at this thread's x_{rS+tid}, out at its output slot.
// When QN = Q the last slot is the round's tail and only lanes with
// last_lane set keep its result.
template <int T, int Q, int QN, int DT, bool CS = false>
__device__ __forceinline__ void round_slots(const GenCtx &g, uint32_t *x, uint32_t (&prev)[Q],
                                            uint32_t *__restrict__ out, bool last_lane)
{
    if constexpr (QN > 0) {
        const uint32_t *xt_p = x + (g.M - 1u);
        uint32_t *xn_p = x + g.N;
        uint32_t a[QN], b[QN], c[QN], u[QN];
#pragma unroll
        for (int q = 0; q < QN; ++q) {         // shared loads: x_i, x_{i+1}, x_{M-1+i}
            a[q] = x[q * T];
            b[q] = x[q * T + 1];
            c[q] = xt_p[q * T];
        }
#pragma unroll
        for (int q = 0; q < QN; ++q) {
            const uint32_t t = b[q] ^ (a[q] & g.mask);
            if constexpr (CS)                  // the shifts of Sec. 5, sh1 = 13, sh2 = 4, as constants
                u[q] = t ^ (t << 13) ^ (prev[q] >> 4);
            else
                u[q] = t ^ (t << g.sh1) ^ (prev[q] >> g.sh2);
        }
#pragma unroll
        for (int q = 0; q < QN; ++q)
            b[q] = __shfl_sync(0xffffffffu, g.rec_r, (int)u[q], 16);
        const uint32_t tbl = out_table<DT>(g);
#pragma unroll
        for (int q = 0; q < QN; ++q) {
            uint32_t s = c[q] ^ (c[q] >> 16);
            s ^= s >> 8;
            c[q] = __shfl_sync(0xffffffffu, tbl, (int)s, 16);
        }
#pragma unroll
        for (int q = 0; q < QN; ++q) {
            const uint32_t xn = u[q] ^ b[q];
            if (q + 1 < QN || QN < Q || last_lane) {
                xn_p[q * T] = xn;
                prev[q] = xn;
                __stcs(out + q * T, finish_entry<DT>(xn, c[q]));
            }
        }
    }
}

// A full round of S words whose outputs all belong to one blocked segment of
// dtype DT.  Q = ceil(S / T): slots 0 .. Q-2 are full for every thread; slot
// Q-1 holds the last S - (Q-1) T columns.  Two schedules for the tail slot:
//   IL (interleaved): warps with tail columns run all Q slots as one chain
//     of dependent steps -- the shortest round, for launches with fewer work
//     items than SMs, where each block's round latency is the time;
//   otherwise (separate): every warp runs Q-1 slots, then warps with tail
//     columns run the tail slot -- measured faster when many blocks share
//     each SM.  The two are separate kernels: one kernel with a run-time
//     choice measured slower than either.
template <int T, int Q, int DT, bool IL, bool CS = false>
__device__ __forceinline__ void round_fast(const GenCtx &g, uint32_t *x, uint32_t (&prev)[Q],
                                           uint32_t *__restrict__ out, bool tail_warp, bool tail_lane)
{
    if constexpr (IL) {
        if (tail_warp)
            round_slots<T, Q, Q, DT, CS>(g, x, prev, out, tail_lane);
        else
            round_slots<T, Q, Q - 1, DT, CS>(g, x, prev, out, true);
        return;
    }
    round_slots<T, Q, Q - 1, DT, CS>(g, x, prev, out, true);
    if (tail_warp) {
        constexpr int q = Q - 1;
        const uint32_t *xt_p = x + (g.M - 1u);
        uint32_t *xn_p = x + g.N;
        const uint32_t a0 = x[q * T], b0 = x[q * T + 1], c0 = xt_p[q * T];
        const uint32_t t = b0 ^ (a0 & g.mask);
        const uint32_t uu = CS ? t ^ (t << 13) ^ (prev[q] >> 4) : t ^ (t << g.sh1) ^ (prev[q] >> g.sh2);
        const uint32_t xn = uu ^ __shfl_sync(0xffffffffu, g.rec_r, (int)uu, 16);
        uint32_t s = c0 ^ (c0 >> 16);
        s ^= s >> 8;
        const uint32_t v = __shfl_sync(0xffffffffu, out_table<DT>(g), (int)s, 16);
        if (tail_lane) {
            xn_p[q * T] = xn;
            prev[q] = xn;
            __stcs(out + q * T, finish_entry<DT>(xn, v));
        }
    }
}

// Runs `rounds` full rounds inside one blocked segment of dtype DT.
template <int T, int Q, int DT, bool IL, bool CS = false>
__device__ __forceinline__ void run_fast(const GenCtx &g, uint32_t *buf, uint32_t B, uint32_t &rel,
                                         uint32_t (&prev)[Q], uint32_t rounds, uint32_t *out)
{
    const uint32_t tid = threadIdx.x;
    const bool tail_warp = (uint32_t)(Q - 1) * T + (tid & ~31u) < g.S;
    const bool tail_lane = (uint32_t)(Q - 1) * T + tid < g.S;
    out += tid;
    const uint32_t span = g.N + (uint32_t)(Q * T) + 32u;   // words a round at rel reads and writes
    uint32_t r = 0;
    // Rounds in groups of U with one compaction check, when the buffer holds
    // U - 1 rounds past the single-round bound: compaction then still finds
    // rel >= N, so the live words move without overlap.
    constexpr uint32_t U = 2u;        // measured: 3 and 4 lose on short work items
    if (B >= g.N + span + (U - 1u) * g.S) {
        for (; r + U <= rounds; r += U) {
            if (rel + span + (U - 1u) * g.S > B) {
                for (uint32_t j = tid; j < g.N; j += T) buf[j] = buf[rel + j];
                round_sync<T>();
                rel = 0;
            }
#pragma unroll
            for (uint32_t k = 0; k < U; ++k) {
                round_fast<T, Q, DT, IL, CS>(g, buf + rel + k * g.S + tid, prev, out + k * g.S, tail_warp, tail_lane);
                round_sync<T>();
            }
            rel += U * g.S;
            out += U * g.S;
        }
    }
    for (; r < rounds; ++r) {
        if (rel + span > B) {                               // compaction: live words to the front
            for (uint32_t j = tid; j < g.N; j += T) buf[j] = buf[rel + j];
            round_sync<T>();
            rel = 0;
        }
        round_fast<T, Q, DT, IL, CS>(g, buf + rel + tid, prev, out, tail_warp, tail_lane);
        round_sync<T>();
        rel += g.S;
        out += g.S;
    }
}

// One word of the recursion (Sec. 3.6) from x0 = x_i, x1 = x_{i+1}, xm = x_{M+i},
// and its tempered output (Sec. 3.7) from xt = x_{M-1+i}.
__device__ __forceinline__ void step(const GenCtx &g, uint32_t x0, uint32_t x1, uint32_t xm,
                                     uint32_t xt, uint32_t &xn, uint32_t &o)
{
    const uint32_t t = x1 ^ (x0 & g.mask);
    const uint32_t u = t ^ (t << g.sh1) ^ (xm >> g.sh2);
    xn = u ^ __shfl_sync(0xffffffffu, g.rec_r, (int)u, 16);
    uint32_t s = xt ^ (xt >> 16);
    s ^= s >> 8;
    o = xn ^ __shfl_sync(0xffffffffu, g.tmp_r, (int)s, 16);
}

// A round that may be partial (S_r < S words) or span several segments of
// any layout and dtype: each output finds its segment on its own.
template <int T, int Q>
__device__ __forceinline__ void round_general(const GenCtx &g, uint32_t *x, uint32_t (&prev)[Q],
                                              uint32_t S_r, uint64_t k0, const DevSeg *segs,
                                              uint32_t si, uint64_t seg_start, uint32_t *out)
{
    const uint32_t tid = threadIdx.x, wbase = tid & ~31u;
    const uint32_t *xt_p = x + (g.M - 1u);
    uint32_t *xn_p = x + g.N;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (q * T + wbase < S_r) {
            const uint32_t a = x[q * T], b = x[q * T + 1], c = xt_p[q * T];
            uint32_t xn, o;
            step(g, a, b, prev[q], c, xn, o);
            if (q * T + tid < S_r) {
                xn_p[q * T] = xn;
                prev[q] = xn;
                const uint64_t k = k0 + q * T + tid;
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
                                         : (kk >> sg.chunk_log2) * sg.stride + (kk & ((1ull << sg.chunk_log2) - 1ull));
                __stcs(out + sg.out_off + idx, finish(sg.dtype, o));
            }
        }
    }
}

// Moves the N live words x_{rS} .. x_{rS+N-1} to the front of the buffer when
// the next round would run past its end (the caller guarantees rel >= N then,
// so source and destination never overlap).
template <int T, int Q>
__device__ __forceinline__ void maybe_compact(const GenCtx &g, uint32_t *buf, uint32_t B, uint32_t &rel)
{
    if (rel + g.N + (uint32_t)(Q * T) + 32u > B) {
        for (uint32_t j = threadIdx.x; j < g.N; j += T) buf[j] = buf[rel + j];
        round_sync<T>();
        rel = 0;
    }
}

// All rounds of one work item (a generator's consecutive segments), with
// Q = ceil(S / T) column slots per thread; IL selects the tail schedule of
// round_fast.
template <int T, int Q, bool IL>
__device__ __forceinline__ void run_item(const GenCtx g, uint32_t *buf, uint32_t B, const DevWork w,
                                      const DevSeg *segs, uint32_t *out_base, uint32_t *st)
{
    const uint32_t tid = threadIdx.x;
    uint32_t prev[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q)                          // x_{c+M}, c = column
        prev[q] = (q * T + tid < g.S) ? buf[q * T + tid + g.M] : 0u;
    // parameter sets with the Sec. 5 shifts run full rounds with the shifts as
    // constants (slot counts of MTGPs 11213, 23209, 44497 in 128-thread blocks)
    constexpr bool kCS = T == 128 && (Q == 3 || Q == 6 || Q == 11);
    const bool cs = kCS && g.sh1 == 13u && g.sh2 == 4u;
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
            if (cs) {
                if (sg.dtype == 0u)
                    run_fast<T, Q, 0, IL, kCS>(g, buf, B, rel, prev, rounds, out);
                else if (sg.dtype == 1u)
                    run_fast<T, Q, 1, IL, kCS>(g, buf, B, rel, prev, rounds, out);
                else
                    run_fast<T, Q, 2, IL, kCS>(g, buf, B, rel, prev, rounds, out);
            } else {
                if (sg.dtype == 0u)
                    run_fast<T, Q, 0, IL>(g, buf, B, rel, prev, rounds, out);
                else if (sg.dtype == 1u)
                    run_fast<T, Q, 1, IL>(g, buf, B, rel, prev, rounds, out);
                else
                    run_fast<T, Q, 2, IL>(g, buf, B, rel, prev, rounds, out);
            }
            k0 += (uint64_t)rounds * g.S;
        } else {
            maybe_compact<T, Q>(g, buf, B, rel);
            const uint32_t S_r = (uint32_t)min((uint64_t)g.S, w.total - k0);
            round_general<T, Q>(g, buf + rel + tid, prev, S_r, k0, segs, si, seg_start, out_base);
            round_sync<T>();
            rel += S_r;
            k0 += S_r;
        }
    }
    if (st)                                              // state write-back (Sec. 8)
        for (uint32_t j = tid; j < g.N; j += T) st[j] = buf[rel + j];
}

// Runs the work item with the slot count Q = ceil(S / T) it needs, searching
// the compiled counts QMAX, QMAX-1, ..., 1.  Returns false if none matches.
template <int T, int QMAX, bool IL>
__device__ __forceinline__ bool dispatch_slots(uint32_t nq, const GenCtx &g, uint32_t *buf, uint32_t B,
                                               const DevWork &w, const DevSeg *segs, uint32_t *out,
                                               uint32_t *st)
{
    if (nq == (uint32_t)QMAX) {
        run_item<T, QMAX, IL>(g, buf, B, w, segs, out, st);
        return true;
    }
    if constexpr (QMAX > 1)
        return dispatch_slots<T, QMAX - 1, IL>(nq, g, buf, B, w, segs, out, st);
    else
        return false;
}

// ---------------------------------------------------------------------------
// Warp-specialised form.  A block of 2 RT threads runs one generator with two
// groups: the first RT threads (recursion group) compute the rounds of the
// recursion (Sec. 3.6) into the shared buffer; the other RT threads (output
// group) temper (Sec. 3.7), convert (Sec. 6) and store the words of rounds
// the recursion group has finished.  The recursion group's critical path per
// round is then two shared loads, four integer operations, one table
// shuffle, one shared store and a barrier among its own warps; the output
// group's work has no dependence between words or rounds.
//
// Hand-off, with named barriers (ids: 1 recursion-group barrier; 2 .. 2+K-1
// FULL; 2+K .. 2+2K-1 EMPTY; K = kRing):
//   recursion, round r: if the buffer must be compacted, sync EMPTY of every
//     round not yet drained, then compact; otherwise, if r - K >= drained,
//     sync EMPTY[(r-K) % K]; compute round r; sync the recursion barrier;
//     arrive FULL[r % K].  After the last round, sync EMPTY of every round not
//     yet drained.
//   output, round r: sync FULL[r % K]; temper, convert, store; arrive
//     EMPTY[r % K].
// Every arrival is matched by exactly one sync of the other group, no group
// arrives twice at a barrier before it completes, and the recursion group
// overwrites buffer words (compaction) only after the output group consumed
// every earlier round (checked by the CPU model in tests).
constexpr uint32_t kRing = 4;
constexpr uint32_t kBarRec = 1;

// Named-barrier operations are warp-aligned: the warp is reconverged first.
__device__ __forceinline__ void nb_sync(uint32_t id, uint32_t n)
{
    __syncwarp();
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void nb_arrive(uint32_t id, uint32_t n)
{
    __syncwarp();
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ uint32_t bar_full(uint32_t r) { return 2u + r % kRing; }
__device__ __forceinline__ uint32_t bar_empty(uint32_t r) { return 2u + kRing + r % kRing; }

// Recursion group: all rounds of one work item.  rt = thread index in the group.
template <int RT, int Q>
__device__ __forceinline__ void split_recursion(const GenCtx &g, uint32_t *buf, uint32_t B, uint64_t total,
                                                uint32_t rt, uint32_t *st)
{
    constexpr int F = Q - 1;
    constexpr uint32_t ALL = 2u * RT;
    const bool tail_warp = (uint32_t)F * RT + (rt & ~31u) < g.S;
    uint32_t prev[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q)                              // x_{c+M}, c = column
        prev[q] = (q * RT + rt < g.S) ? buf[q * RT + rt + g.M] : 0u;
    const uint32_t rounds = (uint32_t)((total + g.S - 1u) / g.S);
    uint32_t rel = 0, drained = 0;
    uint64_t k0 = 0;
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t S_r = (uint32_t)min((uint64_t)g.S, total - k0);
        if (rel + g.N + (uint32_t)(Q * RT) + 32u > B) {      // compaction
            for (uint32_t j = (r > drained + kRing ? r - kRing : drained); j < r; ++j)
                nb_sync(bar_empty(j), ALL);
            drained = r;
            for (uint32_t j = rt; j < g.N; j += RT) buf[j] = buf[rel + j];
            nb_sync(kBarRec, RT);
            rel = 0;
        } else if (r >= drained + kRing) {
            nb_sync(bar_empty(r - kRing), ALL);
        }
        const uint32_t *x = buf + rel + rt;
        uint32_t *xn_p = buf + rel + rt + g.N;
        uint32_t a[Q], b[Q];
#pragma unroll
        for (int q = 0; q < F; ++q) {
            a[q] = x[q * RT];
            b[q] = x[q * RT + 1];
        }
#pragma unroll
        for (int q = 0; q < F; ++q) {
            const uint32_t t = b[q] ^ (a[q] & g.mask);
            a[q] = t ^ (t << g.sh1) ^ (prev[q] >> g.sh2);
        }
#pragma unroll
        for (int q = 0; q < F; ++q) {
            const uint32_t xn = a[q] ^ __shfl_sync(0xffffffffu, g.rec_r, (int)a[q], 16);
            if (q * RT + rt < S_r) xn_p[q * RT] = xn;
            prev[q] = xn;
        }
        if (tail_warp) {
            const uint32_t a0 = x[F * RT], b0 = x[F * RT + 1];
            const uint32_t t = b0 ^ (a0 & g.mask);
            const uint32_t u = t ^ (t << g.sh1) ^ (prev[F] >> g.sh2);
            const uint32_t xn = u ^ __shfl_sync(0xffffffffu, g.rec_r, (int)u, 16);
            if (F * RT + rt < S_r) {
                xn_p[F * RT] = xn;
                prev[F] = xn;
            }
        }
        nb_sync(kBarRec, RT);
        __threadfence_block();
        nb_arrive(bar_full(r), ALL);
        rel += S_r;
        k0 += S_r;
    }
    for (uint32_t j = (rounds > drained + kRing ? rounds - kRing : drained); j < rounds; ++j)
        nb_sync(bar_empty(j), ALL);
    if (st)                                              // state write-back (Sec. 8)
        for (uint32_t j = rt; j < g.N; j += RT) st[j] = buf[rel + j];
}

// Output group: one round's Q slots inside one blocked segment of dtype DT.
template <int RT, int Q, int DT>
__device__ __forceinline__ void split_out_fast(const GenCtx &g, const uint32_t *x, uint32_t *__restrict__ out,
                                               bool tail_warp, bool tail_lane)
{
    constexpr int F = Q - 1;
    const uint32_t *xt_p = x + (g.M - 1u);
    const uint32_t *xn_p = x + g.N;
    uint32_t a[Q], c[Q];
#pragma unroll
    for (int q = 0; q < F; ++q) {
        a[q] = xn_p[q * RT];
        c[q] = xt_p[q * RT];
    }
#pragma unroll
    for (int q = 0; q < F; ++q) {
        uint32_t s = c[q] ^ (c[q] >> 16);
        s ^= s >> 8;
        c[q] = s;
    }
#pragma unroll
    for (int q = 0; q < F; ++q)
        __stcs(out + q * RT, finish(DT, a[q] ^ __shfl_sync(0xffffffffu, g.tmp_r, (int)c[q], 16)));
    if (tail_warp) {
        const uint32_t xn = xn_p[F * RT], xt = xt_p[F * RT];
        uint32_t s = xt ^ (xt >> 16);
        s ^= s >> 8;
        const uint32_t v = __shfl_sync(0xffffffffu, g.tmp_r, (int)s, 16);
        if (tail_lane) __stcs(out + F * RT, finish(DT, xn ^ v));
    }
}

// Output group: full rounds inside one blocked segment of dtype DT.  Only the
// shared reads of a round must be finished before EMPTY is signalled, and
// they are (the stores consume their values), so no fence is needed here.
template <int RT, int Q, int DT>
__device__ __forceinline__ void split_out_run(const GenCtx &g, const uint32_t *buf, uint32_t B, uint32_t &rel,
                                              uint32_t &r, uint32_t rounds, uint32_t *out, uint32_t rt)
{
    constexpr int F = Q - 1;
    constexpr uint32_t ALL = 2u * RT;
    const bool tail_warp = (uint32_t)F * RT + (rt & ~31u) < g.S;
    const bool tail_lane = (uint32_t)F * RT + rt < g.S;
    out += rt;
    for (uint32_t i = 0; i < rounds; ++i, ++r) {
        if (rel + g.N + (uint32_t)(Q * RT) + 32u > B) rel = 0;   // same rule as the recursion group
        nb_sync(bar_full(r), ALL);
        split_out_fast<RT, Q, DT>(g, buf + rel + rt, out, tail_warp, tail_lane);
        nb_arrive(bar_empty(r), ALL);
        rel += g.S;
        out += g.S;
    }
}

// Output group: all rounds of one work item.
template <int RT, int Q>
__device__ __forceinline__ void split_output(const GenCtx &g, uint32_t *buf, uint32_t B, const DevWork &w,
                                             const DevSeg *segs, uint32_t *out_base, uint32_t rt)
{
    constexpr uint32_t ALL = 2u * RT;
    uint32_t rel = 0, si = 0, r = 0;
    uint64_t k0 = 0, seg_start = 0, seg_end = segs[0].n;
    while (k0 < w.total) {
        while (k0 >= seg_end) {                              // skip finished segments
            ++si;
            seg_start = seg_end;
            seg_end += segs[si].n;
        }
        const DevSeg sg = segs[si];
        const uint64_t full = (seg_end - k0) / g.S;          // whole rounds inside this segment
        if (full > 0 && sg.chunk_log2 == kBlocked) {
            uint32_t *out = out_base + sg.out_off + (k0 - seg_start);
            const uint32_t rounds = (uint32_t)min(full, (uint64_t)0x7FFFFFFFu);
            if (sg.dtype == 0u)
                split_out_run<RT, Q, 0>(g, buf, B, rel, r, rounds, out, rt);
            else if (sg.dtype == 1u)
                split_out_run<RT, Q, 1>(g, buf, B, rel, r, rounds, out, rt);
            else
                split_out_run<RT, Q, 2>(g, buf, B, rel, r, rounds, out, rt);
            k0 += (uint64_t)rounds * g.S;
            continue;
        }
        // a round that is partial or spans segments (any layout): per-word routing
        const uint32_t S_r = (uint32_t)min((uint64_t)g.S, w.total - k0);
        if (rel + g.N + (uint32_t)(Q * RT) + 32u > B) rel = 0;
        nb_sync(bar_full(r), ALL);
        const uint32_t *x = buf + rel + rt;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q * RT + (rt & ~31u) < S_r) {
                const uint32_t xn = x[g.N + q * RT], xt = x[g.M - 1u + q * RT];
                uint32_t s = xt ^ (xt >> 16);
                s ^= s >> 8;
                const uint32_t o = xn ^ __shfl_sync(0xffffffffu, g.tmp_r, (int)s, 16);
                if (q * RT + rt < S_r) {
                    const uint64_t k = k0 + q * RT + rt;
                    uint32_t s2 = si;
                    uint64_t start = seg_start, end = seg_end;
                    while (k >= end) {
                        ++s2;
                        start = end;
                        end += segs[s2].n;
                    }
                    const DevSeg sg2 = segs[s2];
                    const uint64_t kk = k - start;
                    const uint64_t idx = sg2.chunk_log2 == kBlocked
                                             ? kk
                                             : (kk >> sg2.chunk_log2) * sg2.stride +
                                                   (kk & ((1ull << sg2.chunk_log2) - 1ull));
                    __stcs(out_base + sg2.out_off + idx, finish(sg2.dtype, o));
                }
            }
        }
        nb_arrive(bar_empty(r), ALL);
        ++r;
        rel += S_r;
        k0 += S_r;
    }
}

template <int RT, int Q>
__device__ __forceinline__ void run_item_split(const GenCtx &g, uint32_t *buf, uint32_t B, const DevWork &w,
                                               const DevSeg *segs, uint32_t *out, uint32_t *st)
{
    const uint32_t tid = threadIdx.x;
    if (tid < (uint32_t)RT)
        split_recursion<RT, Q>(g, buf, B, w.total, tid, st);
    else
        split_output<RT, Q>(g, buf, B, w, segs, out, tid - RT);
}

template <int RT, int QMAX>
__device__ __forceinline__ bool dispatch_split(uint32_t nq, const GenCtx &g, uint32_t *buf, uint32_t B,
                                               const DevWork &w, const DevSeg *segs, uint32_t *out, uint32_t *st)
{
    if (nq == (uint32_t)QMAX) {
        run_item_split<RT, QMAX>(g, buf, B, w, segs, out, st);
        return true;
    }
    if constexpr (QMAX > 1)
        return dispatch_split<RT, QMAX - 1>(nq, g, buf, B, w, segs, out, st);
    else
        return false;
}

// Warp-specialised generation kernel: blocks of 2 RT threads.
template <int RT, int QMAX>
__global__ void __launch_bounds__(2 * RT, (2 * RT) >= 512 ? 1 : 512 / (2 * RT)) k_split(const LaunchArgs a)
{
    extern __shared__ __align__(16) uint32_t buf[];
    __shared__ uint32_t s_item;
    constexpr uint32_t T = 2u * RT;
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint32_t B = a.buf_words;
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
        GenCtx g;
        g.N = gd.N;
        g.M = gd.M;
        g.mask = gd.mask;
        g.sh1 = gd.sh1;
        g.sh2 = gd.sh2;
        g.S = g.N - g.M;
        g.rec_r = gd.rec[lane & 15u];
        g.tmp_r = gd.tmp[lane & 15u];
        g.tmpf_r = 0x3F800000u | (g.tmp_r >> 9);
        const uint32_t nq = (g.S + RT - 1u) / RT;
        bool ok = nq <= (uint32_t)QMAX && 2u * g.N + nq * RT + 32u <= B;
        if (ok) {
            uint32_t *st = a.state + gd.state_off;
            const bool piece = (w.flags & kItemPiece) != 0u;   // jump-ahead piece (Sec. 7)
            const uint32_t *ld = piece ? a.jstate + w.src : st;
            if (piece && !(w.flags & kItemLast)) st = nullptr;
            for (uint32_t j = tid; j < g.N; j += T) buf[j] = ld[j];
            __syncthreads();
            ok = dispatch_split<RT, QMAX>(nq, g, buf, B, w, a.segs + w.seg_begin, out, st);
            if (ok && tid == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&gd.count), (unsigned long long)w.total);
        }
        if (!ok && tid == 0) atomicOr(a.err, kErrBuffer);
        __syncthreads();                                     // buffer and s_item reuse
        if (!a.persistent) break;
    }
}

template <int T, int QMAX, bool IL = false>
__global__ void __launch_bounds__(T, QMAX <= 6 ? 512 / T : (T >= 256 ? 1 : 256 / T)) k_generate(const LaunchArgs a)
{
    extern __shared__ __align__(16) uint32_t buf[];
    __shared__ uint32_t s_item;
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint32_t B = a.buf_words;
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
        GenCtx g;
        g.N = gd.N;
        g.M = gd.M;
        g.mask = gd.mask;
        g.sh1 = gd.sh1;
        g.sh2 = gd.sh2;
        g.S = g.N - g.M;
        g.rec_r = gd.rec[lane & 15u];
        g.tmp_r = gd.tmp[lane & 15u];
        g.tmpf_r = 0x3F800000u | (g.tmp_r >> 9);
        const uint32_t nq = (g.S + T - 1u) / T;
        bool ok = nq <= (uint32_t)QMAX && 2u * g.N + nq * T + 32u <= B;
        if (ok) {
            uint32_t *st = a.state + gd.state_off;
            const bool piece = (w.flags & kItemPiece) != 0u;   // jump-ahead piece (Sec. 7)
            const uint32_t *ld = piece ? a.jstate + w.src : st;
            if (piece && !(w.flags & kItemLast)) st = nullptr;
            for (uint32_t j = tid; j < g.N; j += T) buf[j] = ld[j];
            __syncthreads();
            ok = dispatch_slots<T, QMAX, IL>(nq, g, buf, B, w, a.segs + w.seg_begin, out, st);
            if (ok && tid == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&gd.count), (unsigned long long)w.total);
        }
        if (!ok && tid == 0) atomicOr(a.err, kErrBuffer);
        __syncthreads();                                     // buffer and s_item reuse
        if (!a.persistent) break;
    }
}

// ---------------------------------------------------------------------------
// Flow form.  Same two groups as the split form (blocks of 2 W warps: W
// recursion warps, W output warps), but without a barrier per round.  Round r,
// column c reads x_{rS+c} and x_{rS+c+1}, i.e. columns c-M and c-M+1 of round
// r-1 (of round r-2 when c < M, Sec. 3.2), and its own output of round r-1.
// Recursion warp w owns the 32 C consecutive columns [32 C w, 32 C (w+1)) and,
// before round r, waits only until the warps holding those input columns have
// published round r-1 (or r-2) in a per-warp progress counter in shared
// memory; it publishes its own counter with a release store after the round.
// Output warp w waits for recursion warp w's round r and for the column to its
// left of round r-1 (the tempering word x_{M-1+i}, Sec. 3.7), then tempers,
// converts and stores.  The recursion warps never store to global memory, so
// their release stores do not wait on HBM writes.  A block barrier is taken
// only every E rounds, when the buffer is compacted, and at the end of a work
// item.  Every wait is bounded: after kSpinLimit polls (or the launch's
// LaunchArgs::spin_limit) the warp records kErrTimeout and stops waiting
// (results are then invalid, the kernel still ends).
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t ld_acquire_shared(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];"
                 : "=r"(v)
                 : "r"((uint32_t)__cvta_generic_to_shared(p))
                 : "memory");
    return v;
}

__device__ __forceinline__ void st_release_shared(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v)
                 : "memory");
}

// Where a run-out wait reports (kErrTimeout) and how many polls it makes.
struct FlowWait {
    unsigned *err;
    uint32_t limit;
};

// Waits (warp-uniformly) until *ctr >= need, at most fw.limit polls.
// `failed` turns every later wait of this warp into a no-op once one has run
// out.
__device__ __forceinline__ void wait_progress(const uint32_t *ctr, uint32_t need, bool &failed, const FlowWait &fw)
{
    if (failed) return;
    uint32_t spins = 0;
    while (ld_acquire_shared(ctr) < need) {
        if (++spins > fw.limit) {
            failed = true;
            if ((threadIdx.x & 31u) == 0) atomicOr(fw.err, kErrTimeout);
            return;
        }
    }
}

// Input dependencies of one recursion warp: up to two ranges of warps, each
// at a fixed round offset d (the warps must have published round r - d).
struct FlowDeps {
    uint32_t lo[2], hi[2], d[2];
    uint32_t n;
};

// Dependencies of recursion warp w owning columns [lo, hi] of rounds of S
// words, with `active` warps of `span` columns each (Sec. 3.2 indices).
__device__ __forceinline__ FlowDeps flow_deps(uint32_t w, uint32_t lo, uint32_t hi, uint32_t S, uint32_t M,
                                              uint32_t active, uint32_t span)
{
    FlowDeps f;
    f.n = 0;
    if (M > S) {                                   // inputs may lie several rounds back:
        f.lo[0] = 0;                               // wait for every warp's round r-1
        f.hi[0] = active - 1u;
        f.d[0] = 1;
        f.n = 1;
        return f;
    }
    const int a = (int)lo - (int)M, b = (int)hi - (int)M + 1;
    if (b >= 0) {                                  // columns [max(a,0), b] of round r-1
        f.lo[f.n] = (uint32_t)(a > 0 ? a : 0) / span;
        f.hi[f.n] = (uint32_t)b / span;
        f.d[f.n] = 1;
        ++f.n;
    }
    if (a < 0) {                                   // columns [a+S, min(b,-1)+S] of round r-2
        f.lo[f.n] = (uint32_t)(a + (int)S) / span;
        f.hi[f.n] = (uint32_t)((b < 0 ? b : -1) + (int)S) / span;
        f.d[f.n] = 2;
        ++f.n;
    }
    (void)w;
    return f;
}

// Recursion warp w: rounds [r0, re) of an epoch whose first round starts at
// buffer position rel0.  prev holds x_{N+(r-1)S+c} for each owned column.
template <int C>
__device__ __forceinline__ void flow_recursion(const GenCtx &g, uint32_t *buf, uint32_t rel0, uint32_t r0,
                                               uint32_t re, uint64_t total, uint32_t w, uint32_t lane,
                                               const FlowDeps &dep, uint32_t (&prev)[C], uint32_t *prog,
                                               bool &failed, const FlowWait &fw)
{
    const uint32_t base = 32u * C * w + lane;       // column of chunk 0
    for (uint32_t r = r0; r < re; ++r) {
        const uint64_t k0 = (uint64_t)r * g.S;
        const uint32_t S_r = (uint32_t)min((uint64_t)g.S, total - k0);
        for (uint32_t i = 0; i < dep.n; ++i) {
            if (r < dep.d[i]) continue;
            const uint32_t need = r - dep.d[i] + 1u;
            for (uint32_t v = dep.lo[i]; v <= dep.hi[i]; ++v)
                if (v != w) wait_progress(prog + v, need, failed, fw);
        }
        const uint32_t *x = buf + rel0 + (r - r0) * g.S + base;
        uint32_t *xn_p = buf + rel0 + (r - r0) * g.S + base + g.N;
        uint32_t a[C], b[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            a[j] = x[32 * j];
            b[j] = x[32 * j + 1];
        }
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const uint32_t t = b[j] ^ (a[j] & g.mask);
            a[j] = t ^ (t << g.sh1) ^ (prev[j] >> g.sh2);
        }
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const uint32_t xn = a[j] ^ __shfl_sync(0xffffffffu, g.rec_r, (int)a[j], 16);
            if (base + 32u * j < S_r) xn_p[32 * j] = xn;
            prev[j] = xn;
        }
        __syncwarp();
        st_release_shared(prog + w, r + 1u);
    }
}

// Output routing of one work item, carried by each output warp: the segment
// holding word index k and that segment's fields.
struct SegCursor {
    const DevSeg *segs;
    uint32_t si, nseg;
    uint64_t start, end;
    DevSeg cur;
};

// Advances to the segment holding word k (k below the item's total; the
// cursor never moves past the item's last segment).
__device__ __forceinline__ void seg_seek(SegCursor &sc, uint64_t k)
{
    while (k >= sc.end && sc.si + 1u < sc.nseg) {
        ++sc.si;
        sc.start = sc.end;
        sc.cur = sc.segs[sc.si];
        sc.end += sc.cur.n;
    }
}

// Output warp w: rounds [r0, re) of an epoch (same positions as the
// recursion warps).  Tempering (Sec. 3.7), conversion (Sec. 6), store.
template <int C>
__device__ __forceinline__ void flow_output(const GenCtx &g, const uint32_t *buf, uint32_t rel0, uint32_t r0,
                                            uint32_t re, uint64_t total, uint32_t w, uint32_t lane,
                                            uint32_t active, const uint32_t *prog, SegCursor &sc,
                                            uint32_t *out_base, bool &failed, const FlowWait &fw)
{
    const uint32_t lo = 32u * C * w, base = lo + lane;
    const uint32_t hi = min(lo + 32u * C, g.S) - 1u;
    for (uint32_t r = r0; r < re; ++r) {
        const uint64_t k0 = (uint64_t)r * g.S;
        const uint32_t S_r = (uint32_t)min((uint64_t)g.S, total - k0);
        if (lo >= S_r) continue;                                      // no column of this warp in the round
        wait_progress(prog + w, r + 1u, failed, fw);                  // x_{N+i} of round r
        if (lo > 0)                                                   // x_{M-1+i} of column lo-1
            wait_progress(prog + (lo - 1u) / (32u * C), r, failed, fw);
        else if (r >= 2)
            wait_progress(prog + active - 1u, r - 1u, failed, fw);
        const uint32_t *x = buf + rel0 + (r - r0) * g.S + base;
        uint32_t xn[C], xt[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            xn[j] = x[g.N + 32 * j];
            xt[j] = x[g.M - 1u + 32 * j];
        }
#pragma unroll
        for (int j = 0; j < C; ++j) {
            uint32_t s = xt[j] ^ (xt[j] >> 16);
            s ^= s >> 8;
            xn[j] ^= __shfl_sync(0xffffffffu, g.tmp_r, (int)s, 16);
        }
        const uint64_t kf = k0 + lo, kl = k0 + min(hi, S_r - 1u);
        seg_seek(sc, kf);
        if (kl < sc.end && sc.cur.chunk_log2 == kBlocked) {           // whole warp in one segment
            uint32_t *o = out_base + sc.cur.out_off + (kf - sc.start) + lane;
            const uint32_t dt = sc.cur.dtype;
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (base + 32u * j < S_r) __stcs(o + 32 * j, finish(dt, xn[j]));
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (base + 32u * j >= S_r) continue;
                const uint64_t k = k0 + base + 32u * j;
                SegCursor t = sc;
                seg_seek(t, k);
                const uint64_t kk = k - t.start;
                const uint64_t idx = t.cur.chunk_log2 == kBlocked
                                         ? kk
                                         : (kk >> t.cur.chunk_log2) * t.cur.stride +
                                               (kk & ((1ull << t.cur.chunk_log2) - 1ull));
                __stcs(out_base + t.cur.out_off + idx, finish(t.cur.dtype, xn[j]));
            }
        }
    }
}

// All rounds of one work item in the flow form, C chunks of 32 columns per
// recursion warp.  Epochs of E rounds between block barriers; at each epoch
// end the N newest words move to the front of the buffer.
template <int W, int C>
__device__ __forceinline__ void run_item_flow(const GenCtx &g, uint32_t *buf, uint32_t B, const DevWork &w,
                                              const DevSeg *segs, uint32_t *out, uint32_t *st, uint32_t *prog,
                                              const FlowWait &fw)
{
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t span = 32u * C;
    const uint32_t active = (g.S + span - 1u) / span;
    const bool is_rec = warp < (uint32_t)W;
    const uint32_t wg = is_rec ? warp : warp - W;                     // warp index in its group
    const bool working = wg < active;
    const uint32_t rounds = (uint32_t)((w.total + g.S - 1u) / g.S);
    const uint32_t margin = span + 32u;
    uint32_t E = (B - g.N - margin) / g.S;
    if (E < 1u) E = 1u;
    bool failed = false;
    uint32_t prev[C];
    FlowDeps dep{};
    if (is_rec && working) {
#pragma unroll
        for (int j = 0; j < C; ++j) {                                  // x_{c+M}, c = column
            const uint32_t c = wg * span + 32u * j + lane;
            prev[j] = c < g.S ? buf[c + g.M] : 0u;
        }
        dep = flow_deps(wg, wg * span, min(wg * span + span, g.S) - 1u, g.S, g.M, active, span);
    }
    SegCursor sc;
    sc.segs = segs;
    sc.nseg = w.seg_count;
    sc.si = 0;
    sc.start = 0;
    sc.cur = segs[0];
    sc.end = sc.cur.n;
    uint32_t rel = 0;
    for (uint32_t r0 = 0; r0 < rounds; r0 += E) {
        const uint32_t re = min(rounds, r0 + E);
        if (working) {
            if (is_rec)
                flow_recursion<C>(g, buf, rel, r0, re, w.total, wg, lane, dep, prev, prog, failed, fw);
            else
                flow_output<C>(g, buf, rel, r0, re, w.total, wg, lane, active, prog, sc, out, failed, fw);
        }
        const uint32_t words = (uint32_t)(min((uint64_t)re * g.S, w.total) - (uint64_t)r0 * g.S);
        __syncthreads();
        if (re < rounds) {                                              // compaction (words >= N)
            for (uint32_t j = tid; j < g.N; j += 64u * W) buf[j] = buf[rel + words + j];
            __syncthreads();
            rel = 0;
        } else {
            rel += words;
        }
    }
    if (st)                                              // state write-back (Sec. 8)
        for (uint32_t j = tid; j < g.N; j += 64u * W) st[j] = buf[rel + j];
}

template <int W, int CMAX>
__device__ __forceinline__ bool dispatch_flow(uint32_t nc, const GenCtx &g, uint32_t *buf, uint32_t B,
                                              const DevWork &w, const DevSeg *segs, uint32_t *out, uint32_t *st,
                                              uint32_t *prog, const FlowWait &fw)
{
    if (nc == (uint32_t)CMAX) {
        run_item_flow<W, CMAX>(g, buf, B, w, segs, out, st, prog, fw);
        return true;
    }
    if constexpr (CMAX > 1)
        return dispatch_flow<W, CMAX - 1>(nc, g, buf, B, w, segs, out, st, prog, fw);
    else
        return false;
}

// Flow-form generation kernel: blocks of 2 W warps (64 W threads).
template <int W, int CMAX>
__global__ void __launch_bounds__(64 * W, (64 * W) >= 512 ? 1 : 512 / (64 * W)) k_flow(const LaunchArgs a)
{
    extern __shared__ __align__(16) uint32_t buf[];
    __shared__ uint32_t s_item;
    __shared__ uint32_t prog[W];
    constexpr uint32_t T = 64u * W;
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint32_t B = a.buf_words;
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
        GenCtx g;
        g.N = gd.N;
        g.M = gd.M;
        g.mask = gd.mask;
        g.sh1 = gd.sh1;
        g.sh2 = gd.sh2;
        g.S = g.N - g.M;
        g.rec_r = gd.rec[lane & 15u];
        g.tmp_r = gd.tmp[lane & 15u];
        g.tmpf_r = 0x3F800000u | (g.tmp_r >> 9);
        const uint32_t nc = (g.S + 32u * W - 1u) / (32u * W);          // chunks per recursion warp
        const uint32_t span = 32u * nc;
        bool ok = nc <= (uint32_t)CMAX && 2u * g.N + 2u * g.S + span + 32u <= B;
        if (ok) {
            uint32_t *st = a.state + gd.state_off;
            const bool piece = (w.flags & kItemPiece) != 0u;   // jump-ahead piece (Sec. 7)
            const uint32_t *ld = piece ? a.jstate + w.src : st;
            if (piece && !(w.flags & kItemLast)) st = nullptr;
            for (uint32_t j = tid; j < g.N; j += T) buf[j] = ld[j];
            if (tid < (uint32_t)W) prog[tid] = 0u;
            __syncthreads();
            const FlowWait fw{a.err, a.spin_limit ? a.spin_limit : kSpinLimit};
            ok = dispatch_flow<W, CMAX>(nc, g, buf, B, w, a.segs + w.seg_begin, out, st, prog, fw);
            if (ok && tid == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&gd.count), (unsigned long long)w.total);
        }
        if (!ok && tid == 0) atomicOr(a.err, kErrBuffer);
        __syncthreads();                                     // buffer, counters and s_item reuse
        if (!a.persistent) break;
    }
}

}  // namespace dev
}  // namespace mtgp
