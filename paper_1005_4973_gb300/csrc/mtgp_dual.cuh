// Dual form of the generation kernel (form 5): each 128-thread block runs two
// work items at once, round against round, so that one block barrier and one
// round's bookkeeping serve the rounds of two generators and every warp has
// two independent chains of work between barriers.
//
// Each item ("lane") keeps the plain form's round structure (Sec. 3.2: rounds
// of S = N - M words, column c owned by one thread in every round, the
// recursion input x_{M+i} in a register; Sec. 3.6, 3.7, 6 as in
// mtgp_device.cuh) in its own half of the shared buffer.  Lane B numbers its
// threads backwards (column slot q*T + (T-1-tid)), so the round tails of the
// two lanes, which the plain form gives to the first warps, land on opposite
// warps.  Full rounds of both lanes run in pairs while both are inside a
// blocked segment (of any two dtypes); everything else (rounds that end a
// segment or an item, other layouts, one lane with the Sec. 5 shifts as
// constants and the other without) runs lane by lane.
// Every item of a launch must need Q column slots per thread.
#pragma once

#include "mtgp_device.cuh"

namespace mtgp {
namespace dev {

template <int Q>
struct DualLane {
    GenCtx g;
    uint32_t *buf;                  // this lane's half of the shared buffer
    uint32_t B, rel, t;             // half size, buffer index of x_{k0}, logical thread index
    uint32_t prev[Q];
    DevWork w;
    DevGen *gd;
    const DevSeg *segs;
    uint32_t *st;                   // state write-back (nullptr for a piece that is not the last)
    uint64_t k0, seg_start, seg_end;
    uint32_t si;
    bool active, cs;
};

// Takes the next work item from the launch's counter into lane L and loads
// its state; false when none is left.
template <int T, int Q>
__device__ __forceinline__ bool dual_fetch(const LaunchArgs &a, DualLane<Q> &L, uint32_t *s_item, uint32_t nwork)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    if (tid == 0) *s_item = atomicAdd(a.counter, 1u);
    __syncthreads();
    const uint32_t item = *s_item;
    __syncthreads();                                 // s_item reuse
    L.active = false;
    if (item >= nwork) return false;
    L.w = a.work[item];
    L.gd = &a.gens[L.w.gen];
    DevGen &gd = *L.gd;
    L.g.N = gd.N;
    L.g.M = gd.M;
    L.g.mask = gd.mask;
    L.g.sh1 = gd.sh1;
    L.g.sh2 = gd.sh2;
    L.g.S = L.g.N - L.g.M;
    L.g.rec_r = gd.rec[lane & 15u];
    L.g.tmp_r = gd.tmp[lane & 15u];
    L.g.tmpf_r = 0x3F800000u | (L.g.tmp_r >> 9);
    L.cs = L.g.sh1 == 13u && L.g.sh2 == 4u;
    const uint32_t nq = (L.g.S + T - 1u) / T;
    if (nq != (uint32_t)Q || 2u * L.g.N + (uint32_t)(Q * T) + 32u > L.B) {
        if (tid == 0) atomicOr(a.err, kErrBuffer);  // the host plans only items of Q slots
        return true;                                 // skipped; the caller fetches again
    }
    uint32_t *st = a.state + gd.state_off;
    const bool piece = (L.w.flags & kItemPiece) != 0u;
    const uint32_t *ld = piece ? a.jstate + L.w.src : st;
    L.st = (piece && !(L.w.flags & kItemLast)) ? nullptr : st;
    for (uint32_t j = tid; j < L.g.N; j += T) L.buf[j] = ld[j];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q)                      // x_{c+M}, c = column
        L.prev[q] = (q * T + L.t < L.g.S) ? L.buf[q * T + L.t + L.g.M] : 0u;
    L.segs = a.segs + L.w.seg_begin;
    L.rel = 0;
    L.si = 0;
    L.k0 = 0;
    L.seg_start = 0;
    L.seg_end = L.segs[0].n;
    L.active = true;
    return true;
}

// A round of lane L that may be partial or span segments (round_general with
// the lane's logical thread index).
template <int T, int Q>
__device__ __forceinline__ void dual_round_general(DualLane<Q> &L, uint32_t S_r, uint32_t *out)
{
    const GenCtx &g = L.g;
    const uint32_t t = L.t, wbase = t & ~31u;
    uint32_t *x = L.buf + L.rel + t;
    const uint32_t *xt_p = x + (g.M - 1u);
    uint32_t *xn_p = x + g.N;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (q * T + wbase < S_r) {
            const uint32_t a = x[q * T], b = x[q * T + 1], c = xt_p[q * T];
            uint32_t xn, o;
            step(g, a, b, L.prev[q], c, xn, o);
            if (q * T + t < S_r) {
                xn_p[q * T] = xn;
                L.prev[q] = xn;
                const uint64_t k = L.k0 + q * T + t;
                uint32_t s = L.si;
                uint64_t start = L.seg_start, end = L.seg_start + L.segs[L.si].n;
                while (k >= end) {
                    ++s;
                    start = end;
                    end += L.segs[s].n;
                }
                const DevSeg sg = L.segs[s];
                const uint64_t kk = k - start;
                const uint64_t idx = sg.chunk_log2 == kBlocked
                                         ? kk
                                         : (kk >> sg.chunk_log2) * sg.stride + (kk & ((1ull << sg.chunk_log2) - 1ull));
                __stcs(out + sg.out_off + idx, finish(sg.dtype, o));
            }
        }
    }
}

template <int T, int Q>
__device__ __forceinline__ void dual_compact(DualLane<Q> &L)
{
    for (uint32_t j = threadIdx.x; j < L.g.N; j += T) L.buf[j] = L.buf[L.rel + j];
    __syncthreads();
    L.rel = 0;
}

// Brings lane L to the start of a run of full rounds inside a blocked
// segment: runs the rounds that end a segment or an item (general rounds),
// writes a finished item's state back and takes the next item.  Returns the
// full rounds available (0: the lane has no more work).
template <int T, int Q>
__device__ __forceinline__ uint32_t dual_prepare(const LaunchArgs &a, DualLane<Q> &L, uint32_t *s_item,
                                                 uint32_t nwork, uint32_t *out_base)
{
    while (L.active) {
        if (L.k0 >= L.w.total) {                     // item done: state write-back (Sec. 8)
            if (L.st)
                for (uint32_t j = threadIdx.x; j < L.g.N; j += T) L.st[j] = L.buf[L.rel + j];
            if (threadIdx.x == 0)
                atomicAdd(reinterpret_cast<unsigned long long *>(&L.gd->count), (unsigned long long)L.w.total);
            __syncthreads();                         // buffer reuse
            while (dual_fetch<T, Q>(a, L, s_item, nwork) && !L.active) {
            }
            continue;
        }
        while (L.k0 >= L.seg_end) {                  // skip finished segments
            ++L.si;
            L.seg_start = L.seg_end;
            L.seg_end += L.segs[L.si].n;
        }
        const DevSeg sg = L.segs[L.si];
        const uint64_t full = (L.seg_end - L.k0) / L.g.S;
        if (full > 0 && sg.chunk_log2 == kBlocked) return (uint32_t)min(full, (uint64_t)0x7FFFFFFFu);
        if (L.rel + L.g.N + (uint32_t)(Q * T) + 32u > L.B) dual_compact<T, Q>(L);
        const uint32_t S_r = (uint32_t)min((uint64_t)L.g.S, L.w.total - L.k0);
        dual_round_general<T, Q>(L, S_r, out_base);
        __syncthreads();
        L.rel += S_r;
        L.k0 += S_r;
    }
    return 0;
}

// Output pointer of lane L's current run (its first column's output).
template <int Q>
__device__ __forceinline__ uint32_t *dual_out(const DualLane<Q> &L, uint32_t *out_base)
{
    const DevSeg sg = L.segs[L.si];
    return out_base + sg.out_off + (L.k0 - L.seg_start) + L.t;
}

// `rounds` full rounds of lane L alone (dtype DT).
template <int T, int Q, int DT, bool CS>
__device__ __forceinline__ void dual_single(DualLane<Q> &L, uint32_t rounds, uint32_t *out_base)
{
    const bool tail_warp = (uint32_t)(Q - 1) * T + (L.t & ~31u) < L.g.S;
    const bool tail_lane = (uint32_t)(Q - 1) * T + L.t < L.g.S;
    uint32_t *out = dual_out(L, out_base);
    const uint32_t span = L.g.N + (uint32_t)(Q * T) + 32u;
    for (uint32_t r = 0; r < rounds; ++r) {
        if (L.rel + span > L.B) dual_compact<T, Q>(L);
        round_fast<T, Q, DT, false, CS>(L.g, L.buf + L.rel + L.t, L.prev, out, tail_warp, tail_lane);
        __syncthreads();
        L.rel += L.g.S;
        out += L.g.S;
    }
    L.k0 += (uint64_t)rounds * L.g.S;
}

// Shared-memory word at byte address a + OFF (a register address and an
// immediate offset; asm volatile keeps the order the code gives).
template <int OFF>
__device__ __forceinline__ uint32_t dlds(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF) : "memory");
    return v;
}

template <int OFF>
__device__ __forceinline__ void dsts(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0+%1], %2;" ::"r"(a), "n"(OFF), "r"(v) : "memory");
}

// Byte addresses of one lane's round: x = this thread's x_{rS+t}, xt =
// x_{rS+t+M-1} (tempering, Sec. 3.7), xn = x_{rS+t+N} (the new word).
struct DualAddr {
    uint32_t x, xt, xn;
};

__device__ __forceinline__ DualAddr dual_addr(uint32_t x, uint32_t mt4, uint32_t n4) { return {x, x + mt4, x + n4}; }

// The tail slot Q-1 of one lane's full round (the plain form's separate
// schedule): warps with tail columns only.
template <int T, int Q, int DT, bool CS>
__device__ __forceinline__ void dual_tail(const GenCtx &g, const DualAddr &ad, uint32_t (&prev)[Q],
                                          uint32_t *__restrict__ out, bool tail_lane)
{
    constexpr int q = Q - 1;
    constexpr int o = 4 * q * T;
    const uint32_t a0 = dlds<o>(ad.x), b0 = dlds<o + 4>(ad.x), c0 = dlds<o>(ad.xt);
    const uint32_t t = b0 ^ (a0 & g.mask);
    const uint32_t uu = CS ? t ^ (t << 13) ^ (prev[q] >> 4) : t ^ (t << g.sh1) ^ (prev[q] >> g.sh2);
    const uint32_t xn = uu ^ __shfl_sync(0xffffffffu, g.rec_r, (int)uu, 16);
    uint32_t s = c0 ^ (c0 >> 16);
    s ^= s >> 8;
    const uint32_t v = __shfl_sync(0xffffffffu, out_table<DT>(g), (int)s, 16);
    if (tail_lane) {
        dsts<o>(ad.xn, xn);
        prev[q] = xn;
        __stcs(out + q * T, finish_entry<DT>(xn, v));
    }
}

// The Q-1 full slots of one lane, step by step (K = slot), for the phased
// round below: loads, recursion, look-ups, stores.
template <int T, int Q, int K>
__device__ __forceinline__ void dual_loads(const DualAddr &ad, uint32_t (&a0)[Q], uint32_t (&a1)[Q], uint32_t (&at)[Q])
{
    if constexpr (K < Q - 1) {
        constexpr int o = 4 * K * T;
        a0[K] = dlds<o>(ad.x);
        a1[K] = dlds<o + 4>(ad.x);
        at[K] = dlds<o>(ad.xt);
        dual_loads<T, Q, K + 1>(ad, a0, a1, at);
    }
}

template <int T, int Q, int K>
__device__ __forceinline__ void dual_sts(const DualAddr &ad, const uint32_t (&xn)[Q])
{
    if constexpr (K < Q - 1) {
        dsts<4 * K * T>(ad.xn, xn[K]);
        dual_sts<T, Q, K + 1>(ad, xn);
    }
}

// One full round of each lane, the Q-1 full slots of both in one phased
// sequence -- every shared load of both lanes, the recursion (Sec. 3.6), the
// table look-ups, the tempering (Sec. 3.7), then every store -- so that the
// two lanes' dependency chains overlap (their halves of the buffer are
// disjoint).  The tail slots follow; lane B's tail columns sit on the other
// warps.  DTA and DTB are the lanes' output dtypes.
template <int T, int Q, int DTA, int DTB, bool CS>
__device__ __forceinline__ void dual_round2(const GenCtx &ga, const DualAddr &xa, uint32_t (&pa)[Q],
                                            uint32_t *__restrict__ oa, bool twa, bool tla, const GenCtx &gb,
                                            const DualAddr &xb, uint32_t (&pb)[Q], uint32_t *__restrict__ ob,
                                            bool twb, bool tlb)
{
    constexpr int F = Q - 1;
    if constexpr (F > 0) {
        uint32_t a0[Q], a1[Q], at[Q], b0[Q], b1[Q], bt[Q];
        dual_loads<T, Q, 0>(xa, a0, a1, at);
        dual_loads<T, Q, 0>(xb, b0, b1, bt);
#pragma unroll
        for (int q = 0; q < F; ++q) {
            const uint32_t ta = a1[q] ^ (a0[q] & ga.mask), tb = b1[q] ^ (b0[q] & gb.mask);
            if constexpr (CS) {
                a0[q] = ta ^ (ta << 13) ^ (pa[q] >> 4);
                b0[q] = tb ^ (tb << 13) ^ (pb[q] >> 4);
            } else {
                a0[q] = ta ^ (ta << ga.sh1) ^ (pa[q] >> ga.sh2);
                b0[q] = tb ^ (tb << gb.sh1) ^ (pb[q] >> gb.sh2);
            }
        }
#pragma unroll
        for (int q = 0; q < F; ++q) {
            a1[q] = __shfl_sync(0xffffffffu, ga.rec_r, (int)a0[q], 16);
            b1[q] = __shfl_sync(0xffffffffu, gb.rec_r, (int)b0[q], 16);
        }
        const uint32_t tbla = out_table<DTA>(ga), tblb = out_table<DTB>(gb);
#pragma unroll
        for (int q = 0; q < F; ++q) {
            uint32_t sa = at[q] ^ (at[q] >> 16), sb = bt[q] ^ (bt[q] >> 16);
            sa ^= sa >> 8;
            sb ^= sb >> 8;
            at[q] = __shfl_sync(0xffffffffu, tbla, (int)sa, 16);
            bt[q] = __shfl_sync(0xffffffffu, tblb, (int)sb, 16);
        }
#pragma unroll
        for (int q = 0; q < F; ++q) {
            pa[q] = a0[q] ^ a1[q];
            pb[q] = b0[q] ^ b1[q];
        }
        dual_sts<T, Q, 0>(xa, pa);
        dual_sts<T, Q, 0>(xb, pb);
#pragma unroll
        for (int q = 0; q < F; ++q) {
            __stcs(oa + q * T, finish_entry<DTA>(pa[q], at[q]));
            __stcs(ob + q * T, finish_entry<DTB>(pb[q], bt[q]));
        }
    }
    if (twa) dual_tail<T, Q, DTA, CS>(ga, xa, pa, oa, tla);
    if (twb) dual_tail<T, Q, DTB, CS>(gb, xb, pb, ob, tlb);
}

// Moves lane L's N live words (from buffer index rel) to the front of its half.
template <int T>
__device__ __forceinline__ void dual_compact_at(uint32_t *buf, uint32_t N, uint32_t rel)
{
    for (uint32_t j = threadIdx.x; j < N; j += T) buf[j] = buf[rel + j];
    __syncthreads();
}

// `rounds` full rounds of both lanes, a round of A and a round of B between
// barriers (dtypes DTA, DTB).  When both halves hold a round more than the
// one-round bound, the rounds go in groups of two with one compaction check
// (compaction then still finds rel >= N).
template <int T, int Q, int DTA, int DTB, bool CS>
__device__ __forceinline__ void dual_pair(DualLane<Q> &A, DualLane<Q> &Bl, uint32_t rounds, uint32_t *out_base)
{
    const bool twA = (uint32_t)(Q - 1) * T + (A.t & ~31u) < A.g.S, tlA = (uint32_t)(Q - 1) * T + A.t < A.g.S;
    const bool twB = (uint32_t)(Q - 1) * T + (Bl.t & ~31u) < Bl.g.S, tlB = (uint32_t)(Q - 1) * T + Bl.t < Bl.g.S;
    uint32_t *outA = dual_out(A, out_base), *outB = dual_out(Bl, out_base);
    const uint32_t SA = A.g.S, SB = Bl.g.S;
    const uint32_t limA = A.B - (A.g.N + (uint32_t)(Q * T) + 32u), limB = Bl.B - (Bl.g.N + (uint32_t)(Q * T) + 32u);
    const uint32_t baseA = (uint32_t)__cvta_generic_to_shared(A.buf + A.t);
    const uint32_t baseB = (uint32_t)__cvta_generic_to_shared(Bl.buf + Bl.t);
    const uint32_t mtA = 4u * (A.g.M - 1u), ntA = 4u * A.g.N, mtB = 4u * (Bl.g.M - 1u), ntB = 4u * Bl.g.N;
    uint32_t relA = A.rel, relB = Bl.rel, r = 0;
    if (limA >= A.g.N + SA && limB >= Bl.g.N + SB) {
        for (; r + 2u <= rounds; r += 2u) {
            if (relA > limA - SA) {
                dual_compact_at<T>(A.buf, A.g.N, relA);
                relA = 0;
            }
            if (relB > limB - SB) {
                dual_compact_at<T>(Bl.buf, Bl.g.N, relB);
                relB = 0;
            }
            const uint32_t xa = baseA + 4u * relA, xb = baseB + 4u * relB;
            dual_round2<T, Q, DTA, DTB, CS>(A.g, dual_addr(xa, mtA, ntA), A.prev, outA, twA, tlA, Bl.g,
                                            dual_addr(xb, mtB, ntB), Bl.prev, outB, twB, tlB);
            __syncthreads();
            dual_round2<T, Q, DTA, DTB, CS>(A.g, dual_addr(xa + 4u * SA, mtA, ntA), A.prev, outA + SA, twA, tlA,
                                            Bl.g, dual_addr(xb + 4u * SB, mtB, ntB), Bl.prev, outB + SB, twB, tlB);
            __syncthreads();
            relA += 2u * SA;
            relB += 2u * SB;
            outA += 2u * SA;
            outB += 2u * SB;
        }
    }
    for (; r < rounds; ++r) {
        if (relA > limA) {
            dual_compact_at<T>(A.buf, A.g.N, relA);
            relA = 0;
        }
        if (relB > limB) {
            dual_compact_at<T>(Bl.buf, Bl.g.N, relB);
            relB = 0;
        }
        dual_round2<T, Q, DTA, DTB, CS>(A.g, dual_addr(baseA + 4u * relA, mtA, ntA), A.prev, outA, twA, tlA, Bl.g,
                                        dual_addr(baseB + 4u * relB, mtB, ntB), Bl.prev, outB, twB, tlB);
        __syncthreads();
        relA += SA;
        relB += SB;
        outA += SA;
        outB += SB;
    }
    A.rel = relA;
    Bl.rel = relB;
    A.k0 += (uint64_t)rounds * SA;
    Bl.k0 += (uint64_t)rounds * SB;
}

// dual_pair with the lanes' dtypes as compile-time values (nine pairs).
template <int T, int Q, bool CS, int DTA>
__device__ __forceinline__ void dual_pair_b(DualLane<Q> &A, DualLane<Q> &Bl, uint32_t rounds, uint32_t *out_base)
{
    const uint32_t dt = Bl.segs[Bl.si].dtype;
    if (dt == 0u) dual_pair<T, Q, DTA, 0, CS>(A, Bl, rounds, out_base);
    else if (dt == 1u) dual_pair<T, Q, DTA, 1, CS>(A, Bl, rounds, out_base);
    else dual_pair<T, Q, DTA, 2, CS>(A, Bl, rounds, out_base);
}

template <int T, int Q, bool CS>
__device__ __forceinline__ void dual_pair_any(DualLane<Q> &A, DualLane<Q> &Bl, uint32_t rounds, uint32_t *out_base)
{
    const uint32_t dt = A.segs[A.si].dtype;
    if (dt == 0u) dual_pair_b<T, Q, CS, 0>(A, Bl, rounds, out_base);
    else if (dt == 1u) dual_pair_b<T, Q, CS, 1>(A, Bl, rounds, out_base);
    else dual_pair_b<T, Q, CS, 2>(A, Bl, rounds, out_base);
}

template <int T, int Q>
__device__ __forceinline__ void dual_single_any(DualLane<Q> &L, uint32_t rounds, uint32_t *out_base)
{
    const uint32_t dt = L.segs[L.si].dtype;
    if (L.cs) {
        if (dt == 0u) dual_single<T, Q, 0, true>(L, rounds, out_base);
        else if (dt == 1u) dual_single<T, Q, 1, true>(L, rounds, out_base);
        else dual_single<T, Q, 2, true>(L, rounds, out_base);
    } else {
        if (dt == 0u) dual_single<T, Q, 0, false>(L, rounds, out_base);
        else if (dt == 1u) dual_single<T, Q, 1, false>(L, rounds, out_base);
        else dual_single<T, Q, 2, false>(L, rounds, out_base);
    }
}

// Dual-form kernel: a persistent grid of 128-thread blocks, two items each.
template <int T, int Q>
__global__ void __launch_bounds__(T, 7) k_dual(const LaunchArgs a)
{
    extern __shared__ __align__(16) uint32_t buf[];
    __shared__ uint32_t s_item;
    const uint32_t nwork = a.nwork_dev ? *a.nwork_dev : a.nwork;
    uint32_t *const out = a.out_dev ? *a.out_dev : a.out;
    const uint32_t half = a.buf_words / 2u;
    DualLane<Q> A, Bl;
    A.buf = buf;
    Bl.buf = buf + half;
    A.B = Bl.B = half;
    A.t = threadIdx.x;
    Bl.t = T - 1u - threadIdx.x;
    while (dual_fetch<T, Q>(a, A, &s_item, nwork) && !A.active) {
    }
    while (dual_fetch<T, Q>(a, Bl, &s_item, nwork) && !Bl.active) {
    }
    for (;;) {
        const uint32_t ra = dual_prepare<T, Q>(a, A, &s_item, nwork, out);
        const uint32_t rb = dual_prepare<T, Q>(a, Bl, &s_item, nwork, out);
        if (!ra && !rb) break;
        if (ra && rb && A.cs == Bl.cs) {
            const uint32_t r = min(ra, rb);
            if (A.cs)
                dual_pair_any<T, Q, true>(A, Bl, r, out);
            else
                dual_pair_any<T, Q, false>(A, Bl, r, out);
        } else {
            if (ra) dual_single_any<T, Q>(A, ra, out);
            if (rb) dual_single_any<T, Q>(Bl, rb, out);
        }
    }
}

}  // namespace dev
}  // namespace mtgp
