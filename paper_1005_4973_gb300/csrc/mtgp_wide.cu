// Wide form of the generation kernel (form 3): each thread owns groups of 4
// adjacent columns of a round, so that the words x_i .. x_{i+4} and
// x_{M-1+i} .. x_{M+3+i} it reads serve four outputs at once (x_{i+1} of one
// column is x_i of the next; x_{M+i} of one column is the tempering word
// x_{M-1+i} of the next), and its four outputs leave in one 16-byte store.
//
// Rounds.  Any n <= S = N - M consecutive words of the recursion (Sec. 3.2,
// 3.6) are independent: word x_{N+i} reads x_i, x_{i+1}, x_{M+i} only.  A
// round here computes n = min(R, words left in the segment) of them (R = S,
// or the launch's mtgp_config.round_words if smaller); the
// next round starts where it ended, so segments need no separate tail path.
//
// Shared memory.  The recent words sit in four interleaved sub-buffers of P
// words each: the word at linear position L lives at X[(L & 3) P + (L >> 2)].
// Every shared access of a round is then stride-1 across the lanes of a warp
// (one sub-buffer, consecutive positions) and free of bank conflicts, whatever
// the offsets M - 1 and N of the windows.
//
// Alignment.  The block keeps the linear position of x_{N+k} congruent, mod
// 4, to the word address of output k (a "residue").  A group then covers the
// four linear positions 4q .. 4q+3 and the four outputs at a 16-byte aligned
// address.  The residue is fixed when the state is loaded; a later segment
// whose output address has another residue shifts the live words by 1..3
// positions first.
#include "mtgp_internal.h"

namespace mtgp {
namespace {

struct WideCtx {
    uint32_t N, S, R, mask, sh1, sh2, P;   // R: words per round, R <= S
    uint32_t rec_r, tmp_r, tmpf_r;      // this lane's table entries (index lane & 15)
    // byte offsets (the same for every thread) of the words at linear
    // positions 4q - N + k and 4q - S - 1 + k (k = 0 .. 4), and 4q + j
    // (j = 0 .. 3), from the shared address of X + q (mod 2^32)
    uint32_t offa[5], offw[5], offs[4];
    uint32_t xs;                        // shared address of X
};

__device__ __forceinline__ uint32_t at(uint32_t P, uint32_t L) { return (L & 3u) * P + (L >> 2); }

// 32-bit shared-window accesses: the offsets of a round's windows are
// run-time values, and a generic 64-bit address per access would cost more
// than the access.  The loads may not move across the stores or barriers
// around them ("memory").
__device__ __forceinline__ uint32_t lds(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void sts(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Offset of linear position 4q + e from X + q (e may be negative).
__device__ __forceinline__ int32_t rel_off(uint32_t P, int32_t e) { return (int32_t)((uint32_t)e & 3u) * (int32_t)P + (e >> 2); }

template <int DT>
__device__ __forceinline__ uint32_t table_of(const WideCtx &g) { return DT == 0 ? g.tmp_r : g.tmpf_r; }

// Output of dtype DT from the new word xn and its entry v of table_of<DT>: for
// floats v is 0x3F800000 | (tmp >> 9) (Sec. 6), and (xn >> 9) ^ v has the
// bits of 0x3F800000 | ((xn ^ tmp) >> 9).
template <int DT>
__device__ __forceinline__ uint32_t finish_w(uint32_t xn, uint32_t v)
{
    if constexpr (DT == 0) return xn ^ v;
    const uint32_t f12 = (xn >> 9) ^ v;
    if constexpr (DT == 1) return f12;
    return __float_as_uint(__fsub_rn(__uint_as_float(f12), 1.0f));
}

// One round of n <= S words (Sec. 3.6 recursion, Sec. 3.7 tempering, Sec. 6
// conversion) starting at linear position rel; out0 = address of the round's
// first output, congruent to rel + N mod 4 words.
template <int T, int QW, int DT>
__device__ __forceinline__ void wide_round(const WideCtx &g, uint32_t *X, uint32_t rel, uint32_t n, uint32_t *out0)
{
    const uint32_t W0 = rel + g.N, q0 = W0 >> 2, h = W0 & 3u;
    const uint32_t G = (h + n + 3u) >> 2;                   // groups: the first covers h unused places
    const uint32_t hl = h + n - 4u * (G - 1u);               // used places of the last group, 1 .. 4
    uint32_t *const outg = out0 - h;                         // 16-byte aligned
    const uint32_t tbl = table_of<DT>(g);
#pragma unroll
    for (int k = 0; k < QW; ++k) {
        const uint32_t grp = threadIdx.x + (uint32_t)k * (uint32_t)T;
        if ((grp & ~31u) >= G) break;                        // whole warp idle (and every later slot)
        const bool live = grp < G;
        const uint32_t xr = g.xs + 4u * (q0 + min(grp, G - 1u));   // idle lanes read the last group's words
        uint32_t a[5], w[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            a[j] = lds(xr + g.offa[j]);
            w[j] = lds(xr + g.offw[j]);
        }
        uint32_t u[4], xn[4], v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t t = a[j + 1] ^ (a[j] & g.mask);
            u[j] = t ^ (t << g.sh1) ^ (w[j + 1] >> g.sh2);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) xn[j] = u[j] ^ __shfl_sync(0xffffffffu, g.rec_r, (int)u[j], 16);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t s = w[j] ^ (w[j] >> 16);
            s ^= s >> 8;
            v[j] = finish_w<DT>(xn[j], __shfl_sync(0xffffffffu, tbl, (int)s, 16));
        }
        const uint32_t lo = grp == 0u ? h : 0u, hi = grp == G - 1u ? hl : 4u;
        if (live && lo == 0u && hi == 4u) {
#pragma unroll
            for (int j = 0; j < 4; ++j) sts(xr + g.offs[j], xn[j]);
            __stcs(reinterpret_cast<uint4 *>(outg + 4u * grp), make_uint4(v[0], v[1], v[2], v[3]));
        } else if (live) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((uint32_t)j >= lo && (uint32_t)j < hi) {
                    sts(xr + g.offs[j], xn[j]);
                    __stcs(outg + 4u * grp + (uint32_t)j, v[j]);
                }
        }
    }
}

// Moves the live words [rel, rel + N) by d in {1, 2, 3} positions up, in
// chunks of T from the top (each chunk read completely before it is written).
template <int T>
__device__ __forceinline__ void shift_up(uint32_t *X, uint32_t P, uint32_t rel, uint32_t N, uint32_t d)
{
    for (int32_t top = (int32_t)N; top > 0; top -= T) {
        const int32_t j = top - T + (int32_t)threadIdx.x;
        uint32_t v = 0u;
        if (j >= 0) v = X[at(P, rel + (uint32_t)j)];
        __syncthreads();
        if (j >= 0) X[at(P, rel + (uint32_t)j + d)] = v;
        __syncthreads();
    }
}

// Copies the live words [rel, rel + N) down to [to, to + N), to = rel mod 4,
// to + N <= rel: same sub-buffers, no overlap.
template <int T>
__device__ __forceinline__ void compact(uint32_t *X, uint32_t P, uint32_t rel, uint32_t to, uint32_t N)
{
    for (uint32_t j = threadIdx.x; j < N; j += T) X[at(P, to + j)] = X[at(P, rel + j)];
    __syncthreads();
}

// Rounds of one blocked segment of dtype DT: n words from output address out.
template <int T, int QW, int DT>
__device__ __forceinline__ bool wide_segment(const WideCtx &g, uint32_t *X, uint32_t cap, uint32_t &rel, uint64_t n,
                                             uint32_t *out)
{
    while (n > 0u) {
        const uint32_t nr = (uint32_t)min((uint64_t)g.R, n);
        if (rel + g.N + nr + 8u > cap) {                     // compaction: live words to the front
            const uint32_t to = 4u + (rel & 3u);
            if (to + g.N > rel) return false;                // buffer too small (checked by the host)
            compact<T>(X, g.P, rel, to, g.N);
            rel = to;
        }
        wide_round<T, QW, DT>(g, X, rel, nr, out);
        __syncthreads();
        rel += nr;
        out += nr;
        n -= nr;
    }
    return true;
}

template <int T, int QW>
__global__ void __launch_bounds__(T, (QW == 1 ? 960 : 640) / T) k_wide(const LaunchArgs a)
{
    extern __shared__ __align__(16) uint32_t X[];
    __shared__ uint32_t s_item;
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint32_t P = a.buf_words >> 2, cap = 4u * P;
    uint32_t item = blockIdx.x;
    const uint32_t nwork = a.nwork_dev ? *a.nwork_dev : a.nwork;
    uint32_t *const out_base = a.out_dev ? *a.out_dev : a.out;
    for (;;) {
        if (a.persistent) {
            if (tid == 0) s_item = atomicAdd(a.counter, 1u);
            __syncthreads();
            item = s_item;
        }
        if (item >= nwork) break;
        const DevWork w = a.work[item];
        DevGen &gd = a.gens[w.gen];
        WideCtx g;
        g.N = gd.N;
        g.S = gd.N - gd.M;
        g.R = a.round_words && a.round_words < g.S ? a.round_words : g.S;   // words per round
        g.mask = gd.mask;
        g.sh1 = gd.sh1;
        g.sh2 = gd.sh2;
        g.P = P;
        g.rec_r = gd.rec[lane & 15u];
        g.tmp_r = gd.tmp[lane & 15u];
        g.tmpf_r = 0x3F800000u | (g.tmp_r >> 9);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            g.offa[j] = 4u * (uint32_t)rel_off(P, j - (int32_t)g.N);
            g.offw[j] = 4u * (uint32_t)rel_off(P, j - (int32_t)g.S - 1);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) g.offs[j] = 4u * (uint32_t)j * P;
        g.xs = (uint32_t)__cvta_generic_to_shared(X);
        const DevSeg *segs = a.segs + w.seg_begin;
        const uint32_t groups = (g.S + 6u) / 4u + 1u;
        bool ok = groups <= (uint32_t)(QW * T) && 2u * g.N + g.S + 24u <= cap;
        for (uint32_t si = 0; ok && si < w.seg_count; ++si) ok = segs[si].chunk_log2 == kBlocked;
        if (ok) {
            uint32_t *st = a.state + gd.state_off;
            const bool piece = (w.flags & kItemPiece) != 0u;   // jump-ahead piece (Sec. 7)
            const uint32_t *ld = piece ? a.jstate + w.src : st;
            if (piece && !(w.flags & kItemLast)) st = nullptr;
            // residue of the first output address; x_{N} goes to a congruent linear position
            uint32_t r0 = 0u;
            for (uint32_t si = 0; si < w.seg_count; ++si)
                if (segs[si].n) {
                    r0 = (uint32_t)(reinterpret_cast<uintptr_t>(out_base + segs[si].out_off) >> 2) & 3u;
                    break;
                }
            uint32_t rel = 4u + ((r0 - g.N) & 3u);
            for (uint32_t j = tid; j < g.N; j += T) X[at(P, rel + j)] = ld[j];
            __syncthreads();
            uint64_t k0 = 0;
            for (uint32_t si = 0; ok && si < w.seg_count && k0 < w.total; ++si) {
                const DevSeg sg = segs[si];
                const uint64_t n = min(sg.n, w.total - k0);
                if (n == 0u) continue;
                uint32_t *out = out_base + sg.out_off;
                const uint32_t r = (uint32_t)(reinterpret_cast<uintptr_t>(out) >> 2) & 3u;
                const uint32_t d = (r - (rel + g.N)) & 3u;
                if (d) {
                    if (rel + d + g.N + 8u > cap) {               // room above: compact first
                        const uint32_t to = 4u + (rel & 3u);
                        compact<T>(X, P, rel, to, g.N);
                        rel = to;
                    }
                    shift_up<T>(X, P, rel, g.N, d);
                    rel += d;
                }
                if (sg.dtype == 0u)
                    ok = wide_segment<T, QW, 0>(g, X, cap, rel, n, out);
                else if (sg.dtype == 1u)
                    ok = wide_segment<T, QW, 1>(g, X, cap, rel, n, out);
                else
                    ok = wide_segment<T, QW, 2>(g, X, cap, rel, n, out);
                k0 += n;
            }
            if (ok && st)                                     // state write-back (Sec. 8)
                for (uint32_t j = tid; j < g.N; j += T) st[j] = X[at(P, rel + j)];
            if (ok && tid == 0)
                atomicAdd(reinterpret_cast<unsigned long long *>(&gd.count), (unsigned long long)w.total);
        }
        if (!ok && tid == 0) atomicOr(a.err, kErrBuffer);
        __syncthreads();                                     // buffer and s_item reuse
        if (!a.persistent) break;
    }
}

}  // namespace

GenKernel wide_kernel(uint32_t threads, uint32_t qw)
{
    switch (threads) {
    case 96:
        return qw == 1u ? k_wide<96, 1> : qw == 2u ? k_wide<96, 2> : qw == 4u ? k_wide<96, 4> : nullptr;
    case 192:
        return qw == 1u ? k_wide<192, 1> : qw == 2u ? k_wide<192, 2> : nullptr;
    case 128:
        return qw == 1u ? k_wide<128, 1> : qw == 2u ? k_wide<128, 2> : qw == 3u ? k_wide<128, 3> : nullptr;
    default:
        return nullptr;
    }
}

}  // namespace mtgp
