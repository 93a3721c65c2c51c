// MTGP generation kernels for sm_103a.
//
// One thread block owns one generator at a time (Sec. 3.2).  Its state lives
// in a shared-memory ring X[0 .. L) holding x_k at X[k mod L] (the array of
// Knuth's Algorithm A, Sec. 3.1), with L a power of two >= N + W so that one
// round -- W <= N - M consecutive words x_{N+i}, all independent (Sec. 3.2) --
// never overwrites a word the same round still reads.  A round needs one
// block barrier.  Each output is tempered with x_{M-1+i} (Sec. 3.7) and, for
// float outputs, filled into a float's mantissa (Sec. 6), then streamed to HBM.
//
// GB300 choices (not in the paper, whose GPUs had 16 banks and a texture
// cache): the 16-entry tables are held one entry per lane and read with a
// width-16 warp shuffle, which masks the index to its four LSBs in hardware
// and never conflicts; a round issues all of its shared-memory loads before
// any arithmetic so their latencies overlap; the round size is a whole number
// of warps, and warps with no word in a round skip it; work items (a
// generator's consecutive requests) can be pulled from a device counter by a
// persistent grid, longest first.
#include "mtgp_internal.h"

namespace mtgp {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;   // SplitMix64 Weyl increment

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Seeds generator `first + blockIdx.x`: word j of the state is the low half of
// SplitMix64 output j+1 from (seed ^ key), key = SplitMix64 output 1 from the
// generator ID.  A state whose p effective bits are all zero (a fixed point of
// the linear recursion) gets x_{N-1} = 1.
__global__ void k_seed(DevGen *gens, uint32_t *state, const uint32_t *gen_ids,
                       const uint64_t *seeds, uint32_t first)
{
    const uint32_t g = first + blockIdx.x;
    const uint32_t N = gens[g].N, mask = gens[g].mask;
    const uint64_t s0 = seeds[g] ^ mix64((uint64_t)gen_ids[g] + kGamma);
    uint32_t *st = state + gens[g].state_off;
    uint32_t any = 0;
    for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) {
        const uint32_t w = (uint32_t)mix64(s0 + (uint64_t)(j + 1u) * kGamma);
        st[j] = w;
        any |= (j == 0u) ? (w & mask) : w;
    }
    const int nonzero = __syncthreads_or(any != 0u);
    if (threadIdx.x == 0) {
        if (!nonzero) st[N - 1u] = 1u;
        gens[g].count = 0;
    }
}

// Output of Sec. 3.7 / Sec. 6 from the new word xn and the looked-up table
// entry v (tmptbl for integers, the single-precision table for floats).
template <int DT>
__device__ __forceinline__ uint32_t finish(uint32_t xn, uint32_t v)
{
    if (DT == 0) return xn ^ v;
    const uint32_t bits = (xn >> 9) ^ v;                     // float in [1, 2)
    if (DT == 1) return bits;
    return __float_as_uint(__fsub_rn(__uint_as_float(bits), 1.0f));   // exact
}

// Runs one segment (n numbers of one dtype) of the current work item.
// `base` is the ring index of x_k, the oldest live state word.
template <int QMAX, int DT>
__device__ __forceinline__ void run_segment(uint32_t *ring, uint32_t Lm, uint32_t &base,
                                            uint32_t N, uint32_t M, uint32_t mask,
                                            uint32_t sh1, uint32_t sh2, uint32_t W,
                                            uint32_t rec_r, uint32_t tbl_r, const DevSeg &seg,
                                            uint32_t *out)
{
    const uint32_t T = blockDim.x, tid = threadIdx.x, wbase = tid & ~31u;
    uint32_t *o = out + seg.out_off;
    const bool blocked = seg.chunk_log2 == kBlocked;
    const uint64_t cmask = blocked ? 0ull : ((1ull << seg.chunk_log2) - 1ull);
    for (uint64_t done = 0; done < seg.n; done += W) {
        const uint32_t cnt = (uint32_t)min((uint64_t)W, seg.n - done);
        uint32_t x0[QMAX], x1[QMAX], xm[QMAX], xt[QMAX];
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
            if (q * T + wbase < cnt) {                       // warp-uniform
                const uint32_t i = base + q * T + tid;
                x0[q] = ring[i & Lm];
                x1[q] = ring[(i + 1u) & Lm];
                xm[q] = ring[(i + M) & Lm];
                xt[q] = ring[(i + M - 1u) & Lm];
            }
        }
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
            if (q * T + wbase < cnt) {
                const uint32_t j = q * T + tid;
                // recursion g (Sec. 3.6)
                uint32_t t = x1[q] ^ (x0[q] & mask);
                t ^= t << sh1;
                const uint32_t u = t ^ (xm[q] >> sh2);
                const uint32_t xn = u ^ __shfl_sync(0xffffffffu, rec_r, (int)u, 16);
                // tempering h (Sec. 3.7) with x_{M-1+i}
                uint32_t s = xt[q] ^ (xt[q] >> 16);
                s ^= s >> 8;
                const uint32_t v = __shfl_sync(0xffffffffu, tbl_r, (int)s, 16);
                const uint32_t r = finish<DT>(xn, v);
                if (j < cnt) {
                    ring[(base + j + N) & Lm] = xn;
                    const uint64_t k = done + j;
                    const uint64_t idx = blocked ? k : ((k >> seg.chunk_log2) * seg.stride + (k & cmask));
                    __stcs(o + idx, r);
                }
            }
        }
        base += cnt;
        __syncthreads();
    }
}

template <int QMAX>
__global__ void __launch_bounds__(max_threads_for_q(QMAX)) k_generate(const LaunchArgs a)
{
    extern __shared__ __align__(16) uint32_t ring[];
    __shared__ uint32_t s_item;
    const uint32_t T = blockDim.x, tid = threadIdx.x, lane = tid & 31u;
    const uint32_t Lm = a.ring_words - 1u;
    uint32_t item = blockIdx.x;
    for (;;) {
        if (a.persistent) {
            if (tid == 0) s_item = atomicAdd(a.counter, 1u);
            __syncthreads();
            item = s_item;
        }
        if (item >= a.nwork) break;
        const DevWork w = a.work[item];
        DevGen &g = a.gens[w.gen];
        const uint32_t N = g.N, M = g.M, mask = g.mask, sh1 = g.sh1, sh2 = g.sh2;
        const uint32_t W = round_words(N, M, a.wpr_cap, T, QMAX);
        if (N + W <= a.ring_words && W > 0u) {
            const uint32_t rec_r = g.rec[lane & 15u];
            const uint32_t tmp_r = g.tmp[lane & 15u];
            const uint32_t flt_r = 0x3F800000u | (tmp_r >> 9);  // single-precision table (Sec. 6)
            uint32_t *st = a.state + g.state_off;
            for (uint32_t j = tid; j < N; j += T) ring[j] = st[j];
            __syncthreads();
            uint32_t base = 0;
            for (uint32_t s = 0; s < w.seg_count; ++s) {
                const DevSeg seg = a.segs[w.seg_begin + s];
                if (seg.dtype == 0u)
                    run_segment<QMAX, 0>(ring, Lm, base, N, M, mask, sh1, sh2, W, rec_r, tmp_r, seg, a.out);
                else if (seg.dtype == 1u)
                    run_segment<QMAX, 1>(ring, Lm, base, N, M, mask, sh1, sh2, W, rec_r, flt_r, seg, a.out);
                else
                    run_segment<QMAX, 2>(ring, Lm, base, N, M, mask, sh1, sh2, W, rec_r, flt_r, seg, a.out);
            }
            for (uint32_t j = tid; j < N; j += T) st[j] = ring[(base + j) & Lm];
            if (tid == 0) g.count += w.total;
        } else if (tid == 0) {
            atomicOr(a.err, kErrRing);
        }
        __syncthreads();                                     // ring and s_item reuse
        if (!a.persistent) break;
    }
}

// Write-only bandwidth probe: 16-byte streaming stores over a grid-stride loop.
__global__ void k_fill(uint4 *buf, uint64_t n16, uint32_t pattern)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const uint32_t v = pattern ^ (uint32_t)i;
        __stcs(buf + i, make_uint4(v, v + 1u, v + 2u, v + 3u));
    }
}

template <int Q>
cudaError_t launch_q(const LaunchArgs &a, uint32_t threads, uint32_t grid, cudaStream_t s)
{
    const size_t smem = (size_t)a.ring_words * sizeof(uint32_t);
    k_generate<Q><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_seed(DevGen *gens, uint32_t *state, const uint32_t *gen_ids,
                        const uint64_t *seeds, uint32_t first, uint32_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_seed<<<count, 256, 0, s>>>(gens, state, gen_ids, seeds, first);
    return cudaGetLastError();
}

cudaError_t launch_generate(const LaunchArgs &a, uint32_t threads, uint32_t grid, uint32_t qmax,
                            cudaStream_t s)
{
    switch (qmax) {
    case 1: return launch_q<1>(a, threads, grid, s);
    case 2: return launch_q<2>(a, threads, grid, s);
    case 4: return launch_q<4>(a, threads, grid, s);
    case 8: return launch_q<8>(a, threads, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t generate_occupancy(uint32_t threads, uint32_t qmax, uint32_t ring_words, int *blocks_per_sm)
{
    const size_t smem = (size_t)ring_words * sizeof(uint32_t);
    switch (qmax) {
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_generate<1>, threads, smem);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_generate<2>, threads, smem);
    case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_generate<4>, threads, smem);
    case 8: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_generate<8>, threads, smem);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fill(uint32_t *buf, uint64_t words, uint32_t pattern, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    k_fill<<<(unsigned)sms * 8u, 512, 0, s>>>(reinterpret_cast<uint4 *>(buf), words / 4u, pattern);
    return cudaGetLastError();
}

}  // namespace mtgp
