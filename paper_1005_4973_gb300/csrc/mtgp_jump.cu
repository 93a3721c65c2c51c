// Jump-ahead kernels (Sec. 7).  A state s of the linear transition F
// (Sec. 3.3) jumps J steps as F^J s = g(F) s, g = x^J mod psi with psi(F) s = 0;
// g(F) s = sum_i g_i F^i s is the XOR of the windows x_i .. x_{i+N-1} of the
// recursion's word sequence picked by g's coefficients.  Two kernels, one
// block per job:
//   k_walk      runs the recursion (Sec. 3.6, no tempering) from the job's
//               state and writes the word sequence x_0 .. x_{nseq-1};
//   k_jump_sum  XORs the selected windows, each thread owning R consecutive
//               words of the sum in registers, reading 2R-word windows of the
//               sequence for every R coefficients that select any.
#include "mtgp_internal.h"

namespace mtgp {

namespace {

constexpr uint32_t kJumpThreads = 256;

uint32_t pow2_at_least(uint32_t x)
{
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// One word of the recursion (Sec. 3.6): x_{N+i} from x_i, x_{i+1}, x_{i+M}.
__device__ __forceinline__ uint32_t rec_word(uint32_t a0, uint32_t a1, uint32_t aM, uint32_t mask, uint32_t sh1,
                                             uint32_t sh2, const uint32_t *tbl)
{
    uint32_t t = (a0 & mask) ^ a1;
    t ^= t << sh1;
    const uint32_t u = t ^ (aM >> sh2);
    return u ^ tbl[u & 15u];
}

// Words in rounds of S = N - M, kept in a circular shared buffer of Rb >= N + S
// words (a power of two): round i0 reads x_{i0} .. x_{i0+N-1} and writes
// x_{i0+N} .. x_{i0+N+S-1}.
__global__ void __launch_bounds__(kJumpThreads) k_walk(const DevGen *gens, const uint32_t *src_base,
                                                       uint32_t *seq_base, const DevJump *jobs, uint32_t Rb)
{
    extern __shared__ __align__(16) uint32_t x[];
    __shared__ uint32_t tbl[16];
    const DevJump jb = jobs[blockIdx.x];
    const DevGen &g = gens[jb.gen];
    const uint32_t N = g.N, M = g.M, S = N - M, mask = g.mask, sh1 = g.sh1, sh2 = g.sh2, Rm = Rb - 1u;
    const uint32_t tid = threadIdx.x, nseq = jb.nseq;
    if (tid < 16u) tbl[tid] = g.rec[tid];
    const uint32_t *src = src_base + jb.src;
    uint32_t *seq = seq_base + jb.seq;
    for (uint32_t j = tid; j < N; j += kJumpThreads) {
        const uint32_t v = src[j];
        x[j] = v;
        if (j < nseq) seq[j] = v;
    }
    __syncthreads();
    for (uint32_t i0 = 0; i0 + N < nseq; i0 += S) {
        for (uint32_t c = tid; c < S; c += kJumpThreads) {
            const uint32_t i = i0 + c;
            const uint32_t v = rec_word(x[i & Rm], x[(i + 1u) & Rm], x[(i + M) & Rm], mask, sh1, sh2, tbl);
            x[(i + N) & Rm] = v;
            if (i + N < nseq) seq[i + N] = v;
        }
        __syncthreads();
    }
}

template <int R>
__global__ void __launch_bounds__(kJumpThreads) k_jump_sum(const DevGen *gens, const uint32_t *seq_base,
                                                           uint32_t *dst_base, const DevJump *jobs)
{
    extern __shared__ __align__(16) uint32_t y[];
    __shared__ uint32_t tbl[16];
    const DevJump jb = jobs[blockIdx.x];
    const DevGen &g = gens[jb.gen];
    const uint32_t N = g.N, tid = threadIdx.x, j0 = tid * (uint32_t)R;
    const uint32_t *x = seq_base + jb.seq;
    uint32_t *dst = dst_base + jb.dst;
    if (jb.ncoef == 0u) {                                    // J = 0: the state itself
        for (uint32_t j = tid; j < N; j += kJumpThreads) dst[j] = x[j];
        return;
    }
    if (tid < 16u) tbl[tid] = g.rec[tid];
    uint32_t acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0u;
    if (j0 < N) {
        for (uint32_t i = 0; i < jb.ncoef; i += (uint32_t)R) {
            const uint32_t cb =
                (uint32_t)(__ldg(jb.poly + (i >> 6)) >> (i & 63u)) & (uint32_t)((1ull << R) - 1ull);
            if (!cb) continue;
            uint32_t v[2 * R];
            const uint4 *p4 = reinterpret_cast<const uint4 *>(x + i + j0);
#pragma unroll
            for (int q = 0; q < R / 2; ++q) {
                const uint4 t = __ldg(p4 + q);
                v[4 * q] = t.x;
                v[4 * q + 1] = t.y;
                v[4 * q + 2] = t.z;
                v[4 * q + 3] = t.w;
            }
#pragma unroll
            for (int u = 0; u < R; ++u) {
                if ((cb >> u) & 1u) {
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] ^= v[u + r];
                }
            }
        }
    }
    if (jb.mode == kJumpSum) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (j0 + (uint32_t)r < N) dst[j0 + r] = acc[r];
        return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (j0 + (uint32_t)r < N) y[j0 + r] = acc[r];
    __syncthreads();
    for (uint32_t j = tid; j + 1u < N; j += kJumpThreads) dst[j] = y[j + 1u];
    if (tid == 0u) dst[N - 1u] = rec_word(y[0], y[1], y[g.M], g.mask, g.sh1, g.sh2, tbl);
}

// Walk and sum in one block, the sequence in shared memory: x (seq_cap
// words), then y (the sum, max_N words), then g's coefficients (32-bit
// words).  The sum splits the work two ways: a slice of WS = ceil(N / 32R)
// warps covers the N words, R consecutive words per lane, and the block's
// warps form C = warps / WS slices, each taking a contiguous share of g's
// coefficients; slices XOR their partial sums into y with shared atomics.
// Slices are whole warps, so the coefficient tests branch uniformly.  A lane
// slides a 2R-word window along the sequence: for each R coefficients it
// loads the next R words (R = 12: three 16-byte loads at a 48-byte lane
// stride, which touch every bank exactly once per 8 lanes).
// XORs into acc the windows starting at words U0 + b of (lo, hi) for the set
// bits b of MASK (the compiler folds the chain into 3-input XORs).
template <int R, int U0, int MASK>
__device__ __forceinline__ void xor_windows(uint32_t (&acc)[R], const uint32_t (&lo)[R], const uint32_t (&hi)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint32_t t = acc[r];
        if constexpr ((MASK & 1) != 0) t ^= (U0 + r < R) ? lo[U0 + r] : hi[U0 + r - R];
        if constexpr ((MASK & 2) != 0) t ^= (U0 + 1 + r < R) ? lo[U0 + 1 + r] : hi[U0 + 1 + r - R];
        if constexpr ((MASK & 4) != 0) t ^= (U0 + 2 + r < R) ? lo[U0 + 2 + r] : hi[U0 + 2 + r - R];
        if constexpr ((MASK & 8) != 0) t ^= (U0 + 3 + r < R) ? lo[U0 + 3 + r] : hi[U0 + 3 + r - R];
        acc[r] = t;
    }
}

// The four coefficients U0 .. U0+3 of a group, one warp-uniform branch for
// all sixteen patterns.
template <int R, int U0>
__device__ __forceinline__ void sum_nibble(uint32_t (&acc)[R], const uint32_t (&lo)[R], const uint32_t (&hi)[R],
                                           uint32_t nib)
{
    switch (nib) {
    case 1: xor_windows<R, U0, 1>(acc, lo, hi); break;
    case 2: xor_windows<R, U0, 2>(acc, lo, hi); break;
    case 3: xor_windows<R, U0, 3>(acc, lo, hi); break;
    case 4: xor_windows<R, U0, 4>(acc, lo, hi); break;
    case 5: xor_windows<R, U0, 5>(acc, lo, hi); break;
    case 6: xor_windows<R, U0, 6>(acc, lo, hi); break;
    case 7: xor_windows<R, U0, 7>(acc, lo, hi); break;
    case 8: xor_windows<R, U0, 8>(acc, lo, hi); break;
    case 9: xor_windows<R, U0, 9>(acc, lo, hi); break;
    case 10: xor_windows<R, U0, 10>(acc, lo, hi); break;
    case 11: xor_windows<R, U0, 11>(acc, lo, hi); break;
    case 12: xor_windows<R, U0, 12>(acc, lo, hi); break;
    case 13: xor_windows<R, U0, 13>(acc, lo, hi); break;
    case 14: xor_windows<R, U0, 14>(acc, lo, hi); break;
    case 15: xor_windows<R, U0, 15>(acc, lo, hi); break;
    default: break;
    }
}

// The R coefficients of a group (bits of cb) applied to the sliding window
// (lo, hi): coefficient u selects the words u .. u + R - 1.
template <int R, int T>
__device__ __forceinline__ void sum_group(uint32_t (&acc)[R], const uint32_t (&lo)[R], const uint32_t (&hi)[R],
                                          uint32_t cb)
{
    static_assert(R % 4 == 0, "coefficients go in nibbles");
    sum_nibble<R, 0>(acc, lo, hi, cb & 15u);
    if constexpr (R > 4) sum_nibble<R, 4>(acc, lo, hi, (cb >> 4) & 15u);
    if constexpr (R > 8) sum_nibble<R, 8>(acc, lo, hi, (cb >> 8) & 15u);
    if constexpr (R > 12) sum_nibble<R, 12>(acc, lo, hi, (cb >> 12) & 15u);
}

template <int R>
__device__ __forceinline__ void load_words(uint32_t (&v)[R], const uint32_t *p)
{
    const uint4 *p4 = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
        const uint4 t = p4[q];
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}

// R coefficient bits starting at bit i of the 32-bit coefficient words.
template <int R>
__device__ __forceinline__ uint32_t coef_bits(const uint32_t *cf, uint32_t i)
{
    const uint32_t w = i >> 5, sh = i & 31u;
    const uint32_t v = __funnelshift_r(cf[w], cf[w + 1u], sh);
    return v & ((1u << R) - 1u);
}

// One job: walk, sum and step (Sec. 7) for jb, in the block's shared words.
template <int R, int T>
__device__ __forceinline__ void fused_job(const DevJump jb, const DevGen *gens, const uint32_t *src_base,
                                          uint32_t *dst_base, uint32_t *sm, uint32_t *tbl, uint32_t seq_cap,
                                          uint32_t max_N)
{
    uint32_t *x = sm, *y = sm + seq_cap, *cf = sm + seq_cap + max_N;
    const DevGen &g = gens[jb.gen];
    const uint32_t N = g.N, M = g.M, S = N - M, mask = g.mask, sh1 = g.sh1, sh2 = g.sh2;
    const uint32_t tid = threadIdx.x, ncoef = jb.ncoef;
    uint32_t *dst = dst_base + jb.dst;
    if (tid < 16u) tbl[tid] = g.rec[tid];
    const uint32_t *src = src_base + jb.src;
    for (uint32_t j = tid; j < N; j += T) {
        x[j] = src[j];
        y[j] = 0u;
    }
    const uint32_t cw = (ncoef + 31u) / 32u;
    for (uint32_t w = tid; w < cw + 1u; w += T)           // one zero word past the end
        cf[w] = w < cw ? (uint32_t)(jb.poly[w >> 1] >> (32u * (w & 1u))) : 0u;
    __syncthreads();
    if (ncoef == 0u) {                                      // J = 0: the state itself
        for (uint32_t j = tid; j < N; j += T) dst[j] = x[j];
        return;
    }
    const uint32_t nseq = jb.nseq;
    for (uint32_t i0 = 0; i0 + N < nseq; i0 += S) {
        for (uint32_t c = tid; c < S; c += T) {
            const uint32_t i = i0 + c;
            if (i + N < nseq) x[i + N] = rec_word(x[i], x[i + 1u], x[i + M], mask, sh1, sh2, tbl);
        }
        __syncthreads();
    }
    constexpr uint32_t kWarps = T / 32u;
    const uint32_t WS = (N + 32u * (uint32_t)R - 1u) / (32u * (uint32_t)R), C = kWarps / WS;
    const uint32_t warp = tid >> 5, cs = warp / WS;
    const uint32_t j0 = ((warp % WS) * 32u + (tid & 31u)) * (uint32_t)R;
    if (cs < C && j0 < N) {
        uint32_t acc[R], va[R], vb[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0u;
        const uint32_t ng = (ncoef + (uint32_t)R - 1u) / (uint32_t)R;
        const uint32_t g0 = (uint32_t)((uint64_t)ng * cs / C), g1 = (uint32_t)((uint64_t)ng * (cs + 1u) / C);
        uint32_t gi = g0;
        if (gi < g1) load_words<R>(va, x + gi * (uint32_t)R + j0);
        while (gi < g1) {                                   // windows (va, vb), then (vb, va)
            uint32_t i = gi * (uint32_t)R;
            load_words<R>(vb, x + i + (uint32_t)R + j0);
            sum_group<R, T>(acc, va, vb, coef_bits<R>(cf, i));
            if (++gi >= g1) break;
            i += (uint32_t)R;
            load_words<R>(va, x + i + (uint32_t)R + j0);
            sum_group<R, T>(acc, vb, va, coef_bits<R>(cf, i));
            ++gi;
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (j0 + (uint32_t)r < N && acc[r]) atomicXor(&y[j0 + r], acc[r]);
    }
    __syncthreads();
    if (jb.mode == kJumpSum) {
        for (uint32_t j = tid; j < N; j += T) dst[j] = y[j];
        return;
    }
    for (uint32_t j = tid; j + 1u < N; j += T) dst[j] = y[j + 1u];
    if (tid == 0u) dst[N - 1u] = rec_word(y[0], y[1], y[M], mask, sh1, sh2, tbl);
}

// One job per block and round of the grid: jobs blockIdx.x, blockIdx.x +
// gridDim.x, ... below njobs, or below *njobs_dev when that is set (a
// captured launch, whose grid is fixed while its job count is not).
template <int R, int T>
__global__ void __launch_bounds__(T, T >= 1024 ? 1 : 2) k_jump_fused(const DevGen *gens, const uint32_t *src_base,
                                                    uint32_t *dst_base, const DevJump *jobs, uint32_t seq_cap,
                                                    uint32_t max_N, uint32_t njobs, const uint32_t *njobs_dev)
{
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint32_t tbl[16];
    const uint32_t n = njobs_dev ? *njobs_dev : njobs;
    for (uint32_t job = blockIdx.x; job < n; job += gridDim.x) {
        fused_job<R, T>(jobs[job], gens, src_base, dst_base, sm, tbl, seq_cap, max_N);
        __syncthreads();                                    // shared words reused by the next job
    }
}

constexpr uint32_t kFusedThreads = 512;
constexpr uint32_t kFusedThreadsBig = 1024;   // when one block fills an SM's shared memory
constexpr uint32_t kFusedR = 12;
constexpr size_t kFusedSmemMax = 200u * 1024u;
constexpr size_t kFusedTwoBlocks = 113u * 1024u;  // two blocks of this much fit on an SM

// Sequence window: the sum reads up to word ncoef - 1 + R + (N rounded up to
// a lane's R words) + R - 1 < ncoef + N + 3R.
size_t fused_smem(uint32_t seq_cap, uint32_t max_N, uint32_t max_ncoef)
{
    return sizeof(uint32_t) * ((size_t)seq_cap + max_N + (max_ncoef + 31u) / 32u + 4u);
}

}  // namespace

bool jump_fused_fits(uint32_t max_N, uint32_t max_nseq, uint32_t max_ncoef)
{
    return max_N <= kFusedR * kFusedThreads && fused_smem((max_nseq + 3u) & ~3u, max_N, max_ncoef) <= kFusedSmemMax;
}

namespace {

// The fused kernel for a launch whose blocks need smem bytes: 512 threads
// when two blocks fit on an SM, else 1024 (one block, twice the warps to hide
// the sum's latency; measured on MTGP44497-sized jobs).
void (*fused_kernel(size_t smem))(const DevGen *, const uint32_t *, uint32_t *, const DevJump *, uint32_t, uint32_t,
                                  uint32_t, const uint32_t *)
{
    return smem > kFusedTwoBlocks ? k_jump_fused<kFusedR, kFusedThreadsBig> : k_jump_fused<kFusedR, kFusedThreads>;
}

}  // namespace

cudaError_t prepare_jump_fused(uint32_t max_N, uint32_t max_nseq, uint32_t max_ncoef)
{
    if (max_N < 3u || !jump_fused_fits(max_N, max_nseq, max_ncoef)) return cudaErrorInvalidValue;
    const uint32_t seq_cap = (max_nseq + 3u) & ~3u;
    const size_t smem = fused_smem(seq_cap, max_N, max_ncoef);
    return raise_smem_limit((const void *)fused_kernel(smem), smem);
}

cudaError_t launch_jump_fused(const DevGen *gens, const uint32_t *src_base, uint32_t *dst_base, const DevJump *jobs,
                              uint32_t njobs, uint32_t max_N, uint32_t max_nseq, uint32_t max_ncoef, cudaStream_t s,
                              const uint32_t *njobs_dev, uint32_t grid)
{
    if (!njobs) return cudaSuccess;
    if (!grid || grid > njobs) grid = njobs;
    if (max_N < 3u || !jump_fused_fits(max_N, max_nseq, max_ncoef)) return cudaErrorInvalidValue;
    const uint32_t seq_cap = (max_nseq + 3u) & ~3u;
    const size_t smem = fused_smem(seq_cap, max_N, max_ncoef);
    auto k = fused_kernel(smem);
    const uint32_t threads = smem > kFusedTwoBlocks ? kFusedThreadsBig : kFusedThreads;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusNone) {
        e = raise_smem_limit((const void *)k, smem);
        if (e != cudaSuccess) return e;
    }
    clear_stale_error();
    k<<<grid, threads, smem, s>>>(gens, src_base, dst_base, jobs, seq_cap, max_N, njobs, njobs_dev);
    return cudaGetLastError();
}

cudaError_t launch_walk(const DevGen *gens, const uint32_t *src_base, uint32_t *seq_base, const DevJump *jobs,
                        uint32_t njobs, uint32_t max_N, cudaStream_t s)
{
    if (!njobs) return cudaSuccess;
    if (max_N < 3u || max_N > 4096u) return cudaErrorInvalidValue;
    const uint32_t Rb = pow2_at_least(2u * max_N);              // >= N + S for every job
    clear_stale_error();
    k_walk<<<njobs, kJumpThreads, Rb * sizeof(uint32_t), s>>>(gens, src_base, seq_base, jobs, Rb);
    return cudaGetLastError();
}

cudaError_t launch_jump_sum(const DevGen *gens, const uint32_t *seq_base, uint32_t *dst_base, const DevJump *jobs,
                            uint32_t njobs, uint32_t max_N, cudaStream_t s)
{
    if (!njobs) return cudaSuccess;
    if (max_N < 3u || max_N > 4096u) return cudaErrorInvalidValue;
    const size_t smem = (size_t)max_N * sizeof(uint32_t);
    clear_stale_error();
    if (max_N <= 8u * kJumpThreads)
        k_jump_sum<8><<<njobs, kJumpThreads, smem, s>>>(gens, seq_base, dst_base, jobs);
    else
        k_jump_sum<16><<<njobs, kJumpThreads, smem, s>>>(gens, seq_base, dst_base, jobs);
    return cudaGetLastError();
}

}  // namespace mtgp
