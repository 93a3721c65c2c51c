// Berlekamp-Massey over F2 on the GPU, one warp per bit sequence: the
// characteristic-polynomial step of the MTGPDC recursion search (Sec. 5),
// run for a batch of candidates at once.
//
// For s_0 .. s_{n-1} the algorithm keeps a connection polynomial
// C(x) = 1 + c_1 x + .. + c_L x^L with s_k + c_1 s_{k-1} + .. + c_L s_{k-L} = 0
// for the terms seen so far, and the previous C as B.  At term k the
// discrepancy d = sum_{i=0..L} c_i s_{k-i} decides: d = 0 keeps C; else
// C += x^m B, and when 2L <= k the length becomes k + 1 - L and B the old C.
// The warp holds C, B and a spare in shared memory as bit arrays; d is a
// parity over the words of C AND a window of the reversed sequence (word j
// of a lane's share, a funnel shift aligning the window), reduced with one
// ballot.  The result leaves in annihilator form psi(x) = x^L C(1/x)
// (sum_j psi_j s_{k+j} = 0), as the host routine f2::minpoly returns it.
#include "mtgp_internal.h"

namespace mtgp {
namespace {

// Bit b of the bit array a (word b / 32).
__device__ __forceinline__ uint32_t bit_at(const uint32_t *a, uint32_t b) { return (a[b >> 5] >> (b & 31u)) & 1u; }

// 32 bits of a starting at bit offset o (o may be unaligned; a must hold the
// word after).
__device__ __forceinline__ uint32_t bits32(const uint32_t *a, uint32_t o)
{
    const uint32_t w = o >> 5, sh = o & 31u;
    return __funnelshift_r(a[w], a[w + 1u], sh);
}

// One block = one warp = one sequence.  seq: nseq bit sequences of n bits,
// `words` 32-bit words each (bit i of word i / 32); out: the annihilators,
// `owords` words each; len: their degrees L (0xFFFFFFFF if the linear
// complexity exceeds what the buffers hold, about n / 2, or owords).  Shared
// memory: the reversed sequence (words + 2) and three polynomial buffers (pw
// words each).
__global__ void __launch_bounds__(32) k_bm(const uint32_t *__restrict__ seq, uint32_t nseq, uint32_t n,
                                           uint32_t words, uint32_t pw, uint32_t *__restrict__ out,
                                           uint32_t owords, uint32_t *__restrict__ len)
{
    extern __shared__ uint32_t sm[];
    const uint32_t lane = threadIdx.x, q = blockIdx.x;
    if (q >= nseq) return;
    uint32_t *r = sm;                              // r_j = s_{n-1-j}, words + 2 words
    uint32_t *buf[3] = {sm + words + 2u, sm + words + 2u + pw, sm + words + 2u + 2u * pw};
    const uint32_t *s = seq + (size_t)q * words;
    for (uint32_t w = lane; w < words + 2u; w += 32u) r[w] = 0u;
    for (uint32_t w = lane; w < 3u * pw; w += 32u) buf[0][w] = 0u;
    __syncwarp();
    for (uint32_t j = lane; j < n; j += 32u)       // reverse the sequence
        if (bit_at(s, n - 1u - j)) atomicOr(&r[j >> 5], 1u << (j & 31u));
    __syncwarp();
    uint32_t *C = buf[0], *B = buf[1], *T = buf[2];
    if (lane == 0) {
        C[0] = 1u;
        B[0] = 1u;
    }
    __syncwarp();
    uint32_t L = 0, m = 1;
    for (uint32_t k = 0; k < n; ++k) {
        // d = sum_{i=0..L} c_i s_{k-i} = sum_i c_i r_{n-1-k+i}
        const uint32_t o = n - 1u - k, nw = (L >> 5) + 1u;
        uint32_t acc = 0;
        for (uint32_t w = lane; w < nw; w += 32u) acc ^= C[w] & bits32(r, o + 32u * w);
        const uint32_t d = __popc(__ballot_sync(0xffffffffu, __popc(acc) & 1u)) & 1u;
        if (!d) {
            ++m;
            continue;
        }
        // C' = C + x^m B over the words that can change (deg B + m <= the
        // larger of the two lengths, which stays below pw * 32)
        const uint32_t Lb = k + 1u - L;            // length after a change (if 2L <= k)
        const bool grow = 2u * L <= k;
        if (grow && (Lb >> 5) + 2u >= pw) {        // complexity above the buffers (n / 2): give up
            if (lane == 0) len[q] = 0xFFFFFFFFu;
            return;
        }
        const uint32_t top = ((grow ? Lb : L) >> 5) + 2u;
        const uint32_t ws = m >> 5, bs = m & 31u;
        uint32_t *D = grow ? T : C;                // grow: C' to the spare, B becomes the old C
        for (uint32_t w = lane; w < top && w < pw; w += 32u) {
            uint32_t bsh = 0;
            if (w >= ws) {
                const uint32_t hi = B[w - ws];
                const uint32_t lo = w > ws ? B[w - ws - 1u] : 0u;
                bsh = bs ? __funnelshift_l(lo, hi, bs) : hi;
            }
            D[w] = C[w] ^ bsh;
        }
        __syncwarp();
        if (grow) {
            uint32_t *oldB = B;
            B = C;
            C = T;
            T = oldB;
            // the spare's words above `top` must be zero for the next use
            for (uint32_t w = top + lane; w < pw; w += 32u) T[w] = 0u;
            L = Lb;
            m = 1;
        } else {
            ++m;
        }
        __syncwarp();
    }
    // psi_j = c_{L-j}
    if ((L >> 5) >= owords) {
        if (lane == 0) len[q] = 0xFFFFFFFFu;
        return;
    }
    uint32_t *o = out + (size_t)q * owords;
    for (uint32_t w = lane; w < owords; w += 32u) o[w] = 0u;
    __syncwarp();
    for (uint32_t j = lane; j <= L; j += 32u)
        if (bit_at(C, L - j)) atomicOr(&o[j >> 5], 1u << (j & 31u));
    if (lane == 0) len[q] = L;
}

}  // namespace

cudaError_t launch_bm(const uint32_t *seq, uint32_t nseq, uint32_t n, uint32_t words, uint32_t *out,
                      uint32_t owords, uint32_t *len, cudaStream_t s)
{
    if (nseq == 0) return cudaSuccess;
    const uint32_t pw = (n / 2u + 1u) / 32u + 4u;      // degree <= n / 2 for the searches here
    const size_t smem = ((size_t)words + 2u + 3u * (size_t)pw) * sizeof(uint32_t);
    cudaError_t e = raise_smem_limit((const void *)k_bm, smem);
    if (e != cudaSuccess) return e;
    clear_stale_error();
    k_bm<<<nseq, 32, smem, s>>>(seq, nseq, n, words, pw, out, owords, len);
    return cudaGetLastError();
}

}  // namespace mtgp
