// Irreducibility over F2 of polynomials of prime degree p on the GPU, one
// block per polynomial: the acceptance test of the Sec. 5 recursion search.
// A parameter set has full period when the characteristic polynomial of its
// recursion has degree p = mexp and is irreducible (2^p - 1 is a Mersenne
// prime, so irreducible means primitive).
//
// For prime p, phi of degree p is irreducible iff phi has no root in F2 and
// x^(2^p) = x (mod phi): the only proper divisor of p is 1 (Rabin's test).
// Before the p squarings a sieve rejects most reducible phi: with
// acc = prod_{K/2 < k <= K} (x^(2^k) - x) mod phi, gcd(phi, acc) != 1 exactly
// when phi has an irreducible factor of degree <= K (every d <= K divides
// some k in (K/2, K]), and x^(2^k) = x for some k < p also means a factor of
// degree < p.  The verdicts equal the host's test (mtgp_search.cpp), which
// sieves with the product over all k <= K.
//
// Arithmetic: polynomials are bit arrays of 32-bit words in shared memory
// (bit j of word j/32 = coefficient of x^j).  Squaring spreads bits; a
// product is a sum of 32 x 32 carry-less word products.  Reduction modulo a
// divisor b of degree db runs from the top in 32-bit windows [db + 32k,
// db + 32k + 32): the window's bits w determine the 32-bit quotient digit q
// by the triangular system w = q ^ ((q (x) h) >> 32), (x) the carry-less
// product and h the 32 coefficients of b below its leading one; then
// a ^= (q (x) b) x^(32k) clears the window.  For phi the map w -> q (linear)
// is tabulated once per block, four byte-indexed tables; for the gcd's
// changing divisors warp 0 solves it bit by bit.
#include "mtgp_internal.h"

namespace mtgp {
namespace {

constexpr uint32_t kIrrThreads = 512;

// 64-bit carry-less product of two 32-bit words.
__device__ __forceinline__ uint64_t clmul32(uint32_t a, uint32_t b)
{
    uint64_t r = 0;
    const uint64_t bb = b;
#pragma unroll
    for (int i = 0; i < 32; ++i) r ^= (bb << i) & (0ull - (uint64_t)((a >> i) & 1u));
    return r;
}

// Carry-less product of a word q and a nibble n.
__device__ __forceinline__ uint64_t clmul_nibble(uint32_t q, uint32_t n)
{
    const uint64_t qq = q;
    return ((n & 1u) ? qq : 0ull) ^ ((n & 2u) ? qq << 1 : 0ull) ^ ((n & 4u) ? qq << 2 : 0ull) ^
           ((n & 8u) ? qq << 3 : 0ull);
}

// Carry-less product of the window's digit q (tabulated: tq[n] = q * n for
// n < 16) and a word w.
__device__ __forceinline__ uint64_t clmul_q(const uint64_t *tq, uint32_t w)
{
    uint64_t r = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) r ^= tq[(w >> (4 * j)) & 15u] << (4 * j);
    return r;
}

// 32 bits of the array a from bit offset o (a must hold word o / 32 + 1).
__device__ __forceinline__ uint32_t bits32_at(const uint32_t *a, uint32_t o)
{
    const uint32_t w = o >> 5, sh = o & 31u;
    return __funnelshift_r(a[w], a[w + 1u], sh);
}

// The 32 coefficients of b just below its leading one (degree db >= 1), bit
// m = coefficient of x^(db - 32 + m) (zero below x^0).
__device__ __forceinline__ uint32_t top32_below(const uint32_t *b, uint32_t db)
{
    if (db >= 32u) return bits32_at(b, db - 32u);
    return b[0] << (32u - db);
}

// The quotient digit q of a window w under top coefficients h, bit by bit
// (the same in every thread that calls it with the same arguments).
__device__ __forceinline__ uint32_t solve_digit(uint32_t w, uint32_t h)
{
    uint32_t q = 0;
#pragma unroll
    for (int i = 31; i >= 1; --i) {
        const uint32_t bit = (w >> i) & 1u;
        q |= bit << i;
        w ^= (h >> (32 - i)) & (0u - bit);
    }
    return q | (w & 1u);
}

// Degree of a whose bits above maxdeg are zero (-1 for zero), computed by
// every thread alike from the top word down.
__device__ __forceinline__ int top_degree(const uint32_t *a, int maxdeg)
{
    for (int w = maxdeg / 32; w >= 0; --w) {
        const uint32_t v = a[w];
        if (v) return 32 * w + 31 - __clz(v);
    }
    return -1;
}

// Shared scratch of one block.
struct IrrShared {
    uint64_t *V;       // 2W products of a multiplication
    uint64_t *tq;      // 2 x 16: q * n, by window parity
    uint32_t *phi;     // W (+2)
    uint32_t *r;       // W: x^(2^k) mod phi
    uint32_t *acc;     // W: the sieve's product
    uint32_t *t;       // 2W + 2: products before reduction
    uint32_t *ga, *gb; // W + 2 each: the gcd's pair
    uint32_t *qt;      // 1024: quotient-digit tables for phi (4 x 256)
    uint32_t *col;     // 32: the digits of single-bit windows
    uint32_t *sq;      // 2: the window's digit, by window parity
    uint32_t W;
};

// Warp 0: the quotient digit of the window at bit s of a and its nibble
// table, published in the slots of parity `par`.
__device__ __forceinline__ void publish_digit(const IrrShared &S, const uint32_t *a, uint32_t s, uint32_t h,
                                              bool fixed, uint32_t par)
{
    const uint32_t lane = threadIdx.x;
    const uint32_t w = bits32_at(a, s);
    const uint32_t q = fixed ? S.qt[w & 255u] ^ S.qt[256u + ((w >> 8) & 255u)] ^ S.qt[512u + ((w >> 16) & 255u)] ^
                                   S.qt[768u + (w >> 24)]
                             : solve_digit(w, h);
    if (lane < 16u) S.tq[16u * par + lane] = clmul_nibble(q, lane);
    if (lane == 0u) S.sq[par] = q;
}

// a mod b in place: a of degree <= da, b of degree db >= 1, a's array holding
// word (da - db) / 32 + db / 32 + 1.  Afterwards a has degree < db.  With
// `fixed`, b is phi and the digit comes from the tables; otherwise it is
// solved bit by bit.  Thread t updates the words Wb - t, Wb - t - 512, ... of
// the window's product (Wb = db / 32 + 1), so the two words that hold the
// next window's bits are written by warp 0 alone: warp 0 finds the next digit
// as soon as its own writes are done, while the other warps finish theirs,
// and one block barrier per window publishes the digit (digit and nibble
// table alternate between two slots by window parity).
__device__ void blk_reduce(const IrrShared &S, uint32_t *a, int da, const uint32_t *b, uint32_t db, bool fixed)
{
    const uint32_t tid = threadIdx.x;
    if (da < (int)db) return;
    const uint32_t h = top32_below(b, db);
    const uint32_t Wb = db / 32u + 1u;
    const int kmax = (int)((uint32_t)da - db) / 32;
    if (tid < 32u) publish_digit(S, a, db + 32u * (uint32_t)kmax, h, fixed, (uint32_t)kmax & 1u);
    __syncthreads();
    for (int k = kmax; k >= 0; --k) {
        const uint32_t par = (uint32_t)k & 1u;
        const uint32_t q = S.sq[par];                          // uniform
        if (q != 0u) {                                         // a ^= (q b) x^(32 k)
            const uint64_t *tq = S.tq + 16u * par;
            for (uint32_t i = tid; i <= Wb; i += kIrrThreads) {
                const uint32_t m = Wb - i;
                uint32_t v = 0;
                if (m < Wb) v = (uint32_t)clmul_q(tq, b[m]);
                if (m > 0u) v ^= (uint32_t)(clmul_q(tq, b[m - 1u]) >> 32);
                a[(uint32_t)k + m] ^= v;
            }
        }
        if (k > 0 && tid < 32u) {                              // the next window's bits: warp 0's words
            __syncwarp();
            publish_digit(S, a, db + 32u * (uint32_t)(k - 1), h, fixed, par ^ 1u);
        }
        __syncthreads();
    }
}

// t = r^2 (r of degree < p), words 0 .. 2W+1.
__device__ void blk_square(const IrrShared &S, const uint32_t *r)
{
    const uint32_t W = S.W;
    for (uint32_t i = threadIdx.x; i < W + 1u; i += kIrrThreads) {
        uint32_t lo = 0, hi = 0;
        if (i < W) {
            lo = r[i] & 0xFFFFu;
            hi = r[i] >> 16;
            lo = (lo | (lo << 8)) & 0x00FF00FFu;
            lo = (lo | (lo << 4)) & 0x0F0F0F0Fu;
            lo = (lo | (lo << 2)) & 0x33333333u;
            lo = (lo | (lo << 1)) & 0x55555555u;
            hi = (hi | (hi << 8)) & 0x00FF00FFu;
            hi = (hi | (hi << 4)) & 0x0F0F0F0Fu;
            hi = (hi | (hi << 2)) & 0x33333333u;
            hi = (hi | (hi << 1)) & 0x55555555u;
        }
        S.t[2u * i] = lo;
        S.t[2u * i + 1u] = hi;
    }
    __syncthreads();
}

// t = a b (a, b of degree < p), words 0 .. 2W+1.
__device__ void blk_mul(const IrrShared &S, const uint32_t *a, const uint32_t *b)
{
    const uint32_t W = S.W;
    for (uint32_t j = threadIdx.x; j + 1u < 2u * W; j += kIrrThreads) {
        const uint32_t i0 = j >= W ? j - W + 1u : 0u, i1 = j < W ? j : W - 1u;
        uint64_t v = 0;
        for (uint32_t i = i0; i <= i1; ++i) v ^= clmul32(a[i], b[j - i]);
        S.V[j] = v;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < 2u * W + 2u; j += kIrrThreads) {
        uint32_t v = 0;
        if (j + 1u < 2u * W) v = (uint32_t)S.V[j];
        if (j >= 1u && j < 2u * W) v ^= (uint32_t)(S.V[j - 1u] >> 32);
        S.t[j] = v;
    }
    __syncthreads();
}

__device__ void blk_copy(uint32_t *dst, const uint32_t *src, uint32_t n)
{
    for (uint32_t i = threadIdx.x; i < n; i += kIrrThreads) dst[i] = src[i];
    __syncthreads();
}

// One block per polynomial.  polys: count polynomials of `words` 32-bit words
// each; deg: their degrees (nullptr: read from the words).  Stage 0 (the
// sieve) sets verdict[j] = 0 for a polynomial found reducible (degree other
// than p, a root, a factor of degree <= K) and kSurvivor otherwise; stage 1
// runs the p squarings for the survivors and sets 1 (irreducible) or 0.  A
// nonzero *abort (host memory the caller may set while stage 1 runs; nullptr
// for none) ends stage 1 early, every 32 squarings, with verdict 0.
constexpr uint32_t kSurvivor = 2u;

__global__ void __launch_bounds__(kIrrThreads, 2) k_irr(const uint32_t *__restrict__ polys, uint32_t words,
                                                     const uint32_t *__restrict__ deg, uint32_t p, uint32_t K,
                                                     uint32_t stage, const uint32_t *abort,
                                                     uint32_t *__restrict__ verdict)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t tid = threadIdx.x, j = blockIdx.x;
    const uint32_t W = p / 32u + 1u;
    if (stage == 1u && verdict[j] != kSurvivor) return;          // the same word for every thread
    IrrShared S;
    S.W = W;
    S.V = reinterpret_cast<uint64_t *>(smem);
    S.tq = S.V + 2u * W;
    S.phi = reinterpret_cast<uint32_t *>(S.tq + 32);
    S.r = S.phi + W + 2u;
    S.acc = S.r + W;
    S.t = S.acc + W;
    S.ga = S.t + 2u * W + 2u;
    S.gb = S.ga + W + 2u;
    S.qt = S.gb + W + 2u;
    S.col = S.qt + 1024u;
    S.sq = S.col + 32u;
    const uint32_t *src = polys + (size_t)j * words;
    __shared__ int s_ok;
    if (tid == 0) s_ok = deg ? (deg[j] == p) : 1;
    for (uint32_t w = tid; w < W + 2u; w += kIrrThreads) S.phi[w] = w < W ? src[w] : 0u;
    __syncthreads();
    // degree exactly p, no root 0 (phi(0) = 1), no root 1 (odd weight)
    uint32_t par = 0, high = 0;
    for (uint32_t w = tid; w < words; w += kIrrThreads) {
        const uint32_t v = src[w];
        par ^= (uint32_t)__popc(v) & 1u;
        if (w > p / 32u) high |= v;
        if (w == p / 32u) high |= v & ~((2u << (p & 31u)) - 1u);   // bits above p
    }
    const int odd = __syncthreads_count(par) & 1;
    const int over = __syncthreads_or(high != 0u);
    const bool lead = (S.phi[p / 32u] >> (p & 31u)) & 1u;
    if (!s_ok || over || !lead || !(S.phi[0] & 1u) || !odd) {
        if (tid == 0) verdict[j] = 0u;
        return;
    }
    // quotient-digit tables for phi
    const uint32_t h = top32_below(S.phi, p);
    if (tid < 32u) S.col[tid] = solve_digit(1u << tid, h);
    __syncthreads();
    for (uint32_t e = tid; e < 1024u; e += kIrrThreads) {
        const uint32_t c = e >> 8, v = e & 255u;
        uint32_t q = 0;
        for (uint32_t i = 0; i < 8u; ++i)
            if ((v >> i) & 1u) q ^= S.col[8u * c + i];
        S.qt[e] = q;
    }
    for (uint32_t w = tid; w < W; w += kIrrThreads) {
        S.r[w] = w == 0 ? 2u : 0u;                               // x
        S.acc[w] = w == 0 ? 1u : 0u;                             // 1
    }
    __syncthreads();
    if (stage == 1u) {                                           // x^(2^p) = x mod phi
        __shared__ uint32_t s_abort;
        for (uint32_t k = 1; k <= p; ++k) {
            if (abort && (k & 31u) == 0u) {
                if (tid == 0) s_abort = *(volatile const uint32_t *)abort;
                __syncthreads();
                if (s_abort) {                                   // uniform: read after the barrier
                    if (tid == 0) verdict[j] = 0u;
                    return;
                }
            }
            blk_square(S, S.r);
            blk_reduce(S, S.t, 2 * (int)p - 2, S.phi, p, true);
            blk_copy(S.r, S.t, W);
        }
        uint32_t nz = 0;
        for (uint32_t w = tid; w < W; w += kIrrThreads) nz |= w == 0 ? (S.r[0] ^ 2u) : S.r[w];
        const int differs = __syncthreads_or(nz != 0u);
        if (tid == 0) verdict[j] = differs ? 0u : 1u;
        return;
    }
    const uint32_t Kc = K < p - 1u ? K : p - 1u;
    bool reducible = false;
    for (uint32_t k = 1; k <= Kc && !reducible; ++k) {
        blk_square(S, S.r);                                      // x^(2^k)
        blk_reduce(S, S.t, 2 * (int)p - 2, S.phi, p, true);
        blk_copy(S.r, S.t, W);
        // x^(2^k) - x = 0 mod phi: all factors of degree | k < p
        uint32_t nz = 0;
        for (uint32_t w = tid; w < W; w += kIrrThreads) nz |= w == 0 ? (S.r[0] ^ 2u) : S.r[w];
        if (!__syncthreads_or(nz != 0u)) {
            reducible = true;
            break;
        }
        if (2u * k > Kc) {                                       // k in (K/2, K]: acc *= x^(2^k) - x
            if (tid == 0) S.r[0] ^= 2u;
            __syncthreads();
            blk_mul(S, S.acc, S.r);
            if (tid == 0) S.r[0] ^= 2u;
            blk_reduce(S, S.t, 2 * (int)p - 2, S.phi, p, true);
            blk_copy(S.acc, S.t, W);
        }
    }
    if (!reducible) {                                            // gcd(phi, acc)
        blk_copy(S.ga, S.phi, W + 2u);
        for (uint32_t w = tid; w < W + 2u; w += kIrrThreads) S.gb[w] = w < W ? S.acc[w] : 0u;
        __syncthreads();
        uint32_t *a = S.ga, *b = S.gb;
        int da = (int)p, db = top_degree(b, (int)p - 1);
        while (db > 0) {
            blk_reduce(S, a, da, b, (uint32_t)db, false);        // a = a mod b
            da = top_degree(a, db - 1);
            uint32_t *tp = a;
            a = b;
            b = tp;
            const int td = da;
            da = db;
            db = td;
        }
        reducible = db < 0;                                      // b = 0: gcd = a of degree >= 1
    }
    if (tid == 0) verdict[j] = reducible ? 0u : kSurvivor;
}

}  // namespace

size_t irr_smem_bytes(uint32_t p)
{
    const size_t W = p / 32u + 1u;
    return 8u * (2u * W + 32u) + 4u * ((W + 2u) + W + W + (2u * W + 2u) + 2u * (W + 2u) + 1024u + 32u + 2u);
}

cudaError_t launch_irr(const uint32_t *polys, uint32_t count, uint32_t words, const uint32_t *deg, uint32_t p,
                       uint32_t K, uint32_t stage, const uint32_t *abort, uint32_t *verdict, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    if (p < 33u || words < p / 32u + 1u || stage > 1u) return cudaErrorInvalidValue;
    const size_t smem = irr_smem_bytes(p);
    cudaError_t e = raise_smem_limit((const void *)k_irr, smem);
    if (e != cudaSuccess) return e;
    clear_stale_error();
    k_irr<<<count, kIrrThreads, smem, s>>>(polys, words, deg, p, K, stage, abort, verdict);
    return cudaGetLastError();
}

}  // namespace mtgp
