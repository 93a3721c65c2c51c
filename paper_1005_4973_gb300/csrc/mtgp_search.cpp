// Recursion-parameter search of MTGPDC (Sec. 5), on the host cores.
//
// Candidate t is the parameter set mtgp_params_draw(mexp, seed0 + t, id): the
// ID embedded in R, random LSB blocks with R4 + I invertible, sh1 = 13,
// sh2 = 4, M in Sec. 5's range.  Its characteristic polynomial phi is the
// Berlekamp-Massey polynomial of the MSB sequence of 2 mexp words of the
// recursion (Sec. 3.6) from a nonzero state; the candidate is accepted when
// deg phi = mexp and phi is irreducible, hence primitive as mexp is a
// Mersenne exponent (Sec. 3.3, Sec. 5).  Irreducibility for prime degree p:
// gcd(phi, x^2 - x) = 1 and x^(2^p) = x mod phi; the squarings run anyway, so
// after the first K of them a gcd with prod_{k <= K} (x^(2^k) - x) rejects
// every phi with an irreducible factor of degree <= K early.
#include "mtgp.h"
#include "mtgp_f2.h"
#include "mtgp_internal.h"

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <exception>
#include <limits>
#include <thread>
#include <vector>

namespace mtgp {
namespace {

constexpr uint64_t kGammaS = 0x9E3779B97F4A7C15ull;

uint64_t mix64s(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// MSB sequence of the words x_N .. x_{N+nb-1} from a SplitMix64-filled state.
void msb_sequence(const mtgp_params &p, uint64_t state_seed, uint64_t nb, std::vector<uint64_t> &bits)
{
    const uint32_t N = p.N, M = p.pos;
    std::vector<uint32_t> x((size_t)N + (size_t)nb);
    const uint64_t s0 = state_seed ^ mix64s(kGammaS);
    uint32_t any = 0;
    for (uint32_t j = 0; j < N; ++j) {
        x[j] = (uint32_t)mix64s(s0 + (uint64_t)(j + 1u) * kGammaS);
        any |= (j == 0u) ? (x[j] & p.mask) : x[j];
    }
    if (!any) x[N - 1u] = 1u;
    bits.assign((size_t)(nb / 64u) + 1u, 0u);
    for (uint64_t k = 0; k < nb; ++k) {
        uint32_t t = (x[k] & p.mask) ^ x[k + 1u];
        t ^= t << p.sh1;
        const uint32_t u = t ^ (x[k + M] >> p.sh2);
        const uint32_t v = u ^ p.rec_tbl[u & 15u];
        x[N + k] = v;
        bits[k >> 6] |= (uint64_t)(v >> 31) << (k & 63u);
    }
}

bool irreducible_prime_degree(const f2::Poly &phi, uint64_t p, uint32_t sieve)
{
    if (f2::degree(phi) != (int64_t)p || !(phi[0] & 1u)) return false;      // degree, root 0
    unsigned ones = 0;
    for (uint64_t w : phi) ones ^= (unsigned)__builtin_parityll(w);
    if (!ones) return false;                                              // root 1
    const f2::Modulus M = f2::make_modulus(phi);
    const f2::Poly x{2u};
    f2::Poly r = x, acc{1u};
    const uint64_t K = std::min<uint64_t>(sieve, p - 1u);
    for (uint64_t k = 1; k <= p; ++k) {
        r = f2::sqrmod(r, M);                                             // x^(2^k)
        if (k <= K) {
            f2::Poly d = r;
            d.resize(std::max<size_t>(d.size(), 1u), 0u);
            d[0] ^= 2u;                                                   // x^(2^k) - x
            f2::trim(d);
            if (d.empty()) return false;                                  // a factor of degree | k < p
            acc = f2::mulmod(acc, d, M);
            if (k == K) {
                const f2::Poly g = f2::gcd(phi, acc);
                if (f2::degree(g) > 0) return false;
            }
        }
    }
    f2::trim(r);
    return r == x;
}

}  // namespace
}  // namespace mtgp

extern "C" mtgp_status mtgp_params_search(uint32_t mexp, uint64_t seed0, uint32_t id, uint64_t max_tries,
                                          uint32_t threads, mtgp_params *out, uint64_t *found_seed,
                                          uint64_t *tries, uint64_t *charpoly, uint32_t charpoly_words)
{
    using namespace mtgp;
    if (!out || !found_seed || !tries) return (mtgp_status)report_error(MTGP_EINVAL, "search: NULL argument");
    if (charpoly && charpoly_words < mexp / 64u + 1u)
        return (mtgp_status)report_error(MTGP_EINVAL, "search: charpoly needs mexp / 64 + 1 words");
    mtgp_params probe;
    mtgp_status st = mtgp_params_draw(mexp, seed0, id, &probe);
    if (st != MTGP_OK) return st;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nt = threads ? threads : hw;
    std::atomic<uint64_t> next{0}, best{std::numeric_limits<uint64_t>::max()};
    std::atomic<bool> oom{false};
    std::vector<f2::Poly> found_phi(nt);
    std::vector<uint64_t> found_t(nt, std::numeric_limits<uint64_t>::max());
    auto worker = [&](unsigned w) {
        try {
            std::vector<uint64_t> bits;
            for (;;) {
                const uint64_t t = next.fetch_add(1);
                if (t >= max_tries || t >= best.load()) return;
                mtgp_params p;
                if (mtgp_params_draw(mexp, seed0 + t, id, &p) != MTGP_OK) return;
                msb_sequence(p, 12345u + t, 2ull * mexp, bits);
                f2::Poly phi = f2::minpoly(bits.data(), 2ull * mexp);
                if (f2::degree(phi) != (int64_t)mexp) continue;
                if (!irreducible_prime_degree(phi, mexp, 40u)) continue;
                if (t < found_t[w]) {
                    found_t[w] = t;
                    found_phi[w] = phi;
                }
                uint64_t b = best.load();
                while (t < b && !best.compare_exchange_weak(b, t)) {
                }
                return;
            }
        } catch (const std::exception &) {
            oom = true;
        }
    };
    std::vector<std::thread> pool;
    try {
        for (unsigned w = 0; w < nt; ++w) pool.emplace_back(worker, w);
    } catch (const std::exception &) {
        oom = true;
    }
    for (auto &th : pool) th.join();
    if (oom) return (mtgp_status)report_error(MTGP_ENOMEM, "search: host allocation or thread start failed");
    const uint64_t t = best.load();
    if (t == std::numeric_limits<uint64_t>::max())
        return (mtgp_status)report_error(MTGP_EINVAL, "search: no full-period set within max_tries");
    unsigned w = 0;
    while (found_t[w] != t) ++w;
    st = mtgp_params_draw(mexp, seed0 + t, id, out);
    if (st != MTGP_OK) return st;
    *found_seed = seed0 + t;
    *tries = t + 1u;
    if (charpoly) {
        std::memset(charpoly, 0, sizeof(uint64_t) * charpoly_words);
        std::copy(found_phi[w].begin(), found_phi[w].end(), charpoly);
    }
    return MTGP_OK;
}

// The same search with the Berlekamp-Massey step on the GPU: candidates run in
// batches; the host draws each candidate and walks its MSB sequence (threads
// over candidates), one warp per candidate finds the sequence's minimal
// polynomial (mtgp_bm.cu), and the host tests the ones of degree mexp for
// irreducibility in candidate order (threads over candidates).  The first
// accepted candidate is the host search's.
extern "C" mtgp_status mtgp_params_search_gpu(uint32_t mexp, uint64_t seed0, uint32_t id, uint64_t max_tries,
                                              uint32_t threads, void *stream, mtgp_params *out,
                                              uint64_t *found_seed, uint64_t *tries, uint64_t *charpoly,
                                              uint32_t charpoly_words)
{
    using namespace mtgp;
    if (!out || !found_seed || !tries) return (mtgp_status)report_error(MTGP_EINVAL, "search: NULL argument");
    if (charpoly && charpoly_words < mexp / 64u + 1u)
        return (mtgp_status)report_error(MTGP_EINVAL, "search: charpoly needs mexp / 64 + 1 words");
    mtgp_params probe;
    mtgp_status st = mtgp_params_draw(mexp, seed0, id, &probe);
    if (st != MTGP_OK) return st;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nt = threads ? threads : hw;
    const uint64_t n = 2ull * mexp;
    const uint32_t w64 = (uint32_t)(n / 64u) + 1u, words = 2u * w64;   // msb_sequence's layout
    const uint32_t owords = mexp / 32u + 2u;
    const uint64_t batch = std::min<uint64_t>(4096u, max_tries);
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *d_seq = nullptr, *d_out = nullptr, *d_len = nullptr;
    auto cleanup = [&] {
        cudaFree(d_seq);
        cudaFree(d_out);
        cudaFree(d_len);
        (void)cudaGetLastError();
    };
    auto cuda_err = [&](cudaError_t e, const char *what) {
        cleanup();
        char buf[200];
        snprintf(buf, sizeof buf, "search: %s: %s", what, cudaGetErrorString(e));
        return (mtgp_status)report_error(e == cudaErrorMemoryAllocation ? MTGP_ENOMEM : MTGP_ECUDA, buf);
    };
    cudaError_t e = cudaMalloc(&d_seq, (size_t)batch * words * 4u);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)batch * owords * 4u);
    if (e == cudaSuccess) e = cudaMalloc(&d_len, (size_t)batch * 4u);
    if (e != cudaSuccess) return cuda_err(e, "cudaMalloc");
    try {
        std::vector<uint64_t> seq((size_t)batch * w64);
        std::vector<uint32_t> polys((size_t)batch * owords), lens(batch);
        for (uint64_t base = 0; base < max_tries; base += batch) {
            const uint64_t nb = std::min<uint64_t>(batch, max_tries - base);
            std::atomic<uint64_t> next{0};
            std::atomic<bool> bad{false};
            auto walker = [&] {
                try {
                    std::vector<uint64_t> bits;
                    for (uint64_t j; (j = next.fetch_add(1)) < nb;) {
                        mtgp_params p;
                        if (mtgp_params_draw(mexp, seed0 + base + j, id, &p) != MTGP_OK) {
                            bad = true;
                            return;
                        }
                        msb_sequence(p, 12345u + base + j, n, bits);
                        std::copy(bits.begin(), bits.begin() + w64, seq.begin() + (ptrdiff_t)(j * w64));
                    }
                } catch (const std::exception &) {
                    bad = true;
                }
            };
            std::vector<std::thread> pool;
            for (unsigned t = 0; t < nt; ++t) pool.emplace_back(walker);
            for (auto &th : pool) th.join();
            if (bad) {
                cleanup();
                return (mtgp_status)report_error(MTGP_ENOMEM, "search: host allocation failed");
            }
            e = cudaMemcpyAsync(d_seq, seq.data(), (size_t)nb * w64 * 8u, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = launch_bm(d_seq, (uint32_t)nb, (uint32_t)n, words, d_out, owords, d_len, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(lens.data(), d_len, (size_t)nb * 4u, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(polys.data(), d_out, (size_t)nb * owords * 4u, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_err(e, "Berlekamp-Massey batch");
            // candidates of degree mexp, in order; the smallest irreducible wins
            std::vector<uint64_t> cand;
            for (uint64_t j = 0; j < nb; ++j)
                if (lens[j] == mexp) cand.push_back(j);
            std::atomic<size_t> ci{0};
            std::atomic<uint64_t> best{std::numeric_limits<uint64_t>::max()};
            auto tester = [&] {
                try {
                    for (size_t i; (i = ci.fetch_add(1)) < cand.size();) {
                        const uint64_t j = cand[i];
                        if (j >= best.load()) return;
                        f2::Poly phi((size_t)(mexp / 64u) + 1u, 0u);
                        for (uint32_t b = 0; b <= mexp; ++b)
                            if ((polys[(size_t)j * owords + (b >> 5)] >> (b & 31u)) & 1u)
                                phi[b >> 6] |= 1ull << (b & 63u);
                        if (!irreducible_prime_degree(phi, mexp, 40u)) continue;
                        uint64_t b0 = best.load();
                        while (j < b0 && !best.compare_exchange_weak(b0, j)) {
                        }
                    }
                } catch (const std::exception &) {
                    bad = true;
                }
            };
            pool.clear();
            for (unsigned t = 0; t < nt; ++t) pool.emplace_back(tester);
            for (auto &th : pool) th.join();
            if (bad) {
                cleanup();
                return (mtgp_status)report_error(MTGP_ENOMEM, "search: host allocation failed");
            }
            const uint64_t j = best.load();
            if (j == std::numeric_limits<uint64_t>::max()) continue;
            cleanup();
            st = mtgp_params_draw(mexp, seed0 + base + j, id, out);
            if (st != MTGP_OK) return st;
            *found_seed = seed0 + base + j;
            *tries = base + j + 1u;
            if (charpoly) {
                std::memset(charpoly, 0, sizeof(uint64_t) * charpoly_words);
                for (uint32_t b = 0; b <= mexp; ++b)
                    if ((polys[(size_t)j * owords + (b >> 5)] >> (b & 31u)) & 1u) charpoly[b >> 6] |= 1ull << (b & 63u);
            }
            return MTGP_OK;
        }
    } catch (const std::exception &) {
        cleanup();
        return (mtgp_status)report_error(MTGP_ENOMEM, "search: host allocation or thread start failed");
    }
    cleanup();
    return (mtgp_status)report_error(MTGP_EINVAL, "search: no full-period set within max_tries");
}
