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

// The same search with the polynomial work on the GPU.  Candidates run in
// batches of up to 4096: the host draws each candidate and walks its MSB
// sequence (threads over candidates), one warp per candidate finds the
// sequence's minimal polynomial (mtgp_bm.cu), and one block per candidate of
// degree mexp runs the irreducibility sieve (mtgp_irr.cu, stage 0) on the
// caller's stream.  The few survivors' p squarings (stage 1) take far longer
// than a batch's sieve, so they run on a stream of their own per batch (up to
// kIrrSlots batches in flight) while later batches are walked and sieved;
// batches are settled in order, so the first accepted candidate is the host
// search's.
namespace {
constexpr uint32_t kIrrSieve = 40;   // factors of degree <= 40 found before the squarings
constexpr uint32_t kIrrSlots = 4;    // batches whose squarings may run at once
}  // namespace

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
    if (mexp < 33u) return (mtgp_status)report_error(MTGP_EINVAL, "search: the GPU search needs mexp > 32");
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nt = threads ? threads : hw;
    const uint64_t n = 2ull * mexp;
    const uint32_t w64 = (uint32_t)(n / 64u) + 1u, words = 2u * w64;   // msb_sequence's layout
    const uint32_t owords = mexp / 32u + 2u;
    const uint64_t batch = std::min<uint64_t>(4096u, max_tries);
    cudaStream_t s = (cudaStream_t)stream;
    struct Slot {
        uint32_t *d_out = nullptr, *d_len = nullptr, *d_ver = nullptr, *h_ver = nullptr;
        cudaStream_t sf = nullptr;
        cudaEvent_t sieved = nullptr, settled = nullptr;
        bool pending = false;
        uint64_t base = 0, nb = 0;
    };
    Slot slot[kIrrSlots];
    uint32_t *d_seq = nullptr;
    uint32_t *h_abort = nullptr, *d_abort = nullptr;   // set once the result is known: later squarings stop
    auto cleanup = [&] {
        if (h_abort) *(volatile uint32_t *)h_abort = 1u;
        (void)cudaStreamSynchronize(s);
        for (Slot &q : slot) {
            if (q.sf) (void)cudaStreamSynchronize(q.sf);
            cudaFree(q.d_out);
            cudaFree(q.d_len);
            cudaFree(q.d_ver);
            cudaFreeHost(q.h_ver);
            if (q.sieved) cudaEventDestroy(q.sieved);
            if (q.settled) cudaEventDestroy(q.settled);
            if (q.sf) cudaStreamDestroy(q.sf);
        }
        cudaFree(d_seq);
        if (h_abort) cudaFreeHost(h_abort);
        (void)cudaGetLastError();
    };
    auto cuda_err = [&](cudaError_t e, const char *what) {
        cleanup();
        char buf[200];
        snprintf(buf, sizeof buf, "search: %s: %s", what, cudaGetErrorString(e));
        return (mtgp_status)report_error(e == cudaErrorMemoryAllocation ? MTGP_ENOMEM : MTGP_ECUDA, buf);
    };
    cudaError_t e = cudaMalloc(&d_seq, (size_t)batch * words * 4u);
    if (e == cudaSuccess) e = cudaHostAlloc(&h_abort, sizeof(uint32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *(volatile uint32_t *)h_abort = 0u;
        e = cudaHostGetDevicePointer(&d_abort, h_abort, 0);
    }
    for (Slot &q : slot) {
        if (e == cudaSuccess) e = cudaMalloc(&q.d_out, (size_t)batch * owords * 4u);
        if (e == cudaSuccess) e = cudaMalloc(&q.d_len, (size_t)batch * 4u);
        if (e == cudaSuccess) e = cudaMalloc(&q.d_ver, (size_t)batch * 4u);
        if (e == cudaSuccess) e = cudaHostAlloc(&q.h_ver, (size_t)batch * 4u, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q.sf, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.sieved, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.settled, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_err(e, "allocation");
    // Settles the batch in slot q (waits for its squarings): the index of its
    // first accepted candidate, or UINT64_MAX.
    auto settle = [&](Slot &q, uint64_t *j_out) -> cudaError_t {
        *j_out = std::numeric_limits<uint64_t>::max();
        if (!q.pending) return cudaSuccess;
        q.pending = false;
        const cudaError_t r = cudaEventSynchronize(q.settled);
        if (r != cudaSuccess) return r;
        for (uint64_t j = 0; j < q.nb; ++j)
            if (q.h_ver[j] == 1u) {
                *j_out = j;
                break;
            }
        return cudaSuccess;
    };
    // Reports the accepted candidate j of slot q.
    auto accept = [&](Slot &q, uint64_t j) -> mtgp_status {
        std::vector<uint32_t> poly(owords);
        cudaError_t r = cudaMemcpy(poly.data(), q.d_out + (size_t)j * owords, (size_t)owords * 4u,
                                   cudaMemcpyDeviceToHost);
        if (r != cudaSuccess) return cuda_err(r, "copy of the accepted polynomial");
        const uint64_t cand = q.base + j;
        cleanup();
        const mtgp_status r2 = mtgp_params_draw(mexp, seed0 + cand, id, out);
        if (r2 != MTGP_OK) return r2;
        *found_seed = seed0 + cand;
        *tries = cand + 1u;
        if (charpoly) {
            std::memset(charpoly, 0, sizeof(uint64_t) * charpoly_words);
            for (uint32_t b = 0; b <= mexp; ++b)
                if ((poly[b >> 5] >> (b & 31u)) & 1u) charpoly[b >> 6] |= 1ull << (b & 63u);
        }
        return MTGP_OK;
    };
    try {
        std::vector<uint64_t> seq((size_t)batch * w64);
        uint64_t bi = 0;
        for (uint64_t base = 0; base < max_tries; base += batch, ++bi) {
            Slot &q = slot[bi % kIrrSlots];
            uint64_t j = 0;
            e = settle(q, &j);                                    // the batch kIrrSlots back, in order
            if (e != cudaSuccess) return cuda_err(e, "irreducibility squarings");
            if (j != std::numeric_limits<uint64_t>::max()) return accept(q, j);
            const uint64_t nb = std::min<uint64_t>(batch, max_tries - base);
            std::atomic<uint64_t> next{0};
            std::atomic<bool> bad{false};
            auto walker = [&] {
                try {
                    std::vector<uint64_t> bits;
                    for (uint64_t t; (t = next.fetch_add(1)) < nb;) {
                        mtgp_params p;
                        if (mtgp_params_draw(mexp, seed0 + base + t, id, &p) != MTGP_OK) {
                            bad = true;
                            return;
                        }
                        msb_sequence(p, 12345u + base + t, n, bits);
                        std::copy(bits.begin(), bits.begin() + w64, seq.begin() + (ptrdiff_t)(t * w64));
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
            if (e == cudaSuccess) e = launch_bm(d_seq, (uint32_t)nb, (uint32_t)n, words, q.d_out, owords, q.d_len, s);
            if (e == cudaSuccess)
                e = launch_irr(q.d_out, (uint32_t)nb, owords, q.d_len, mexp, kIrrSieve, 0u, nullptr, q.d_ver, s);
            if (e == cudaSuccess) e = cudaEventRecord(q.sieved, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(q.sf, q.sieved, 0);
            if (e == cudaSuccess)
                e = launch_irr(q.d_out, (uint32_t)nb, owords, q.d_len, mexp, kIrrSieve, 1u, d_abort, q.d_ver, q.sf);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(q.h_ver, q.d_ver, (size_t)nb * 4u, cudaMemcpyDeviceToHost, q.sf);
            if (e == cudaSuccess) e = cudaEventRecord(q.settled, q.sf);
            if (e != cudaSuccess) return cuda_err(e, "Berlekamp-Massey and irreducibility batch");
            q.pending = true;
            q.base = base;
            q.nb = nb;
        }
        for (uint64_t k = 0; k < kIrrSlots; ++k) {                // the batches still in flight, in order
            Slot &q = slot[(bi + k) % kIrrSlots];
            uint64_t j = 0;
            e = settle(q, &j);
            if (e != cudaSuccess) return cuda_err(e, "irreducibility squarings");
            if (j != std::numeric_limits<uint64_t>::max()) return accept(q, j);
        }
    } catch (const std::exception &) {
        cleanup();
        return (mtgp_status)report_error(MTGP_ENOMEM, "search: host allocation or thread start failed");
    }
    cleanup();
    return (mtgp_status)report_error(MTGP_EINVAL, "search: no full-period set within max_tries");
}

// Irreducibility of host polynomials of prime degree p on the GPU (the
// search's acceptance test, for callers and tests).
extern "C" mtgp_status mtgp_f2_irreducible_gpu(const uint64_t *polys, uint32_t count, uint32_t words, uint32_t p,
                                               void *stream, uint8_t *verdicts)
{
    using namespace mtgp;
    if (!polys || !verdicts || count == 0)
        return (mtgp_status)report_error(MTGP_EINVAL, "irreducible: NULL pointer or count 0");
    bool prime = p > 32u;
    for (uint32_t d = 2; prime && (uint64_t)d * d <= p; ++d) prime = p % d != 0u;
    if (!prime) return (mtgp_status)report_error(MTGP_EINVAL, "irreducible: p must be a prime > 32");
    if (words < p / 64u + 1u) return (mtgp_status)report_error(MTGP_EINVAL, "irreducible: words < p / 64 + 1");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *d_polys = nullptr, *d_ver = nullptr;
    auto fail_cuda = [&](cudaError_t e, const char *what) {
        cudaFree(d_polys);
        cudaFree(d_ver);
        (void)cudaGetLastError();
        char buf[200];
        snprintf(buf, sizeof buf, "irreducible: %s: %s", what, cudaGetErrorString(e));
        return (mtgp_status)report_error(e == cudaErrorMemoryAllocation ? MTGP_ENOMEM : MTGP_ECUDA, buf);
    };
    // 64-bit little-endian words are pairs of 32-bit words in the same order
    const size_t bytes = (size_t)count * words * 8u;
    cudaError_t e = cudaMalloc(&d_polys, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d_ver, (size_t)count * 4u);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc");
    try {
        std::vector<uint32_t> ver(count);
        e = cudaMemcpyAsync(d_polys, polys, bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = launch_irr(d_polys, count, 2u * words, nullptr, p, kIrrSieve, 0u, nullptr, d_ver, s);
        if (e == cudaSuccess)
            e = launch_irr(d_polys, count, 2u * words, nullptr, p, kIrrSieve, 1u, nullptr, d_ver, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ver.data(), d_ver, (size_t)count * 4u, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail_cuda(e, "test");
        for (uint32_t j = 0; j < count; ++j) verdicts[j] = ver[j] ? 1u : 0u;
    } catch (const std::exception &) {
        cudaFree(d_polys);
        cudaFree(d_ver);
        return (mtgp_status)report_error(MTGP_ENOMEM, "irreducible: host allocation failed");
    }
    cudaFree(d_polys);
    cudaFree(d_ver);
    return MTGP_OK;
}
