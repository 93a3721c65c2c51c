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

namespace mtgp {
namespace {

// The recursion's words x_0 .. x_{N+L-1} (Sec. 3.6) from a SplitMix64-filled
// nonzero state.
void raw_sequence(const mtgp_params &p, uint64_t L, std::vector<uint32_t> &x)
{
    const uint32_t N = p.N, M = p.pos;
    x.assign((size_t)N + (size_t)L, 0u);
    const uint64_t s0 = 0x5EEDull ^ mix64s(kGammaS);
    uint32_t any = 0;
    for (uint32_t j = 0; j < N; ++j) {
        x[j] = (uint32_t)mix64s(s0 + (uint64_t)(j + 1u) * kGammaS);
        any |= (j == 0u) ? (x[j] & p.mask) : x[j];
    }
    if (!any) x[N - 1u] = 1u;
    for (uint64_t i = 0; i < L; ++i) {
        uint32_t t = (x[i] & p.mask) ^ x[i + 1u];
        t ^= t << p.sh1;
        const uint32_t u = t ^ (x[i + M] >> p.sh2);
        x[N + i] = u ^ p.rec_tbl[u & 15u];
    }
}

// Tempered outputs o_0 .. o_{L-1} (Sec. 3.7) with the table tmp, as 32 bit
// planes of L bits each (plane b = bit b).
void output_planes(const mtgp_params &p, const uint32_t tmp[16], const std::vector<uint32_t> &x, uint64_t L,
                   std::vector<std::vector<uint64_t>> &planes)
{
    const uint32_t N = p.N, M = p.pos;
    planes.assign(32, std::vector<uint64_t>((size_t)(L / 64u) + 2u, 0u));
    for (uint64_t i = 0; i < L; ++i) {
        const uint32_t y = x[M - 1u + i];
        uint32_t z = y ^ (y >> 16);
        z ^= z >> 8;
        const uint32_t o = x[N + i] ^ tmp[z & 15u];
        for (uint32_t b = 0; b < 32u; ++b)
            planes[b][i >> 6] |= (uint64_t)((o >> b) & 1u) << (i & 63u);
    }
}

// k(v) by row echelon over the basis F^j s (j < p): row (i, b) = bits
// i .. i+p-1 of plane b; rows are added output by output, MSB first, until
// the first dependent one.  The basis is kept by lowest set bit, so a
// reduction only touches words at and above the current lowest bit.
uint32_t kv_one(const std::vector<std::vector<uint64_t>> &planes, uint32_t p, uint32_t v)
{
    const size_t W = (p + 63u) / 64u;
    std::vector<uint64_t> basis((size_t)p * W), row(W + 1u);
    std::vector<int32_t> piv(p, -1);
    uint32_t rank = 0, k = 0;
    const uint32_t kmax = p / v + 1u;
    for (uint32_t i = 0; i < kmax; ++i) {
        for (uint32_t t = 0; t < v; ++t) {                    // bits 31, 30, ..., 32 - v
            const std::vector<uint64_t> &pl = planes[31u - t];
            const uint32_t q = i >> 6, sh = i & 63u;
            for (size_t w = 0; w < W; ++w)
                row[w] = sh ? (pl[q + w] >> sh) | (pl[q + w + 1u] << (64u - sh)) : pl[q + w];
            if (p & 63u) row[W - 1u] &= (1ull << (p & 63u)) - 1u;
            size_t w0 = 0;
            for (;;) {
                while (w0 < W && !row[w0]) ++w0;
                if (w0 == W) return k;                        // dependent: k(v) = outputs so far
                const uint32_t c = (uint32_t)(64u * w0) + (uint32_t)__builtin_ctzll(row[w0]);
                if (piv[c] < 0) {
                    std::copy(row.begin(), row.begin() + (ptrdiff_t)W, basis.begin() + (ptrdiff_t)((size_t)rank * W));
                    piv[c] = (int32_t)rank++;
                    break;
                }
                const uint64_t *r = &basis[(size_t)piv[c] * W];
                for (size_t w = w0; w < W; ++w) row[w] ^= r[w];
            }
        }
        k = i + 1u;
    }
    return k;
}

}  // namespace
}  // namespace mtgp

namespace mtgp {
namespace {

// k(v), v = 1 .. 32, of the outputs with tempering table tmp; threads over v.
// Returns false on an allocation failure.
bool all_kv(const mtgp_params &p, const uint32_t tmp[16], const std::vector<uint32_t> &x, unsigned nt,
            uint32_t kv[32])
{
    std::vector<std::vector<uint64_t>> planes;
    output_planes(p, tmp, x, 2ull * p.mexp + 64u, planes);
    std::atomic<uint32_t> next{1};
    std::atomic<bool> oom{false};
    auto worker = [&] {
        try {
            for (uint32_t v; (v = next.fetch_add(1)) <= 32u;) kv[v - 1u] = kv_one(planes, p.mexp, v);
        } catch (const std::exception &) {
            oom = true;
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (auto &th : pool) th.join();
    return !oom;
}

uint32_t total_defect(uint32_t mexp, const uint32_t kv[32])
{
    uint32_t d = 0;
    for (uint32_t v = 1; v <= 32u; ++v) d += mexp / v - kv[v - 1u];
    return d;
}

unsigned thread_count(uint32_t threads)
{
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    return std::min<unsigned>(32u, threads ? threads : hw);
}

}  // namespace
}  // namespace mtgp

extern "C" mtgp_status mtgp_params_equidistribution(const mtgp_params *p, uint32_t threads, uint32_t *kv,
                                                    uint32_t *delta)
{
    using namespace mtgp;
    if (!p || !kv) return (mtgp_status)report_error(MTGP_EINVAL, "equidistribution: NULL argument");
    mtgp_status st = mtgp_params_validate(p);
    if (st != MTGP_OK) return st;
    try {
        std::vector<uint32_t> x;
        raw_sequence(*p, 2ull * p->mexp + 64u, x);
        uint32_t k[32];
        if (!all_kv(*p, p->tmp_tbl, x, thread_count(threads), k))
            return (mtgp_status)report_error(MTGP_ENOMEM, "equidistribution: host allocation failed");
        std::copy(k, k + 32, kv);
        if (delta) *delta = total_defect(p->mexp, k);
        return MTGP_OK;
    } catch (const std::exception &) {
        return (mtgp_status)report_error(MTGP_ENOMEM, "equidistribution: host allocation or thread start failed");
    }
}

// Tempering search (Sec. 5 says MTGPDC searches a tempering set after the
// recursion set but not how): candidate 0 is the input's table, candidate t
// >= 1 the table of four rows drawn by SplitMix64 from seed + t (Sec. 3.7:
// tmptbl[b] = b T with bit 3 of b selecting row 0); the smallest total defect
// wins, the earliest candidate on ties.
extern "C" mtgp_status mtgp_params_temper_search(const mtgp_params *in, uint64_t seed, uint32_t tries,
                                                 uint32_t threads, mtgp_params *out, uint32_t *delta)
{
    using namespace mtgp;
    if (!in || !out) return (mtgp_status)report_error(MTGP_EINVAL, "temper search: NULL argument");
    mtgp_status st = mtgp_params_validate(in);
    if (st != MTGP_OK) return st;
    try {
        std::vector<uint32_t> x;
        raw_sequence(*in, 2ull * in->mexp + 64u, x);
        const unsigned nt = thread_count(threads);
        uint32_t best_tbl[16], k[32];
        std::copy(in->tmp_tbl, in->tmp_tbl + 16, best_tbl);
        if (!all_kv(*in, in->tmp_tbl, x, nt, k))
            return (mtgp_status)report_error(MTGP_ENOMEM, "temper search: host allocation failed");
        uint32_t best = total_defect(in->mexp, k);
        for (uint32_t t = 1; t <= tries; ++t) {
            uint64_t s = seed + t;
            uint32_t rows[4], tbl[16];
            for (uint32_t &r : rows) {
                s += kGammaS;
                r = (uint32_t)mix64s(s);
            }
            for (uint32_t b = 0; b < 16u; ++b) {
                uint32_t v = 0;
                if (b & 8u) v ^= rows[0];
                if (b & 4u) v ^= rows[1];
                if (b & 2u) v ^= rows[2];
                if (b & 1u) v ^= rows[3];
                tbl[b] = v;
            }
            if (!all_kv(*in, tbl, x, nt, k))
                return (mtgp_status)report_error(MTGP_ENOMEM, "temper search: host allocation failed");
            const uint32_t d = total_defect(in->mexp, k);
            if (d < best) {
                best = d;
                std::copy(tbl, tbl + 16, best_tbl);
            }
        }
        *out = *in;
        std::copy(best_tbl, best_tbl + 16, out->tmp_tbl);
        if (delta) *delta = best;
        return MTGP_OK;
    } catch (const std::exception &) {
        return (mtgp_status)report_error(MTGP_ENOMEM, "temper search: host allocation or thread start failed");
    }
}

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
