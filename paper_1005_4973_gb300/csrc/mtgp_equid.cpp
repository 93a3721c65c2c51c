// Dimensions of equidistribution by lattice reduction, and the tempering
// search of Sec. 5.  See mtgp_equid.h.
#include "mtgp_equid.h"

#include <algorithm>
#include <utility>

namespace mtgp {
namespace eq {

namespace {

// a ^= b << s over F2, growing a as needed; db = degree of b (>= 0).
void xor_shl(Poly &a, const Poly &b, int64_t db, uint64_t s)
{
    const size_t nb = (size_t)(db / 64) + 1u;
    const size_t need = (size_t)((db + (int64_t)s) / 64) + 1u;
    if (a.size() < need) a.resize(need, 0u);
    uint64_t *d = a.data() + (s >> 6);
    const unsigned sh = (unsigned)(s & 63u);
    const size_t room = a.size() - (size_t)(s >> 6);
    if (!sh) {
        for (size_t k = 0; k < nb && k < room; ++k) d[k] ^= b[k];
        return;
    }
    uint64_t carry = 0;
    size_t k = 0;
    for (; k < nb && k < room; ++k) {
        d[k] ^= (b[k] << sh) | carry;
        carry = b[k] >> (64u - sh);
    }
    if (k < room) d[k] ^= carry;
}

// Degree of a, searching down from the word holding bit `hint` (a >= hint).
int64_t degree_from(const Poly &a, int64_t hint)
{
    size_t w = std::min(a.size(), (size_t)(hint / 64) + 1u);
    while (w-- > 0)
        if (a[w]) return (int64_t)(w * 64u) + 63 - (int64_t)__builtin_clzll(a[w]);
    return -1;
}

}  // namespace

Poly invmod(const Poly &a, const Poly &m)
{
    // u = su a, v = sv a (mod m) throughout; reduce the higher-degree one by
    // a shifted copy of the other until one of them is 1 (or 0: no inverse)
    Poly u = m, v = a, su, sv{1u};
    f2::trim(v);
    int64_t du = f2::degree(u), dv = f2::degree(v);
    if (dv < 0) return {};
    while (dv > 0 && du > 0) {
        if (du < dv) {
            std::swap(u, v);
            std::swap(su, sv);
            std::swap(du, dv);
        }
        const uint64_t s = (uint64_t)(du - dv);
        xor_shl(u, v, dv, s);
        const int64_t dsv = f2::degree(sv);
        if (dsv >= 0) xor_shl(su, sv, dsv, s);
        du = degree_from(u, du);
    }
    Poly r;
    if (dv == 0) r = sv;
    else if (du == 0) r = su;
    else return {};
    const f2::Modulus M = f2::make_modulus(m);
    f2::reduce(r, M);
    f2::trim(r);
    return r;
}

Poly numerator(const Poly &P, const uint64_t *bits, uint64_t p)
{
    Poly rev((size_t)(p / 64u) + 1u, 0u);
    for (uint64_t i = 0; i < p; ++i)
        if ((bits[i >> 6] >> (i & 63u)) & 1u) {
            const uint64_t j = p - 1u - i;
            rev[j >> 6] |= 1ull << (j & 63u);
        }
    const Poly prod = f2::mul(P, rev);
    Poly h((size_t)(p / 64u) + 1u, 0u);
    for (uint64_t j = 0; j < p; ++j) {
        const uint64_t k = p + j;
        if ((k >> 6) < prod.size() && ((prod[k >> 6] >> (k & 63u)) & 1u)) h[j >> 6] |= 1ull << (j & 63u);
    }
    f2::trim(h);
    return h;
}

bool KvLattice::start(const Poly &P, const Poly &h1)
{
    P_ = P;
    f2::trim(P_);
    h1inv_ = invmod(h1, P_);
    if (h1inv_.empty()) return false;
    mod_ = f2::make_modulus(P_);
    basis_.clear();
    bypiv_.assign(1, -1);
    dim_ = 1;
    Vec w;
    w.c.assign(1, P_);
    w.cd.assign(1, f2::degree(P_));
    refresh(w);
    insert(std::move(w));
    return true;
}

void KvLattice::refresh(Vec &w) const
{
    w.deg = -1;
    w.piv = -1;
    for (size_t b = 0; b < w.cd.size(); ++b)
        if (w.cd[b] >= 0 && w.cd[b] >= w.deg) {
            w.deg = w.cd[b];
            w.piv = (int)b;
        }
}

void KvLattice::add_shifted(Vec &w, const Vec &u, uint64_t s) const
{
    for (size_t b = 0; b < u.c.size(); ++b) {
        if (u.cd[b] < 0) continue;
        xor_shl(w.c[b], u.c[b], u.cd[b], s);
        w.cd[b] = degree_from(w.c[b], std::max<int64_t>(w.cd[b], u.cd[b] + (int64_t)s));
    }
    refresh(w);
}

// Adds w to the basis keeping the pivots distinct (Mulders-Storjohann): on a
// clash, the vector of higher degree is reduced by a shifted copy of the
// other, which lowers its degree or moves its pivot left.
void KvLattice::insert(Vec w)
{
    for (;;) {
        if (w.deg < 0) return;
        const int idx = bypiv_[(size_t)w.piv];
        if (idx < 0) {
            bypiv_[(size_t)w.piv] = (int)basis_.size();
            basis_.push_back(std::move(w));
            return;
        }
        Vec &u = basis_[(size_t)idx];
        if (u.deg > w.deg) std::swap(u, w);
        add_shifted(w, u, (uint64_t)(w.deg - u.deg));
    }
}

uint32_t KvLattice::add(const Poly &h)
{
    for (Vec &u : basis_) {                  // the new coordinate is zero in the old vectors
        u.c.emplace_back();
        u.cd.push_back(-1);
    }
    bypiv_.push_back(-1);
    Vec w;
    w.c.assign(dim_ + 1u, Poly());
    w.cd.assign(dim_ + 1u, -1);
    w.c[0] = f2::mulmod(h, h1inv_, mod_);    // c = h / h1 mod P
    f2::trim(w.c[0]);
    w.cd[0] = f2::degree(w.c[0]);
    w.c[dim_] = Poly{1u};
    w.cd[dim_] = 0;
    ++dim_;
    refresh(w);
    insert(std::move(w));
    return kmin();
}

uint32_t KvLattice::kmin() const
{
    int64_t m = -1;
    for (const Vec &u : basis_)
        if (m < 0 || u.deg < m) m = u.deg;
    return (uint32_t)std::max<int64_t>(m, 0);
}

}  // namespace eq
}  // namespace mtgp

// ---------------------------------------------------------------------------
// k(v) of parameter sets, and the Sec. 5 tempering search
// ---------------------------------------------------------------------------
#include "mtgp_internal.h"

#include <atomic>
#include <cstdio>
#include <cstring>
#include <exception>
#include <string>
#include <thread>

namespace mtgp {
namespace {

constexpr uint64_t kGammaE = 0x9E3779B97F4A7C15ull;

uint64_t mix64e(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The recursion's words x_0 .. x_{N+L-1} (Sec. 3.6) from a SplitMix64-filled
// nonzero state.
void raw_sequence(const mtgp_params &p, uint64_t L, std::vector<uint32_t> &x)
{
    const uint32_t N = p.N, M = p.pos;
    x.assign((size_t)N + (size_t)L, 0u);
    const uint64_t s0 = 0x5EEDull ^ mix64e(kGammaE);
    uint32_t any = 0;
    for (uint32_t j = 0; j < N; ++j) {
        x[j] = (uint32_t)mix64e(s0 + (uint64_t)(j + 1u) * kGammaE);
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

// Tempering index (Sec. 3.7) of the word y.
uint32_t temper_index(uint32_t y)
{
    uint32_t z = y ^ (y >> 16);
    z ^= z >> 8;
    return z & 15u;
}

// Tempered outputs o_0 .. o_{L-1} (Sec. 3.7) with the table tmp, as 32 bit
// planes of L bits each (plane b = bit b).
void output_planes(const mtgp_params &p, const uint32_t tmp[16], const std::vector<uint32_t> &x, uint64_t L,
                   std::vector<std::vector<uint64_t>> &planes)
{
    const uint32_t N = p.N, M = p.pos;
    planes.assign(32, std::vector<uint64_t>((size_t)(L / 64u) + 2u, 0u));
    for (uint64_t i = 0; i < L; ++i) {
        const uint32_t o = x[N + i] ^ tmp[temper_index(x[M - 1u + i])];
        for (uint32_t b = 0; b < 32u; ++b)
            planes[b][i >> 6] |= (uint64_t)((o >> b) & 1u) << (i & 63u);
    }
}

// k(v) by row echelon over the basis F^j s (j < p): row (i, b) = bits
// i .. i+p-1 of plane b; rows are added output by output, bit order
// `bits[0 .. v)`, until the first dependent one.  The basis is kept by lowest
// set bit, so a reduction only touches words at and above it.  Used where
// the lattice method does not apply (characteristic polynomial of degree
// below p, as for sets that are not of full period).
uint32_t kv_rowechelon(const std::vector<std::vector<uint64_t>> &planes, uint32_t p, const uint32_t *bits, uint32_t v)
{
    const size_t W = (p + 63u) / 64u;
    std::vector<uint64_t> basis((size_t)p * W), row(W + 1u);
    std::vector<int32_t> piv(p, -1);
    uint32_t rank = 0, k = 0;
    const uint32_t kmax = p / v + 1u;
    for (uint32_t i = 0; i < kmax; ++i) {
        for (uint32_t t = 0; t < v; ++t) {
            const std::vector<uint64_t> &pl = planes[bits[t]];
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

unsigned thread_count(uint32_t threads)
{
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    return std::min<unsigned>(64u, threads ? threads : hw);
}

// Tempering rows from a linear table (Sec. 3.7 convention: bit 3 of the
// index selects row 0), and back.
void table_rows(const uint32_t tbl[16], uint32_t rows[4])
{
    for (uint32_t r = 0; r < 4u; ++r) rows[r] = tbl[1u << (3u - r)];
}

void rows_table(const uint32_t rows[4], uint32_t tbl[16])
{
    for (uint32_t b = 0; b < 16u; ++b) {
        uint32_t v = 0;
        for (uint32_t r = 0; r < 4u; ++r)
            if ((b >> (3u - r)) & 1u) v ^= rows[r];
        tbl[b] = v;
    }
}

// Everything about a parameter set's recursion that the output bit planes
// need: its characteristic polynomial, the bit planes of the recursion's
// words x_{N+i} (i < p) and the row selectors of the tempering words.
struct Setup {
    uint32_t p = 0;
    f2::Poly P;
    size_t W = 0;                                        // words per plane
    std::vector<std::vector<uint64_t>> X;                // X[b]: bit b of x_{N+i}
    std::vector<std::vector<uint64_t>> J;                // J[r]: row r selected for o_i
};

// False when the lattice method does not apply (the MSB sequence's
// polynomial has degree below p: not a full-period set).
bool make_setup(const mtgp_params &p, Setup &S)
{
    const uint32_t P = p.mexp, N = p.N, M = p.pos;
    std::vector<uint32_t> x;
    raw_sequence(p, 2ull * P + 64u, x);
    std::vector<uint64_t> msb((size_t)(2u * P) / 64u + 1u, 0u);
    for (uint64_t i = 0; i < 2ull * P; ++i) msb[i >> 6] |= (uint64_t)(x[N + i] >> 31) << (i & 63u);
    S.P = f2::minpoly(msb.data(), 2ull * P);
    f2::trim(S.P);
    if (f2::degree(S.P) != (int64_t)P) return false;
    S.p = P;
    S.W = (size_t)P / 64u + 1u;
    S.X.assign(32, std::vector<uint64_t>(S.W, 0u));
    S.J.assign(4, std::vector<uint64_t>(S.W, 0u));
    for (uint32_t i = 0; i < P; ++i) {
        const uint32_t y = x[N + i], idx = temper_index(x[M - 1u + i]);
        const uint64_t bit = 1ull << (i & 63u);
        for (uint32_t b = 0; b < 32u; ++b)
            if ((y >> b) & 1u) S.X[b][i >> 6] |= bit;
        for (uint32_t r = 0; r < 4u; ++r)
            if ((idx >> (3u - r)) & 1u) S.J[r][i >> 6] |= bit;
    }
    return true;
}

// Numerator h of bit b of the outputs o_i = x_{N+i} ^ (rows selected by the
// tempering index of x_{M-1+i}).
f2::Poly plane_numerator(const Setup &S, const uint32_t rows[4], uint32_t b)
{
    std::vector<uint64_t> a = S.X[b];
    for (uint32_t r = 0; r < 4u; ++r)
        if ((rows[r] >> b) & 1u)
            for (size_t w = 0; w < S.W; ++w) a[w] ^= S.J[r][w];
    return eq::numerator(S.P, a.data(), S.p);
}

// k(1 .. nb) for the bits `bits` (in order) of the outputs with tempering
// rows `rows`, by lattice reduction; false if the first plane's numerator is
// not invertible.
bool lattice_kv(const Setup &S, const uint32_t rows[4], const uint32_t *bits, uint32_t nb, uint32_t *kv)
{
    eq::KvLattice L;
    if (!L.start(S.P, plane_numerator(S, rows, bits[0]))) return false;
    kv[0] = L.kmin();
    for (uint32_t v = 1; v < nb; ++v) kv[v] = L.add(plane_numerator(S, rows, bits[v]));
    return true;
}

void msb_bits(uint32_t *bits)
{
    for (uint32_t v = 0; v < 32u; ++v) bits[v] = 31u - v;
}

void lsb_bits(uint32_t *bits)
{
    for (uint32_t v = 0; v < 32u; ++v) bits[v] = v;
}

// k(v), v = 1 .. 32, of the bits `bits` of the outputs with table tbl: the
// lattice method for full-period sets, else row echelon (threads over v).
bool kv_all(const mtgp_params &p, const uint32_t tbl[16], const uint32_t *bits, unsigned nt, uint32_t kv[32])
{
    Setup S;
    uint32_t rows[4];
    table_rows(tbl, rows);
    if (make_setup(p, S) && lattice_kv(S, rows, bits, 32u, kv)) return true;
    std::vector<uint32_t> x;
    raw_sequence(p, 2ull * p.mexp + 64u, x);
    std::vector<std::vector<uint64_t>> planes;
    output_planes(p, tbl, x, 2ull * p.mexp + 64u, planes);
    std::atomic<uint32_t> next{1};
    std::atomic<bool> oom{false};
    auto worker = [&] {
        try {
            for (uint32_t v; (v = next.fetch_add(1)) <= 32u;) kv[v - 1u] = kv_rowechelon(planes, p.mexp, bits, v);
        } catch (const std::exception &) {
            oom = true;
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (auto &th : pool) th.join();
    return !oom;
}

uint32_t defect_sum(uint32_t p, const uint32_t *kv, uint32_t v0, uint32_t v1)   // v0 .. v1-1, 1-based v
{
    uint32_t d = 0;
    for (uint32_t v = v0; v < v1; ++v) d += p / v - kv[v - 1u];
    return d;
}

}  // namespace
}  // namespace mtgp

namespace mtgp {
namespace {

// The pattern q in [0, 2^w) of bits shift .. shift+w-1 of tempering row i
// with the least sum of dimension defects d(j+1) + .. + d(e) of the bits
// bits[0 .. e) (d(1) .. d(j) do not depend on q: those output bits do not
// see the window), the smallest q on ties (Sec. 5).  The lattice of the
// first j bits is reduced once and extended per pattern.
bool best_pattern(const Setup &S, uint32_t rows[4], uint32_t i, uint32_t shift, uint32_t w, const uint32_t *bits,
                  uint32_t j, uint32_t e, unsigned nt)
{
    eq::KvLattice base;
    if (j > 0) {
        if (!base.start(S.P, plane_numerator(S, rows, bits[0]))) return false;
        for (uint32_t v = 1; v < j; ++v) base.add(plane_numerator(S, rows, bits[v]));
    }
    const uint32_t npat = 1u << w, wmask = (npat - 1u) << shift;
    std::vector<uint64_t> score(npat, ~0ull);
    std::atomic<uint32_t> next{0};
    std::atomic<bool> oom{false};
    auto worker = [&] {
        try {
            for (uint32_t q; (q = next.fetch_add(1)) < npat;) {
                uint32_t r[4] = {rows[0], rows[1], rows[2], rows[3]};
                r[i] = (r[i] & ~wmask) | (q << shift);
                eq::KvLattice L;
                uint32_t v = j;
                if (j > 0) {
                    L = base;
                } else {
                    if (!L.start(S.P, plane_numerator(S, r, bits[0]))) continue;
                    v = 1;
                    if (e == 1) {
                        score[q] = S.p - L.kmin();
                        continue;
                    }
                }
                uint64_t d = 0;
                if (j == 0) d += S.p - L.kmin();                 // d(1)
                for (; v < e; ++v) {
                    const uint32_t k = L.add(plane_numerator(S, r, bits[v]));
                    d += S.p / (v + 1u) - k;
                }
                score[q] = d;
            }
        } catch (const std::exception &) {
            oom = true;
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < std::min<unsigned>(nt, npat); ++t) pool.emplace_back(worker);
    for (auto &th : pool) th.join();
    if (oom) throw std::bad_alloc();
    uint32_t best = 0;
    for (uint32_t q = 1; q < npat; ++q)
        if (score[q] < score[best]) best = q;
    if (score[best] == ~0ull) return false;
    rows[i] = (rows[i] & ~wmask) | (best << shift);
    return true;
}

// SHA-1 (FIPS 180-4) of a byte string, as 40 lowercase hexadecimal digits.
void sha1_hex(const std::string &msg, char out[41])
{
    uint32_t h[5] = {0x67452301u, 0xEFCDAB89u, 0x98BADCFEu, 0x10325476u, 0xC3D2E1F0u};
    std::string m = msg;
    const uint64_t bitlen = (uint64_t)msg.size() * 8u;
    m.push_back((char)0x80);
    while (m.size() % 64u != 56u) m.push_back('\0');
    for (int k = 7; k >= 0; --k) m.push_back((char)((bitlen >> (8 * k)) & 0xFFu));
    auto rotl = [](uint32_t x, unsigned n) { return (x << n) | (x >> (32u - n)); };
    for (size_t blk = 0; blk < m.size(); blk += 64u) {
        uint32_t w[80];
        for (unsigned t = 0; t < 16u; ++t) {
            const unsigned char *c = (const unsigned char *)m.data() + blk + 4u * t;
            w[t] = ((uint32_t)c[0] << 24) | ((uint32_t)c[1] << 16) | ((uint32_t)c[2] << 8) | (uint32_t)c[3];
        }
        for (unsigned t = 16; t < 80u; ++t) w[t] = rotl(w[t - 3] ^ w[t - 8] ^ w[t - 14] ^ w[t - 16], 1);
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4];
        for (unsigned t = 0; t < 80u; ++t) {
            uint32_t f, k;
            if (t < 20u) {
                f = (b & c) | (~b & d);
                k = 0x5A827999u;
            } else if (t < 40u) {
                f = b ^ c ^ d;
                k = 0x6ED9EBA1u;
            } else if (t < 60u) {
                f = (b & c) | (b & d) | (c & d);
                k = 0x8F1BBCDCu;
            } else {
                f = b ^ c ^ d;
                k = 0xCA62C1D6u;
            }
            const uint32_t tmp = rotl(a, 5) + f + e + k + w[t];
            e = d;
            d = c;
            c = rotl(b, 30);
            b = a;
            a = tmp;
        }
        h[0] += a;
        h[1] += b;
        h[2] += c;
        h[3] += d;
        h[4] += e;
    }
    for (unsigned k = 0; k < 5u; ++k) snprintf(out + 8u * k, 9, "%08x", h[k]);
}

mtgp_status fail_eq(mtgp_status st, const char *msg) { return (mtgp_status)report_error(st, msg); }

}  // namespace
}  // namespace mtgp

extern "C" mtgp_status mtgp_params_equidistribution(const mtgp_params *p, uint32_t threads, uint32_t *kv,
                                                    uint32_t *delta)
{
    using namespace mtgp;
    if (!p || !kv) return fail_eq(MTGP_EINVAL, "equidistribution: NULL argument");
    mtgp_status st = mtgp_params_validate(p);
    if (st != MTGP_OK) return st;
    try {
        uint32_t bits[32], k[32];
        msb_bits(bits);
        if (!kv_all(*p, p->tmp_tbl, bits, thread_count(threads), k))
            return fail_eq(MTGP_ENOMEM, "equidistribution: host allocation failed");
        std::copy(k, k + 32, kv);
        if (delta) *delta = defect_sum(p->mexp, k, 1u, 33u);
        return MTGP_OK;
    } catch (const std::exception &) {
        return fail_eq(MTGP_ENOMEM, "equidistribution: host allocation or thread start failed");
    }
}

extern "C" mtgp_status mtgp_params_equidistribution_lsb(const mtgp_params *p, uint32_t threads, uint32_t *kv,
                                                        uint32_t *delta)
{
    using namespace mtgp;
    if (!p || !kv) return fail_eq(MTGP_EINVAL, "equidistribution: NULL argument");
    mtgp_status st = mtgp_params_validate(p);
    if (st != MTGP_OK) return st;
    try {
        uint32_t bits[32], k[32];
        lsb_bits(bits);
        if (!kv_all(*p, p->tmp_tbl, bits, thread_count(threads), k))
            return fail_eq(MTGP_ENOMEM, "equidistribution: host allocation failed");
        std::copy(k, k + 32, kv);
        if (delta) *delta = defect_sum(p->mexp, k, 1u, 33u);
        return MTGP_OK;
    } catch (const std::exception &) {
        return fail_eq(MTGP_ENOMEM, "equidistribution: host allocation or thread start failed");
    }
}

// The tempering search of Sec. 5, in the paper's order: all four rows from
// zero; for each row, the 23 MSBs in windows of 5 bits from the top (the
// last window 3 bits), each window set to the pattern with the least
// d(1) + .. + d(e) over the MSBs; then, for each row, the 9 LSBs in windows
// of 5 and 4 bits from the bottom, against the defects d'(1) + .. + d'(e) of
// the v least significant bits.
extern "C" mtgp_status mtgp_params_temper_search(const mtgp_params *in, uint32_t threads, mtgp_params *out,
                                                 uint32_t *delta)
{
    using namespace mtgp;
    if (!in || !out) return fail_eq(MTGP_EINVAL, "temper search: NULL argument");
    mtgp_status st = mtgp_params_validate(in);
    if (st != MTGP_OK) return st;
    try {
        Setup S;
        if (!make_setup(*in, S))
            return fail_eq(MTGP_EINVAL, "temper search: the recursion is not of full period (characteristic "
                                        "polynomial of degree below mexp)");
        const unsigned nt = thread_count(threads);
        uint32_t rows[4] = {0u, 0u, 0u, 0u}, bits[32];
        msb_bits(bits);
        for (uint32_t i = 0; i < 4u; ++i)
            for (uint32_t j = 0; j < 23u; j += 5u) {             // MSB positions j .. e-1
                const uint32_t e = std::min(j + 5u, 23u);
                if (!best_pattern(S, rows, i, 32u - e, e - j, bits, j, e, nt))
                    return fail_eq(MTGP_EINVAL, "temper search: a characteristic polynomial factor blocks the "
                                                "lattice method");
            }
        lsb_bits(bits);
        for (uint32_t i = 0; i < 4u; ++i)
            for (uint32_t j = 0; j < 9u; j += 5u) {              // LSB positions j .. e-1
                const uint32_t e = std::min(j + 5u, 9u);
                if (!best_pattern(S, rows, i, j, e - j, bits, j, e, nt))
                    return fail_eq(MTGP_EINVAL, "temper search: a characteristic polynomial factor blocks the "
                                                "lattice method");
            }
        mtgp_params r = *in;
        rows_table(rows, r.tmp_tbl);
        uint32_t k[32];
        msb_bits(bits);
        if (!lattice_kv(S, rows, bits, 32u, k)) return fail_eq(MTGP_EINVAL, "temper search: lattice failed");
        *out = r;
        if (delta) *delta = defect_sum(in->mexp, k, 1u, 33u);
        return MTGP_OK;
    } catch (const std::exception &) {
        return fail_eq(MTGP_ENOMEM, "temper search: host allocation or thread start failed");
    }
}

extern "C" mtgp_status mtgp_params_report(const mtgp_params *p, uint32_t threads, char *buf, size_t len)
{
    using namespace mtgp;
    if (!p || !buf || !len) return fail_eq(MTGP_EINVAL, "report: NULL argument");
    uint32_t k[32], total = 0;
    mtgp_status st = mtgp_params_equidistribution(p, threads, k, &total);
    if (st != MTGP_OK) return st;
    std::string s = "   v     k(v)   d(v)   r(v)%\n";
    char line[96];
    for (uint32_t v = 1; v <= 32u; ++v) {
        const uint32_t d = p->mexp / v - k[v - 1u];
        snprintf(line, sizeof line, "%4u %8u %6u %7.2f\n", v, k[v - 1u], d,
                 100.0 * (double)d / (double)(k[v - 1u] + d));
        s += line;
    }
    snprintf(line, sizeof line, "total dimension defect %u", total);
    s += line;
    if (s.size() + 1u > len) return fail_eq(MTGP_EINVAL, "report: buffer too small");
    std::memcpy(buf, s.c_str(), s.size() + 1u);
    return MTGP_OK;
}

extern "C" mtgp_status mtgp_params_record(const mtgp_params *p, const uint64_t *charpoly, uint32_t charpoly_words,
                                          uint32_t threads, char *buf, size_t len)
{
    using namespace mtgp;
    if (!p || !charpoly || !buf || !len) return fail_eq(MTGP_EINVAL, "record: NULL argument");
    if (charpoly_words < p->mexp / 64u + 1u) return fail_eq(MTGP_EINVAL, "record: charpoly needs mexp / 64 + 1 words");
    try {
        uint32_t k[32], total = 0;
        mtgp_status st = mtgp_params_equidistribution(p, threads, k, &total);
        if (st != MTGP_OK) return st;
        std::string coef;
        uint32_t terms = 0;
        for (uint32_t i = 0; i <= p->mexp; ++i) {
            const bool c = (charpoly[i >> 6] >> (i & 63u)) & 1u;
            coef.push_back(c ? '1' : '0');
            terms += c;
        }
        char sha[41];
        sha1_hex(coef, sha);
        std::string s;
        char f[32];
        const uint32_t head[6] = {p->mexp, p->N, p->pos, p->sh1, p->sh2, p->id};
        for (uint32_t v : head) {
            snprintf(f, sizeof f, "%u,", v);
            s += f;
        }
        for (uint32_t v : p->rec_tbl) {
            snprintf(f, sizeof f, "%08x,", v);
            s += f;
        }
        for (uint32_t v : p->tmp_tbl) {
            snprintf(f, sizeof f, "%08x,", v);
            s += f;
        }
        s += sha;
        snprintf(f, sizeof f, ",%u,%u", terms, total);
        s += f;
        if (s.size() + 1u > len) return fail_eq(MTGP_EINVAL, "record: buffer too small");
        std::memcpy(buf, s.c_str(), s.size() + 1u);
        return MTGP_OK;
    } catch (const std::exception &) {
        return fail_eq(MTGP_ENOMEM, "record: host allocation failed");
    }
}
