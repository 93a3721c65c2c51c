// F2[x] arithmetic for jump-ahead (Sec. 7).  See mtgp_f2.h.
#include "mtgp_f2.h"

#include <algorithm>

namespace mtgp {
namespace f2 {

namespace {

inline unsigned clz64(uint64_t v) { return (unsigned)__builtin_clzll(v); }
inline unsigned parity64(uint64_t v) { return (unsigned)__builtin_parityll(v); }

// a[...] ^= b[0 .. nb) << s (bits); a must hold word (s / 64) + nb.
void xor_shifted(uint64_t *a, const uint64_t *b, size_t nb, uint64_t s)
{
    uint64_t *d = a + (s >> 6);
    const unsigned sh = (unsigned)(s & 63u);
    if (!sh) {
        for (size_t k = 0; k < nb; ++k) d[k] ^= b[k];
        return;
    }
    uint64_t carry = 0;
    for (size_t k = 0; k < nb; ++k) {
        d[k] ^= (b[k] << sh) | carry;
        carry = b[k] >> (64u - sh);
    }
    d[nb] ^= carry;
}

// Spreads the 32 bits of v to the even bit positions of a 64-bit word
// (squaring over F2 doubles every exponent), by the usual mask-and-shift
// interleave.
inline uint64_t spread32(uint32_t v)
{
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

inline uint32_t byte_at(const Poly &a, uint64_t t)   // bits [t, t + 8)
{
    const size_t w = (size_t)(t >> 6);
    const unsigned sh = (unsigned)(t & 63u);
    uint64_t v = w < a.size() ? a[w] >> sh : 0u;
    if (sh > 56u && w + 1 < a.size()) v |= a[w + 1] << (64u - sh);
    return (uint32_t)(v & 0xFFu);
}

}  // namespace

int64_t degree(const Poly &a)
{
    for (size_t w = a.size(); w-- > 0;)
        if (a[w]) return (int64_t)(w * 64u + 63u - clz64(a[w]));
    return -1;
}

void trim(Poly &a)
{
    while (!a.empty() && !a.back()) a.pop_back();
}

// Berlekamp-Massey over F2.  C is the connection polynomial (C_0 = 1) with
// s_k = sum_{i=1..L} C_i s_{k-i}; B is C before the last length change, m the
// steps since then.  The discrepancy sum_{i=0..L} C_i s_{k-i} is a masked
// parity against the sequence stored reversed (bit j = s_{n-1-j}), so the
// window for step k starts at bit n-1-k and runs upward.
Poly minpoly(const uint64_t *bits, uint64_t n)
{
    const size_t W = (size_t)(n >> 6) + 3u;
    std::vector<uint64_t> rev(W + 1u, 0u), C(W, 0u), B(W, 0u), T(W, 0u);
    for (uint64_t j = 0; j < n; ++j) {
        const uint64_t i = n - 1u - j;
        if ((bits[i >> 6] >> (i & 63u)) & 1u) rev[j >> 6] |= 1ull << (j & 63u);
    }
    C[0] = B[0] = 1u;
    uint64_t L = 0, Lb = 0, m = 1;
    for (uint64_t k = 0; k < n; ++k) {
        const uint64_t o = n - 1u - k;
        const size_t q = (size_t)(o >> 6), cw = (size_t)(L >> 6) + 1u;
        const unsigned sh = (unsigned)(o & 63u);
        uint64_t acc = 0;
        if (sh) {
            for (size_t w = 0; w < cw; ++w) acc ^= C[w] & ((rev[q + w] >> sh) | (rev[q + w + 1u] << (64u - sh)));
        } else {
            for (size_t w = 0; w < cw; ++w) acc ^= C[w] & rev[q + w];
        }
        if (!parity64(acc)) {
            ++m;
            continue;
        }
        const size_t bw = (size_t)(Lb >> 6) + 1u;
        if (2u * L <= k) {
            const size_t nw = std::max(cw, bw);
            std::copy(C.begin(), C.begin() + (ptrdiff_t)nw, T.begin());
            xor_shifted(C.data(), B.data(), bw, m);
            std::copy(T.begin(), T.begin() + (ptrdiff_t)nw, B.begin());
            Lb = L;
            L = k + 1u - L;
            m = 1;
        } else {
            xor_shifted(C.data(), B.data(), bw, m);
            ++m;
        }
    }
    Poly psi((size_t)(L >> 6) + 1u, 0u);
    for (uint64_t j = 0; j <= L; ++j) {
        const uint64_t i = L - j;
        if ((C[i >> 6] >> (i & 63u)) & 1u) psi[j >> 6] |= 1ull << (j & 63u);
    }
    trim(psi);
    return psi;
}

// Comb product: rows Q[c] = c(x) a(x) for every byte c, then one row XOR per
// byte of b, accumulated per bit offset (0, 8, .., 56) and shifted once.
Poly mul(const Poly &a0, const Poly &b0)
{
    Poly a = a0, b = b0;
    trim(a);
    trim(b);
    if (a.empty() || b.empty()) return {};
    const size_t nq = a.size() + 1u;
    std::vector<uint64_t> Q(256u * nq, 0u);
    for (unsigned t = 0; t < 8u; ++t) {
        uint64_t *row = &Q[(size_t)(1u << t) * nq];
        xor_shifted(row, a.data(), a.size(), t);
    }
    for (unsigned c = 3; c < 256u; ++c) {
        if (!(c & (c - 1u))) continue;
        const unsigned lo = c & (0u - c);
        const uint64_t *x = &Q[(size_t)(c ^ lo) * nq], *y = &Q[(size_t)lo * nq];
        uint64_t *d = &Q[(size_t)c * nq];
        for (size_t k = 0; k < nq; ++k) d[k] = x[k] ^ y[k];
    }
    const size_t nr = a.size() + b.size() + 1u;
    std::vector<uint64_t> acc(8u * nr, 0u);
    for (size_t w = 0; w < b.size(); ++w) {
        for (unsigned j = 0; j < 8u; ++j) {
            const unsigned c = (unsigned)((b[w] >> (8u * j)) & 0xFFu);
            if (!c) continue;
            uint64_t *r = &acc[j * nr + w];
            const uint64_t *q = &Q[(size_t)c * nq];
            for (size_t k = 0; k < nq; ++k) r[k] ^= q[k];
        }
    }
    Poly res(nr + 1u, 0u);
    for (unsigned j = 0; j < 8u; ++j) xor_shifted(res.data(), &acc[j * nr], nr - 1u, 8u * j);
    trim(res);
    return res;
}

Modulus make_modulus(const Poly &m0)
{
    Modulus M;
    M.m = m0;
    trim(M.m);
    const int64_t D = degree(M.m);
    M.D = D > 0 ? (uint64_t)D : 0u;
    if (D < 1) return M;
    M.np = (size_t)((M.D + 8u) >> 6) + 2u;
    M.P.assign(256u * M.np, 0u);
    for (unsigned t = 0; t < 8u; ++t) xor_shifted(&M.P[(size_t)(1u << t) * M.np], M.m.data(), M.m.size(), t);
    for (unsigned c = 3; c < 256u; ++c) {
        if (!(c & (c - 1u))) continue;
        const unsigned lo = c & (0u - c);
        const uint64_t *x = &M.P[(size_t)(c ^ lo) * M.np], *y = &M.P[(size_t)lo * M.np];
        uint64_t *d = &M.P[(size_t)c * M.np];
        for (size_t k = 0; k < M.np; ++k) d[k] = x[k] ^ y[k];
    }
    // c -> top byte of c(x) m(x) is triangular with a unit diagonal (m is
    // monic), hence a bijection on bytes
    for (unsigned c = 0; c < 256u; ++c) {
        const uint64_t *row = &M.P[(size_t)c * M.np];
        const uint64_t t = M.D;
        const size_t w = (size_t)(t >> 6);
        const unsigned sh = (unsigned)(t & 63u);
        uint64_t v = row[w] >> sh;
        if (sh > 56u) v |= row[w + 1u] << (64u - sh);
        M.inv[v & 0xFFu] = (uint8_t)c;
    }
    const size_t nr = M.np + 1u;
    M.P8.assign(8u * 256u * nr, 0u);
    for (unsigned j = 0; j < 8u; ++j)
        for (unsigned c = 1; c < 256u; ++c)
            xor_shifted(&M.P8[((size_t)j * 256u + c) * nr], &M.P[(size_t)c * M.np], M.np - 1u, 8u * j);
    return M;
}

// Clears the bits at and above D eight at a time, top down: for the byte c at
// [t, t+8), XOR in (c'(x) m(x)) x^(t-D) whose top byte is c.
void reduce(Poly &a, const Modulus &M)
{
    trim(a);
    if (M.D == 0u) {
        a.clear();
        return;
    }
    const int64_t da = degree(a);
    if (da < (int64_t)M.D) return;
    a.resize(std::max(a.size(), (size_t)(((uint64_t)da + 8u) >> 6) + M.np + 2u), 0u);
    const size_t nr = M.np + 1u;
    for (int64_t t = (int64_t)M.D + (da - (int64_t)M.D) / 8 * 8; t >= (int64_t)M.D; t -= 8) {
        const uint32_t c = byte_at(a, (uint64_t)t);
        if (!c) continue;
        const uint64_t sft = (uint64_t)t - M.D;               // a multiple of 8
        const uint64_t *row = &M.P8[((size_t)((sft >> 3) & 7u) * 256u + M.inv[c]) * nr];
        uint64_t *d = a.data() + (sft >> 6);
        for (size_t k = 0; k < nr; ++k) d[k] ^= row[k];
    }
    a.resize((size_t)((M.D + 63u) >> 6));
    trim(a);
}

Poly mulmod(const Poly &a, const Poly &b, const Modulus &M)
{
    Poly r = mul(a, b);
    reduce(r, M);
    return r;
}

Poly sqrmod(const Poly &a, const Modulus &M)
{
    Poly r(2u * a.size(), 0u);
    for (size_t w = 0; w < a.size(); ++w) {
        r[2u * w] = spread32((uint32_t)a[w]);
        r[2u * w + 1u] = spread32((uint32_t)(a[w] >> 32));
    }
    reduce(r, M);
    return r;
}

Poly mulx_mod(Poly a, const Modulus &M)
{
    trim(a);
    if (a.empty()) return a;
    a.push_back(0u);
    for (size_t w = a.size() - 1u; w > 0; --w) a[w] = (a[w] << 1) | (a[w - 1u] >> 63);
    a[0] <<= 1;
    reduce(a, M);
    return a;
}

// Euclid's algorithm, word-level: the remainder step XORs b shifted under
// a's leading term until deg a < deg b.
Poly gcd(Poly a, Poly b)
{
    trim(a);
    trim(b);
    while (!b.empty()) {
        int64_t da = degree(a);
        const int64_t db = degree(b);
        while (da >= db) {
            a.resize(std::max(a.size(), (size_t)((uint64_t)(da - db) / 64u) + b.size() + 1u), 0u);
            xor_shifted(a.data(), b.data(), b.size(), (uint64_t)(da - db));
            trim(a);
            da = degree(a);
            if (da < 0) break;
        }
        a.swap(b);
    }
    return a;
}

Poly xpow_mod(uint64_t e, const Modulus &M)
{
    if (M.D == 0u) return {};
    Poly r{1u};
    for (int b = 63; b >= 0; --b) {
        if (!r.empty() && !(r.size() == 1u && r[0] == 1u)) r = sqrmod(r, M);
        if ((e >> b) & 1u) r = mulx_mod(r, M);
    }
    return r;
}

}  // namespace f2
}  // namespace mtgp
