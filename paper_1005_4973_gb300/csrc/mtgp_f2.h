// Polynomials over F2 for jumping ahead (Sec. 7): a state s of the linear
// transition F (Sec. 3.3) satisfies psi(F) s = 0 for its annihilating
// polynomial psi, so F^J s = g(F) s with g = x^J mod psi, and g(F) s is the
// XOR of the states s, F s, F^2 s, ... picked by g's coefficients.
//
// A polynomial is a little-endian vector of 64-bit words: bit i of word i/64
// is the coefficient of x^i.  Host code only; portable C++ (no intrinsics).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace mtgp {
namespace f2 {

using Poly = std::vector<uint64_t>;

int64_t degree(const Poly &a);            // -1 for the zero polynomial
void trim(Poly &a);                       // drops zero top words

// Minimal polynomial of the bit sequence s_0 .. s_{n-1} (bit i of bits[i/64])
// by Berlekamp-Massey, in annihilator form: psi(x) = sum psi_j x^j with
// sum_j psi_j s_{k+j} = 0 for every k.  Exact when the sequence's linear
// complexity is at most n/2.
Poly minpoly(const uint64_t *bits, uint64_t n);

Poly mul(const Poly &a, const Poly &b);   // plain product

// Reduction modulo a fixed polynomial m of degree D >= 1 (8-bit comb tables).
struct Modulus {
    Poly m;
    uint64_t D = 0;
    size_t np = 0;                        // words per table row
    std::vector<uint64_t> P;              // P[c] = c(x) * m(x), c < 256
    uint8_t inv[256] = {};                // top byte of P[c] -> c
    // P[c] shifted left by 8 j bits (j = 0 .. 7), np + 1 words per row, so
    // that every reduction step XORs whole words
    std::vector<uint64_t> P8;
};
Modulus make_modulus(const Poly &m);
void reduce(Poly &a, const Modulus &M);
Poly mulmod(const Poly &a, const Poly &b, const Modulus &M);
Poly sqrmod(const Poly &a, const Modulus &M);
Poly mulx_mod(Poly a, const Modulus &M);  // x * a mod m
Poly xpow_mod(uint64_t e, const Modulus &M);
Poly gcd(Poly a, Poly b);                 // monic greatest common divisor

}  // namespace f2
}  // namespace mtgp
