// Dimensions of equidistribution k(v) of an F2-linear generator by lattice
// reduction over F2[t] (Sec. 3.4, 3.8; Sec. 5 computes them with a lattice
// method), and the tempering-parameter search of Sec. 5 built on it.
//
// For a full-period generator with characteristic polynomial P of degree p,
// the bit sequence a = (bit b of o_0, o_1, ...) has generating function
// sum_i a_i t^(-i-1) = h_b(t) / P(t) with deg h_b < p.  The v bits b_1 .. b_v
// of k consecutive outputs are equidistributed iff no nonzero (f_1 .. f_v)
// with deg f_j < k has sum_j f_j h_{b_j} = 0 mod P.  These f form an F2[t]
// lattice of rank v, so k(v) is the least max-degree of its nonzero vectors:
// the smallest degree of a basis in weak Popov form.  With c_j = h_{b_j} /
// h_{b_1} mod P the lattice has the basis (P, 0, .., 0), (c_j, 0, .., 1 at
// j, .., 0), j = 2 .. v, so adding bit v+1 adds one vector to a reduced basis
// of the first v bits.  Host code only.
#pragma once

#include <cstdint>
#include <vector>

#include "mtgp.h"
#include "mtgp_f2.h"

namespace mtgp {
namespace eq {

using f2::Poly;

// Inverse of a modulo m over F2 (extended Euclid); empty if gcd(a, m) != 1.
Poly invmod(const Poly &a, const Poly &m);

// Weak-Popov reduced basis of the lattice of the bits added so far.
class KvLattice {
public:
    // P: characteristic polynomial (degree p).  First bit plane: h1 must be
    // invertible mod P (P irreducible and h1 != 0).
    bool start(const Poly &P, const Poly &h1);
    // Adds the next bit with numerator h; returns k for the bits so far.
    uint32_t add(const Poly &h);
    uint32_t dim() const { return dim_; }
    uint32_t kmin() const;

private:
    struct Vec {
        std::vector<Poly> c;            // components, one per bit
        std::vector<int64_t> cd;        // their degrees (-1: zero)
        int64_t deg = -1;
        int piv = -1;                   // rightmost component of degree deg
    };
    void refresh(Vec &w) const;
    void add_shifted(Vec &w, const Vec &u, uint64_t s) const;
    void insert(Vec w);

    Poly P_, h1inv_;
    f2::Modulus mod_;
    std::vector<Vec> basis_;
    std::vector<int> bypiv_;           // pivot -> basis index
    uint32_t dim_ = 0;
};

// Numerator h of the generating function of the bit sequence a_0 .. a_{p-1}
// (bit i of bits[i / 64]) of a sequence with characteristic polynomial P of
// degree p: h = (P * rev_p(a)) >> p.
Poly numerator(const Poly &P, const uint64_t *bits, uint64_t p);

}  // namespace eq
}  // namespace mtgp
