"""The MTGPDC recursion search (Sec. 5) with its polynomial work on the GPU
(Berlekamp-Massey, one warp per candidate; irreducibility, one block per
candidate) against the host search and the oracle's search: the same first
accepted candidate, and a characteristic polynomial equal to the oracle's
Berlekamp-Massey polynomial of the set's MSB sequence.  The GPU
irreducibility test alone against the oracle's plain test (x^(2^p) = x mod
phi, no sieve) on irreducible trinomials, searched characteristic
polynomials, random polynomials and products with factors of every small
degree."""
import time

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_1005_4973_gb300 import build
    build.build()
    O.build()
    assert torch.cuda.is_available()
    import paper_1005_4973_gb300 as M
    return M


@pytest.mark.parametrize("mexp,s0,gid", [(89, 1000, 7), (107, 5, 1), (127, 3, 2), (521, 1000, 7), (607, 31, 12),
                                         (1279, 9, 1)])
def test_gpu_search_equals_host_and_oracle(M, mexp, s0, gid):
    pg, sg, tg, phig = M.mtgp_params_search_gpu(mexp, s0, gid)
    ph, sh, th, phih = M.mtgp_params_search(mexp, s0, gid)
    op, so, _ = O.search_full_period(mexp, s0, gid, max_tries=200000)
    assert sg == sh == so and tg == th
    assert np.array_equal(phig, phih)
    # the oracle's Berlekamp-Massey polynomial of its own MSB sequence of the set
    out = O.generate(op, O.seed_state(op, 4, 9), 2 * mexp + 64, 0)
    assert np.array_equal(O.bm(((out >> 31) & 1).astype(np.uint8)), phig)
    assert O.irreducible_prime_degree(phig)


def test_gpu_search_limits(M):
    with pytest.raises(M.MTGPError):
        M.mtgp_params_search_gpu(1279, 9, 1, max_tries=3)   # the first accepted candidate is number 1184


def test_gpu_search_mtgp11213_timed(M):
    """A full-size MTGP11213 search: the same set as the host search, and
    faster; both times are printed (pytest -s)."""
    t0 = time.perf_counter()
    pg, sg, tg, phig = M.mtgp_params_search_gpu(11213, 1, 0)
    tgpu = time.perf_counter() - t0
    t0 = time.perf_counter()
    ph, sh, th, phih = M.mtgp_params_search(11213, 1, 0)
    thost = time.perf_counter() - t0
    print(f"MTGP11213 search: GPU {tgpu:.2f} s, host {thost:.2f} s, {tg} candidates")
    assert sg == sh and np.array_equal(phig, phih) and phig.size - 1 == 11213
    assert tgpu < thost


# irreducible trinomials x^p + x^k + 1 of Mersenne exponents p
TRINOMIALS = {89: 38, 127: 1, 521: 32, 607: 105, 1279: 216}


def _poly(p, rng, odd_weight=True):
    c = rng.integers(0, 2, size=p + 1).astype(np.uint8)
    c[0] = c[p] = 1
    if odd_weight and c.sum() % 2 == 0:
        c[1 + int(rng.integers(0, p - 1))] ^= 1
    return c


@pytest.mark.parametrize("p", [37, 89, 107, 127, 521, 607, 1279])
def test_gpu_irreducibility_equals_the_oracle(M, p):
    rng = np.random.default_rng(p)
    polys = []
    if p in TRINOMIALS:
        c = np.zeros(p + 1, dtype=np.uint8)
        c[0] = c[TRINOMIALS[p]] = c[p] = 1
        polys.append(c)
    if p >= 89:
        polys.append(M.mtgp_params_search(p, 1000, 7)[3])      # a searched characteristic polynomial
    known = len(polys)                                        # the polynomials above are irreducible
    nrand = 160 if p <= 127 else 24
    polys += [_poly(p, rng) for _ in range(nrand)]
    # products with a factor of each degree 2 .. 45 (the sieve finds those of degree <= 40)
    for d in [d for d in (range(2, 46) if p <= 607 else (2, 17, 40, 41, 45)) if d < p - 1]:
        f, g = _poly(d, rng, False), _poly(p - d, rng, False)
        polys.append((np.convolve(f, g) % 2).astype(np.uint8))
    # degree below p, even weight, no constant term
    low = _poly(p, rng)
    low[p] = 0
    polys.append(low)
    even = _poly(p, rng)
    even[1 + int(np.nonzero(even[1:p])[0][0])] ^= 1
    polys.append(even)
    noc = _poly(p, rng)
    noc[0] = 0
    polys.append(noc)
    got = M.mtgp_f2_irreducible_gpu(polys, p)
    ref = np.array([O.irreducible_prime_degree(c) if c[p] else False for c in polys])
    assert np.array_equal(got, ref), np.nonzero(got != ref)[0]
    assert got[:known].all()
    assert not got[-3:].any()


def test_gpu_irreducibility_rejects_bad_arguments(M):
    c = np.zeros(90, dtype=np.uint8)
    c[0] = c[89] = 1
    with pytest.raises(M.MTGPError):
        M.mtgp_f2_irreducible_gpu([c], 91)                 # not prime
    with pytest.raises(M.MTGPError):
        M.mtgp_f2_irreducible_gpu([c[:32]], 31)            # too small
    with pytest.raises(M.MTGPError):
        M.mtgp_f2_irreducible_gpu([], 89)                  # no polynomial


def test_gpu_irreducibility_of_products_beyond_one_block_pass(M):
    """p = 19937: the polynomial has more words than the block has threads,
    so every reduction window's update loops.  Products with a factor of
    degree 3, 29 and 43 are reducible; a polynomial of degree p + 1 is
    rejected."""
    p = 19937
    rng = np.random.default_rng(7)
    polys = []
    for d in (3, 29, 43):
        f, g = _poly(d, rng), _poly(p - d, rng)
        polys.append((np.convolve(f, g) % 2).astype(np.uint8))
    over = np.zeros(p + 2, dtype=np.uint8)
    over[0] = over[p + 1] = over[5] = 1
    polys.append(over)
    got = M.mtgp_f2_irreducible_gpu(polys, p)
    assert not got.any()
