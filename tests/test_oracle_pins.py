"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each check comes from another
formulation (F2 bit-matrices built from the definitions), a closed form, an
invariant the definitions imply, or brute force on tiny inputs.  A plausible
slip in the oracle (a dropped term, a wrong shift, a transposed table
convention, a wrong tempering word) fails at least one of them.
"""
import hashlib
import itertools
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import f2

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(20240601)


def _sets():
    out = []
    for mexp in (11213, 23209, 44497):
        for seed in (1, 2, 77):
            out.append(O.params_draw(mexp, seed, seed * 1000003 & 0xFFFFFFFF))
    out.append(O.params_draw(11213, 5, 3, random_shifts=True))
    out.append(O.params_draw(23209, 9, 4, random_shifts=True))
    for mexp in (89, 107, 127, 521, 607, 1279):
        out.append(O.params_draw(mexp, 3, 1))
    return out


SETS = _sets()
IDS = [f"p{p.mexp}-M{p.pos}-s{p.sh1}.{p.sh2}" for p in SETS]


# ---------------------------------------------------------------- structure
@pytest.mark.parametrize("mexp,N,r,mask,lo,hi", [
    (11213, 351, 19, 0xFFF80000, 3, 94),     # N = ceil(p/32), r = 32N - p (Sec. 3.3)
    (23209, 726, 23, 0xFF800000, 3, 213),    # M range 2 < M < N - [N]_2 (Sec. 5)
    (44497, 1391, 15, 0xFFFF8000, 3, 366),
    (521, 17, 23, 0xFF800000, 2, 9),         # Sec. 3.5 rule where Sec. 5's is empty
    (607, 19, 1, 0xFFFFFFFE, 2, 3),
    (1279, 40, 1, 0xFFFFFFFE, 3, 7),
])
def test_derived_constants(mexp, N, r, mask, lo, hi):
    p = O.params_draw(mexp, 1, 0)
    assert (p.N, p.r, p.mask) == (N, r, mask)
    assert O.pos_range(N) == (lo, hi)
    ms = {O.params_draw(mexp, s, 0).pos for s in range(400)}
    assert min(ms) == lo and max(ms) == hi


def test_threads_rule_sec35():
    # Sec. 3.5: threads = [N-2]_2 give 256, 512, 1024 for the three exponents,
    # and every drawn M leaves N - M at least that many independent words.
    for mexp, threads in ((11213, 256), (23209, 512), (44497, 1024)):
        for s in range(50):
            p = O.params_draw(mexp, s, s)
            assert p.N - p.pos >= threads


def test_table_row_convention():
    # "(0001)R" is the row vector with only its last (rightmost = LSB) component
    # set, so rectbl[1] is the last row of R and rectbl[8] the first (Sec. 3.6).
    R = [0x80000001, 0x40000002, 0x20000004, 0x10000008]
    t = O.table_from_rows(R)
    assert t[0] == 0 and t[8] == R[0] and t[4] == R[1] and t[2] == R[2] and t[1] == R[3]
    assert t[15] == R[0] ^ R[1] ^ R[2] ^ R[3]


def test_tables_are_linear():
    for p in SETS:
        for tbl in (np.array(p.rectbl), np.array(p.tmptbl)):
            for a, b in itertools.product(range(16), repeat=2):
                assert tbl[a ^ b] == tbl[a] ^ tbl[b]


def test_sngltbl_sec6():
    # nine MSBs 001111111 then the leading tmptbl bits.
    for p in SETS:
        for b in range(16):
            assert p.sngltbl[b] >> 23 == 0b001111111
            assert p.sngltbl[b] & 0x7FFFFF == p.tmptbl[b] >> 9


def test_id_embedding_sec5():
    for gid in (0, 1, 0xFFFFFFFF, 0x12345678, 0xDEADBEEF):
        p = O.params_draw(11213, 42, gid)
        assert p.R[0] >> 16 == gid >> 16                       # 16 MSBs of row 0
        assert (p.R[1] >> 4) & 0xFFFF == gid & 0xFFFF           # MSB positions 13..28 of row 1
        assert O.lsb_block_invertible(list(p.R))               # (4x4) + I invertible
        assert (p.sh1, p.sh2) == (13, 4)


def test_lsb_block_invertibility_bruteforce():
    # I + R4 invertible <=> v -> v ^ (v R4) is a bijection on 4-bit vectors.
    for _ in range(300):
        R = [int(x) for x in rng.integers(0, 2**32, 4, dtype=np.uint64)]
        tbl = O.table_from_rows(R)
        images = {(v ^ int(tbl[v])) & 0xF for v in range(16)}
        assert O.lsb_block_invertible(R) == (len(images) == 16)


# ------------------------------------------------- recursion and tempering
@pytest.mark.parametrize("p", SETS, ids=IDS)
def test_matrix_formulation(p):
    """Word operations of the oracle == products of F2 matrices built from the
    definitions (shifts, mask, 4x32 matrices on the four LSBs)."""
    st = rng.integers(0, 2**32, p.N, dtype=np.uint64).astype(np.uint32)
    n = min(2 * p.N + 5, 900)
    ref, ref_state = f2.simulate(p.N, p.pos, p.mask, p.sh1, p.sh2, list(p.R), list(p.T), st, n)
    s2 = st.copy()
    out = O.generate(p, s2, n, O.U32)
    assert np.array_equal(out, ref)
    assert np.array_equal(s2, ref_state)


@pytest.mark.parametrize("p", SETS[:4] + SETS[-3:], ids=IDS[:4] + IDS[-3:])
def test_f2_linearity(p):
    n = 3 * p.N + 11
    a = rng.integers(0, 2**32, p.N, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, 2**32, p.N, dtype=np.uint64).astype(np.uint32)
    oa = O.generate(p, a.copy(), n)
    ob = O.generate(p, b.copy(), n)
    oab = O.generate(p, a ^ b, n)
    assert np.array_equal(oab, oa ^ ob)
    assert not O.generate(p, np.zeros(p.N, np.uint32), n).any()   # zero is a fixed point


@pytest.mark.parametrize("p", SETS[:4] + SETS[-3:], ids=IDS[:4] + IDS[-3:])
def test_mask_invariance(p):
    # x_0 enters only through its w - r MSBs (Sec. 3.3, 3.6).
    n = 2 * p.N + 3
    a = rng.integers(0, 2**32, p.N, dtype=np.uint64).astype(np.uint32)
    b = a.copy()
    b[0] ^= np.uint32(~p.mask & 0xFFFFFFFF)
    assert np.array_equal(O.generate(p, a.copy(), n), O.generate(p, b.copy(), n))
    if p.r < 32:
        c = a.copy()
        c[0] ^= np.uint32(0x80000000)
        assert not np.array_equal(O.generate(p, a.copy(), n), O.generate(p, c, n))


def test_tempering_word_and_offset():
    # o_{N+k} = x_{N+k} ^ h(x_{M-1+k}) (Sec. 3.7).  With T = 0 the outputs are the
    # recursion words x_{N+k} themselves; with T != 0 their XOR difference must be
    # h applied to the word M-1 places after the k-th word of the array.
    p0 = O.params_draw(11213, 8, 8)
    pz = O.params_from_fields(11213, p0.pos, 13, 4, 8, list(p0.R), [0, 0, 0, 0])
    st = O.seed_state(pz, 0, 99)
    n = 3000
    x = np.concatenate([st, O.generate(pz, st.copy(), n)])
    o = O.generate(p0, st.copy(), n)
    H = f2.tempering_block(list(p0.T))
    M, N = p0.pos, p0.N
    for k in range(0, n, 29):
        assert int(o[k] ^ x[N + k]) == f2.word_of(f2.mm(H, f2.bits_of(int(x[M - 1 + k]))[:, None])[:, 0])


# -------------------------------------------------------------- float Sec. 6
@pytest.mark.parametrize("p", SETS[:3], ids=IDS[:3])
def test_float_closed_forms(p):
    n = 50000
    st = O.seed_state(p, 3, 777)
    u = O.generate(p, st.copy(), n, O.U32)
    f12 = O.generate(p, st.copy(), n, O.F12)
    f01 = O.generate(p, st.copy(), n, O.F01).view(np.float32)
    assert np.array_equal(f12, O.f12_closed_form(u))
    assert np.array_equal(f01, O.f01_closed_form(u))
    v12 = f12.view(np.float32)
    assert v12.min() >= 1.0 and v12.max() < 2.0
    assert f01.min() >= 0.0 and f01.max() < 1.0
    # f01 = f12 - 1 exactly (Sterbenz): it never rounds
    assert np.array_equal(f01.astype(np.float64), v12.astype(np.float64) - 1.0)


# ---------------------------------------------------------- continuation Sec. 8
@pytest.mark.parametrize("splits", [(1, 1), (7, 1000), (351, 352), (1000, 1), (4097, 3)])
def test_continuation(splits):
    p = SETS[0]
    st = O.seed_state(p, 0, 1234)
    whole = O.generate(p, st.copy(), sum(splits))
    s = st.copy()
    parts = np.concatenate([O.generate(p, s, n) for n in splits])
    assert np.array_equal(parts, whole)


def test_seed_state_nonzero_and_distinct():
    p = SETS[0]
    seen = set()
    for gid in range(64):
        st = O.seed_state(p, gid, 1234)
        assert st.any()
        seen.add(st.tobytes())
    assert len(seen) == 64
    assert not np.array_equal(O.seed_state(p, 0, 1), O.seed_state(p, 0, 2))


# --------------------------------------------------- F2 tools vs brute force
def _poly_mod(a: int, m: int) -> int:
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def _irreducible_bruteforce(f: int) -> bool:
    d = f.bit_length() - 1
    for g in range(2, 1 << (d // 2 + 1)):
        if g.bit_length() - 1 <= d // 2 and _poly_mod(f, g) == 0:
            return False
    return True


@pytest.mark.parametrize("deg,count", [(5, 6), (7, 18), (13, 630)])
def test_irreducible_count_gauss(deg, count):
    # number of irreducible polynomials of prime degree d over F2 is (2^d - 2)/d
    found = 0
    for low in range(1 << deg):
        f = (1 << deg) | low
        c = np.array([(f >> i) & 1 for i in range(deg + 1)], dtype=np.uint8)
        ir = O.irreducible_prime_degree(c)
        found += ir
        if deg <= 7:
            assert ir == _irreducible_bruteforce(f)
    assert found == count


def test_bm_recovers_lfsr():
    for _ in range(200):
        L = int(rng.integers(1, 12))
        taps = [int(x) for x in rng.integers(0, 2, L)]
        taps[-1] = 1                                   # c_L = 1
        s = [int(x) for x in rng.integers(0, 2, L)]
        if not any(s):
            s[0] = 1
        for k in range(L, 4 * L + 8):
            s.append(sum(taps[i] * s[k - 1 - i] for i in range(L)) & 1)
        poly = O.bm(s)
        # brute force: the shortest recurrence that generates the whole sequence
        best = None
        for l2 in range(0, L + 1):
            for cs in itertools.product((0, 1), repeat=l2):
                if all(sum(cs[i] * s[k - 1 - i] for i in range(l2)) & 1 == s[k]
                       for k in range(l2, len(s))):
                    best = (l2, cs)
                    break
            if best:
                break
        l2, cs = best
        assert len(poly) - 1 == l2
        assert poly[l2] == 1 and [int(poly[l2 - 1 - i]) for i in range(l2)] == list(cs)


# ------------------------------------------------- period at reduced size
def _golden_sets():
    with open(os.path.join(GOLDEN, "full_period_sets.json")) as f:
        return json.load(f)["sets"]


def _params(d):
    return O.params_from_fields(d["mexp"], d["pos"], d["sh1"], d["sh2"], d["id"], d["R"], d["T"])


@pytest.mark.parametrize("d", [d for d in _golden_sets() if d["mexp"] <= 607],
                         ids=lambda d: f"p{d['mexp']}-seed{d['param_seed']}")
def test_full_period_reduced(d):
    """Sec. 3.3 / Sec. 5: the searched sets have a primitive characteristic
    polynomial: BM degree p and irreducible, phi(F) = 0 for the transition F
    built from the definitions, F^(2^p) = F and F - I invertible, so the period
    is the Mersenne prime 2^p - 1."""
    p = _params(d)
    assert O.params_draw(d["mexp"], d["param_seed"], d["id"]).pos == p.pos
    mexp = d["mexp"]
    # BM on the output MSB sequence (tempering is linear, so the tempered
    # sequence has the same minimal polynomial for a nonzero state).
    out = O.generate(p, O.seed_state(p, 5, 4321), 2 * mexp)
    poly = O.bm((out >> np.uint32(31)).astype(np.uint8))
    assert len(poly) - 1 == mexp and O.irreducible_prime_degree(poly)
    F = f2.transition_matrix(p.N, p.r, p.pos, p.mask, p.sh1, p.sh2, list(p.R))
    assert F.shape == (mexp, mexp)
    Fp = O.pack_f2(F)
    assert not O.f2_polyeval(poly, Fp, mexp).any()
    assert np.array_equal(O.f2_pow2k(Fp, mexp, mexp), Fp)
    FmI = F.copy()
    FmI[np.arange(mexp), np.arange(mexp)] ^= 1
    assert O.f2_rank(O.pack_f2(FmI), mexp) == mexp


def test_reducible_set_fails_period_check():
    # negative control: a drawn set that the search rejected is not full period
    d = [d for d in _golden_sets() if d["mexp"] == 521][0]
    p = O.params_draw(521, d["param_seed"] - 1, d["id"])
    out = O.generate(p, O.seed_state(p, 5, 4321), 2 * 521)
    poly = O.bm((out >> np.uint32(31)).astype(np.uint8))
    assert not (len(poly) - 1 == 521 and O.irreducible_prime_degree(poly))
    F = f2.transition_matrix(p.N, p.r, p.pos, p.mask, p.sh1, p.sh2, list(p.R))
    Fp = O.pack_f2(F)
    assert not np.array_equal(O.f2_pow2k(Fp, 521, 521), Fp)


def test_transition_matrix_matches_oracle_steps():
    # F applied N times to the state vector equals N oracle steps.
    d = [d for d in _golden_sets() if d["mexp"] == 127][0]
    p = _params(d)
    st = O.seed_state(p, 1, 1)
    F = f2.transition_matrix(p.N, p.r, p.pos, p.mask, p.sh1, p.sh2, list(p.R))

    def vec(state):
        bits = np.concatenate([f2.bits_of(int(w)) for w in state])
        return bits[p.r:]

    v = vec(st)
    s2 = st.copy()
    for _ in range(3 * p.N):
        v = (F.astype(np.int64) @ v.astype(np.int64) & 1).astype(np.uint8)
        O.generate(p, s2, 1)
    assert np.array_equal(v, vec(s2))


# ------------------------------------------------------------ stored digests
def test_oracle_digests_unchanged():
    with open(os.path.join(GOLDEN, "oracle_digests.json")) as f:
        g = json.load(f)
    p = O.params_draw(11213, 1, 0)
    for name, dt in (("u32", O.U32), ("f12", O.F12), ("f01", O.F01)):
        st = O.seed_state(p, 0, 1234)
        out = O.generate(p, st, 1 << 20, dt)
        assert hashlib.sha256(out.tobytes()).hexdigest() == g["sha256"][name]
        assert hashlib.sha256(st.tobytes()).hexdigest() == g["sha256"][name + "_state_after"]
    for s, words in g["seed_state_first8"].items():
        assert [int(x) for x in O.seed_state(p, 0, int(s))[:8]] == words


def test_generate_many_matches_single():
    ps = [O.params_draw(11213, s, s) for s in (1, 2, 3)] + [O.params_draw(23209, 4, 4)]
    sts = [O.seed_state(p, i, 1234) for i, p in enumerate(ps)]
    ns = [1000, 2001, 5, 777]
    dts = [O.U32, O.F12, O.F01, O.U32]
    outs = O.generate_many(ps, [s.copy() for s in sts], ns, dts, nthreads=3)
    for p, s, n, dt, o in zip(ps, sts, ns, dts, outs):
        assert np.array_equal(o, O.generate(p, s.copy(), n, dt))
