"""Host-side jump-ahead arithmetic (Sec. 7), no GPU: the library's F2[x]
routines (mtgp_f2_minpoly / mulmod / xpow_mod) against brute force and the
oracle's Berlekamp-Massey, and the jump identity F^J s = (x^J mod psi)(F) s
checked on the oracle's own generator states."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def M():
    from paper_1005_4973_gb300 import build
    build.build()
    O.build()
    import paper_1005_4973_gb300 as M
    return M


# polynomials over F2 as Python ints, bit i = coefficient of x^i
def _clmul(a: int, b: int) -> int:
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def _mod(a: int, m: int) -> int:
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def _to_int(c) -> int:
    return sum(1 << i for i, v in enumerate(c) if v)


def _from_int(a: int) -> np.ndarray:
    return np.array([(a >> i) & 1 for i in range(a.bit_length())], dtype=np.uint8)


def test_mulmod_and_xpow_match_brute_force(M):
    rng = np.random.default_rng(5)
    for _ in range(200):
        dm = int(rng.integers(1, 300))
        m = _to_int(rng.integers(0, 2, dm)) | (1 << dm)
        a = _to_int(rng.integers(0, 2, int(rng.integers(1, 400))))
        b = _to_int(rng.integers(0, 2, int(rng.integers(1, 400))))
        got = _to_int(M.mtgp_f2_mulmod(_from_int(a), _from_int(b), _from_int(m)))
        assert got == _mod(_clmul(_mod(a, m), _mod(b, m)), m)
        e = int(rng.integers(0, 3000))
        want = 1 % m if dm else 0
        for _ in range(e):
            want = _mod(want << 1, m)
        assert _to_int(M.mtgp_f2_xpow_mod(e, _from_int(m))) == want
    # large exponent: x^(2^k) by k squarings, brute-force squaring chain
    m = _to_int(np.random.default_rng(1).integers(0, 2, 127)) | (1 << 127)
    r = 2
    for _ in range(40):
        r = _mod(_clmul(r, r), m)
    assert _to_int(M.mtgp_f2_xpow_mod(1 << 40, _from_int(m))) == r


def test_minpoly_matches_oracle_bm_on_lfsr_sequences(M):
    rng = np.random.default_rng(6)
    for _ in range(120):
        d = int(rng.integers(1, 400))
        c = rng.integers(0, 2, d + 1).astype(np.uint8)
        c[d] = 1
        n = 2 * d + int(rng.integers(0, 40))
        s = np.zeros(n, dtype=np.uint8)
        s[:d] = rng.integers(0, 2, d)
        for k in range(d, n):                           # sum_j c_j s_{k-d+j} = 0
            s[k] = np.bitwise_xor.reduce(c[:d] & s[k - d:k])
        got = M.mtgp_f2_minpoly(s)
        assert np.array_equal(got, O.bm(s))
        # annihilates and divides the generating polynomial
        L = got.size - 1
        for k in range(n - L):
            assert not np.bitwise_xor.reduce(got & s[k:k + L + 1])
        assert _mod(_to_int(c), _to_int(got)) == 0


def test_minpoly_is_minimal_by_enumeration(M):
    rng = np.random.default_rng(7)
    for _ in range(60):
        n = int(rng.integers(1, 13))
        s = rng.integers(0, 2, n).astype(np.uint8)
        got = M.mtgp_f2_minpoly(s)
        L = got.size - 1
        best = None
        for deg in range(0, n + 1):                     # shortest annihilating recurrence
            for low in range(1 << deg):
                cand = [(low >> i) & 1 for i in range(deg)] + [1]
                if all(not (sum(cand[j] & s[k + j] for j in range(deg + 1)) & 1) for k in range(n - deg)):
                    best = deg
                    break
            if best is not None:
                break
        assert L == best


def _state_after(p, st0, k):
    st = st0.copy()
    if k:
        O.generate(p, st, k, 0)
    return st


@pytest.mark.parametrize("mexp,seed", [(521, 3), (607, 4), (1279, 8)])
def test_jump_identity_on_oracle_states(M, mexp, seed):
    """psi from parities of the oracle's outputs, completed until psi(F) s = 0;
    then (x^J mod psi)(F) s equals the oracle's state after J outputs on every
    state bit (the r low bits of the first word are not state)."""
    p = O.params_draw(mexp, seed, seed)
    s0 = O.seed_state(p, seed, 99)
    N, mask = p.N, p.mask
    window = 2 * mexp + 2
    states = [s0.copy()]
    st = s0.copy()
    for _ in range(window + N + 1):
        O.generate(p, st, 1, 0)
        states.append(st.copy())

    def apply(c, base_states):
        acc = np.zeros(N, dtype=np.uint32)
        for i in np.nonzero(c)[0]:
            acc ^= base_states[i]
        return acc

    def nonzero(v):
        return bool((v[0] & mask) or v[1:].any())

    psi = 1
    cur = states
    for fmask in (0xFFFFFFFF, 0x55555555, 0x33333333, 0x0F0F0F0F, 1, 0x80000000):
        bits = np.array([bin(int(c[1]) & fmask).count("1") & 1 for c in cur[:window]], dtype=np.uint8)
        phi = M.mtgp_f2_minpoly(bits)
        psi = _clmul(psi, _to_int(phi))
        v = apply(phi, cur)
        if not nonzero(v):
            break
        # continue on V: its walk is the oracle stream from V
        cur = [v.copy()]
        sv = v.copy()
        for _ in range(window + N + 1):
            O.generate(p, sv, 1, 0)
            cur.append(sv.copy())
    assert not nonzero(apply(_from_int(psi), states)), "psi does not annihilate s"
    assert psi.bit_length() - 1 <= mexp
    for J in (1, 2, N, 3 * N + 5, 4096, 12345):
        g = M.mtgp_f2_xpow_mod(J, _from_int(psi))
        jumped = apply(g, states)
        want = _state_after(p, s0, J)
        assert (jumped[0] & mask) == (want[0] & mask) and np.array_equal(jumped[1:], want[1:]), J
