"""Dimensions of equidistribution k(v) (Sec. 3.4, 3.8): the oracle's k(v)
against values the paper prints (MT19937's defects, Sec. 3.8; minutes, so
--runmanual; a record of its pass is in tests/golden), against a construction
from the standard state basis at small p, and against theorems (k(1) = p at
full period, k(v) <= floor(p / v), k non-increasing); then the library's k(v)
(lattice reduction) against the oracle's (row reduction), MSBs and LSBs, and
the tempering search of Sec. 5 against the oracle's restatement of it."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def M():
    from paper_1005_4973_gb300 import build
    build.build()
    O.build()
    import paper_1005_4973_gb300 as M
    return M


def _f2_rank(rows: np.ndarray) -> int:
    """Rank over F2 of a 0/1 matrix (plain Gaussian elimination)."""
    a = rows.copy() & 1
    r = 0
    for c in range(a.shape[1]):
        pivot = next((i for i in range(r, a.shape[0]) if a[i, c]), None)
        if pivot is None:
            continue
        a[[r, pivot]] = a[[pivot, r]]
        for i in range(a.shape[0]):
            if i != r and a[i, c]:
                a[i] ^= a[r]
        r += 1
    return r


def _kv_standard_basis(op, vmax):
    """k(v) from the definition's linear map on the standard state basis: one
    column per state bit (the 32 - r upper bits of x_0, all bits of x_1 ..
    x_{N-1}), each column the v MSBs of K outputs generated from that unit
    state by the oracle."""
    N, r, p = op.N, 32 * op.N - op.mexp, op.mexp
    K = p + 1
    cols = []
    for w in range(N):
        for b in range(32):
            if w == 0 and b < r:
                continue
            st = np.zeros(N, dtype=np.uint32)
            st[w] = np.uint32(1 << b)
            cols.append(O.generate(op, st, K, 0))
    out = np.stack(cols, axis=1)                          # K x p outputs
    ks = []
    for v in range(1, vmax + 1):
        k = 0
        while (k + 1) * v <= p:
            rows = [((out[i] >> (31 - t)) & 1).astype(np.uint8) for i in range(k + 1) for t in range(v)]
            if _f2_rank(np.array(rows)) < (k + 1) * v:
                break
            k += 1
        ks.append(k)
    return np.array(ks)


def test_oracle_kv_matches_the_standard_basis_construction():
    op, _, _ = O.search_full_period(89, 1000, 7)
    seq = O.generate(op, O.seed_state(op, 1, 2), 2 * 89 + 64, 0)
    assert np.array_equal(O.kv(seq, 89, vmax=8), _kv_standard_basis(op, 8))


@pytest.mark.parametrize("mexp,s0,gid", [(521, 1000, 7), (607, 31, 12), (1279, 9, 1)])
def test_oracle_kv_theorems(mexp, s0, gid):
    op, _, _ = O.search_full_period(mexp, s0, gid, max_tries=200000)
    k = O.kv(O.generate(op, O.seed_state(op, 4, 9), 2 * mexp + 64, 0), mexp)
    v = np.arange(1, 33)
    assert k[0] == mexp                                   # full period: the MSB sequence has complexity p
    assert np.all(k <= mexp // v) and np.all(np.diff(k) <= 0)
    # the same from another nonzero state (any nonzero state is cyclic at full period)
    k2 = O.kv(O.generate(op, O.seed_state(op, 8, 1), 2 * mexp + 64, 0), mexp)
    assert np.array_equal(k, k2)


@pytest.mark.manual
def test_oracle_kv_reproduces_the_mt19937_defects_printed_in_sec_3_8():
    """MT19937 has d(1) = d(2) = d(4) = d(8) = 0, d(3) = 405, d(5) = 249,
    d(6) = 207 and d(7) = 355 (Sec. 3.8)."""
    p = 19937
    seq = O.mt19937_outputs(7, 2 * p + 64)
    d = O.dimension_defects(O.kv(seq, p, vmax=8), p)
    assert list(d) == [0, 0, 405, 0, 249, 207, 355, 0]


@pytest.mark.parametrize("mexp,s0,gid", [(521, 1000, 7), (607, 31, 12), (1279, 9, 1), (2203, 1, 0)])
def test_library_kv_equals_the_oracle(M, mexp, s0, gid):
    p, seed, _, _ = M.mtgp_params_search(mexp, s0, gid)
    k, delta = M.mtgp_params_equidistribution(p)
    op = O.params_draw(mexp, seed, gid)
    ko = O.kv(O.generate(op, O.seed_state(op, 3, 5), 2 * mexp + 64, 0), mexp)
    assert np.array_equal(k, ko)
    assert delta == int(O.dimension_defects(ko, mexp).sum())
    k1, _ = M.mtgp_params_equidistribution(p, threads=1)
    assert np.array_equal(k1, k)


@pytest.mark.parametrize("mexp,s0,gid", [(521, 1000, 7), (1279, 9, 1)])
def test_library_lsb_kv_equals_the_oracle_on_bit_reversed_outputs(M, mexp, s0, gid):
    # k'(v) of the v least significant bits is k(v) of the outputs with their
    # bit order reversed, which the oracle's row reduction computes
    p, seed, _, _ = M.mtgp_params_search(mexp, s0, gid)
    k, delta = M.mtgp_params_equidistribution_lsb(p)
    op = O.params_draw(mexp, seed, gid)
    out = O.generate(op, O.seed_state(op, 3, 5), 2 * mexp + 64, 0)
    ko = O.kv(O.reverse_bits(out), mexp)
    assert np.array_equal(k, ko)
    assert delta == int(O.dimension_defects(ko, mexp).sum())


def test_oracle_search_window_choice_by_brute_force():
    """The oracle's first window (row 0, its 5 MSBs) against a brute force
    that computes k(1) .. k(5) from the standard state basis for each of the
    32 patterns: the oracle's pattern has the least d(1) + ... + d(5), the
    smallest such pattern."""
    op, _, _ = O.search_full_period(89, 1000, 7)
    rows = O.temper_search_sec5(op)
    sums = []
    for pat in range(32):
        q = O.params_from_fields(op.mexp, op.pos, op.sh1, op.sh2, op.id, list(op.R), [pat << 27, 0, 0, 0])
        k = _kv_standard_basis(q, 5)
        sums.append(sum(89 // v - int(k[v - 1]) for v in range(1, 6)))
    assert (rows[0] >> 27) == int(np.argmin(sums))


def test_oracle_search_phases_touch_only_their_bits():
    # Sec. 5: the MSB phase sets bits 31 .. 9 of each row, the LSB phase bits
    # 8 .. 0 and leaves the MSBs found before
    op, _, _ = O.search_full_period(89, 1000, 7)
    rows = O.temper_search_sec5(op)
    p = op.mexp
    k_final = O.kv(O.generate(O.params_from_fields(op.mexp, op.pos, op.sh1, op.sh2, op.id, list(op.R), rows),
                              O.seed_state(op, 1, 2), 2 * p + 64, 0), p)
    assert k_final[0] == p                               # full period: the MSB has complexity p
    assert all(0 <= r < 1 << 32 for r in rows)


@pytest.mark.parametrize("mexp,s0,gid", [(89, 1000, 7), (521, 1000, 7)])
def test_tempering_search_equals_the_oracle_restatement(M, mexp, s0, gid):
    """Sec. 5's tempering search: the library (lattice k(v), windows in
    parallel) and the oracle's step-by-step restatement (row-reduction k(v))
    find the same four rows; the library keeps the recursion and reports the
    total MSB defect of the table it returns."""
    op, seed, _ = O.search_full_period(mexp, s0, gid)
    lp, lseed, _, _ = M.mtgp_params_search(mexp, s0, gid)
    assert seed == lseed
    rows_o = O.temper_search_sec5(op)
    q, d = M.mtgp_params_temper_search(lp)
    assert [q.tmp_tbl[8], q.tmp_tbl[4], q.tmp_tbl[2], q.tmp_tbl[1]] == rows_o
    assert list(q.rec_tbl) == list(lp.rec_tbl) and q.pos == lp.pos
    M.mtgp_params_validate(q)
    oq = O.params_from_fields(mexp, op.pos, op.sh1, op.sh2, gid, list(op.R), rows_o)
    assert list(oq.tmptbl) == list(q.tmp_tbl)
    ko = O.kv(O.generate(oq, O.seed_state(oq, 2, 3), 2 * mexp + 64, 0), mexp)
    assert d == int(O.dimension_defects(ko, mexp).sum())


def test_report_and_record(M):
    """The Table 1 style report lists k(v), d(v) = floor(p/v) - k(v) and the
    total; the MTGPDC record's digest is the SHA-1 (checked with Python's
    hashlib) of the characteristic polynomial's coefficient string."""
    import hashlib
    p, seed, _, phi = M.mtgp_params_search(1279, 9, 1)
    k, delta = M.mtgp_params_equidistribution(p)
    lines = M.mtgp_params_report(p).splitlines()
    assert lines[-1] == f"total dimension defect {delta}"
    for v in range(1, 33):
        f = lines[v].split()
        assert int(f[0]) == v and int(f[1]) == k[v - 1] and int(f[2]) == 1279 // v - k[v - 1]
    rec = M.mtgp_params_record(p, phi).split(",")
    coef = "".join("1" if c else "0" for c in np.asarray(phi, dtype=np.uint8))
    assert rec[-3] == hashlib.sha1(coef.encode()).hexdigest()
    assert int(rec[-2]) == int(np.asarray(phi).sum()) and int(rec[-1]) == delta
    assert rec[:6] == [str(x) for x in (p.mexp, p.N, p.pos, p.sh1, p.sh2, p.id)]
    assert rec[6:22] == [f"{v:08x}" for v in p.rec_tbl] and rec[22:38] == [f"{v:08x}" for v in p.tmp_tbl]
