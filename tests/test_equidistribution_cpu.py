"""Dimensions of equidistribution k(v) (Sec. 3.4, 3.8): the oracle's k(v)
against values the paper prints (MT19937's defects, Sec. 3.8; minutes, so
--runmanual), against a construction from the standard state basis at small
p, and against theorems (k(1) = p at full period, k(v) <= floor(p / v),
k non-increasing); then the library's k(v) against the oracle's."""
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


def test_tempering_search_lowers_the_defect_and_matches_the_oracle(M):
    """The tempering search keeps the recursion, never returns a worse total
    defect than the input's, and the oracle's k(v) for the returned table
    (rebuilt from its four rows, Sec. 3.7 convention) equals the library's."""
    p, seed, _, _ = M.mtgp_params_search(1279, 9, 1)
    _, d0 = M.mtgp_params_equidistribution(p)
    q, d1 = M.mtgp_params_temper_search(p, 100, 40)
    assert d1 <= d0
    assert list(q.rec_tbl) == list(p.rec_tbl) and q.pos == p.pos
    M.mtgp_params_validate(q)
    kq, dq = M.mtgp_params_equidistribution(q)
    assert dq == d1
    rows_r = [p.rec_tbl[8], p.rec_tbl[4], p.rec_tbl[2], p.rec_tbl[1]]
    rows_t = [q.tmp_tbl[8], q.tmp_tbl[4], q.tmp_tbl[2], q.tmp_tbl[1]]
    oq = O.params_from_fields(q.mexp, q.pos, q.sh1, q.sh2, q.id, rows_r, rows_t)
    assert list(oq.rectbl) == list(q.rec_tbl) and list(oq.tmptbl) == list(q.tmp_tbl)
    ko = O.kv(O.generate(oq, O.seed_state(oq, 2, 3), 2 * 1279 + 64, 0), 1279)
    assert np.array_equal(kq, ko)
    table = M.equidistribution_table(q, kq)
    assert table.splitlines()[-1] == f"total dimension defect {d1}"
