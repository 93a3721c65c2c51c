"""MTGPDC's recursion-parameter search (Sec. 5) in the library against the
oracle's own search: the same candidate order, so both must accept the same
first candidate; the polynomial returned must be irreducible by the oracle's
test and must be the minimal polynomial of the oracle's output sequence."""
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


@pytest.mark.parametrize("mexp,seed0,gen_id", [(89, 1000, 7), (107, 5, 0), (127, 77, 3), (521, 1000, 7),
                                               (607, 31, 12), (1279, 9, 1)])
def test_search_accepts_the_oracles_first_candidate(M, mexp, seed0, gen_id):
    p, seed, tries, phi = M.mtgp_params_search(mexp, seed0, gen_id)
    op, oseed, otries = O.search_full_period(mexp, seed0, gen_id, max_tries=200000)
    assert (seed, tries) == (oseed, otries)
    assert (p.pos, p.sh1, p.sh2) == (op.pos, op.sh1, op.sh2)
    assert list(p.rec_tbl) == list(op.rectbl)
    assert phi.size - 1 == mexp and O.irreducible_prime_degree(phi)


def test_search_result_does_not_depend_on_threads(M):
    a = M.mtgp_params_search(607, 400, 2, threads=1)
    b = M.mtgp_params_search(607, 400, 2, threads=0)
    assert a[1:3] == b[1:3] and np.array_equal(a[3], b[3])


def test_searched_polynomial_is_the_minimal_polynomial_of_the_oracle_stream(M):
    """The accepted polynomial annihilates the oracle's output (tempered words,
    every bit) from another seed: it is the characteristic polynomial of F."""
    p, seed, _, phi = M.mtgp_params_search(521, 1000, 7)
    op = O.params_draw(521, seed, 7)
    st = O.seed_state(op, 3, 99)
    o = O.generate(op, st, 2 * 521 + 200, 0)
    sel = np.nonzero(phi)[0]
    for k in range(0, 200, 3):
        assert np.bitwise_xor.reduce(o[k + sel]) == 0
    bits = (o >> 17) & 1
    assert np.array_equal(O.bm(bits.astype(np.uint8)), phi)


def test_search_limits_and_record(M):
    with pytest.raises(M.MTGPError):
        M.mtgp_params_search(1279, 9, 1, max_tries=3)      # the first accepted candidate is number 1184
    p, seed, tries, phi = M.mtgp_params_search(89, 1000, 7)
    rec = M.mtgp_params_record(p, phi).split(",")
    _, delta = M.mtgp_params_equidistribution(p)
    assert rec[0] == "89" and len(rec) == 6 + 32 + 3 and len(rec[-3]) == 40
    assert int(rec[-2]) == int(phi.sum()) and int(rec[-1]) == delta


@pytest.mark.manual
def test_full_size_mtgp11213_search(M):
    """A full-size search (about a minute of 16 cores): the polynomial has
    degree 11213, the oracle's irreducibility test agrees, and it annihilates
    the oracle's output."""
    p, seed, tries, phi = M.mtgp_params_search(11213, 1, 0)
    assert phi.size - 1 == 11213
    assert O.irreducible_prime_degree(phi)
    op = O.params_draw(11213, seed, 0)
    o = O.generate(op, O.seed_state(op, 0, 5), 11213 + 64, 0)
    sel = np.nonzero(phi)[0]
    for k in range(0, 64, 9):
        assert np.bitwise_xor.reduce(o[k + sel]) == 0
