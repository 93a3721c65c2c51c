"""The MTGPDC recursion search (Sec. 5) with Berlekamp-Massey on the GPU (one
warp per candidate) against the host search and the oracle's search: the same
first accepted candidate, and a characteristic polynomial equal to the
oracle's Berlekamp-Massey polynomial of the set's MSB sequence, which
annihilates the oracle's outputs."""
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
    """A full-size MTGP11213 search: the same set as the host search; both
    times are printed (pytest -s)."""
    t0 = time.perf_counter()
    pg, sg, tg, phig = M.mtgp_params_search_gpu(11213, 1, 0)
    tgpu = time.perf_counter() - t0
    t0 = time.perf_counter()
    ph, sh, th, phih = M.mtgp_params_search(11213, 1, 0)
    thost = time.perf_counter() - t0
    print(f"MTGP11213 search: GPU Berlekamp-Massey {tgpu:.2f} s, host {thost:.2f} s, {tg} candidates")
    assert sg == sh and np.array_equal(phig, phih) and phig.size - 1 == 11213
