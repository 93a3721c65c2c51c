"""Seeded random cases across every kernel form against the CPU oracle, bit
for bit: random parameter sets (exponents 521 .. 23209, drawn or random
M and shifts), random request lists (lengths 0 .. 40000, every dtype, several
requests per generator, random gaps between outputs), blocked or interleaved
layouts, persistent or not, jump-ahead pieces on or off, two calls in a row
(the second continues the streams).  Each case is small enough for the
oracle; the seeds make every failure reproducible."""
import numpy as np
import pytest

import oracle as O
from tests.helpers import as_u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (threads, form): plain, split, flow, wide, pairs, dual
FORMS = [(128, 0), (256, 0), (256, 1), (512, 2), (128, 3), (128, 4), (128, 5)]


@pytest.fixture(scope="module")
def M():
    from paper_1005_4973_gb300 import build
    build.build()
    O.build()
    assert torch.cuda.is_available()
    import paper_1005_4973_gb300 as M
    return M


def _sets(M, rng, form, count):
    """count parameter sets usable by the form (library and oracle copies)."""
    ps, ops = [], []
    for i in range(count):
        if form == 5:                                    # rounds of 257 .. 384 words
            mexp, S = 11213, int(rng.integers(257, 349))
        else:
            mexp = int(rng.choice([521, 1279, 11213, 23209]))
            S = None
        seed, gid = int(rng.integers(1, 1 << 30)), int(rng.integers(0, 1 << 16))
        lp = M.mtgp_params_draw(mexp, seed, gid)
        o = O.params_draw(mexp, seed, gid)
        pos = o.pos if S is None else o.N - S
        sh1, sh2 = o.sh1, o.sh2
        if rng.random() < 0.3:                           # shifts other than Sec. 5's
            sh1, sh2 = int(rng.integers(1, 32)), int(rng.integers(1, 32))
        lp.pos, lp.sh1, lp.sh2 = pos, sh1, sh2
        M.mtgp_params_validate(lp)
        ps.append(lp)
        ops.append(O.params_from_fields(mexp, pos, sh1, sh2, gid, list(o.R), list(o.T)))
    return ps, ops


@pytest.mark.parametrize("case", range(70))
def test_random_case(M, case):
    rng = np.random.default_rng(1000 + case)
    threads, form = FORMS[case % len(FORMS)]
    ngen = int(rng.integers(1, 9))
    ps, ops = _sets(M, rng, form, ngen)
    layout = int(rng.random() < 0.3)
    chunk = int(rng.choice([32, 256, 1024]))
    pieces = int(rng.choice([0, 1, 3]))
    cfg = dict(threads=threads, form=form, persistent=int(rng.integers(0, 2)), chunk=chunk, pieces=pieces,
               piece_log2=10 if pieces else 0)
    seeds = [int(s) for s in rng.integers(1, 1 << 40, size=ngen)]
    pool = M.Pool(ps, list(range(ngen)), seeds)
    pool.set_config(**cfg)
    states = [O.seed_state(ops[g], g, seeds[g]) for g in range(ngen)]
    for call in range(2):
        if layout == 0:
            reqs, off = [], int(rng.integers(0, 5))
            for _ in range(int(rng.integers(1, 12))):
                g, n = int(rng.integers(0, ngen)), int(rng.integers(0, 40000))
                reqs.append((g, int(rng.integers(0, 3)), n, off))
                off += n + int(rng.integers(0, 3))
            total = off
        else:                                            # one request per generator, equal lengths
            n = int(rng.integers(1, 30000))
            reqs = [(g, int(rng.integers(0, 3)), n, 0) for g in range(ngen)]
            total = ngen * -(-n // chunk) * chunk
        out = torch.full((total + 4,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        pool.generate(reqs, out, layout=layout)
        torch.cuda.synchronize()
        got = as_u32(out)
        for j, (g, dt, n, off) in enumerate(reqs):
            ref = O.generate(ops[g], states[g], n, dt)   # advances the oracle's state
            if layout == 0:
                assert np.array_equal(got[off:off + n], ref), (case, call, j, cfg)
            else:
                idx = np.arange(n)
                pos = (idx // chunk) * (len(reqs) * chunk) + j * chunk + idx % chunk
                assert np.array_equal(got[pos], ref), (case, call, j, cfg)
        assert int(got[total]) == 0x5A5A5A5A
    assert pool.errors() == 0
    for g in range(ngen):
        assert np.array_equal(pool.read_state(g), states[g]), (case, g)
    pool.close()
