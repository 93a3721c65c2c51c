"""The pair form of the generation kernel (form 4: two adjacent columns per
thread, the shared buffer split into even and odd halves, 8-byte output
stores) against the CPU oracle, bit for bit.

Cases aimed at what is particular to the form:
- rounds of odd and even size S = N - M, so that the round's start parity and
  the output address's 8-byte alignment alternate or stay fixed, and the
  round's last pair is half when S is odd;
- output offsets of either parity, and segments that end inside a round
  (the general round);
- parameter sets with the Sec. 5 shifts (13, 4; compile-time path) and with
  other shifts (run-time path);
- the smallest buffers (compaction from an odd buffer index), interleaved
  layouts, and every pair-slot count.
"""
import numpy as np
import pytest

import oracle as O
from paper_1005_4973_gb300 import workloads as WL
from tests.helpers import as_u32

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


def _sets(M, specs):
    """Library and oracle parameter sets for (mexp, param_seed, id, S, sh1, sh2)
    with M = N - S (None keeps the drawn value)."""
    ps, ops = [], []
    for mexp, seed, gid, S, sh1, sh2 in specs:
        lp = M.mtgp_params_draw(mexp, seed, gid)
        o = O.params_draw(mexp, seed, gid)
        pos = o.pos if S is None else o.N - S
        s1 = o.sh1 if sh1 is None else sh1
        s2 = o.sh2 if sh2 is None else sh2
        lp.pos, lp.sh1, lp.sh2 = pos, s1, s2
        M.mtgp_params_validate(lp)
        ps.append(lp)
        ops.append(O.params_from_fields(mexp, pos, s1, s2, gid, list(o.R), list(o.T)))
    return ps, ops


def _check(M, ps, ops, reqs, config, layout=0, seed=5):
    pool = M.Pool(ps, list(range(len(ps))), [seed] * len(ps))
    pool.set_config(**config)
    if layout == 0:
        total = max(off + n for _, _, n, off in reqs)
    else:                                            # whole chunks per request
        c = config.get("chunk", 256)
        total = len(reqs) * -(-reqs[0][2] // c) * c
    out = torch.full((total + 3,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out, layout=layout)
    torch.cuda.synchronize()
    got = as_u32(out)
    by_gen = {}
    for j, (g, dt, n, off) in enumerate(reqs):
        by_gen.setdefault(g, []).append((j, dt, n, off))
    for g, segs in by_gen.items():
        st = O.seed_state(ops[g], g, seed)
        for j, dt, n, off in segs:
            ref = O.generate(ops[g], st, n, dt)          # advances st in place
            if layout == 0:
                assert np.array_equal(got[off:off + n], ref), (g, dt, n, off)
            else:
                c = config.get("chunk", 256)
                idx = np.arange(n)
                pos = (idx // c) * (len(reqs) * c) + j * c + idx % c
                assert np.array_equal(got[pos], ref), (g, dt, n)
        assert np.array_equal(pool.read_state(g), st), g
    pool.close()


# S odd and even for each exponent; (13, 4) and other shifts
SPECS = [(11213, 1, 0, 300, None, None), (11213, 2, 1, 301, None, None), (11213, 3, 2, 257, None, None),
         (11213, 4, 3, 348, 7, 19), (23209, 5, 4, 513, None, None), (23209, 6, 5, 722, 3, 30),
         (44497, 7, 6, 1025, None, None), (44497, 8, 7, 1387, None, None), (521, 9, 8, None, None, None),
         (89, 10, 9, None, None, None)]


@pytest.mark.parametrize("persistent", [0, 1])
def test_pairs_odd_and_even_rounds_any_output_parity(M, persistent):
    ps, ops = _sets(M, SPECS)
    reqs, off = [], 1                                # offset 1: every generator starts misaligned
    lens = [1, 2, 3, 255, 256, 257, 1000, 4097, 30001, 99999]
    for g in range(len(ps)):
        for k in range(3):
            n = lens[(g + 3 * k) % len(lens)] + k
            reqs.append((g, (g + k) % 3, n, off))
            off += n
    _check(M, ps, ops, reqs, dict(threads=128, form=4, persistent=persistent, blocks_per_sm=persistent))


@pytest.mark.parametrize("extra", [0, 1, 2, 33, 700])
def test_pairs_smallest_buffers(M, extra):
    # compaction every round or few rounds, from buffer indexes of both parities
    ps, ops = _sets(M, SPECS[:4] + SPECS[6:7])
    need = max(2 * p.N + 256 * -(-(p.N - p.pos) // 256) + 32 for p in ps)
    reqs = [(g, g % 3, 20011 + g, 21000 * g + (g & 1)) for g in range(len(ps))]
    _check(M, ps, ops, reqs, dict(threads=128, form=4, buffer_words=need + extra))


@pytest.mark.parametrize("chunk", [32, 1024])
def test_pairs_interleaved_layout(M, chunk):
    ps, ops = _sets(M, SPECS[:3])
    reqs = [(g, (2 * g) % 3, 12345, 0) for g in range(3)]
    _check(M, ps, ops, reqs, dict(threads=128, form=4, chunk=chunk), layout=1)


def test_pairs_every_slot_count(M):
    # S = 256 q and 256 q - 31 for q = 1 .. 6 pair slots (fullest and emptiest
    # tail slot), shifts (13, 4) and others
    specs = []
    for q in range(1, 7):
        for S in (256 * q, 256 * q - 31):
            N = S + 2 + q % 5
            specs.append((32 * N - 17, q, q, S, None if q % 2 else 5, None if q % 2 else 9))
    ps, ops = _sets(M, specs)
    reqs = [(i, i % 3, 5003, 5010 * i + (i & 1)) for i in range(len(ps))]
    _check(M, ps, ops, reqs, dict(threads=128, form=4))


def test_pairs_equal_the_plain_form_on_c2_shapes(M):
    # the C2 parameter sets (drawn M, shifts 13 / 4) with jump-ahead pieces:
    # pair form and plain form give the same outputs and states
    wl = WL.c2(n=1 << 18)
    gens = wl.gens[:48]
    ps = [M.mtgp_params_draw(g.mexp, g.param_seed, g.id) for g in gens]
    reqs = [(i, r[1], r[2], r[3]) for i, r in enumerate(wl.requests[:48])]
    total = max(off + n for _, _, n, off in reqs)
    outs, states = [], []
    for form in (0, 4):
        pool = M.Pool(ps, [g.gen_id for g in gens], [g.seed for g in gens])
        pool.set_config(threads=128, form=form, pieces=5, piece_log2=14)
        out = torch.zeros(total, dtype=torch.int32, device="cuda")
        pool.generate(reqs, out)
        pool.generate(reqs, out)                     # second call continues the streams
        torch.cuda.synchronize()
        outs.append(out.clone())
        states.append([pool.read_state(i) for i in range(len(ps))])
        pool.close()
    assert torch.equal(outs[0], outs[1])
    for a, b in zip(states[0], states[1]):
        assert np.array_equal(a, b)
