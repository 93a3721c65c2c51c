"""The dual form of the generation kernel (form 5: two work items per
128-thread block, a round of each between block barriers) against the CPU
oracle, bit for bit.

Cases aimed at what is particular to the form:
- odd and even item counts (the last block's second item slot stays empty),
  items of very different lengths (one slot refills while the other runs),
  neighbouring items of different dtypes (rounds run one item at a time);
- rounds of odd and even size S in 257 .. 348 (MTGP 11213), the Sec. 5
  shifts (13, 4; compile-time path) and other shifts (run-time path);
- segments that end inside a round, the smallest buffers (compaction every
  round), interleaved layouts, jump-ahead pieces and the graph-captured
  launch;
- a launch with a generator whose rounds need another slot count is
  refused before anything runs.
"""
import numpy as np
import pytest

import oracle as O
from paper_1005_4973_gb300 import workloads as WL
from tests.helpers import as_u32, lib_pool, oracle_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DUAL = dict(threads=128, form=5)


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


def _check(M, ps, ops, reqs, config, layout=0, seed=5, calls=1):
    pool = M.Pool(ps, list(range(len(ps))), [seed] * len(ps))
    pool.set_config(**config)
    sts = {g: O.seed_state(ops[g], g, seed) for g in range(len(ps))}
    for _ in range(calls):                           # later calls continue the streams
        if layout == 0:
            total = max(off + n for _, _, n, off in reqs)
        else:                                        # whole chunks per request
            c = config.get("chunk", 256)
            total = len(reqs) * -(-reqs[0][2] // c) * c
        out = torch.full((total + 3,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        pool.generate(reqs, out, layout=layout)
        torch.cuda.synchronize()
        got = as_u32(out)
        for j, (g, dt, n, off) in enumerate(reqs):
            ref = O.generate(ops[g], sts[g], n, dt)  # advances the state in place
            if layout == 0:
                assert np.array_equal(got[off:off + n], ref), (g, dt, n, off)
            else:
                c = config.get("chunk", 256)
                idx = np.arange(n)
                pos = (idx // c) * (len(reqs) * c) + j * c + idx % c
                assert np.array_equal(got[pos], ref), (g, dt, n)
        assert int(got[total]) == 0x5A5A5A5A        # nothing written past the end
    for g in range(len(ps)):
        assert np.array_equal(pool.read_state(g), sts[g]), g
    pool.close()


# MTGP 11213 (N = 351): S odd and even, (13, 4) and other shifts
SPECS = [(11213, 1, 0, 300, None, None), (11213, 2, 1, 301, None, None), (11213, 3, 2, 257, None, None),
         (11213, 4, 3, 348, 7, 19), (11213, 5, 4, 299, 13, 4), (11213, 6, 5, 258, 3, 30),
         (11213, 7, 6, None, None, None)]


@pytest.mark.parametrize("count", [1, 2, 7, 13])
@pytest.mark.parametrize("bps", [0, 1, 3])
def test_dual_item_counts_lengths_and_dtypes(M, count, bps):
    specs = [SPECS[i % len(SPECS)][:1] + (10 + i, i) + SPECS[i % len(SPECS)][3:] for i in range(count)]
    ps, ops = _sets(M, specs)
    lens = [1, 2, 299, 300, 301, 1000, 4097, 30001, 99999, 250000]
    reqs, off = [], 1
    for g in range(count):
        for k in range(1 + g % 3):                   # 1 .. 3 segments per item
            n = lens[(3 * g + k) % len(lens)] + k
            reqs.append((g, (g + k) % 3, n, off))
            off += n
    _check(M, ps, ops, reqs, dict(DUAL, blocks_per_sm=bps), calls=2)


def test_dual_same_dtype_pairs_run_together(M):
    # every item one blocked segment of one dtype: full rounds of both items
    # share barriers; lengths differ so that pairs break up and re-form
    ps, ops = _sets(M, SPECS)
    reqs, off = [], 0
    for g in range(len(ps)):
        n = 40000 + 7919 * g
        reqs.append((g, 2, n, off))
        off += n
    for bps in (1, 0):
        _check(M, ps, ops, reqs, dict(DUAL, blocks_per_sm=bps))


@pytest.mark.parametrize("extra", [0, 2, 33, 700])
def test_dual_smallest_buffers(M, extra):
    ps, ops = _sets(M, SPECS)
    need = max(2 * (2 * p.N + 3 * 128 + 32) for p in ps)
    reqs = [(g, g % 3, 20011 + g, 21000 * g + (g & 1)) for g in range(len(ps))]
    _check(M, ps, ops, reqs, dict(DUAL, buffer_words=need + extra))


@pytest.mark.parametrize("chunk", [32, 1024])
def test_dual_interleaved_layout(M, chunk):
    ps, ops = _sets(M, SPECS[:5])
    reqs = [(g, (2 * g) % 3, 12345, 0) for g in range(5)]
    _check(M, ps, ops, reqs, dict(DUAL, chunk=chunk), layout=1)


def test_dual_refuses_other_slot_counts(M):
    # MTGP 521 (S < 257) and MTGP 23209 (S > 384) need other slot counts
    for mexp in (521, 23209):
        ps, _ = _sets(M, [SPECS[0], (mexp, 9, 9, None, None, None)])
        pool = M.Pool(ps, [0, 1], [1, 1])
        pool.set_config(**DUAL)
        out = torch.zeros(2000, dtype=torch.int32, device="cuda")
        with pytest.raises(M.MTGPError) as e:
            pool.generate([(0, 0, 1000, 0), (1, 0, 1000, 1000)], out)
        assert "form 5" in str(e.value)
        pool.close()


def test_dual_equals_the_plain_form_on_c2_shapes(M):
    # the C2 parameter sets with jump-ahead pieces, two calls: dual form and
    # plain form give the same outputs and states
    wl = WL.c2(n=1 << 18)
    gens = wl.gens[:48] + wl.gens[128:176] + wl.gens[256:304]
    ps = [M.mtgp_params_draw(g.mexp, g.param_seed, g.id) for g in gens]
    reqs, off = [], 0
    for i, g in enumerate(gens):
        n = (1 << 18) - 977 * (i % 5)
        reqs.append((i, i // 48, n, off))
        off += n
    outs, states = [], []
    for form in (0, 5):
        pool = M.Pool(ps, [g.gen_id for g in gens], [g.seed for g in gens])
        pool.set_config(threads=128, form=form, pieces=5, piece_log2=14)
        res = []
        for _ in range(2):                           # the second call continues the streams
            out = torch.zeros(off, dtype=torch.int32, device="cuda")
            pool.generate(reqs, out)
            torch.cuda.synchronize()
            res.append(out)
        outs.append(res)
        states.append([pool.read_state(i) for i in range(len(ps))])
        pool.close()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    for a, b in zip(states[0], states[1]):
        assert np.array_equal(a, b)


def test_dual_first_call_matches_the_oracle_on_c2_sets(M):
    wl = WL.c2(n=1 << 14)
    gens = wl.gens[::37]
    pool = lib_pool(gens)
    pool.set_config(**DUAL)
    reqs, off = [], 0
    for i, g in enumerate(gens):
        reqs.append((i, i % 3, 16384 + i, off))
        off += 16384 + i
    out = torch.zeros(off, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    got = as_u32(out)
    for i, g in enumerate(gens):
        p, st = oracle_state(g)
        ref = O.generate(p, st, 16384 + i, i % 3)
        assert np.array_equal(got[reqs[i][3]:reqs[i][3] + 16384 + i], ref), i
        assert np.array_equal(pool.read_state(i), st), i
    pool.close()


def test_dual_graph_replays_with_changing_work(M):
    gens = [WL.GenSpec(11213, i + 1, i, i, 100 + i) for i in range(9)]
    pool = lib_pool(gens)
    pool.set_config(**DUAL)
    graph = M.Graph(pool, max_items=len(gens))
    rng = np.random.default_rng(3)
    launches = []
    for rep in range(4):
        sel = sorted(rng.choice(len(gens), size=int(rng.integers(1, len(gens) + 1)), replace=False).tolist())
        reqs, off = [], 0
        for g in sel:
            n = int(rng.integers(1, 30000))
            reqs.append((g, int(rng.integers(0, 3)), n, off))
            off += n
        out = torch.zeros(off, dtype=torch.int32, device="cuda")
        graph.set_requests(reqs, out)
        for _ in range(1 + rep % 2):
            graph.launch()
            torch.cuda.synchronize()
            launches.append((reqs, as_u32(out).copy()))
    assert graph.errors() == 0
    states = {g: oracle_state(gens[g]) for g in range(len(gens))}
    for reqs, o in launches:
        for g, dt, n, off in reqs:
            p, st = states[g]
            assert np.array_equal(o[off:off + n], O.generate(p, st, n, dt)), (g, dt, n)
    graph.close()
