"""The wide form of the generation kernel (form 3: four adjacent columns per
thread, four interleaved shared sub-buffers, 16-byte output stores) against the
CPU oracle, bit for bit.

The cases aim at its own edges:
- output addresses of every residue mod 4, including several segments per
  generator whose residues differ (the live words move by 1-3 places);
- rounds shorter than S (segment tails), and requests of 1 to 3 numbers;
- shared buffers at their minimum (compaction every round);
- every group count a block size compiles;
- jump-ahead pieces, persistent grids, the graph form, and interleaved
  layouts (which run in the plain form).
"""
import numpy as np
import pytest

import oracle as O
from paper_1005_4973_gb300 import workloads as WL
from tests.helpers import as_u32, lib_pool, oracle_params, oracle_stream

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WIDE = [96, 128, 192]
QW_MAX = {96: 4, 128: 3, 192: 2}
MIXED = [WL.GenSpec(11213, 1, 0, 0), WL.GenSpec(23209, 2, 1, 1), WL.GenSpec(44497, 3, 2, 2),
         WL.GenSpec(521, 4, 3, 3), WL.GenSpec(89, 5, 4, 4), WL.GenSpec(1279, 6, 5, 5),
         WL.GenSpec(11213, 7, 0xFFFF0001, 6, 99)]
RAGGED = [1, 2, 3, 5, 31, 33, 255, 257, 1000, 4097, 12345]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1005_4973_gb300 import build
    build.build()
    O.build()
    assert torch.cuda.is_available()


def _fits(spec, threads):
    p = oracle_params(spec)
    return (p.N - p.pos + 6) // 4 + 1 <= threads * QW_MAX[threads]


def _check(gens, reqs, out, pool, base=0):
    by_gen = {}
    for g, dt, n, off in reqs:
        by_gen.setdefault(g, []).append((dt, n, off))
    for g, segs in by_gen.items():
        outs, st = oracle_stream(gens[g], [(dt, n) for dt, n, _ in segs])
        for (dt, n, off), ref in zip(segs, outs):
            assert np.array_equal(out[base + off:base + off + n], ref), (gens[g], dt, n, off)
        assert np.array_equal(pool.read_state(g), st), gens[g]
        assert pool.position(g) == sum(n for _, n, _ in segs)


def _ragged_requests(ngens, seed):
    rng = np.random.default_rng(seed)
    reqs, off = [], int(rng.integers(0, 4))
    for g in range(ngens):
        for _ in range(int(rng.integers(1, 5))):
            n = int(rng.choice(RAGGED))
            reqs.append((g, int(rng.integers(0, 3)), n, off))
            off += n + int(rng.integers(0, 4))        # gaps give every residue mod 4
    return reqs, off


@pytest.mark.parametrize("threads", WIDE)
@pytest.mark.parametrize("persistent", [0, 1])
def test_ragged_segments_every_residue(threads, persistent):
    gens = [g for g in MIXED if _fits(g, threads)]
    pool = lib_pool(gens)
    pool.set_config(threads=threads, form=3, persistent=persistent, blocks_per_sm=persistent)
    reqs, total = _ragged_requests(len(gens), 17 + threads + persistent)
    out = torch.full((total + 8,), 0x5A, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    _check(gens, reqs, as_u32(out), pool)
    assert pool.errors() == 0


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_output_pointer_not_16_byte_aligned(shift):
    # the output tensor starts 4, 8 or 12 bytes past a 16-byte boundary
    gens = MIXED[:2]
    pool = lib_pool(gens)
    pool.set_config(threads=96, form=3)
    reqs = [(0, 0, 5000, 0), (1, 2, 7001, 5000), (0, 1, 3, 12001)]
    buf = torch.zeros(12004 + 8, dtype=torch.int32, device="cuda")
    out = buf[shift:]
    assert out.data_ptr() % 16 == 4 * shift
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    _check(gens, reqs, as_u32(out), pool)


@pytest.mark.parametrize("threads", WIDE)
def test_every_group_count(threads):
    """Synthetic sets whose round size S gives each group count per thread,
    with the last slot as full and as empty as it gets."""
    import paper_1005_4973_gb300 as M
    ps, ops, n = [], [], 2503
    for qw in range(1, QW_MAX[threads] + 1):
        for G in sorted({threads * qw, threads * (qw - 1) + 1}):
            S = max(1, 4 * (G - 1) - 6)                  # (S + 6) / 4 + 1 = G at most
            if (S + 6) // 4 + 1 > threads * QW_MAX[threads]:
                continue
            N = S + 3 + (qw % 4)
            mexp = 32 * N - 17
            if N > 4096:
                continue
            lp = M.mtgp_params_draw(mexp, qw, qw)
            o = O.params_draw(mexp, qw, qw)
            lp.pos = N - S
            ops.append(O.params_from_fields(mexp, N - S, o.sh1, o.sh2, qw, list(o.R), list(o.T)))
            ps.append(lp)
    pool = M.Pool(ps, list(range(len(ps))), [13] * len(ps))
    pool.set_config(threads=threads, form=3)
    out = torch.zeros((n + 4) * len(ps), dtype=torch.int32, device="cuda")
    pool.generate([(i, i % 3, n, i * (n + 4) + (i % 4)) for i in range(len(ps))], out)
    o = as_u32(out)
    for i, op in enumerate(ops):
        st = O.seed_state(op, i, 13)
        off = i * (n + 4) + (i % 4)
        assert np.array_equal(o[off:off + n], O.generate(op, st, n, i % 3)), (op.N, op.pos)
        assert np.array_equal(pool.read_state(i), st)


@pytest.mark.parametrize("extra", [0, 1, 5, 300])
@pytest.mark.parametrize("threads", [96, 192])
def test_minimum_buffers_compact_every_round(extra, threads):
    gens = MIXED[:3] if threads == 192 else [MIXED[0], MIXED[3], MIXED[6]]
    ps = [oracle_params(g) for g in gens]
    need = max(2 * p.N + (p.N - p.pos) + 24 for p in ps)
    need = -(-need // 4) * 4                          # whole sub-buffer rows
    pool = lib_pool(gens)
    pool.set_config(threads=threads, form=3, buffer_words=need + extra)
    reqs, total = _ragged_requests(len(gens), 99 + extra)
    reqs += [(g, g % 3, 20011, total + 20011 * g + g) for g in range(len(gens))]
    total += 20011 * len(gens) + len(gens)
    out = torch.zeros(total + 8, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    _check(gens, reqs, as_u32(out), pool)


def test_buffer_below_minimum_rejected():
    import paper_1005_4973_gb300 as M
    p = oracle_params(MIXED[0])
    pool = lib_pool(MIXED[:1])
    pool.set_config(threads=96, form=3, buffer_words=2 * p.N + (p.N - p.pos) + 23)
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MTGPError):
        pool.generate([(0, 0, 64, 0)], out)


@pytest.mark.parametrize("threads", WIDE)
def test_jump_ahead_pieces(threads):
    gens = [g for g in MIXED if _fits(g, threads)][:4]
    pool = lib_pool(gens)
    pool.set_config(threads=threads, form=3, pieces=5, piece_log2=10)
    reqs, off = [], 1
    for g in range(len(gens)):
        reqs.append((g, g % 3, 30001 + 7 * g, off))
        off += 30001 + 7 * g + 1
    out = torch.zeros(off + 4, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    pool.generate(reqs, out)                          # second call continues the streams
    torch.cuda.synchronize()
    o = as_u32(out)
    assert pool.launch_count() >= 4
    for g, dt, n, off in reqs:
        outs, st = oracle_stream(gens[g], [(dt, n), (dt, n)])
        assert np.array_equal(o[off:off + n], outs[1])
        assert np.array_equal(pool.read_state(g), st)


def test_interleaved_layout_runs_plain():
    gens = MIXED[:3]
    pool = lib_pool(gens)
    chunk, n = 64, 5000
    pool.set_config(threads=96, form=3, chunk=chunk)
    reqs = [(g, g % 3, n, 0) for g in range(3)]
    out = torch.zeros(3 * n + 3 * chunk, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out, layout=1)
    torch.cuda.synchronize()
    o = as_u32(out)
    k = np.arange(n)
    for g in range(3):
        (ref,), _ = oracle_stream(gens[g], [(g % 3, n)])
        assert np.array_equal(o[(k // chunk) * (3 * chunk) + g * chunk + k % chunk], ref)


def test_graph_form_replays_and_rejects_interleaved():
    import paper_1005_4973_gb300 as M
    gens = MIXED[:4]
    pool = lib_pool(gens)
    pool.set_config(threads=96, form=3)
    g = M.Graph(pool, 64)
    reqs, total = _ragged_requests(len(gens), 7)
    out = torch.zeros(total + 8, dtype=torch.int32, device="cuda")
    g.set_requests(reqs, out)
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    o = as_u32(out)
    for gi in range(len(gens)):
        segs = [(dt, n, off) for gg, dt, n, off in reqs if gg == gi]
        outs, st = oracle_stream(gens[gi], [(dt, n) for dt, n, _ in segs] * 2)
        for (dt, n, off), ref in zip(segs, outs[len(segs):]):
            assert np.array_equal(o[off:off + n], ref)
        assert np.array_equal(pool.read_state(gi), st)
    with pytest.raises(M.MTGPError):
        g.set_requests([(0, 0, 64, 0), (1, 0, 64, 0)], out, layout=1)


def test_c2_instances_in_full():
    """Three C2 instances (one per dtype) at the full 2^24 numbers, pieces auto."""
    wl = WL.c2()
    idx = [0, 200, 383]
    gens = [wl.gens[i] for i in idx]
    n = 1 << 24
    pool = lib_pool(gens)
    pool.set_config(threads=96, form=3)
    reqs = [(k, wl.requests[i][1], n, k * n) for k, i in enumerate(idx)]
    out = torch.zeros(3 * n, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    _check(gens, reqs, as_u32(out), pool)


@pytest.mark.parametrize("round_words", [8, 12, 128, 256])
def test_rounds_shorter_than_s(round_words):
    """mtgp_config.round_words: the wide form runs rounds of fewer than S
    words (any n <= S consecutive words are independent, Sec. 3.2); outputs
    and states equal the oracle's, ragged segments of every residue."""
    gens = [g for g in MIXED if _fits(g, 128)]
    pool = lib_pool(gens)
    pool.set_config(threads=128, form=3, round_words=round_words)
    reqs, total = _ragged_requests(len(gens), 1000 + round_words)
    out = torch.full((total + 8,), 0x5A, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    _check(gens, reqs, as_u32(out), pool)
    assert pool.errors() == 0
