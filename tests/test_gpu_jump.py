"""Jump-ahead on the GPU (Sec. 7) against the oracle's sequential streams: a
generator's work split into pieces that start from jumped states must give
exactly the numbers, final state and position of the unsplit stream; an
explicit jump must land on the oracle's state after that many outputs; and the
annihilating polynomial the library finds must annihilate the oracle's output
sequence."""
import numpy as np
import pytest

import oracle as O
from paper_1005_4973_gb300 import workloads as WL
from tests.helpers import as_u32, lib_pool, oracle_state, oracle_stream

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = [dict(threads=128, form=0), dict(threads=256, form=1), dict(threads=256, form=2),
         dict(threads=128, form=0, persistent=1, blocks_per_sm=1), dict(threads=128, form=4),
         dict(threads=128, form=4, persistent=1, blocks_per_sm=1)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1005_4973_gb300 import build
    build.build()
    O.build()
    assert torch.cuda.is_available()


def _gens(mexps, seed0=1):
    return [WL.GenSpec(m, seed0 + i, 40 + i, i, 500 + i) for i, m in enumerate(mexps)]


def _check(gens, reqs, out, pool):
    by_gen = {}
    for g, dt, n, off in reqs:
        by_gen.setdefault(g, []).append((dt, n, off))
    for g, segs in by_gen.items():
        outs, st = oracle_stream(gens[g], [(dt, n) for dt, n, _ in segs])
        for (dt, n, off), ref in zip(segs, outs):
            got = out[off:off + n]
            if not np.array_equal(got, ref):
                bad = np.nonzero(got != ref)[0]
                raise AssertionError(f"gen {g} ({gens[g].mexp}) dtype {dt} n {n}: {bad.size} differ, "
                                     f"first at {bad[0]}")
        assert np.array_equal(pool.read_state(g), st), f"state of gen {g}"
        assert pool.position(g) == sum(n for _, n, _ in segs)


def _blocked(spec):
    reqs, off = [], 0
    for g, dt, n in spec:
        reqs.append((g, dt, n, off))
        off += n
    return reqs, off


@pytest.mark.parametrize("cfg", FORMS, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_pieces_equal_the_sequential_stream(cfg):
    gens = _gens([11213, 23209, 44497, 521, 607, 11213])
    spec = [(0, 0, 9000), (1, 2, 20011), (2, 1, 7777), (3, 0, 40000), (4, 2, 1025), (5, 0, 65536)]
    reqs, total = _blocked(spec)
    pool = lib_pool(gens)
    pool.set_config(pieces=8, piece_log2=10, **cfg)
    before = pool.launch_count()
    out = torch.full((total,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    assert pool.launch_count() - before in (2, 3)     # fused jump (or walk + sum), generation
    assert pool.errors() == 0
    _check(gens, reqs, as_u32(out), pool)


def test_pieces_across_segments_and_calls():
    """Several requests of one generator in a call (piece boundaries fall inside
    and between segments, dtypes change across them), repeated calls continuing
    the streams, and piece counts from 2 to 64."""
    gens = _gens([11213, 521, 23209])
    pool = lib_pool(gens)
    hist = {0: [], 1: [], 2: []}
    rng = np.random.default_rng(17)
    for call, k in enumerate((2, 3, 7, 64, 5)):
        pool.set_config(pieces=k, piece_log2=10)
        spec = []
        for g in (0, 1, 2, 0, 1):
            spec.append((g, int(rng.integers(0, 3)), int(rng.integers(1, 30000))))
        reqs, total = _blocked(spec)
        out = torch.full((total,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        pool.generate(reqs, out)
        torch.cuda.synchronize()
        got = as_u32(out)
        for g, dt, n, off in reqs:
            hist[g].append((dt, n, got[off:off + n].copy()))
    for g in hist:
        outs, st = oracle_stream(gens[g], [(dt, n) for dt, n, _ in hist[g]])
        for (dt, n, mine), ref in zip(hist[g], outs):
            assert np.array_equal(mine, ref), (g, dt, n)
        assert np.array_equal(pool.read_state(g), st)
        assert pool.position(g) == sum(n for _, n, _ in hist[g])


def test_automatic_pieces_of_long_items_in_a_launch_of_few_items():
    """Fewer work items than SMs, each long enough for the normal piece rule
    to give more pieces than the few-item rule (100 items of 5 x 2^20 + 777
    numbers of MTGP11213: 5 pieces each, not 4): sampled generators' streams,
    states and positions equal the oracle's, over two calls."""
    n = 5 * (1 << 20) + 777
    gens = _gens([11213] * 100)
    pool = lib_pool(gens)
    spec = [(g, g % 3, n) for g in range(100)]
    reqs, total = _blocked(spec)
    out = torch.full((total,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    sample = (0, 1, 2, 37, 98, 99)
    got = {g: [] for g in sample}
    for _ in range(2):
        pool.generate(reqs, out)
        torch.cuda.synchronize()
        o = as_u32(out)
        for g in sample:
            off = reqs[g][3]
            got[g].append(o[off:off + n].copy())
    assert pool.errors() == 0
    for g in sample:
        outs, st = oracle_stream(gens[g], [(g % 3, n), (g % 3, n)])
        for mine, ref in zip(got[g], outs):
            assert np.array_equal(mine, ref), g
        assert np.array_equal(pool.read_state(g), st), g
        assert pool.position(g) == 2 * n


def test_split_and_unsplit_calls_interleave():
    gens = _gens([44497, 11213])
    pool = lib_pool(gens)
    segs = {0: [], 1: []}
    outs_all = {0: [], 1: []}
    for pieces, n in ((1, 30000), (16, 70001), (0, 5000), (4, 1 << 16)):
        pool.set_config(pieces=pieces, piece_log2=10)
        reqs, total = _blocked([(0, 2, n), (1, 0, n + 3)])
        out = torch.zeros(total, dtype=torch.int32, device="cuda")
        pool.generate(reqs, out)
        torch.cuda.synchronize()
        got = as_u32(out)
        for g, dt, m, off in reqs:
            segs[g].append((dt, m))
            outs_all[g].append(got[off:off + m].copy())
    for g in (0, 1):
        ref, st = oracle_stream(gens[g], segs[g])
        for a, b in zip(outs_all[g], ref):
            assert np.array_equal(a, b)
        assert np.array_equal(pool.read_state(g), st)


def test_pieces_of_a_state_too_large_for_the_fused_jump():
    """mexp 86243 (N = 2696): the walked sequence does not fit in shared
    memory, so the jump runs as the walk and sum kernels over a scratch."""
    gens = _gens([86243, 11213])
    reqs, total = _blocked([(0, 0, 300000), (1, 2, 50000)])
    pool = lib_pool(gens)
    pool.set_config(pieces=3, piece_log2=10, threads=512)     # rounds of 2328 words
    before = pool.launch_count()
    out = torch.zeros(total, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    assert pool.launch_count() - before == 3
    _check(gens, reqs, as_u32(out), pool)


@pytest.mark.parametrize("mexp", [521, 11213, 23209, 44497, 86243])
def test_explicit_jump_lands_on_the_oracle_state(mexp):
    gens = _gens([mexp, mexp], seed0=mexp % 97)
    threads = 512 if mexp > 50000 else 128
    pool = lib_pool(gens)
    pool.set_config(threads=threads)
    for J in (1, 2, 3, 1000, 123457):
        p, st = oracle_state(gens[0])
        O.generate(p, st, J, 0)                      # oracle state after J outputs
        pool2 = lib_pool(gens)
        pool2.set_config(threads=threads)
        pool2.jump(0, J)
        assert pool2.position(0) == J
        assert np.array_equal(pool2.read_state(0), st), J
        out = torch.zeros(5000, dtype=torch.int32, device="cuda")
        pool2.generate([(0, 1, 5000, 0)], out)
        torch.cuda.synchronize()
        assert np.array_equal(as_u32(out), O.generate(p, st, 5000, 1))
        pool2.close()
    # jumps compose with generation on the same generator
    p, st = oracle_state(gens[1])
    pool.jump(1, 777)
    out = torch.zeros(3000, dtype=torch.int32, device="cuda")
    pool.generate([(1, 0, 3000, 0)], out)
    pool.jump(1, 1 << 20)
    pool.generate([(1, 2, 1000, 0)], out)
    torch.cuda.synchronize()
    O.generate(p, st, 777, 0)
    O.generate(p, st, 3000, 0)
    O.generate(p, st, 1 << 20, 0)
    assert np.array_equal(as_u32(out)[:1000], O.generate(p, st, 1000, 2))
    assert pool.position(1) == 777 + 3000 + (1 << 20) + 1000


def test_state_api_jump():
    import paper_1005_4973_gb300 as M
    spec = WL.GenSpec(11213, 9, 3, 3, 77)
    s = M.State(M.mtgp_params_draw(spec.mexp, spec.param_seed, spec.id), spec.gen_id, spec.seed)
    s.jump(50000)
    out = torch.zeros(2048, dtype=torch.int32, device="cuda")
    s.generate(0, out, 2048)
    torch.cuda.synchronize()
    p, st = oracle_state(spec)
    O.generate(p, st, 50000, 0)
    assert np.array_equal(as_u32(out), O.generate(p, st, 2048, 0))
    assert s.position() == 52048


@pytest.mark.parametrize("mexp", [521, 1279, 11213])
def test_annihilator_annihilates_the_oracle_sequence(mexp):
    """Every output bit is a linear functional of the state (Sec. 3.3), so
    sum_j psi_j o_{k+j} = 0 (XOR of 32-bit outputs) for every k."""
    gens = _gens([mexp], seed0=mexp % 31)
    pool = lib_pool(gens)
    psi = pool.annihilator(0)
    assert psi[-1] == 1 and 1 <= psi.size - 1 <= mexp
    p, st = oracle_state(gens[0])
    L = psi.size - 1
    o = O.generate(p, st, L + 600, 0)
    sel = np.nonzero(psi)[0]
    for k in range(0, 600, 7):
        assert np.bitwise_xor.reduce(o[k + sel]) == 0, k
    # it belongs to the stream: still valid after generating and after a jump
    out = torch.zeros(100000, dtype=torch.int32, device="cuda")
    pool.generate([(0, 0, 100000, 0)], out)
    assert np.array_equal(pool.annihilator(0), psi)


def test_checkpoint_load_forgets_annihilators():
    gens = _gens([11213, 23209])
    pool = lib_pool(gens)
    blob = pool.save()
    pool.set_config(pieces=4, piece_log2=10)
    out = torch.zeros(200000, dtype=torch.int32, device="cuda")
    pool.generate([(0, 0, 100000, 0), (1, 0, 100000, 100000)], out)
    pool.load(blob)                                  # back to the seeded states
    pool.generate([(0, 0, 100000, 0), (1, 0, 100000, 100000)], out)
    torch.cuda.synchronize()
    reqs = [(0, 0, 100000, 0), (1, 0, 100000, 100000)]
    _check(gens, reqs, as_u32(out), pool)


def test_searched_full_period_set_on_the_gpu():
    """A set from the Sec. 5 search (mexp 4423): its generation matches the
    oracle, and the annihilator the GPU walk finds for a seeded state is the
    searched characteristic polynomial itself (irreducible, so every nonzero
    state has it)."""
    import paper_1005_4973_gb300 as M
    p, seed, _, phi = M.mtgp_params_search(4423, 1, 0)
    pool = M.Pool([p, p], [0, 1], [77, 78])
    pool.set_config(pieces=4, piece_log2=12)
    assert np.array_equal(pool.annihilator(0), phi)
    assert np.array_equal(pool.annihilator(1), phi)
    out = torch.zeros(100000, dtype=torch.int32, device="cuda")
    pool.generate([(0, 2, 100000, 0)], out)
    torch.cuda.synchronize()
    op = O.params_draw(4423, seed, 0)
    st = O.seed_state(op, 0, 77)
    assert np.array_equal(as_u32(out), O.generate(op, st, 100000, 2))
    assert np.array_equal(pool.read_state(0), st)


def test_autotune_leaves_streams_untouched_and_keeps_parity():
    """mtgp_autotune times candidate configurations (forms, block sizes,
    persistence, pieces on/off) and restores every state afterwards: the
    positions are back to zero and the next call under the chosen
    configuration still equals the oracle."""
    gens = _gens([11213, 23209, 521])
    reqs, total = _blocked([(0, 0, 200000), (1, 2, 150000), (2, 1, 90000)])
    pool = lib_pool(gens)
    scratch = torch.zeros(total, dtype=torch.int32, device="cuda")
    best, ms, layout = pool.autotune(reqs, scratch)
    assert ms > 0 and best.threads in (32, 64, 96, 128, 192, 256, 512, 1024) and best.pieces in (0, 1)
    assert layout == 0 and best.form in (0, 1, 2, 3, 4)
    assert [pool.position(g) for g in range(3)] == [0, 0, 0]
    out = torch.zeros(total, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    _check(gens, reqs, as_u32(out), pool)


def test_pool_call_on_a_stream_under_capture_is_refused():
    """A pool call on a stream that the caller is capturing into a CUDA graph
    is refused before it touches the stream (its work list would be copied
    from a buffer that later calls reuse); the pool is unchanged, the next
    call continues the streams exactly, and no error is left behind for the
    next launch."""
    from paper_1005_4973_gb300 import mtgp as L
    gens = _gens([11213, 521])
    pool = lib_pool(gens)
    pool.set_config(pieces=4, piece_log2=10)
    reqs, total = _blocked([(0, 0, 40000), (1, 2, 30000)])
    out = torch.zeros(total, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    pool.generate(reqs, out, stream=s)
    s.synchronize()
    first = as_u32(out).copy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        with pytest.raises(L.MTGPError, match="captur"):
            pool.generate(reqs, out, stream=s)
        with pytest.raises(L.MTGPError, match="captur"):
            pool.jump(0, 1000, stream=s)
        torch.zeros(4, device="cuda").add_(1)        # keeps the captured graph non-empty
    assert [pool.position(i) for i in range(2)] == [40000, 30000]
    pool.generate(reqs, out, stream=s)
    s.synchronize()
    second = as_u32(out).copy()
    for g_, (dt, n, off) in ((0, (0, 40000, 0)), (1, (2, 30000, 40000))):
        ref, _ = oracle_stream(gens[g_], [(dt, n), (dt, n)])
        assert np.array_equal(first[off:off + n], ref[0])
        assert np.array_equal(second[off:off + n], ref[1])
    fresh = lib_pool(gens)                           # a launch right after reports itself only
    fresh.generate(reqs, out)
    torch.cuda.synchronize()


def test_autotune_picks_a_layout_and_the_output_follows_it():
    """With the interleaved layout allowed (equal lengths, distinct
    generators) the autotuner returns the layout it timed fastest, with its
    chunk in the configuration; generating in that layout equals the oracle."""
    gens = _gens([11213, 11213, 23209, 11213])
    n = 1 << 16
    reqs = [(g, g % 3, n, g * n) for g in range(4)]
    pool = lib_pool(gens)
    scratch = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    best, ms, layout = pool.autotune(reqs, scratch, layouts=3)
    assert layout in (0, 1) and ms > 0
    assert [pool.position(g) for g in range(4)] == [0, 0, 0, 0]
    out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out, layout=layout)
    torch.cuda.synchronize()
    o = as_u32(out)
    c = best.chunk
    for j, (g, dt, nn, off) in enumerate(reqs):
        p, st = oracle_state(gens[g])
        ref = O.generate(p, st, nn, dt)
        if layout == 0:
            assert np.array_equal(o[off:off + nn], ref)
        else:
            idx = np.arange(nn)
            assert np.array_equal(o[(idx // c) * (4 * c) + j * c + idx % c], ref)
