"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every output is an exact integer or float bit pattern, so every comparison is
bit-exact (the method's arithmetic is integer; the one float subtraction of
Sec. 6 is exact).  Small cases compare everything; full-size cases compare
sampled generators in full, every generator's prefix, every final state where
the oracle can afford it, and closed-form relations between dtypes.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1005_4973_gb300 import workloads as WL
from tests.helpers import as_u32, lib_pool, oracle_params, oracle_state, oracle_stream

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1005_4973_gb300 import build
    build.build()
    O.build()
    assert torch.cuda.is_available()


def _run(gens, reqs, layout=0, config=None, total=None):
    pool = lib_pool(gens)
    if config:
        pool.set_config(**config)
    if total is None:
        total = sum(r[2] for r in reqs) if layout == 0 else len(reqs) * (reqs[0][2] if reqs else 0)
    out = torch.full((max(total, 1),), 0xA5, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out, layout=layout)
    torch.cuda.synchronize()
    return pool, as_u32(out)[:total]


def _check_blocked(gens, reqs, out, pool=None):
    by_gen = {}
    for g, dt, n, off in reqs:
        by_gen.setdefault(g, []).append((dt, n, off))
    for g, segs in by_gen.items():
        outs, st = oracle_stream(gens[g], [(dt, n) for dt, n, _ in segs])
        for (dt, n, off), ref in zip(segs, outs):
            assert np.array_equal(out[off:off + n], ref), (gens[g], dt, n)
        if pool is not None:
            assert np.array_equal(pool.read_state(g), st), gens[g]
            assert pool.position(g) == sum(n for _, n, _ in segs)


# ---------------------------------------------------------------- seeding
def test_seed_state_matches_oracle():
    gens = [WL.GenSpec(m, s, s * 7 + 1, gid, seed) for m in (89, 11213, 23209, 44497)
            for s, gid, seed in ((1, 0, 1234), (2, 5, 0), (3, 2**31, 2**63 + 17))]
    pool = lib_pool(gens)
    for i, g in enumerate(gens):
        _, st = oracle_state(g)
        assert np.array_equal(pool.read_state(i), st), g
        assert pool.position(i) == 0


# ------------------------------------------------------------------- C1
@pytest.mark.parametrize("dtype", [WL.U32, WL.F12, WL.F01])
def test_c1_full_size_bitexact(dtype):
    wl = WL.c1(dtype=dtype)
    pool, out = _run(wl.gens, wl.requests)
    _check_blocked(wl.gens, wl.requests, out, pool)


# -------------------------------------------------- launch-shape sweep
MIXED = [WL.GenSpec(11213, 1, 0, 0), WL.GenSpec(23209, 2, 1, 1), WL.GenSpec(44497, 3, 2, 2),
         WL.GenSpec(521, 4, 3, 3), WL.GenSpec(89, 5, 4, 4), WL.GenSpec(1279, 6, 5, 5),
         WL.GenSpec(11213, 7, 0xFFFF0001, 6, 99)]
RAGGED = [1, 31, 33, 255, 257, 1000, 4097, 12345]


def _round_size(spec):
    p = oracle_params(spec)
    return p.N - p.pos


FORMS = [(32, 0), (64, 0), (128, 0), (256, 0), (512, 0), (128, 1), (256, 1), (512, 1), (1024, 1),
         (128, 2), (256, 2), (512, 2), (1024, 2), (128, 4)]
FORM_ID = lambda f: f"{f[0]}{'psfwq'[f[1]]}"


def _need(p, threads, fm):
    """Smallest buffer_words for parameter set p (see mtgp_config.buffer_words)."""
    owners = _owners(threads, fm)
    S = p.N - p.pos
    nq = -(-S // owners)
    return 2 * p.N + 2 * S + 32 * nq + 32 if fm == 2 else 2 * p.N + nq * owners + 32


def _owners(threads, form):
    """Columns one slot covers: a column per thread (plain), per thread of the
    recursion half (split, flow), two per thread (pairs)."""
    return 2 * threads if form == 4 else threads // 2 if form else threads


def _max_slots(threads, form):
    from paper_1005_4973_gb300._lib import MAX_SLOTS, MAX_SLOTS_FLOW, MAX_SLOTS_PAIRS, MAX_SLOTS_SPLIT
    return (MAX_SLOTS_SPLIT if form == 1 else MAX_SLOTS_FLOW if form == 2 else MAX_SLOTS_PAIRS if form == 4
            else MAX_SLOTS)[threads]


@pytest.mark.parametrize("form", FORMS, ids=FORM_ID)
@pytest.mark.parametrize("persistent", [0, 1])
def test_launch_shapes(form, persistent):
    threads, fm = form
    gens = [g for g in MIXED if _round_size(g) <= _owners(threads, fm) * _max_slots(threads, fm)]
    reqs, off = [], 0
    for g in range(len(gens)):
        for k, n in enumerate(RAGGED[g % 3::3] + [RAGGED[(g + 1) % len(RAGGED)]]):
            reqs.append((g, (g + k) % 3, n, off))
            off += n
    # persistent: one block per SM, so that the blocks pull several items from
    # the work counter (with blocks_per_sm = 0 a launch whose items fit in one
    # wave runs one block per item)
    cfg = dict(threads=threads, form=fm, persistent=persistent, blocks_per_sm=persistent)
    pool, out = _run(gens, reqs, config=cfg)
    _check_blocked(gens, reqs, out, pool)


@pytest.mark.parametrize("form", FORMS, ids=FORM_ID)
def test_every_slot_count(form):
    """Generators whose round size S = N - M needs each slot count 1 .. max:
    synthetic sets with M chosen to hit S = owners q and S = owners q - 31
    (fullest and emptiest last slot)."""
    import paper_1005_4973_gb300 as M
    threads, fm = form
    owners = _owners(threads, fm)
    ps, ops, n = [], [], 3001
    for q in range(1, _max_slots(threads, fm) + 1):
        for S in sorted({owners * q, max(1, owners * q - 31)}):
            N = S + 2 + (q % 5)
            mexp = 32 * N - 17
            if N > 4096:
                continue
            lp = M.mtgp_params_draw(mexp, q, q)
            o = O.params_draw(mexp, q, q)
            lp.pos = N - S
            ops.append(O.params_from_fields(mexp, N - S, o.sh1, o.sh2, q, list(o.R), list(o.T)))
            ps.append(lp)
    pool = M.Pool(ps, list(range(len(ps))), [11] * len(ps))
    pool.set_config(threads=threads, form=fm)
    out = torch.zeros(n * len(ps), dtype=torch.int32, device="cuda")
    pool.generate([(i, i % 3, n, i * n) for i in range(len(ps))], out)
    o = as_u32(out)
    for i, op in enumerate(ops):
        st = O.seed_state(op, i, 11)
        assert np.array_equal(o[i * n:(i + 1) * n], O.generate(op, st, n, i % 3)), (op.N, op.pos)
        assert np.array_equal(pool.read_state(i), st)


@pytest.mark.parametrize("tail", [1, 5, 31, 33, 97])
def test_flow_partial_last_round_with_idle_warps(tail):
    # 1024-thread flow blocks give a 300-word round to ten 32-column warps; a
    # final round of `tail` words leaves most of them without a column, and
    # their output warps must neither route nor store anything for it
    g = [WL.GenSpec(11213, 1, 0, 0)]
    S = _round_size(g[0])
    n1, n2 = 7 * S + tail, 3 * S + tail
    reqs = [(0, 0, n1, 0), (0, 2, n2, n1)]
    pool, out = _run(g, reqs, config=dict(threads=1024, form=2))
    _check_blocked(g, reqs, out, pool)


@pytest.mark.parametrize("extra", [0, 1, 7, 300, 2000])
@pytest.mark.parametrize("form", [(128, 0), (256, 1), (256, 2), (1024, 2), (128, 4)], ids=FORM_ID)
def test_small_buffers_force_compaction(extra, form):
    # buffer_words at (or just above) its minimum: compaction every round or
    # few rounds (split form: every compaction drains the hand-off ring; flow
    # form: every epoch ends at a block barrier)
    threads, fm = form
    gens = MIXED[:3]
    ps = [oracle_params(g) for g in gens]
    need = max(_need(p, threads, fm) for p in ps)
    reqs = [(g, g % 3, 20011, 20011 * g) for g in range(3)]
    reqs += [(g, (g + 1) % 3, 777, 60033 + 777 * g) for g in range(3)]
    pool, out = _run(gens, reqs, config=dict(threads=threads, form=fm, buffer_words=need + extra))
    _check_blocked(gens, reqs, out, pool)


def test_too_small_buffer_rejected():
    import paper_1005_4973_gb300 as M
    pool = lib_pool(MIXED[:1])
    p = oracle_params(MIXED[0])
    pool.set_config(buffer_words=2 * p.N + -(-(p.N - p.pos) // 128) * 128 + 31)
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MTGPError):
        pool.generate([(0, 0, 16, 0)], out)
    pool.set_config(buffer_words=0, threads=32)
    # S > 32 x 11: no 32-thread kernel; the plain form runs the launch with the
    # next block size that has one, and the output is the oracle's
    big = lib_pool([MIXED[2]])
    big.set_config(threads=32)
    out2 = torch.zeros(5000, dtype=torch.int32, device="cuda")
    big.generate([(0, 0, 5000, 0)], out2)
    p2, st2 = oracle_state(MIXED[2])
    assert np.array_equal(as_u32(out2), O.generate(p2, st2, 5000, 0))
    big.set_config(threads=128, form=5)             # the dual form has no kernel for these rounds
    with pytest.raises(M.MTGPError):
        big.generate([(0, 0, 16, 0)], out)


@pytest.mark.parametrize("form", [(128, 0), (128, 4)], ids=FORM_ID)
def test_random_shift_sets(form):
    # sh1, sh2 over [1, 31] exercise every shift path; the shift values are
    # recipe inputs (numpy RNG) applied to each side's own drawn set.
    import paper_1005_4973_gb300 as M
    rng = np.random.default_rng(5)
    shifts = rng.integers(1, 32, size=(8, 2))
    ps, ops = [], []
    for s in range(8):
        mexp = 11213 if s % 2 else 23209
        lp = M.mtgp_params_draw(mexp, 100 + s, s)
        lp.sh1, lp.sh2 = int(shifts[s, 0]), int(shifts[s, 1])
        M.mtgp_params_validate(lp)
        o = O.params_draw(mexp, 100 + s, s)
        ops.append(O.params_from_fields(mexp, o.pos, int(shifts[s, 0]), int(shifts[s, 1]), s, list(o.R), list(o.T)))
        ps.append(lp)
    pool = M.Pool(ps, list(range(8)), [7] * 8)
    pool.set_config(threads=form[0], form=form[1])
    reqs = [(i, i % 3, 7777, i * 7777) for i in range(8)]
    out = torch.zeros(8 * 7777, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    o = as_u32(out)
    for i, op in enumerate(ops):
        st = O.seed_state(op, i, 7)
        assert np.array_equal(o[i * 7777:(i + 1) * 7777], O.generate(op, st, 7777, i % 3)), shifts[i]


# ------------------------------------------------------------ edge cases
def test_zero_length_and_empty():
    pool = lib_pool(MIXED[:2])
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    pool.generate([], out)
    pool.generate([(0, 0, 0, 0), (1, 2, 0, 0)], out)
    torch.cuda.synchronize()
    assert pool.position(0) == 0 and pool.position(1) == 0
    assert not out.any()


@pytest.mark.parametrize("splits", [(1, 1, 1), (255, 257, 31), (351, 352), (1000, 1, 4097), (65536, 3)])
def test_continuation_across_calls(splits):
    g = WL.GenSpec(11213, 9, 9, 9)
    pool = lib_pool([g])
    parts = []
    for k, n in enumerate(splits):
        out = torch.zeros(n, dtype=torch.int32, device="cuda")
        pool.generate([(0, k % 3, n, 0)], out)
        parts.append(as_u32(out))
    outs, st = oracle_stream(g, [(k % 3, n) for k, n in enumerate(splits)])
    for a, b in zip(parts, outs):
        assert np.array_equal(a, b)
    assert np.array_equal(pool.read_state(0), st)


def test_same_generator_many_requests_in_one_call():
    g = [WL.GenSpec(23209, 4, 4, 4), WL.GenSpec(11213, 5, 5, 5)]
    reqs = [(0, 0, 100, 0), (1, 1, 50, 100), (0, 2, 3000, 150), (0, 1, 1, 3150), (1, 0, 999, 3151)]
    pool, out = _run(g, reqs)
    _check_blocked(g, reqs, out, pool)


@pytest.mark.parametrize("chunk", [32, 256, 4096])
def test_interleaved_layout(chunk):
    gens = [WL.GenSpec(11213 if i % 2 else 44497, i + 1, i, i) for i in range(5)]
    n = 3 * chunk + 17
    reqs = [(i, i % 3, n, 0) for i in range(5)]
    pool = lib_pool(gens)
    pool.set_config(chunk=chunk)
    total = 5 * n + 5 * chunk
    out = torch.zeros(total, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out, layout=1)
    torch.cuda.synchronize()
    o = as_u32(out)
    for j, g in enumerate(gens):
        (ref,), _ = oracle_stream(g, [(j % 3, n)])
        k = np.arange(n)
        idx = (k // chunk) * (5 * chunk) + j * chunk + k % chunk
        assert np.array_equal(o[idx], ref)


def test_bad_requests_rejected():
    import paper_1005_4973_gb300 as M
    pool = lib_pool(MIXED[:2])
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    for reqs, layout in (([(2, 0, 4, 0)], 0), ([(0, 3, 4, 0)], 0), ([(0, 0, 4, 0), (1, 0, 5, 0)], 1),
                         ([(0, 0, 4, 0), (0, 0, 4, 0)], 1)):
        with pytest.raises(M.MTGPError):
            pool.generate(reqs, out, layout=layout)
    with pytest.raises(M.MTGPError):
        pool.set_config(threads=48)
    with pytest.raises(M.MTGPError):
        pool.set_config(threads=1024)
    with pytest.raises(M.MTGPError):
        pool.set_config(chunk=100)


# ------------------------------------------------------ checkpoint / e2e
def test_checkpoint_save_load():
    gens = MIXED[:3]
    pool = lib_pool(gens)
    out = torch.zeros(3 * 5000, dtype=torch.int32, device="cuda")
    pool.generate([(i, 0, 5000, 5000 * i) for i in range(3)], out)
    blob = pool.save()
    pool.generate([(i, 1, 5000, 5000 * i) for i in range(3)], out)
    first = as_u32(out).copy()
    pool.load(blob)
    pool.generate([(i, 1, 5000, 5000 * i) for i in range(3)], out)
    assert np.array_equal(as_u32(out), first)
    for i, g in enumerate(gens):
        outs, st = oracle_stream(g, [(0, 5000), (1, 5000)])
        assert np.array_equal(first[5000 * i:5000 * (i + 1)], outs[1])
        assert pool.position(i) == 10000


def test_state_object_and_checkpoint():
    import paper_1005_4973_gb300 as M
    g = WL.GenSpec(11213, 1, 0, 0)
    s = M.State(M.mtgp_params_draw(g.mexp, g.param_seed, g.id), g.gen_id, g.seed)
    out = torch.zeros(70000, dtype=torch.int32, device="cuda")
    s.generate(0, out, 30000)
    blob = s.save()
    s.generate(2, out[30000:], 40000)
    torch.cuda.synchronize()
    full = as_u32(out).copy()
    assert s.position() == 70000
    outs, _ = oracle_stream(g, [(0, 30000), (2, 40000)])
    assert np.array_equal(full, np.concatenate(outs))
    s.load(blob)
    s.generate(2, out, 40000)
    assert np.array_equal(as_u32(out)[:40000], outs[1])


def test_generate_host_end_to_end():
    gens = MIXED[:4]
    reqs = [(0, 0, 300000, 0), (1, 2, 123457, 300000), (2, 1, 5, 423457), (3, 0, 77777, 423462)]
    pool = lib_pool(gens)
    host = torch.zeros(501239, dtype=torch.int32).pin_memory()
    pool.generate_host(reqs, host, staging_bytes=1 << 18)      # forces many slices
    o = host.numpy().view(np.uint32)
    _check_blocked(gens, reqs, o, pool)


# ------------------------------------------- reduced exponents, full period
def test_full_period_sets_on_gpu():
    import paper_1005_4973_gb300 as M
    with open(os.path.join(GOLDEN, "full_period_sets.json")) as f:
        sets = json.load(f)["sets"]
    ps, ops = [], []
    for d in sets:
        ops.append(O.params_from_fields(d["mexp"], d["pos"], d["sh1"], d["sh2"], d["id"], d["R"], d["T"]))
        ps.append(M.mtgp_params_draw(d["mexp"], d["param_seed"], d["id"]))
    pool = M.Pool(ps, list(range(len(ps))), [3] * len(ps))
    n = 20011
    out = torch.zeros(n * len(ps), dtype=torch.int32, device="cuda")
    pool.generate([(i, i % 3, n, i * n) for i in range(len(ps))], out)
    o = as_u32(out)
    for i, op in enumerate(ops):
        st = O.seed_state(op, i, 3)
        assert np.array_equal(o[i * n:(i + 1) * n], O.generate(op, st, n, i % 3)), sets[i]["mexp"]


# ----------------------------------------------------- full-size configs
def _oracle_final_states(gens, n, dtype, nthreads=None, rows=None):
    """Oracle streams of many generators in chunks; returns final states and
    the first `keep` outputs of each.  With rows (a device tensor, one row per
    generator) every stream is also compared with its row in full."""
    keep = 1 << 16
    states, heads = [], []
    batch = 8
    for b in range(0, len(gens), batch):
        ps, sts = [], []
        for g in gens[b:b + batch]:
            p, st = oracle_state(g)
            ps.append(p)
            sts.append(st)
        outs = O.generate_many(ps, sts, [n] * len(ps), [dtype] * len(ps), nthreads)
        if rows is not None:
            got = as_u32(rows[b:b + len(ps)])
            for k, o in enumerate(outs):
                if not np.array_equal(got[k], o):
                    bad = np.nonzero(got[k] != o)[0]
                    raise AssertionError(f"generator {b + k}: {bad.size} outputs differ, first at {bad[0]}")
        states += sts
        heads += [o[:keep].copy() for o in outs]
        del outs
    return states, heads


def test_c2_full_size():
    """C2: 128 sets x 2^24 x {u32, f12, f01}, the bench's launch (default
    configuration: each instance split into jump-ahead pieces).  Every uint32
    stream is compared in full; the float runs by the Sec. 6 closed forms."""
    wl = WL.c2()
    n = 1 << 24
    pool = lib_pool(wl.gens)
    out = torch.empty(wl.total_numbers, dtype=torch.int32, device="cuda")
    pool.generate(wl.requests, out)
    torch.cuda.synchronize()
    u = out[: 128 * n].view(128, n)
    f12 = out[128 * n: 256 * n].view(128, n)
    f01 = out[256 * n:].view(128, n)
    # Sec. 6 closed forms relate the three runs of each set at full size
    assert torch.equal(f12, (u >> 9) & 0x7FFFFF | 0x3F800000)
    ff = f12.view(torch.float32) - 1.0
    assert torch.equal(f01.view(torch.float32), ff)
    # every uint32 stream in full, every final state, against the oracle
    states, heads = _oracle_final_states(wl.gens[:128], n, WL.U32, rows=u)
    for i in range(128):
        assert np.array_equal(pool.read_state(i), states[i]), i
        assert np.array_equal(pool.read_state(256 + i), states[i]), i
        assert pool.position(i) == n


@pytest.mark.parametrize("mexp", [23209, 44497])
def test_c3_full_size(mexp):
    wl = WL.c3(mexps=(mexp,))
    n = 1 << 26
    pool = lib_pool(wl.gens)
    out = torch.empty(wl.total_numbers, dtype=torch.int32, device="cuda")
    pool.generate(wl.requests, out)
    torch.cuda.synchronize()
    f = out.view(128, n)
    fv = f.view(torch.float32)
    assert float(fv.min()) >= 0.0 and float(fv.max()) < 1.0
    # f01 * 2^23 is an exact integer < 2^23
    assert torch.equal(torch.floor(fv * 8388608.0), fv * 8388608.0)
    heads_ref = []
    for i in range(128):
        p, st = oracle_state(wl.gens[i])
        heads_ref.append(O.generate(p, st, 1 << 14, WL.F01))
    fh = as_u32(f[:, : 1 << 14])
    for i in range(128):
        assert np.array_equal(fh[i], heads_ref[i]), i
    for i in (5, 100):
        (ref,), st = oracle_stream(wl.gens[i], [(WL.F01, n)])
        assert np.array_equal(as_u32(f[i]), ref)
        assert np.array_equal(pool.read_state(i), st)


@pytest.mark.parametrize("dtype", [WL.U32, WL.F12, WL.F01])
def test_paper_workload_in_full(dtype):
    """Sec. 4.4's workload (5e7 numbers from 108 MTGP11213 generators) in the
    bench's launch (default configuration, pieces for the idle SMs), every
    output and final state against the oracle."""
    wl = WL.paper(dtype=dtype)
    pool = lib_pool(wl.gens)
    out = torch.empty(wl.total_numbers, dtype=torch.int32, device="cuda")
    pool.generate(wl.requests, out)
    torch.cuda.synchronize()
    got = as_u32(out)
    ps, sts = [], []
    for g in wl.gens:
        p, st = oracle_state(g)
        ps.append(p)
        sts.append(st)
    refs = O.generate_many(ps, sts, [r[2] for r in wl.requests], [dtype] * len(ps))
    for (g, _, n, off), ref in zip(wl.requests, refs):
        assert np.array_equal(got[off:off + n], ref), g
        assert np.array_equal(pool.read_state(g), sts[g]), g


def test_c4_batched_sampled():
    """C4: 8192 generators, mixed exponents, log-uniform lengths, in the
    persistent longest-first launch; sampled generators in full, all prefixes."""
    wl = WL.c4()
    pool = lib_pool(wl.gens)
    pool.set_config(persistent=1)
    out = torch.empty(wl.total_numbers, dtype=torch.int32, device="cuda")
    pool.generate(wl.requests, out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    sample = sorted(set(rng.integers(0, 8192, 24).tolist()) | {int(np.argmax([r[2] for r in wl.requests]))})
    for g in sample:
        _, dt, n, off = wl.requests[g]
        (ref,), st = oracle_stream(wl.gens[g], [(dt, n)])
        assert np.array_equal(as_u32(out[off:off + n]), ref), g
        assert np.array_equal(pool.read_state(g), st), g
    for g in range(0, 8192, 16):
        _, dt, n, off = wl.requests[g]
        k = min(n, 1024)
        p, st = oracle_state(wl.gens[g])
        assert np.array_equal(as_u32(out[off:off + k]), O.generate(p, st, k, dt)), g


def test_flow_form_bounded_wait_runs_out_and_reports():
    """The flow form's waits between warps are bounded.  With a limit of two
    polls some wait runs out: the launch still ends, bit 1 of the error word
    (a wait ran out) comes back, and the next launch with the default limit
    continues bit-exact on the same pool (the context stays usable)."""
    g = [WL.GenSpec(11213, 1, 0, 0)]
    pool = lib_pool(g)
    pool.set_config(threads=256, form=2)
    out = torch.zeros(1 << 18, dtype=torch.int32, device="cuda")
    pool.set_spin_limit(2)
    pool.generate([(0, 0, 1 << 18, 0)], out)
    torch.cuda.synchronize()
    assert pool.errors() & 2
    pool.set_spin_limit(0)
    p, st = oracle_state(g[0])
    fresh = lib_pool(g)                                  # the failed call's state is unspecified
    fresh.set_config(threads=256, form=2)
    fresh.generate([(0, 1, 4097, 0)], out)
    torch.cuda.synchronize()
    assert fresh.errors() == 0
    assert np.array_equal(as_u32(out)[:4097], O.generate(p, st, 4097, 1))
    pool.generate([(0, 0, 1000, 0)], out)               # the first pool also runs again, without errors
    torch.cuda.synchronize()
    assert pool.errors() == 0


def test_more_than_2_32_numbers_in_one_request():
    """One request of 2^32 + 12345 numbers (16 GiB of output, split into
    jump-ahead pieces): positions, output offsets and the state write-back
    past 32 bits.  The last 2^20 numbers and the final state equal the
    oracle's, which generates the whole stream in 2^28-number parts."""
    n = (1 << 32) + 12345
    g = WL.GenSpec(11213, 21, 21, 21)
    pool = lib_pool([g])
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    pool.generate([(0, WL.U32, n, 0)], out)
    torch.cuda.synchronize()
    tail = as_u32(out[n - (1 << 20):])
    head = as_u32(out[:4096])
    del out
    torch.cuda.empty_cache()
    p, st = oracle_state(g)
    first = O.generate(p, st, 4096, WL.U32)
    left = n - 4096
    while left > (1 << 20):
        k = min(1 << 28, left - (1 << 20))
        O.generate(p, st, k, WL.U32)
        left -= k
    last = O.generate(p, st, left, WL.U32)
    assert np.array_equal(head, first)
    assert np.array_equal(tail, last)
    assert np.array_equal(pool.read_state(0), st)
    assert pool.position(0) == n


@pytest.mark.parametrize("pieces", [1, 0])
def test_zero_state_is_a_fixed_point(pieces):
    """The degenerate case of the recursion: a state whose p effective bits
    are all zero (here with the r bits the mask drops set in x_0) is a fixed
    point; loaded from a checkpoint it generates zero words, 1.0f and 0.0f, as
    the oracle does, with and without jump-ahead pieces."""
    import paper_1005_4973_gb300 as M
    gens = [WL.GenSpec(11213, 31, 31, 31), WL.GenSpec(23209, 32, 32, 32)]
    pool = lib_pool(gens)
    pool.set_config(pieces=pieces)
    blob = bytearray(pool.save())
    nst = sum((oracle_params(g).N + 3) & ~3 for g in gens)   # states start 16-byte aligned
    words = np.frombuffer(blob, dtype=np.uint32, count=nst, offset=len(blob) - 4 * nst).copy()
    ops, off = [], 0
    for g in gens:
        p = oracle_params(g)
        words[off:off + p.N] = 0
        words[off] = ~np.uint32(p.mask)                  # bits outside the p effective ones
        ops.append((p, words[off:off + p.N].copy()))
        off += (p.N + 3) & ~3
    blob[len(blob) - 4 * nst:] = words.tobytes()
    pool.load(bytes(blob))
    n = 1 << 20
    reqs = [(0, WL.U32, n, 0), (1, WL.F12, n, n), (0, WL.F01, n, 2 * n)]
    out = torch.full((3 * n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    torch.cuda.synchronize()
    got = as_u32(out)
    assert pool.errors() == 0
    st0, st1 = ops[0][1].copy(), ops[1][1].copy()
    ref = [O.generate(ops[0][0], st0, n, WL.U32), O.generate(ops[1][0], st1, n, WL.F12),
           O.generate(ops[0][0], st0, n, WL.F01)]
    assert not ref[0].any() and (ref[1] == 0x3F800000).all() and not ref[2].any()
    for (g, dt, k, o), r in zip(reqs, ref):
        assert np.array_equal(got[o:o + k], r), (g, dt)


@pytest.mark.parametrize("pieces", [0, 1])
def test_largest_exponents_with_the_default_configuration(pieces):
    """MTGP86243 and MTGP110503 (N = 2696 and 3454: rounds longer than the
    128-thread kernels cover) generate with the default configuration (the
    plain form moves to a larger block size), mixed with an MTGP11213
    generator, over two calls, with jump-ahead pieces (the few-item rule
    splits these launches) and without, and match the oracle."""
    gens = [WL.GenSpec(86243, 3, 3, 3), WL.GenSpec(110503, 4, 4, 4), WL.GenSpec(11213, 5, 5, 5)]
    pool = lib_pool(gens)
    pool.set_config(pieces=pieces)
    spec = [(0, WL.U32, 300001), (1, WL.F01, 250003), (2, WL.F12, 99999), (1, WL.U32, 7)]
    reqs, off = [], 0
    for g, dt, n in spec:
        reqs.append((g, dt, n, off))
        off += n
    out = torch.full((off,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    pool.generate(reqs, out)
    pool.generate(reqs, out)                             # the second call continues the streams
    torch.cuda.synchronize()
    got = as_u32(out)
    sts = {g: oracle_state(gens[g]) for g in range(3)}
    for rep in range(2):
        for g, dt, n, o in reqs:
            p, st = sts[g]
            ref = O.generate(p, st, n, dt)
            if rep == 1:
                assert np.array_equal(got[o:o + n], ref), (g, dt, n)
    for g in range(3):
        assert np.array_equal(pool.read_state(g), sts[g][1])
