"""Batched and served forms (§8 row a9) against the oracle: the graph-captured
persistent launch replayed with changing work lists, and the continuous-
batching server.  A served result must equal what the same generator's
requests give alone, in submission order."""
import numpy as np
import pytest

import oracle as O
from paper_1005_4973_gb300 import workloads as WL
from tests.helpers import as_u32, lib_pool, oracle_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GENS = [WL.GenSpec([11213, 23209, 44497, 521][i % 4], i + 1, i, i, 100 + i) for i in range(12)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1005_4973_gb300 import build
    build.build()
    O.build()


def _oracle_streams(gens, per_gen):
    """per_gen[g] = list of (dtype, n) in order -> list of outputs per request."""
    res = {}
    for g, segs in per_gen.items():
        p, st = oracle_state(gens[g])
        res[g] = [O.generate(p, st, n, dt) for dt, n in segs]
    return res


@pytest.mark.parametrize("form", [(128, 0), (256, 1), (256, 2), (128, 4)])
def test_graph_replays_with_changing_work(form):
    """One captured launch, replayed with new work lists (and twice with the
    same list, which continues the streams); every replay's output matches the
    oracle streams of the generators involved, in order."""
    import paper_1005_4973_gb300 as M
    pool = lib_pool(GENS)
    pool.set_config(threads=form[0], form=form[1])
    graph = M.Graph(pool, max_items=len(GENS))
    rng = np.random.default_rng(1)
    launches = []
    for rep in range(4):
        gens = sorted(rng.choice(len(GENS), size=int(rng.integers(1, len(GENS) + 1)), replace=False).tolist())
        reqs, off = [], 0
        for g in gens:
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
    per_gen = {}
    for reqs, _ in launches:
        for g, dt, n, _ in reqs:
            per_gen.setdefault(g, []).append((dt, n))
    ref = _oracle_streams(GENS, per_gen)
    cursor = {g: 0 for g in per_gen}
    for reqs, o in launches:
        for g, dt, n, off in reqs:
            assert np.array_equal(o[off:off + n], ref[g][cursor[g]]), (g, dt, n)
            cursor[g] += 1
    graph.close()


@pytest.mark.parametrize("max_items", [256, None])
def test_graph_replays_with_jump_ahead_pieces(max_items):
    """The captured launch holds a jump kernel (Sec. 7) before the generation
    kernel: long requests run as pieces whose start states each replay
    computes from the generators' current states.  With room for only the
    unsplit items (max_items = None: as many as the largest list), the plan
    falls back to whole items.  Either way every replay matches the oracle
    streams, in order."""
    import paper_1005_4973_gb300 as M
    pool = lib_pool(GENS)
    pool.set_config(pieces=4, piece_log2=10)
    rng = np.random.default_rng(7)
    lists = []
    for rep in range(3):
        gens = sorted(rng.choice(len(GENS), size=int(rng.integers(3, len(GENS) + 1)), replace=False).tolist())
        reqs, off = [], int(rng.integers(0, 4))
        for g in gens:
            n = int(rng.integers(1000, 120000))
            reqs.append((g, int(rng.integers(0, 3)), n, off))
            off += n + int(rng.integers(0, 4))
        lists.append((reqs, off))
    graph = M.Graph(pool, max_items=max_items or max(len(r) for r, _ in lists))
    launches = []
    for rep, (reqs, total) in enumerate(lists):
        out = torch.zeros(total, dtype=torch.int32, device="cuda")
        graph.set_requests(reqs, out)
        for _ in range(1 + rep % 2):
            before = pool.launch_count()
            graph.launch()
            torch.cuda.synchronize()
            assert pool.launch_count() - before == 2          # jump, generation
            launches.append((reqs, as_u32(out).copy()))
    assert graph.errors() == 0
    per_gen = {}
    for reqs, _ in launches:
        for g, dt, n, _ in reqs:
            per_gen.setdefault(g, []).append((dt, n))
    ref = _oracle_streams(GENS, per_gen)
    cursor = {g: 0 for g in per_gen}
    for reqs, o in launches:
        for g, dt, n, off in reqs:
            assert np.array_equal(o[off:off + n], ref[g][cursor[g]]), (g, dt, n)
            cursor[g] += 1
    graph.close()


def test_graph_set_requests_error_empties_the_list():
    """After a failed set_requests the graph's list is empty: a replay then
    writes nothing and advances no stream."""
    import paper_1005_4973_gb300 as M
    pool = lib_pool(GENS[:4])
    pool.set_config(pieces=4, piece_log2=10)
    graph = M.Graph(pool, max_items=64)
    out = torch.zeros(50000, dtype=torch.int32, device="cuda")
    graph.set_requests([(0, 0, 30000, 0), (1, 1, 20000, 30000)], out)
    graph.launch()
    torch.cuda.synchronize()
    pos = [pool.position(i) for i in range(4)]
    assert pos[:2] == [30000, 20000]
    with pytest.raises(M.MTGPError):
        graph.set_requests([(0, 0, 10, 0), (9, 0, 10, 10)], out)     # generator 9 is not in the pool
    out.fill_(7)
    graph.launch()
    torch.cuda.synchronize()
    assert [pool.position(i) for i in range(4)] == pos
    assert bool((out == 7).all())
    graph.close()


def test_pool_load_empties_graph_lists_with_pieces():
    """mtgp_pool_load replaces the states the graph's jump jobs were planned
    for: the graph's list is emptied (a replay writes nothing), and a new
    set_requests continues from the loaded states exactly."""
    import paper_1005_4973_gb300 as M
    gens = GENS[:3]
    pool = lib_pool(gens)
    pool.set_config(pieces=4, piece_log2=10)
    saved = pool.save()
    graph = M.Graph(pool, max_items=64)
    reqs = [(0, 0, 40000, 0), (1, 2, 30000, 40000), (2, 1, 20000, 70000)]
    out = torch.zeros(90000, dtype=torch.int32, device="cuda")
    graph.set_requests(reqs, out)
    graph.launch()
    torch.cuda.synchronize()
    first = as_u32(out).copy()
    pool.load(saved)                                     # back to the seeded states
    out.fill_(7)
    graph.launch()
    torch.cuda.synchronize()
    assert bool((out == 7).all()) and [pool.position(i) for i in range(3)] == [0, 0, 0]
    graph.set_requests(reqs, out)
    graph.launch()
    torch.cuda.synchronize()
    assert np.array_equal(as_u32(out), first)            # the same numbers again from the same states
    graph.close()


class _DevView:
    """Zero-copy int32 view of n words of device memory (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _serve(pool, requests, arena_bytes, chunk, max_active=0, polls_between=0):
    """Submits `requests` (gen, dtype, n), polling between submissions so later
    requests arrive while earlier ones are on the GPU; returns the tickets in
    submission order, {ticket: host array} and the final stats."""
    import paper_1005_4973_gb300 as M
    srv = M.Server(pool, arena_bytes=arena_bytes, chunk=chunk, max_active=max_active)
    tickets, results = [], {}

    def collect(block=False):
        for c in srv.poll(block=block):
            view = torch.as_tensor(_DevView(c.dev_out, c.n), device="cuda")
            results[c.ticket] = view.cpu().numpy().view(np.uint32).copy()
            srv.release(c.ticket)

    for i, (g, dt, n) in enumerate(requests):
        tickets.append(srv.submit(g, dt, n))
        for _ in range(polls_between):
            collect()
    while len(results) < len(tickets):
        collect(block=True)
    stats = srv.stats()
    srv.close()
    return tickets, results, stats


def _check_served(requests, tickets, results):
    per_gen = {}
    for g, dt, n in requests:
        per_gen.setdefault(g, []).append((dt, n))
    ref = _oracle_streams(GENS, per_gen)
    cursor = {g: 0 for g in per_gen}
    for (g, dt, n), t in zip(requests, tickets):
        want = ref[g][cursor[g]]
        cursor[g] += 1
        assert np.array_equal(results[t], want), (g, dt, n)


def _random_requests(seed, count, max_len):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(0, len(GENS))), int(rng.integers(0, 3)), int(rng.integers(1, max_len)))
            for _ in range(count)]


@pytest.mark.parametrize("form", [(128, 0), (256, 2), (128, 4)])
def test_server_mix_equals_alone(form):
    """Requests of 12 generators arrive while others are being generated; every
    result equals the oracle stream of its generator's requests in order."""
    pool = lib_pool(GENS)
    pool.set_config(threads=form[0], form=form[1])
    reqs = _random_requests(7, 60, 70000)
    tickets, results, stats = _serve(pool, reqs, arena_bytes=64 << 20, chunk=4096, polls_between=2)
    _check_served(reqs, tickets, results)
    assert stats["pending"] == 0 and stats["active"] == 0
    assert stats["ticks"] > 1 and stats["numbers_completed"] == sum(r[2] for r in reqs)
    assert stats["arena_free_bytes"] == 64 << 20
    assert pool.errors() == 0


def test_server_admission_by_memory():
    """An arena that holds only a few outputs at once: requests wait for
    memory, complete, free it, and the rest are admitted; results unchanged."""
    pool = lib_pool(GENS)
    reqs = _random_requests(11, 40, 40000)
    tickets, results, stats = _serve(pool, reqs, arena_bytes=3 * 40000 * 4, chunk=1000, polls_between=1)
    _check_served(reqs, tickets, results)
    assert stats["arena_free_bytes"] == (3 * 40000 * 4 + 255) // 256 * 256


def test_server_slot_limit_and_single_generator_order():
    pool = lib_pool(GENS)
    reqs = [(3, k % 3, 1000 + 17 * k) for k in range(8)] + _random_requests(5, 20, 5000)
    tickets, results, _ = _serve(pool, reqs, arena_bytes=16 << 20, chunk=333, max_active=2, polls_between=1)
    _check_served(reqs, tickets, results)


def test_server_rejects_bad_requests():
    import paper_1005_4973_gb300 as M
    pool = lib_pool(GENS[:2])
    srv = M.Server(pool, arena_bytes=1 << 20)
    for g, dt, n in ((2, 0, 10), (0, 3, 10), (0, 0, 0), (0, 0, (1 << 20) // 4 + 1)):
        with pytest.raises(M.MTGPError):
            srv.submit(g, dt, n)
    srv.close()


def test_server_native_trace_loop():
    """mtgp_server_run_trace over a Poisson trace: every request completes with
    a positive latency, the counters agree with the trace, and each generator's
    state has advanced exactly as the oracle's stream over the same lengths."""
    import paper_1005_4973_gb300 as M
    pool = lib_pool(GENS)
    arrivals = WL.c5_arrivals(20000.0, 300, pool_size=len(GENS), lo=4.0, hi=15.0, seed=21)
    srv = M.Server(pool, arena_bytes=64 << 20, chunk=4096, max_active=6, max_inflight=2)
    lat, done = srv.run_trace(arrivals)
    st = srv.stats()
    srv.close()
    assert np.all(lat > 0) and np.all(done > 0)
    assert st["numbers_completed"] == sum(a[3] for a in arrivals)
    assert st["pending"] == 0 and st["active"] == 0
    for g in range(len(GENS)):
        n = sum(a[3] for a in arrivals if a[1] == g)
        assert pool.position(g) == n
        p, st = oracle_state(GENS[g])
        O.generate(p, st, n, 0)                        # advances st in place
        assert np.array_equal(pool.read_state(g), st)
