"""Python face of libmtgp.  Same names as the C ABI (include/mtgp.h), plus small
owner classes (Pool, State, Graph, Server) that free their handles.  Marshalling only:
every number is produced by the CUDA kernels behind the C ABI.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L
from ._lib import (MTGP_F32_01, MTGP_F32_12, MTGP_LAYOUT_BLOCKED, MTGP_LAYOUT_INTERLEAVED,  # noqa: F401
                   MTGP_MAX_N, MTGP_U32, MTGPError, mtgp_config, mtgp_params, mtgp_request)


def mtgp_version() -> str:
    return L.LIB.mtgp_version().decode()


def mtgp_params_draw(mexp: int, param_seed: int, gen_id: int) -> mtgp_params:
    p = mtgp_params()
    L.check(L.LIB.mtgp_params_draw(mexp, param_seed, gen_id, ctypes.byref(p)))
    return p


def mtgp_params_search(mexp: int, seed0: int, gen_id: int, max_tries: int = 1 << 20, threads: int = 0):
    """Sec. 5 recursion-parameter search; returns (params, found_seed, tries,
    characteristic polynomial as a coefficient array)."""
    p = mtgp_params()
    found, tries = ctypes.c_uint64(), ctypes.c_uint64()
    words = np.zeros(mexp // 64 + 1, dtype=np.uint64)
    L.check(L.LIB.mtgp_params_search(mexp, seed0, gen_id, max_tries, threads, ctypes.byref(p), ctypes.byref(found),
                                     ctypes.byref(tries), words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                     words.size))
    return p, found.value, tries.value, poly_from_words(words, mexp)


def mtgp_params_search_gpu(mexp: int, seed0: int, gen_id: int, max_tries: int = 1 << 20, threads: int = 0,
                           stream=None):
    """The Sec. 5 recursion-parameter search with its polynomial work on the
    GPU (Berlekamp-Massey, one warp per candidate; irreducibility, one block
    per candidate); the same result as mtgp_params_search."""
    p = mtgp_params()
    found, tries = ctypes.c_uint64(), ctypes.c_uint64()
    words = np.zeros(mexp // 64 + 1, dtype=np.uint64)
    L.check(L.LIB.mtgp_params_search_gpu(mexp, seed0, gen_id, max_tries, threads, L.stream_handle(stream),
                                         ctypes.byref(p), ctypes.byref(found), ctypes.byref(tries),
                                         words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), words.size))
    return p, found.value, tries.value, poly_from_words(words, mexp)


def mtgp_params_equidistribution(p: mtgp_params, threads: int = 0):
    """k(v) for v = 1..32 (index v - 1) and the total dimension defect
    (Sec. 3.4, 3.8) of a full-period parameter set."""
    kv = (ctypes.c_uint32 * 32)()
    delta = ctypes.c_uint32()
    L.check(L.LIB.mtgp_params_equidistribution(ctypes.byref(p), threads, kv, ctypes.byref(delta)))
    return np.array(list(kv), dtype=np.int64), delta.value


def mtgp_params_equidistribution_lsb(p: mtgp_params, threads: int = 0):
    """k'(v) for v = 1..32 (the v least significant bits) and their total defect."""
    kv = (ctypes.c_uint32 * 32)()
    delta = ctypes.c_uint32()
    L.check(L.LIB.mtgp_params_equidistribution_lsb(ctypes.byref(p), threads, kv, ctypes.byref(delta)))
    return np.array(list(kv), dtype=np.int64), delta.value


def mtgp_params_temper_search(p: mtgp_params, threads: int = 0):
    """Tempering search of Sec. 5: returns (params with the table found, its total defect)."""
    out = mtgp_params()
    delta = ctypes.c_uint32()
    L.check(L.LIB.mtgp_params_temper_search(ctypes.byref(p), threads, ctypes.byref(out), ctypes.byref(delta)))
    return out, delta.value


def mtgp_params_report(p: mtgp_params, threads: int = 0) -> str:
    """Table 1 style report (Sec. 3.8): v, k(v), d(v), r(v) and the total defect."""
    buf = ctypes.create_string_buffer(4096)
    L.check(L.LIB.mtgp_params_report(ctypes.byref(p), threads, buf, len(buf)))
    return buf.value.decode()


def mtgp_params_record(p: mtgp_params, charpoly, threads: int = 0) -> str:
    """MTGPDC record of a searched set (Sec. 5), charpoly as a coefficient array."""
    w = poly_to_words(charpoly)
    need = p.mexp // 64 + 1
    if w.size < need:
        w = np.concatenate([w, np.zeros(need - w.size, dtype=np.uint64)])
    buf = ctypes.create_string_buffer(4096)
    L.check(L.LIB.mtgp_params_record(ctypes.byref(p), _u64p(w), w.size, threads, buf, len(buf)))
    return buf.value.decode()


def mtgp_params_validate(p: mtgp_params) -> None:
    L.check(L.LIB.mtgp_params_validate(ctypes.byref(p)))


def mtgp_fill_probe(dev_buf, words: int, pattern: int = 0x9E3779B9, stream=None) -> None:
    L.check(L.LIB.mtgp_fill_probe(L.ptr(dev_buf), words, pattern, L.stream_handle(stream)))


# -- F2[x] routines behind jump-ahead (coefficient arrays: index = power of x) --
def poly_to_words(c) -> np.ndarray:
    c = np.asarray(c, dtype=np.uint8) & 1
    w = np.zeros(max(1, (c.size + 63) // 64), dtype=np.uint64)
    for i in np.nonzero(c)[0]:
        w[i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return w


def poly_from_words(w, deg: int) -> np.ndarray:
    if deg < 0:
        return np.zeros(0, dtype=np.uint8)
    w = np.asarray(w, dtype=np.uint64)
    i = np.arange(deg + 1)
    return ((w[i // 64] >> (i % 64).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def mtgp_f2_minpoly(bits) -> np.ndarray:
    bits = np.asarray(bits, dtype=np.uint8) & 1
    w = poly_to_words(bits) if bits.size else np.zeros(1, dtype=np.uint64)
    out = np.zeros(bits.size // 64 + 3, dtype=np.uint64)
    d = ctypes.c_int64()
    L.check(L.LIB.mtgp_f2_minpoly(_u64p(w), bits.size, _u64p(out), out.size, ctypes.byref(d)))
    return poly_from_words(out, d.value)


def mtgp_f2_irreducible_gpu(polys, p: int, stream=None) -> np.ndarray:
    """GPU irreducibility test (degree exactly p, p a prime > 32) of each
    coefficient array in polys; returns a bool array."""
    words = p // 64 + 1
    arr = np.zeros((len(polys), words), dtype=np.uint64)
    for j, c in enumerate(polys):
        w = poly_to_words(c)
        if w.size > words:
            if np.any(w[words:]):
                raise ValueError("polynomial of degree above p")
            w = w[:words]
        arr[j, :w.size] = w
    ver = np.zeros(len(polys), dtype=np.uint8)
    L.check(L.LIB.mtgp_f2_irreducible_gpu(_u64p(arr), len(polys), words, p, L.stream_handle(stream),
                                          ver.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return ver.astype(bool)


def mtgp_f2_mulmod(a, b, m) -> np.ndarray:
    aw, bw, mw = poly_to_words(a), poly_to_words(b), poly_to_words(m)
    out = np.zeros(mw.size + 1, dtype=np.uint64)
    d = ctypes.c_int64()
    L.check(L.LIB.mtgp_f2_mulmod(_u64p(aw), aw.size, _u64p(bw), bw.size, _u64p(mw), mw.size, _u64p(out),
                                 out.size, ctypes.byref(d)))
    return poly_from_words(out, d.value)


def mtgp_f2_xpow_mod(e: int, m) -> np.ndarray:
    mw = poly_to_words(m)
    out = np.zeros(mw.size + 1, dtype=np.uint64)
    d = ctypes.c_int64()
    L.check(L.LIB.mtgp_f2_xpow_mod(e, _u64p(mw), mw.size, _u64p(out), out.size, ctypes.byref(d)))
    return poly_from_words(out, d.value)


class Pool:
    """Device-resident generators (mtgp_pool_*)."""

    def __init__(self, params, gen_ids, seeds, stream=None):
        params = list(params)
        n = len(params)
        parr = (mtgp_params * n)(*params)
        ids = (ctypes.c_uint32 * n)(*[int(i) for i in gen_ids])
        sds = (ctypes.c_uint64 * n)(*[int(s) for s in seeds])
        h = ctypes.c_void_p()
        L.check(L.LIB.mtgp_pool_create(parr, ids, sds, n, L.stream_handle(stream), ctypes.byref(h)))
        self.handle = h
        self.params = params
        self.count = n

    # -- generation ---------------------------------------------------------
    def generate(self, reqs, out, layout=MTGP_LAYOUT_BLOCKED, stream=None) -> None:
        arr = L.requests_array(reqs)
        L.check(L.LIB.mtgp_pool_generate(self.handle, arr, len(reqs), L.ptr(out), layout,
                                         L.stream_handle(stream)))

    def generate_host(self, reqs, host_out, layout=MTGP_LAYOUT_BLOCKED, staging_bytes=0, stream=None) -> None:
        arr = L.requests_array(reqs)
        L.check(L.LIB.mtgp_pool_generate_host(self.handle, arr, len(reqs), L.ptr(host_out), layout,
                                              staging_bytes, L.stream_handle(stream)))

    # -- configuration ------------------------------------------------------
    @property
    def config(self) -> mtgp_config:
        c = mtgp_config()
        L.check(L.LIB.mtgp_pool_get_config(self.handle, ctypes.byref(c)))
        return c

    def set_config(self, **kw) -> mtgp_config:
        c = self.config
        for k, v in kw.items():
            setattr(c, k, int(v))
        L.check(L.LIB.mtgp_pool_set_config(self.handle, ctypes.byref(c)))
        return c

    def autotune(self, reqs, scratch, stream=None, layouts: int = 1):
        """The autotuner (mtgp_autotune): sets and returns (config, ms, layout);
        layouts: bit 0 blocked, bit 1 interleaved allowed."""
        arr = L.requests_array(reqs)
        best, ms, lay = mtgp_config(), ctypes.c_float(), ctypes.c_int()
        L.check(L.LIB.mtgp_autotune(self.handle, arr, len(reqs), L.ptr(scratch), layouts, L.stream_handle(stream),
                                    ctypes.byref(best), ctypes.byref(lay), ctypes.byref(ms)))
        return best, ms.value, lay.value

    # -- state --------------------------------------------------------------
    def position(self, i: int) -> int:
        v = ctypes.c_uint64()
        L.check(L.LIB.mtgp_pool_position(self.handle, i, ctypes.byref(v)))
        return v.value

    def read_state(self, i: int) -> np.ndarray:
        st = np.zeros(self.params[i].N, dtype=np.uint32)
        L.check(L.LIB.mtgp_pool_read_state(self.handle, i, st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
        return st

    def save(self) -> bytes:
        n = ctypes.c_size_t()
        L.check(L.LIB.mtgp_pool_save(self.handle, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        L.check(L.LIB.mtgp_pool_save(self.handle, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob: bytes) -> None:
        L.check(L.LIB.mtgp_pool_load(self.handle, blob, len(blob)))

    def errors(self) -> int:
        """Error word of the last launches (bit 0 shape/buffer, bit 1 wait timeout); clears it."""
        v = ctypes.c_uint32()
        L.check(L.LIB.mtgp_pool_errors(self.handle, ctypes.byref(v)))
        return v.value

    def launch_count(self) -> int:
        v = ctypes.c_uint64()
        L.check(L.LIB.mtgp_pool_launch_count(self.handle, ctypes.byref(v)))
        return v.value

    def set_spin_limit(self, polls: int) -> None:
        """Flow form: polls per bounded wait (0 = default)."""
        L.check(L.LIB.mtgp_pool_set_spin_limit(self.handle, polls))

    def set_timing(self, entries: int) -> None:
        """Record CUDA events around the jump and generation launches of the next calls."""
        L.check(L.LIB.mtgp_pool_set_timing(self.handle, entries))

    def kernel_times(self, count: int):
        """(jump_ms, gen_ms) lists of the last `count` recorded calls, oldest first."""
        a = (ctypes.c_float * max(count, 1))()
        b = (ctypes.c_float * max(count, 1))()
        L.check(L.LIB.mtgp_pool_kernel_times(self.handle, count, a, b))
        return list(a)[:count], list(b)[:count]

    # -- jump-ahead (Sec. 7) ----------------------------------------------------
    def jump(self, i: int, steps: int, stream=None) -> None:
        L.check(L.LIB.mtgp_pool_jump(self.handle, i, steps, L.stream_handle(stream)))

    def annihilator(self, i: int, stream=None) -> np.ndarray:
        """Coefficients (uint8, index = power of x) of generator i's annihilating polynomial."""
        d = ctypes.c_uint32()
        L.check(L.LIB.mtgp_pool_annihilator(self.handle, i, None, 0, ctypes.byref(d), L.stream_handle(stream)))
        words = np.zeros(d.value // 64 + 1, dtype=np.uint64)
        L.check(L.LIB.mtgp_pool_annihilator(self.handle, i, words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                            words.size, ctypes.byref(d), L.stream_handle(stream)))
        return poly_from_words(words, d.value)

    def info(self):
        c, b = ctypes.c_uint32(), ctypes.c_uint64()
        L.check(L.LIB.mtgp_pool_info(self.handle, ctypes.byref(c), ctypes.byref(b)))
        return c.value, b.value

    def close(self) -> None:
        if self.handle:
            L.LIB.mtgp_pool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """One device-resident generator (mtgp_state_*)."""

    def __init__(self, params: mtgp_params, gen_id: int, seed: int, stream=None):
        h = ctypes.c_void_p()
        L.check(L.LIB.mtgp_state_create(ctypes.byref(params), gen_id, seed, L.stream_handle(stream),
                                        ctypes.byref(h)))
        self.handle = h
        self.params = params

    def generate(self, dtype: int, out, n: int, stream=None) -> None:
        L.check(L.LIB.mtgp_generate(self.handle, dtype, L.ptr(out), n, L.stream_handle(stream)))

    def position(self) -> int:
        v = ctypes.c_uint64()
        L.check(L.LIB.mtgp_state_position(self.handle, ctypes.byref(v)))
        return v.value

    def jump(self, steps: int, stream=None) -> None:
        L.check(L.LIB.mtgp_state_jump(self.handle, steps, L.stream_handle(stream)))

    def save(self) -> bytes:
        n = ctypes.c_size_t()
        L.check(L.LIB.mtgp_state_save(self.handle, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        L.check(L.LIB.mtgp_state_save(self.handle, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob: bytes) -> None:
        L.check(L.LIB.mtgp_state_load(self.handle, blob, len(blob)))

    def close(self) -> None:
        if self.handle:
            L.LIB.mtgp_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """Captured persistent launch over a pool (mtgp_graph_*)."""

    def __init__(self, pool: Pool, max_items: int, stream=None):
        h = ctypes.c_void_p()
        L.check(L.LIB.mtgp_graph_create(pool.handle, max_items, L.stream_handle(stream), ctypes.byref(h)))
        self.handle, self.pool = h, pool

    def set_requests(self, reqs, out, layout=MTGP_LAYOUT_BLOCKED, stream=None) -> None:
        arr = L.requests_array(reqs)
        L.check(L.LIB.mtgp_graph_set_requests(self.handle, arr, len(reqs), L.ptr(out), layout,
                                              L.stream_handle(stream)))

    def launch(self, stream=None) -> None:
        L.check(L.LIB.mtgp_graph_launch(self.handle, L.stream_handle(stream)))

    def errors(self) -> int:
        v = ctypes.c_uint32()
        L.check(L.LIB.mtgp_graph_errors(self.handle, ctypes.byref(v)))
        return v.value

    def close(self) -> None:
        if self.handle:
            L.LIB.mtgp_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over a pool (mtgp_server_*)."""

    def __init__(self, pool: Pool, arena_bytes=0, chunk=0, max_active=0, max_inflight=0, stream=None):
        cfg = L.mtgp_server_config(arena_bytes, chunk, max_active, max_inflight)
        h = ctypes.c_void_p()
        L.check(L.LIB.mtgp_server_create(pool.handle, ctypes.byref(cfg), L.stream_handle(stream),
                                         ctypes.byref(h)))
        self.handle, self.pool = h, pool
        self._buf = (L.mtgp_completion * 256)()

    def submit(self, gen: int, dtype: int, n: int) -> int:
        t = ctypes.c_uint64()
        L.check(L.LIB.mtgp_server_submit(self.handle, gen, dtype, n, ctypes.byref(t)))
        return t.value

    def poll(self, block: bool = False):
        nd = ctypes.c_uint32()
        L.check(L.LIB.mtgp_server_poll(self.handle, self._buf, len(self._buf), ctypes.byref(nd), int(block)))
        return [self._buf[i] for i in range(nd.value)]

    def release(self, ticket: int) -> None:
        L.check(L.LIB.mtgp_server_release(self.handle, ticket))

    def run_trace(self, arrivals):
        """arrivals: list of (time_s, gen, dtype, n), sorted by time.  Runs the
        native request loop; returns (latency_s, done_s) numpy arrays."""
        k = len(arrivals)
        a = np.ascontiguousarray([x[0] for x in arrivals], dtype=np.float64)
        g = np.ascontiguousarray([x[1] for x in arrivals], dtype=np.uint32)
        d = np.ascontiguousarray([x[2] for x in arrivals], dtype=np.uint32)
        n = np.ascontiguousarray([x[3] for x in arrivals], dtype=np.uint64)
        lat = np.zeros(k, dtype=np.float64)
        done = np.zeros(k, dtype=np.float64)
        P = ctypes.POINTER
        L.check(L.LIB.mtgp_server_run_trace(
            self.handle, a.ctypes.data_as(P(ctypes.c_double)), g.ctypes.data_as(P(ctypes.c_uint32)),
            d.ctypes.data_as(P(ctypes.c_uint32)), n.ctypes.data_as(P(ctypes.c_uint64)), k,
            lat.ctypes.data_as(P(ctypes.c_double)), done.ctypes.data_as(P(ctypes.c_double))))
        return lat, done

    def stats(self):
        st = L.mtgp_server_stats_t()
        L.check(L.LIB.mtgp_server_stats(self.handle, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in st._fields_}

    def close(self) -> None:
        if self.handle:
            L.LIB.mtgp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
