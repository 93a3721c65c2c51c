"""ctypes binding of libmtgp (include/mtgp.h): argument marshalling only.

Every function keeps the C name; device buffers are passed as torch CUDA
tensors (or raw integer addresses) and streams as torch.cuda.Stream objects
(or raw cudaStream_t integers).  Nothing here computes any part of the
generation path; if the shared library is missing, importing this module
raises ImportError instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libmtgp.so")

MTGP_OK, MTGP_EINVAL, MTGP_ENOMEM, MTGP_ECUDA, MTGP_ETIMEOUT, MTGP_EBUSY = range(6)
MTGP_U32, MTGP_F32_12, MTGP_F32_01 = 0, 1, 2
MTGP_LAYOUT_BLOCKED, MTGP_LAYOUT_INTERLEAVED = 0, 1
MTGP_MAX_N = 4096
MTGP_NOALLOC_SCRATCH_BYTES, MTGP_NOALLOC_MAX_GENS, MTGP_NOALLOC_MAX_REQS = 32768, 64, 64
# block sizes compiled into the library and the column slots per thread each
# supports (mirrors max_slots in the CUDA sources)
MAX_SLOTS = {32: 11, 64: 12, 128: 11, 256: 6, 512: 8}
# split form: block size -> columns per recursion thread (threads / 2 own columns)
MAX_SLOTS_SPLIT = {128: 12, 256: 11, 512: 6, 1024: 3}
# flow form: block size -> chunks of 32 columns per recursion warp (threads / 2 own columns)
MAX_SLOTS_FLOW = {128: 12, 256: 11, 512: 6, 1024: 8}
# wide form: block size -> groups of 4 columns per thread
MAX_SLOTS_WIDE = {96: 4, 128: 3, 192: 2}
# pair form: block size -> slots of two adjacent columns per thread
MAX_SLOTS_PAIRS = {128: 6}
STATUS_NAMES = {0: "MTGP_OK", 1: "MTGP_EINVAL", 2: "MTGP_ENOMEM", 3: "MTGP_ECUDA",
                4: "MTGP_ETIMEOUT", 5: "MTGP_EBUSY"}


class MTGPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class mtgp_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("mexp", "N", "r", "mask", "pos", "sh1", "sh2", "id")] + [
        ("rec_tbl", ctypes.c_uint32 * 16), ("tmp_tbl", ctypes.c_uint32 * 16)]


class mtgp_request(ctypes.Structure):
    _fields_ = [("gen", ctypes.c_uint32), ("dtype", ctypes.c_uint32),
                ("n", ctypes.c_uint64), ("out_offset", ctypes.c_uint64)]


class mtgp_config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("threads", "persistent", "blocks_per_sm", "chunk", "buffer_words", "form", "pieces",
                 "piece_log2", "round_words")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class mtgp_server_config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_uint64), ("chunk", ctypes.c_uint64),
                ("max_active", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32)]


class mtgp_completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("gen", ctypes.c_uint32), ("dtype", ctypes.c_uint32),
                ("n", ctypes.c_uint64), ("dev_out", ctypes.c_void_p), ("submit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class mtgp_server_stats_t(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_uint32), ("active", ctypes.c_uint32), ("inflight_ticks", ctypes.c_uint32),
                ("ticks", ctypes.c_uint64), ("numbers_completed", ctypes.c_uint64),
                ("arena_free_bytes", ctypes.c_uint64), ("now_s", ctypes.c_double)]


_vp, _u32, _u64, _sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
_P = ctypes.POINTER
_SIGS = {
    "mtgp_version": (ctypes.c_char_p, []),
    "mtgp_last_error": (ctypes.c_char_p, []),
    "mtgp_params_draw": (ctypes.c_int, [_u32, _u64, _u32, _P(mtgp_params)]),
    "mtgp_params_validate": (ctypes.c_int, [_P(mtgp_params)]),
    "mtgp_state_create": (ctypes.c_int, [_P(mtgp_params), _u32, _u64, _vp, _P(_vp)]),
    "mtgp_generate": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _u64, _vp]),
    "mtgp_state_save": (ctypes.c_int, [_vp, _vp, _P(_sz)]),
    "mtgp_state_load": (ctypes.c_int, [_vp, _vp, _sz]),
    "mtgp_state_position": (ctypes.c_int, [_vp, _P(_u64)]),
    "mtgp_state_destroy": (None, [_vp]),
    "mtgp_pool_create": (ctypes.c_int, [_P(mtgp_params), _P(_u32), _P(_u64), _u32, _vp, _P(_vp)]),
    "mtgp_pool_info": (ctypes.c_int, [_vp, _P(_u32), _P(_u64)]),
    "mtgp_pool_get_config": (ctypes.c_int, [_vp, _P(mtgp_config)]),
    "mtgp_pool_set_config": (ctypes.c_int, [_vp, _P(mtgp_config)]),
    "mtgp_pool_generate": (ctypes.c_int, [_vp, _P(mtgp_request), _u32, _vp, ctypes.c_int, _vp]),
    "mtgp_pool_generate_host": (ctypes.c_int, [_vp, _P(mtgp_request), _u32, _vp, ctypes.c_int, _u64, _vp]),
    "mtgp_pool_position": (ctypes.c_int, [_vp, _u32, _P(_u64)]),
    "mtgp_pool_read_state": (ctypes.c_int, [_vp, _u32, _P(_u32)]),
    "mtgp_pool_save": (ctypes.c_int, [_vp, _vp, _P(_sz)]),
    "mtgp_pool_load": (ctypes.c_int, [_vp, _vp, _sz]),
    "mtgp_pool_destroy": (None, [_vp]),
    "mtgp_autotune": (ctypes.c_int, [_vp, _P(mtgp_request), _u32, _vp, _u32, _vp, _P(mtgp_config),
                                     _P(ctypes.c_int), _P(ctypes.c_float)]),
    "mtgp_fill_probe": (ctypes.c_int, [_vp, _u64, _u32, _vp]),
    "mtgp_pool_errors": (ctypes.c_int, [_vp, _P(_u32)]),
    "mtgp_pool_launch_count": (ctypes.c_int, [_vp, _P(_u64)]),
    "mtgp_pool_set_timing": (ctypes.c_int, [_vp, _u32]),
    "mtgp_pool_set_spin_limit": (ctypes.c_int, [_vp, _u32]),
    "mtgp_pool_kernel_times": (ctypes.c_int, [_vp, _u32, _P(ctypes.c_float), _P(ctypes.c_float)]),
    "mtgp_pool_jump": (ctypes.c_int, [_vp, _u32, _u64, _vp]),
    "mtgp_state_jump": (ctypes.c_int, [_vp, _u64, _vp]),
    "mtgp_pool_annihilator": (ctypes.c_int, [_vp, _u32, _P(_u64), _u32, _P(_u32), _vp]),
    "mtgp_params_search": (ctypes.c_int, [_u32, _u64, _u32, _u64, _u32, _P(mtgp_params), _P(_u64), _P(_u64),
                                          _P(_u64), _u32]),
    "mtgp_params_search_gpu": (ctypes.c_int, [_u32, _u64, _u32, _u64, _u32, _vp, _P(mtgp_params), _P(_u64),
                                               _P(_u64), _P(_u64), _u32]),
    "mtgp_params_equidistribution": (ctypes.c_int, [_P(mtgp_params), _u32, _P(_u32), _P(_u32)]),
    "mtgp_params_equidistribution_lsb": (ctypes.c_int, [_P(mtgp_params), _u32, _P(_u32), _P(_u32)]),
    "mtgp_params_temper_search": (ctypes.c_int, [_P(mtgp_params), _u32, _P(mtgp_params), _P(_u32)]),
    "mtgp_params_report": (ctypes.c_int, [_P(mtgp_params), _u32, ctypes.c_char_p, _sz]),
    "mtgp_params_record": (ctypes.c_int, [_P(mtgp_params), _P(_u64), _u32, _u32, ctypes.c_char_p, _sz]),
    "mtgp_f2_minpoly": (ctypes.c_int, [_P(_u64), _u64, _P(_u64), _u32, _P(ctypes.c_int64)]),
    "mtgp_f2_irreducible_gpu": (ctypes.c_int, [_P(_u64), _u32, _u32, _u32, _vp, _P(ctypes.c_uint8)]),
    "mtgp_f2_mulmod": (ctypes.c_int, [_P(_u64), _u32, _P(_u64), _u32, _P(_u64), _u32, _P(_u64), _u32,
                                      _P(ctypes.c_int64)]),
    "mtgp_f2_xpow_mod": (ctypes.c_int, [_u64, _P(_u64), _u32, _P(_u64), _u32, _P(ctypes.c_int64)]),
    "mtgp_graph_create": (ctypes.c_int, [_vp, _u32, _vp, _P(_vp)]),
    "mtgp_graph_set_requests": (ctypes.c_int, [_vp, _P(mtgp_request), _u32, _vp, ctypes.c_int, _vp]),
    "mtgp_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "mtgp_graph_errors": (ctypes.c_int, [_vp, _P(_u32)]),
    "mtgp_graph_destroy": (None, [_vp]),
    "mtgp_server_create": (ctypes.c_int, [_vp, _P(mtgp_server_config), _vp, _P(_vp)]),
    "mtgp_server_submit": (ctypes.c_int, [_vp, _u32, _u32, _u64, _P(_u64)]),
    "mtgp_server_poll": (ctypes.c_int, [_vp, _P(mtgp_completion), _u32, _P(_u32), ctypes.c_int]),
    "mtgp_server_release": (ctypes.c_int, [_vp, _u64]),
    "mtgp_server_stats": (ctypes.c_int, [_vp, _P(mtgp_server_stats_t)]),
    "mtgp_server_destroy": (None, [_vp]),
    "mtgp_server_run_trace": (ctypes.c_int, [_vp, _P(ctypes.c_double), _P(_u32), _P(_u32), _P(_u64), _u32,
                                             _P(ctypes.c_double), _P(ctypes.c_double)]),
    "mtgp_generate_noalloc": (ctypes.c_int, [_P(mtgp_params), _u32, _vp, _P(_u64), _P(mtgp_request), _u32,
                                             _vp, _vp]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmtgp is not built ({LIB_PATH} missing); run "
                          f"`python -m paper_1005_4973_gb300.build` first -- there is no fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


LIB = _load()


def exported_symbols():
    return sorted(_SIGS)


def last_error() -> str:
    return LIB.mtgp_last_error().decode()


def check(status: int) -> None:
    if status != MTGP_OK:
        raise MTGPError(status, last_error())


def ptr(x) -> int | None:
    """Device or host address of a torch tensor, numpy array or int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# numpy view of mtgp_request (same field order, sizes and padding)
REQUEST_DTYPE = np.dtype([("gen", "<u4"), ("dtype", "<u4"), ("n", "<u8"), ("out_offset", "<u8")])


def requests_array(reqs) -> ctypes.Array:
    """(gen, dtype, n, out_offset) rows -- a list of tuples, an (n, 4) integer
    array, a REQUEST_DTYPE array or mtgp_request objects -- as a C array of
    mtgp_request.  Rows are converted column-wise by numpy, so a call with
    thousands of requests does not pay a Python loop."""
    n = len(reqs)
    if isinstance(reqs, np.ndarray) and reqs.dtype == REQUEST_DTYPE:
        a = np.ascontiguousarray(reqs) if n else np.zeros(1, dtype=REQUEST_DTYPE)
    else:
        a = np.zeros(max(n, 1), dtype=REQUEST_DTYPE)
        if n and isinstance(reqs[0], mtgp_request):
            for i, r in enumerate(reqs):
                a[i] = (r.gen, r.dtype, r.n, r.out_offset)
        elif n:
            m = np.asarray(reqs, dtype=np.uint64).reshape(n, 4)
            a["gen"][:n] = m[:, 0]
            a["dtype"][:n] = m[:, 1]
            a["n"][:n] = m[:, 2]
            a["out_offset"][:n] = m[:, 3]
    return (mtgp_request * len(a)).from_buffer(a)
