"""MTGP CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct statement of what the MTGP generation path
computes (Saito & Matsumoto, arXiv 1005.4973): the recursion of Sec. 3.6, the
tempering of Sec. 3.7 and the single-precision fill of Sec. 6, on a straight
array with no ring, no blocking and no reordering.  The arithmetic lives in
``mtgp_oracle.c`` (plain C, built with gcc by :func:`build`); this module is
its ctypes wrapper.  ``oracle.f2`` restates the same maps as F2 bit-matrices
built from the definitions, as an independent second formulation.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library and the library never imports it.

What pins each part (tests marked ``not gpu``):
  * recursion + tempering: equal to the bit-matrix formulation of ``oracle.f2``
    on random states; F2-linearity of the output in the state; invariance
    under the r masked LSBs of x_0 (Sec. 3.3, 3.6, 3.7);
  * period structure: for reduced exponents p in {89, 107, 127, 521, 607},
    sets found by the small MTGPDC search have a Berlekamp-Massey minimal
    polynomial of degree p that is irreducible, the transition matrix F built
    from the definitions satisfies phi(F) = 0, F^(2^p) = F and rank(F - I) = p
    (Sec. 3.3, Sec. 5);
  * float output: f12 bits = 0x3F800000 | (u32 >> 9) and f01 = (u32 >> 9) 2^-23
    exactly (Sec. 6);
  * continuation: generate(a) then generate(b) equals generate(a + b) (Sec. 8);
  * Berlekamp-Massey and the irreducibility test: against brute force on
    small polynomials.
Parity unpinned (project definitions of passages the paper leaves open):
``params_draw`` (how sets are drawn) and ``seed_state`` (how a state is seeded).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

U32, F12, F01 = 0, 1, 2
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mtgp_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libmtgp_oracle.so")
_lib = None


class OrcParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("mexp", "N", "r", "mask", "pos", "sh1", "sh2", "id")] + [
        ("R", ctypes.c_uint32 * 4), ("T", ctypes.c_uint32 * 4),
        ("rectbl", ctypes.c_uint32 * 16), ("tmptbl", ctypes.c_uint32 * 16),
        ("sngltbl", ctypes.c_uint32 * 16)]


def build(force: bool = False) -> str:
    """Compiles the C oracle with gcc into oracle/_build (idempotent)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        P = ctypes.POINTER
        u8p, u32p, u64p = P(ctypes.c_uint8), P(ctypes.c_uint32), P(ctypes.c_uint64)
        sig = {
            "orc_mix64": (ctypes.c_uint64, [ctypes.c_uint64]),
            "orc_splitmix64_next": (ctypes.c_uint64, [u64p]),
            "orc_table_from_rows": (None, [u32p, u32p]),
            "orc_derive": (ctypes.c_int, [P(OrcParams)]),
            "orc_pos_range": (None, [ctypes.c_uint32, u32p, u32p]),
            "orc_lsb_block_invertible": (ctypes.c_int, [u32p]),
            "orc_params_draw": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_int, P(OrcParams)]),
            "orc_seed_state": (None, [P(OrcParams), ctypes.c_uint32, ctypes.c_uint64, u32p]),
            "orc_generate": (ctypes.c_int, [P(OrcParams), u32p, ctypes.c_uint64, ctypes.c_int, u32p]),
            "orc_generate_many": (ctypes.c_int, [P(OrcParams), P(u32p), u64p, P(ctypes.c_int),
                                                 P(u32p), ctypes.c_int, ctypes.c_int]),
            "orc_bm": (ctypes.c_int, [u8p, ctypes.c_int, u8p]),
            "orc_poly_irreducible_prime": (ctypes.c_int, [u8p, ctypes.c_int]),
            "orc_f2mat_mul": (None, [u64p, u64p, u64p, ctypes.c_int]),
            "orc_f2mat_rank": (ctypes.c_int, [u64p, ctypes.c_int]),
            "orc_f2mat_pow2k": (None, [u64p, u64p, ctypes.c_int, ctypes.c_int]),
            "orc_f2mat_polyeval": (None, [u8p, ctypes.c_int, u64p, u64p, ctypes.c_int]),
            "orc_search_full_period": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                                      ctypes.c_int, P(OrcParams), u64p]),
            "orc_params_sizeof": (ctypes.c_int, []),
            "orc_kv": (ctypes.c_int, [u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_int)]),
            "orc_mt19937_outputs": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, u32p]),
            "orc_mt19937_init_genrand": (None, [ctypes.c_uint32, u32p]),
            "orc_mt19937_outputs_from": (ctypes.c_int, [u32p, ctypes.c_int, u32p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        assert L.orc_params_sizeof() == ctypes.sizeof(OrcParams)
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# --------------------------------------------------------------------------
# parameter sets and seeding
# --------------------------------------------------------------------------
def params_draw(mexp: int, param_seed: int, gen_id: int, random_shifts: bool = False) -> OrcParams:
    """Synthetic parameter set with MTGPDC's structure (Sec. 5); see the C header."""
    p = OrcParams()
    if lib().orc_params_draw(mexp, param_seed, gen_id, int(random_shifts), ctypes.byref(p)):
        raise ValueError(f"cannot draw a parameter set for mexp={mexp}")
    return p


def params_from_fields(mexp, pos, sh1, sh2, gen_id, R, T) -> OrcParams:
    """Parameter set from explicit fields; derived fields per Sec. 3.3, 3.6, 3.7, 6."""
    p = OrcParams()
    p.mexp, p.pos, p.sh1, p.sh2, p.id = mexp, pos, sh1, sh2, gen_id
    for j in range(4):
        p.R[j], p.T[j] = int(R[j]), int(T[j])
    if lib().orc_derive(ctypes.byref(p)):
        raise ValueError("invalid parameter fields")
    return p


def pos_range(N: int):
    lo, hi = ctypes.c_uint32(), ctypes.c_uint32()
    lib().orc_pos_range(N, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def table_from_rows(rows) -> np.ndarray:
    r = np.asarray(rows, dtype=np.uint32)
    t = np.zeros(16, dtype=np.uint32)
    lib().orc_table_from_rows(_p(r, ctypes.c_uint32), _p(t, ctypes.c_uint32))
    return t


def lsb_block_invertible(R) -> bool:
    r = np.asarray(R, dtype=np.uint32)
    return bool(lib().orc_lsb_block_invertible(_p(r, ctypes.c_uint32)))


def seed_state(p: OrcParams, gen_id: int, seed: int) -> np.ndarray:
    st = np.zeros(p.N, dtype=np.uint32)
    lib().orc_seed_state(ctypes.byref(p), gen_id, seed, _p(st, ctypes.c_uint32))
    return st


def splitmix64(state: int, count: int) -> list[int]:
    s = ctypes.c_uint64(state)
    return [lib().orc_splitmix64_next(ctypes.byref(s)) for _ in range(count)]


# --------------------------------------------------------------------------
# generation
# --------------------------------------------------------------------------
def generate(p: OrcParams, state: np.ndarray, n: int, dtype: int = U32) -> np.ndarray:
    """n outputs (32-bit patterns) of one generator; ``state`` is advanced in place."""
    assert state.dtype == np.uint32 and state.size == p.N and state.flags.c_contiguous
    out = np.zeros(n, dtype=np.uint32)
    if lib().orc_generate(ctypes.byref(p), _p(state, ctypes.c_uint32), n, dtype,
                          _p(out, ctypes.c_uint32)):
        raise MemoryError("oracle allocation failed")
    return out


def generate_many(params, states, ns, dtypes, nthreads: int | None = None):
    """orc_generate for many independent generators, one per host thread."""
    count = len(params)
    nthreads = nthreads or os.cpu_count() or 1
    parr = (OrcParams * count)(*params)
    outs = [np.zeros(int(n), dtype=np.uint32) for n in ns]
    sp = (ctypes.POINTER(ctypes.c_uint32) * count)(*[_p(s, ctypes.c_uint32) for s in states])
    op = (ctypes.POINTER(ctypes.c_uint32) * count)(*[_p(o, ctypes.c_uint32) for o in outs])
    na = np.asarray(ns, dtype=np.uint64)
    da = np.asarray(dtypes, dtype=np.int32)
    if lib().orc_generate_many(parr, sp, _p(na, ctypes.c_uint64), _p(da, ctypes.c_int), op,
                               count, nthreads):
        raise MemoryError("oracle allocation failed")
    return outs


# --------------------------------------------------------------------------
# F2 tools (Sec. 3.3 and Sec. 5 at reduced size)
# --------------------------------------------------------------------------
def bm(bits) -> np.ndarray:
    """Berlekamp-Massey minimal polynomial; returns coefficients c[0..L] (c[i] of x^i)."""
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    poly = np.zeros(b.size + 1, dtype=np.uint8)
    L = lib().orc_bm(_p(b, ctypes.c_uint8), b.size, _p(poly, ctypes.c_uint8))
    return poly[: L + 1].copy()


def irreducible_prime_degree(poly) -> bool:
    c = np.ascontiguousarray(poly, dtype=np.uint8)
    return bool(lib().orc_poly_irreducible_prime(_p(c, ctypes.c_uint8), c.size - 1))


def pack_f2(m: np.ndarray) -> np.ndarray:
    """Dense 0/1 n x n matrix -> rows packed in uint64 words (bit j of row = column j)."""
    n = m.shape[0]
    w = (n + 63) // 64
    pad = np.zeros((n, w * 64), dtype=np.uint8)
    pad[:, :n] = m & 1
    return np.packbits(pad, axis=1, bitorder="little").view(np.uint64).reshape(n, w).copy()


def unpack_f2(pk: np.ndarray, n: int) -> np.ndarray:
    return np.unpackbits(pk.view(np.uint8), axis=1, bitorder="little")[:, :n]


def f2_mul(a_pk: np.ndarray, b_pk: np.ndarray, n: int) -> np.ndarray:
    c = np.zeros_like(a_pk)
    lib().orc_f2mat_mul(_p(a_pk, ctypes.c_uint64), _p(b_pk, ctypes.c_uint64),
                        _p(c, ctypes.c_uint64), n)
    return c


def f2_rank(a_pk: np.ndarray, n: int) -> int:
    return lib().orc_f2mat_rank(_p(np.ascontiguousarray(a_pk), ctypes.c_uint64), n)


def f2_pow2k(a_pk: np.ndarray, n: int, k: int) -> np.ndarray:
    out = np.zeros_like(a_pk)
    lib().orc_f2mat_pow2k(_p(a_pk, ctypes.c_uint64), _p(out, ctypes.c_uint64), n, k)
    return out


def f2_polyeval(poly, a_pk: np.ndarray, n: int) -> np.ndarray:
    c = np.ascontiguousarray(poly, dtype=np.uint8)
    out = np.zeros_like(a_pk)
    lib().orc_f2mat_polyeval(_p(c, ctypes.c_uint8), c.size - 1, _p(a_pk, ctypes.c_uint64),
                             _p(out, ctypes.c_uint64), n)
    return out


def search_full_period(mexp: int, seed0: int, gen_id: int, max_tries: int = 20000):
    """Small-size MTGPDC recursion search (Sec. 5); returns (params, seed, tries)."""
    p = OrcParams()
    found = ctypes.c_uint64()
    t = lib().orc_search_full_period(mexp, seed0, gen_id, max_tries, ctypes.byref(p),
                                     ctypes.byref(found))
    if t < 0:
        raise RuntimeError(f"no full-period set for mexp={mexp} in {max_tries} tries")
    return p, found.value, t


# --------------------------------------------------------------------------
# dimensions of equidistribution (Sec. 3.4, 3.8)
# --------------------------------------------------------------------------
def kv(seq: np.ndarray, p: int, vmax: int = 32) -> np.ndarray:
    """k(v), v = 1..vmax, of the 32-bit output sequence seq (from a nonzero
    state of a full-period generator of state dimension p)."""
    seq = np.ascontiguousarray(seq, dtype=np.uint32)
    out = (ctypes.c_int * vmax)()
    if lib().orc_kv(_p(seq, ctypes.c_uint32), seq.size, p, vmax, out):
        raise MemoryError("oracle allocation failed")
    return np.array(list(out), dtype=np.int64)


def mt19937_outputs(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint32)
    if lib().orc_mt19937_outputs(seed, n, _p(out, ctypes.c_uint32)):
        raise MemoryError("oracle allocation failed")
    return out


def mt19937_outputs_init_genrand(seed: int, n: int) -> np.ndarray:
    """n outputs of MT19937 seeded by the published 32-bit seeding routine."""
    st = np.zeros(624, dtype=np.uint32)
    lib().orc_mt19937_init_genrand(seed, _p(st, ctypes.c_uint32))
    out = np.zeros(n, dtype=np.uint32)
    if lib().orc_mt19937_outputs_from(_p(st, ctypes.c_uint32), n, _p(out, ctypes.c_uint32)):
        raise MemoryError("oracle allocation failed")
    return out


def reverse_bits(words: np.ndarray) -> np.ndarray:
    """Each 32-bit word with its bit order reversed (bit b to bit 31 - b)."""
    words = np.asarray(words, dtype=np.uint32)
    out = np.zeros_like(words)
    for b in range(32):
        out |= ((words >> np.uint32(b)) & np.uint32(1)) << np.uint32(31 - b)
    return out


def temper_search_sec5(op: OrcParams) -> list[int]:
    """The tempering-parameter search of Sec. 5, restated step by step with
    the row-reduction k(v) above: the four tempering rows start at zero; row
    by row, the 23 MSBs are fixed in windows of bits j .. e-1 counted from the
    MSB (j = 0, 5, 10, 15, 20; e = min(j + 5, 23)), each to the pattern with
    the least d(1) + ... + d(e); then, row by row, the 9 LSBs in windows of
    bits j .. e-1 counted from the LSB (j = 0, 5; e = min(j + 5, 9)) against
    d'(1) + ... + d'(e) of the v least significant bits.  Every pattern of a
    window is tried in increasing order and the first least sum kept.
    Returns the four rows (row 0 first).  Full-period sets only."""
    p = op.mexp
    start = seed_state(op, 1, 2)
    n = 2 * p + 64

    def defects(rows, lsb, e):
        q = params_from_fields(op.mexp, op.pos, op.sh1, op.sh2, op.id, list(op.R), rows)
        out = generate(q, start.copy(), n, U32)
        k = kv(reverse_bits(out) if lsb else out, p, vmax=e)
        return sum(p // v - int(k[v - 1]) for v in range(1, e + 1))

    rows = [0, 0, 0, 0]
    for lsb, top in ((False, 23), (True, 9)):
        for i in range(4):
            for j in range(0, top, 5):
                e = min(j + 5, top)
                w = e - j
                shift = j if lsb else 32 - e
                mask = ((1 << w) - 1) << shift
                best = None
                for pat in range(1 << w):
                    r = list(rows)
                    r[i] = (r[i] & ~mask & 0xFFFFFFFF) | (pat << shift)
                    d = defects(r, lsb, e)
                    if best is None or d < best[0]:
                        best = (d, r)
                rows = best[1]
    return rows


def dimension_defects(k: np.ndarray, p: int) -> np.ndarray:
    """d(v) = floor(p / v) - k(v) (Sec. 3.4)."""
    v = np.arange(1, k.size + 1)
    return p // v - k


# --------------------------------------------------------------------------
# closed forms of Sec. 6 (used as pins, not as the definition)
# --------------------------------------------------------------------------
def f12_closed_form(u32: np.ndarray) -> np.ndarray:
    return (np.uint32(0x3F800000) | (u32 >> np.uint32(9))).astype(np.uint32)


def f01_closed_form(u32: np.ndarray) -> np.ndarray:
    return ((u32 >> np.uint32(9)).astype(np.float64) * 2.0 ** -23).astype(np.float32)
