"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/mtgp.h declares, and its host-only calls (parameter drawing and
validation) agree with the oracle and reject bad input."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mtgp.h")


@pytest.fixture(scope="module")
def L():
    from paper_1005_4973_gb300 import build
    build.build()
    from paper_1005_4973_gb300 import _lib
    return _lib


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mtgp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    fns = header_functions()
    for required in ("mtgp_params_draw", "mtgp_params_validate", "mtgp_state_create", "mtgp_generate",
                     "mtgp_state_save", "mtgp_state_load", "mtgp_state_destroy", "mtgp_pool_create",
                     "mtgp_pool_generate", "mtgp_last_error"):
        assert required in fns


def test_library_exports_every_header_symbol(L):
    nm = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True,
                        check=True).stdout
    exported = set(re.findall(r"\b(mtgp_[a-z0-9_]+)\b", nm))
    missing = [f for f in header_functions() if f not in exported]
    assert not missing, missing
    assert sorted(L.exported_symbols()) == header_functions()
    assert L.LIB.mtgp_version().decode().startswith("libmtgp")


def test_no_oracle_in_product():
    # the product path never references the oracle
    pkg = os.path.join(ROOT, "paper_1005_4973_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "orc_" not in text, f


def _lib_params(L, mexp, seed, gid):
    import ctypes
    p = L.mtgp_params()
    L.check(L.LIB.mtgp_params_draw(mexp, seed, gid, ctypes.byref(p)))
    return p


@pytest.mark.parametrize("mexp", [89, 107, 127, 521, 607, 1279, 11213, 23209, 44497, 86243, 110503])
def test_params_draw_matches_oracle(L, mexp):
    for seed in (0, 1, 2, 127, 128, 2**40 + 5):
        for gid in (0, 5, 0xFFFFFFFF, 0x89ABCDEF):
            a = _lib_params(L, mexp, seed, gid)
            b = O.params_draw(mexp, seed, gid)
            assert (a.mexp, a.N, a.r, a.mask, a.pos, a.sh1, a.sh2, a.id) == \
                (b.mexp, b.N, b.r, b.mask, b.pos, b.sh1, b.sh2, b.id)
            assert list(a.rec_tbl) == list(b.rectbl)
            assert list(a.tmp_tbl) == list(b.tmptbl)
            L.check(L.LIB.mtgp_params_validate(__import__("ctypes").byref(a)))


def test_params_validate_rejects(L):
    import ctypes
    base = _lib_params(L, 11213, 1, 0)

    def bad(**kw):
        p = L.mtgp_params()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(base), ctypes.sizeof(p))
        for k, v in kw.items():
            if k in ("rec0", "tmp3"):
                (p.rec_tbl if k == "rec0" else p.tmp_tbl)[0 if k == "rec0" else 3] ^= v
            else:
                setattr(p, k, v)
        st = L.LIB.mtgp_params_validate(ctypes.byref(p))
        assert st == L.MTGP_EINVAL, kw
        assert L.last_error()

    bad(N=350)
    bad(mask=0xFFFFFFFF)
    bad(pos=1)
    bad(pos=351)
    bad(sh1=0)
    bad(sh2=32)
    bad(rec0=1)            # rec_tbl[0] != 0: not linear
    bad(tmp3=0x100)        # breaks tmp[3] = tmp[1] ^ tmp[2]
    bad(mexp=64)
    p = L.mtgp_params()
    assert L.LIB.mtgp_params_draw(200000, 1, 0, ctypes.byref(p)) == L.MTGP_EINVAL   # N > MTGP_MAX_N
    assert L.LIB.mtgp_params_draw(11213, 1, 0, None) == L.MTGP_EINVAL


def test_singular_lsb_block_rejected(L):
    import ctypes
    p = _lib_params(L, 11213, 3, 0)
    # rows with LSB nibbles making I + R4 singular: rows 0 and 1 give the same row of I + R4
    R = [0x10000008 ^ 0x8, 0x20000004 ^ 0x4, 0x40000002, 0x80000001]
    R[1] = (R[1] & ~0xF) | ((R[0] & 0xF) ^ 0x8 ^ 0x4)
    tbl = O.table_from_rows(R)
    assert not O.lsb_block_invertible(R)
    for b in range(16):
        p.rec_tbl[b] = int(tbl[b])
    assert L.LIB.mtgp_params_validate(ctypes.byref(p)) == L.MTGP_EINVAL


def test_import_without_library_fails_loudly(tmp_path):
    # a copy of the binding with no built library raises ImportError on first use
    import shutil
    import sys
    pkg = tmp_path / "paper_1005_4973_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_1005_4973_gb300"), pkg,
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    code = "import paper_1005_4973_gb300 as M\ntry:\n    M.Pool\nexcept ImportError as e:\n    print('IMPORTERROR', e)\n"
    r = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert "IMPORTERROR" in r.stdout and "no fallback" in r.stdout
