"""The oracle's pins discriminate: plausible mistakes planted in a copy of the
oracle (on the CPU, in a temporary directory) each make the pin tests fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "middle-word-off-by-one": ("u = t ^ (x[k + M] >> p->sh2);", "u = t ^ (x[k + M - 1] >> p->sh2);"),
    "mask-dropped": ("t = x[k + 1] ^ (x[k] & p->mask);", "t = x[k + 1] ^ (x[k]);"),
    "sh1-wrong-direction": ("t ^= t << p->sh1;", "t ^= t >> p->sh1;"),
    "tempering-word": ("uint32_t t = x[M - 1 + k] ^ (x[M - 1 + k] >> 16);",
                       "uint32_t t = x[M + k] ^ (x[M + k] >> 16);"),
    "tempering-shift-dropped": ("        t ^= t >> 8;\n        if (dtype", "        if (dtype"),
    "table-bit-order": ("if ((b >> (3u - j)) & 1u) v ^= rows[j];", "if ((b >> j) & 1u) v ^= rows[j];"),
    "lookup-index": ("x[N + k] = u ^ p->rectbl[u & 0xfu];", "x[N + k] = u ^ p->rectbl[(u >> 1) & 0xfu];"),
    "single-table-shift": ("(p->tmptbl[b] >> 9)", "(p->tmptbl[b] >> 8)"),
    "state-write-back": ("memcpy(state, x + n,", "memcpy(state, x + n + 1,"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "mtgp_oracle.c")).read()
    before, after = MUTANTS[name]
    assert before in src
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutants.py"))
    (tmp_path / "oracle" / "mtgp_oracle.c").write_text(src.replace(before, after, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=tmp_path, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, r.stdout[-2000:]
